// walldist.cu -- wall distance d(r) of the volume points (Section 4): the
// distance of each volume point from the nearest surface point, the input of
// the blending function psi (Eq. 23), which the paper takes as given.
//
// The query runs over the mesh's Morton-sorted surface point blocks (128
// consecutive sorted points with their bounding box).  One warp takes 32
// consecutive Morton-sorted volume points (a compact patch), so the warp
// decides together which point blocks to scan; each lane keeps its own
// nearest point.
//
//   pass A (search, FP32): start at the block whose centre is nearest to the
//     patch, then scan every block that may still hold a nearer point (box
//     distance below the lanes' current best).  Coordinates relative to the
//     block origin keep the FP32 error at the block's scale.  The winner's
//     distance, recomputed in FP64, is an upper bound U of the true minimum.
//   pass B (exact): scan the blocks whose box lies within U (conservative
//     box distances with directed rounding); an FP32 filter with a rigorous
//     rounding margin passes every point that may lie within the lane's
//     current minimum, and those are evaluated in FP64.  The result is the
//     minimum over the surface of the FP64 distance sqrt(sum (x_k - s_k)^2)
//     evaluated in axis order without contraction -- bit for bit the value of
//     a plain brute-force minimum, whatever order the points are visited in.
//
// An optional cap c returns min(d, c): the volume update needs d only below
// max_l D_l (volume point reduction), so points farther away finish after the
// box tests.
#include <cmath>

#include "common.cuh"
#include "internal.h"

namespace rbfd {

namespace {

constexpr int kWarps = 4;
constexpr int kThreads = 32 * kWarps;

inline unsigned cdiv(size_t a, size_t b) { return (unsigned)((a + b - 1) / b); }

// Per point block, in FP32: box rounded outward [lo, hi], its centre and the
// block origin (the FP64 box corner rounded to nearest).
__global__ void k_pb_fbox(const double4 *__restrict__ lo, const double4 *__restrict__ hi, int n_pb,
                          float4 *__restrict__ fb) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n_pb) return;
    double4 l = lo[b], h = hi[b];
    fb[b] = make_float4(__double2float_rd(l.x), __double2float_rd(l.y), __double2float_rd(l.z), 0.f);
    fb[n_pb + b] = make_float4(__double2float_ru(h.x), __double2float_ru(h.y), __double2float_ru(h.z), 0.f);
    fb[2 * n_pb + b] = make_float4((float)(0.5 * (l.x + h.x)), (float)(0.5 * (l.y + h.y)), (float)(0.5 * (l.z + h.z)),
                                   0.f);
    // largest coordinate of a point relative to the origin (bounds the FP32 error of the block)
    double ext = fmax(fmax(h.x - l.x, h.y - l.y), h.z - l.z);
    fb[3 * n_pb + b] = make_float4((float)l.x, (float)l.y, (float)l.z, __double2float_ru(ext));
}

struct WallArgs {
    int64_t n;               // volume points (Morton-sorted)
    const double4 *vpos;     // their coordinates (FP64; w unused on input)
    int64_t n_s;
    int n_pb;
    const double4 *xs;       // sorted surface points (FP64)
    const float4 *xs_hi;     // the same relative to the block origin, rounded to FP32
    const double4 *pb_lo;    // block origins (FP64 box corner)
    const float4 *fb;        // [4][n_pb] FP32 boxes (outward), centres, origins + extents
    double cap;              // return min(d, cap); +inf for the plain distance
    double *d_out;           // [n] sorted order, or nullptr:
    double4 *w_out;          //   write vpos[i].w instead
    unsigned long long *pairs;  // [2]: pairs scanned in pass A, pass B (nullable)
};

// Lower bound of the squared distance between the boxes [alo, ahi] and
// [blo, bhi]: each step rounds down, so the result never exceeds the true value.
template <int DIM>
__device__ __forceinline__ float box_gap2_rd(float3 alo, float3 ahi, float4 blo, float4 bhi) {
    float gx = fmaxf(0.f, fmaxf(__fsub_rd(blo.x, ahi.x), __fsub_rd(alo.x, bhi.x)));
    float gy = fmaxf(0.f, fmaxf(__fsub_rd(blo.y, ahi.y), __fsub_rd(alo.y, bhi.y)));
    float s = __fadd_rd(__fmul_rd(gx, gx), __fmul_rd(gy, gy));
    if (DIM == 3) {
        float gz = fmaxf(0.f, fmaxf(__fsub_rd(blo.z, ahi.z), __fsub_rd(alo.z, bhi.z)));
        s = __fadd_rd(s, __fmul_rd(gz, gz));
    }
    return s;
}

__device__ __forceinline__ float warp_max_f(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Stage the relative coordinates of block b in the warp's shared buffer.
__device__ __forceinline__ int stage_block(const WallArgs &a, int b, float4 *sp, int lane) {
    const int64_t base = (int64_t)b * kPB;
    const int cnt = (int)(a.n_s - base < kPB ? a.n_s - base : kPB);
    __syncwarp();
    for (int k = lane; k < cnt; k += 32) sp[k] = a.xs_hi[base + k];
    __syncwarp();
    return cnt;
}

template <int DIM>
__global__ void __launch_bounds__(kThreads) k_wall_dist(WallArgs a) {
    __shared__ float4 s_pts[kWarps][kPB];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * kWarps + warp) * 32;
    if (w0 >= a.n) return;  // whole warp past the end (warp-uniform)
    float4 *sp = s_pts[warp];
    const int64_t i = w0 + lane;
    const bool valid = i < a.n;
    const double4 p = valid ? a.vpos[i] : a.vpos[w0];
    const int n_pb = a.n_pb;
    const float4 *fb_lo = a.fb, *fb_hi = a.fb + n_pb, *fb_c = a.fb + 2 * n_pb, *fb_o = a.fb + 3 * n_pb;

    // the patch's box (rounded outward) and each lane's own point box
    const float3 plo = make_float3(__double2float_rd(p.x), __double2float_rd(p.y), __double2float_rd(p.z));
    const float3 pub = make_float3(__double2float_ru(p.x), __double2float_ru(p.y), __double2float_ru(p.z));
    float3 wlo = valid ? plo : make_float3(INFINITY, INFINITY, INFINITY);
    float3 whi = valid ? pub : make_float3(-INFINITY, -INFINITY, -INFINITY);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        wlo.x = fminf(wlo.x, __shfl_xor_sync(0xffffffffu, wlo.x, o));
        wlo.y = fminf(wlo.y, __shfl_xor_sync(0xffffffffu, wlo.y, o));
        wlo.z = fminf(wlo.z, __shfl_xor_sync(0xffffffffu, wlo.z, o));
        whi.x = fmaxf(whi.x, __shfl_xor_sync(0xffffffffu, whi.x, o));
        whi.y = fmaxf(whi.y, __shfl_xor_sync(0xffffffffu, whi.y, o));
        whi.z = fmaxf(whi.z, __shfl_xor_sync(0xffffffffu, whi.z, o));
    }
    const float pxf = (float)p.x, pyf = (float)p.y, pzf = (float)p.z;
    unsigned long long scanned_a = 0, scanned_b = 0;

    // ---------------------------------------------------------------- pass A
    const float cap2 = isinf(a.cap) ? INFINITY : __double2float_ru(a.cap * a.cap * (1.0 + 0x1p-20));
    float best2 = valid ? cap2 : -1.f;  // lanes past the end never ask for a block
    int64_t bidx = -1;
    auto visit_a = [&](int b) {
        const int cnt = stage_block(a, b, sp, lane);
        const float4 o = fb_o[b];
        const float qx = pxf - o.x, qy = pyf - o.y, qz = pzf - o.z;
        float bb = best2;
        int bk = -1;
#pragma unroll 8
        for (int k = 0; k < cnt; ++k) {
            const float4 s = sp[k];
            const float dx = qx - s.x, dy = qy - s.y;
            float d2 = fmaf(dy, dy, dx * dx);
            if (DIM == 3) {
                const float dz = qz - s.z;
                d2 = fmaf(dz, dz, d2);
            }
            if (d2 < bb) {
                bb = d2;
                bk = k;
            }
        }
        if (valid && bk >= 0) {
            best2 = bb;
            bidx = (int64_t)b * kPB + bk;
        }
        scanned_a += (unsigned long long)cnt;
    };

    // start block: centre nearest to the patch centre (lowest index on ties)
    {
        const float cx = 0.5f * (wlo.x + whi.x), cy = 0.5f * (wlo.y + whi.y), cz = 0.5f * (wlo.z + whi.z);
        float bd = INFINITY;
        int bb = 0x7fffffff;
        for (int b = lane; b < n_pb; b += 32) {
            const float4 c = fb_c[b];
            const float dx = c.x - cx, dy = c.y - cy, dz = (DIM == 3) ? c.z - cz : 0.f;
            const float d = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
            if (d < bd) {
                bd = d;
                bb = b;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float od = __shfl_xor_sync(0xffffffffu, bd, o);
            const int ob = __shfl_xor_sync(0xffffffffu, bb, o);
            if (od < bd || (od == bd && ob < bb)) {
                bd = od;
                bb = ob;
            }
        }
        if (bb >= n_pb) bb = 0;  // every centre distance non-finite: start anywhere
        const int start = bb;
        visit_a(start);
        for (int b0 = 0; b0 < n_pb; b0 += 32) {
            const int b = b0 + lane;
            const float lb = (b < n_pb && b != start) ? box_gap2_rd<DIM>(wlo, whi, fb_lo[b], fb_hi[b]) : INFINITY;
            unsigned mask = __ballot_sync(0xffffffffu, lb < warp_max_f(best2));
            while (mask) {
                const int j = __ffs(mask) - 1;
                mask &= mask - 1;
                const int bj = b0 + j;
                const float lbj = __shfl_sync(0xffffffffu, lb, j);
                if (!(lbj < warp_max_f(best2))) continue;
                const bool want = box_gap2_rd<DIM>(plo, pub, fb_lo[bj], fb_hi[bj]) < best2;
                if (!__any_sync(0xffffffffu, want)) continue;
                visit_a(bj);
            }
        }
    }

    // ---------------------------------------------------------------- pass B
    // dmin: an FP64 distance actually attained (so >= the FP64 minimum), or the cap
    double dmin = a.cap;
    if (valid && bidx >= 0) {
        const double4 x = a.xs[bidx];
        dmin = fmin(dmin, dist_f64<DIM>(p.x, p.y, p.z, x.x, x.y, x.z));
    }
    // squared search radius for the box tests, rounded up with a margin
    auto radius2 = [&]() -> float {
        if (!valid) return -1.f;
        if (isinf(dmin)) return INFINITY;
        return __double2float_ru(dmin * dmin * (1.0 + 0x1p-18));
    };
    float r2 = radius2();
    for (int b0 = 0; b0 < n_pb; b0 += 32) {
        const int b = b0 + lane;
        const float lb = (b < n_pb) ? box_gap2_rd<DIM>(wlo, whi, fb_lo[b], fb_hi[b]) : INFINITY;
        unsigned mask = __ballot_sync(0xffffffffu, lb <= warp_max_f(r2));
        while (mask) {
            const int j = __ffs(mask) - 1;
            mask &= mask - 1;
            const int bj = b0 + j;
            const float lbj = __shfl_sync(0xffffffffu, lb, j);
            if (!(lbj <= warp_max_f(r2))) continue;
            const bool want = box_gap2_rd<DIM>(plo, pub, fb_lo[bj], fb_hi[bj]) <= r2;
            if (!__any_sync(0xffffffffu, want)) continue;
            const int cnt = stage_block(a, bj, sp, lane);
            scanned_b += (unsigned long long)cnt;
            // q = p - origin, rounded once from FP64
            const double4 org = a.pb_lo[bj];
            const float ext = fb_o[bj].w;
            const float qx = __double2float_rn(p.x - org.x), qy = __double2float_rn(p.y - org.y),
                        qz = __double2float_rn(p.z - org.z);
            // Filter threshold.  Per axis the FP32 difference qx - s.x carries
            // three roundings (q, s, the subtraction), each below 2^-24 of
            // |q| + ext, so the computed difference vector is within
            // E = 2^-22 (|q|_1 + DIM ext) of the true one, and the two FMA
            // roundings of the squared sum add a relative 2^-23.  Any point
            // whose true distance is at most dmin therefore has a computed d2
            // below ((dmin + E)(1 + 2^-22))^2; we use twice each margin.
            float T = -1.f;
            if (want) {
                const double q1 = fabs((double)qx) + fabs((double)qy) + (DIM == 3 ? fabs((double)qz) : 0.0);
                const double E = 0x1p-21 * (q1 + DIM * (double)ext);
                const double t = (dmin + E) * (1.0 + 0x1p-21);
                T = isinf(t) ? INFINITY : __double2float_ru(t * t) + 1e-37f;
            }
            const int64_t base = (int64_t)bj * kPB;
#pragma unroll 4
            for (int k = 0; k < cnt; ++k) {
                const float4 s = sp[k];
                const float dx = qx - s.x, dy = qy - s.y;
                float d2 = fmaf(dy, dy, dx * dx);
                if (DIM == 3) {
                    const float dz = qz - s.z;
                    d2 = fmaf(dz, dz, d2);
                }
                if (d2 <= T) {
                    const double4 x = a.xs[base + k];
                    dmin = fmin(dmin, dist_f64<DIM>(p.x, p.y, p.z, x.x, x.y, x.z));
                }
            }
            r2 = radius2();
        }
    }

    if (valid) {
        const double d = fmin(dmin, a.cap);
        if (a.d_out)
            a.d_out[i] = d;
        else
            a.w_out[i].w = d;
    }
    if (a.pairs && lane == 0) {
        // scanned counts are warp-uniform: count them once per warp, times the lanes in use
        const unsigned long long nl = (unsigned long long)(a.n - w0 < 32 ? a.n - w0 : 32);
        atomicAdd(&a.pairs[0], scanned_a * nl);
        atomicAdd(&a.pairs[1], scanned_b * nl);
    }
}

}  // namespace

// Wall distance of n Morton-sorted points vpos (FP64): min(d, cap) into
// d_out[i] (sorted order), or into vpos[i].w when d_out is null.
void wall_distance_sorted(rbfd_mesh *m, int64_t n, double4 *vpos, double cap, double *d_out) {
    if (n <= 0) return;
    cudaStream_t st = m->stream;
    if (!m->d_pb_fbox) {
        m->d_pb_fbox = dalloc<float4>((size_t)4 * m->n_pb, "block boxes (FP32)");
        k_pb_fbox<<<cdiv(m->n_pb, 128), 128, 0, st>>>(m->d_pb_lo, m->d_pb_hi, m->n_pb, m->d_pb_fbox);
        RBFD_CUDA(cudaGetLastError());
        m->stats.launches += 1;
    }
    WallArgs a{};
    a.n = n;
    a.vpos = vpos;
    a.n_s = m->n_s;
    a.n_pb = m->n_pb;
    a.xs = m->d_xs;
    a.xs_hi = m->d_xs_hi;
    a.pb_lo = m->d_pb_lo;
    a.fb = m->d_pb_fbox;
    a.cap = cap;
    a.d_out = d_out;
    a.w_out = d_out ? nullptr : vpos;
    a.pairs = m->d_pairs + 4;
    const unsigned grid = cdiv((size_t)n, (size_t)kThreads);
    cudaEvent_t e0 = m->prof.begin(st);
    if (m->dim == 2)
        k_wall_dist<2><<<grid, kThreads, 0, st>>>(a);
    else
        k_wall_dist<3><<<grid, kThreads, 0, st>>>(a);
    RBFD_CUDA(cudaGetLastError());
    m->prof.end(kProfWall, e0, st, 1);
    m->stats.launches += 1;
}

}  // namespace rbfd
