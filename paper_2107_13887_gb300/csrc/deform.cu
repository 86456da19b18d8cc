// deform.cu -- volume update with volume point reduction (Section 4, Eq. 19
// and Eq. 23):
//
//   dV_v = sum_l psi(d_v / D_l) sum_j alpha_j^(l) phi(|r_v - r_cj^(l)| / R_l),
//   psi(xi) = 1 - xi on [0, 1), 0 beyond,   D_l = k max_i |dS_l,i| (capped at D).
//
// Steps: (1) keep only the volume points with d < max_l D_l (stream
// compaction); (2) Morton-sort those points so that a block of 128
// consecutive points is spatially compact; (3) per level, compact the sorted
// points further to d < D_l and run the fused evaluation: each block takes the
// controls of every cell of the level's uniform grid (cell size R_l) that
// overlaps its bounding box grown by R_l, stages them tile by tile in shared
// memory, and accumulates alpha phi for its points; (4) scatter the blended
// displacement back to the caller's order.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "internal.h"

namespace rbfd {

namespace {

constexpr int kThreads = 128;

inline unsigned cdiv(size_t a, size_t b) { return (unsigned)((a + b - 1) / b); }

__global__ void k_vol_pack(const void *__restrict__ xyz, const void *__restrict__ d, int64_t n, int dim, int f64,
                           double4 *__restrict__ out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double x, y, z = 0.0, w;
    if (f64) {
        const double *p = static_cast<const double *>(xyz) + i * dim;
        x = p[0];
        y = p[1];
        if (dim == 3) z = p[2];
        w = d ? static_cast<const double *>(d)[i] : 0.0;
    } else {
        const float *p = static_cast<const float *>(xyz) + i * dim;
        x = p[0];
        y = p[1];
        if (dim == 3) z = p[2];
        w = d ? static_cast<const float *>(d)[i] : 0.0;
    }
    out[i] = make_double4(x, y, z, w < 0.0 ? 0.0 : w);
}

__global__ void k_flag_below(const double4 *__restrict__ p, const uint32_t *__restrict__ idx, int64_t n, double D,
                             uint32_t *__restrict__ flag, const double *__restrict__ D_dev = nullptr) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (D_dev) D = *D_dev;
    double d = p[idx ? idx[i] : i].w;
    flag[i] = (d < D) ? 1u : 0u;
}

// D_l of levels 0..L-1 on the device, exactly as the host forms it from the
// level's max |dS_l| (k max|dS_l| capped at D when k > 0, else D), and its
// FP32 inverse; flags *mismatch if D_0 differs from d0 (the D_0 a staged
// volume's early level-0 sweep used).
__global__ void k_level_D(const double *__restrict__ hist, int L, double k, double D, double *__restrict__ Dl,
                          float *__restrict__ invDlf, double d0, unsigned *__restrict__ mismatch) {
    const int l = threadIdx.x;
    if (l >= L) return;
    double v = (k > 0.0) ? k * __dsqrt_rn(hist[l]) : D;
    if (k > 0.0 && D > 0.0 && v > D) v = D;
    Dl[l] = v;
    invDlf[l] = v > 0.0 ? (float)(1.0 / v) : 0.f;
    if (l == 0 && mismatch && v != d0) *mismatch = 1u;
}

__global__ void k_compact(const uint32_t *__restrict__ flag, const uint32_t *__restrict__ pos, int64_t n,
                          uint32_t *__restrict__ out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (flag[i]) out[pos[i]] = (uint32_t)i;
}

__global__ void k_bbox_idx(const double4 *__restrict__ p, const uint32_t *__restrict__ idx, int64_t n,
                           double *__restrict__ part) {
    __shared__ double s[6][32];
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double4 q = p[idx[i]];
        lo[0] = fmin(lo[0], q.x); lo[1] = fmin(lo[1], q.y); lo[2] = fmin(lo[2], q.z);
        hi[0] = fmax(hi[0], q.x); hi[1] = fmax(hi[1], q.y); hi[2] = fmax(hi[2], q.z);
    }
    for (int o = 16; o > 0; o >>= 1)
        for (int k = 0; k < 3; ++k) {
            lo[k] = fmin(lo[k], __shfl_xor_sync(0xffffffffu, lo[k], o));
            hi[k] = fmax(hi[k], __shfl_xor_sync(0xffffffffu, hi[k], o));
        }
    int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0)
        for (int k = 0; k < 3; ++k) {
            s[k][w] = lo[k];
            s[3 + k][w] = hi[k];
        }
    __syncthreads();
    if (threadIdx.x < 6) {
        double v = s[threadIdx.x][0];
        for (int j = 1; j < (int)(blockDim.x >> 5); ++j)
            v = threadIdx.x < 3 ? fmin(v, s[threadIdx.x][j]) : fmax(v, s[threadIdx.x][j]);
        part[blockIdx.x * 6 + threadIdx.x] = v;
    }
}

__global__ void k_bbox_partial_v(const double4 *__restrict__ p, int64_t n, double *__restrict__ part) {
    __shared__ double s[6][32];
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double4 q = p[i];
        lo[0] = fmin(lo[0], q.x); lo[1] = fmin(lo[1], q.y); lo[2] = fmin(lo[2], q.z);
        hi[0] = fmax(hi[0], q.x); hi[1] = fmax(hi[1], q.y); hi[2] = fmax(hi[2], q.z);
    }
    for (int o = 16; o > 0; o >>= 1)
        for (int k = 0; k < 3; ++k) {
            lo[k] = fmin(lo[k], __shfl_xor_sync(0xffffffffu, lo[k], o));
            hi[k] = fmax(hi[k], __shfl_xor_sync(0xffffffffu, hi[k], o));
        }
    int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0)
        for (int k = 0; k < 3; ++k) {
            s[k][w] = lo[k];
            s[3 + k][w] = hi[k];
        }
    __syncthreads();
    if (threadIdx.x < 6) {
        double v = s[threadIdx.x][0];
        for (int j = 1; j < (int)(blockDim.x >> 5); ++j)
            v = threadIdx.x < 3 ? fmin(v, s[threadIdx.x][j]) : fmax(v, s[threadIdx.x][j]);
        part[blockIdx.x * 6 + threadIdx.x] = v;
    }
}

// Final box from nb per-block partials [nb][6] (lo xyz, hi xyz): one warp per
// coordinate bound, lanes striding over the partials (min / max are exact, so
// the order does not matter).
__global__ void k_bbox_reduce(const double *__restrict__ part, int nb, double *__restrict__ out) {
    const int q = threadIdx.x >> 5, lane = threadIdx.x & 31;  // 6 warps
    if (q >= 6) return;
    double v = q < 3 ? INFINITY : -INFINITY;
    for (int b = lane; b < nb; b += 32) v = q < 3 ? fmin(v, part[b * 6 + q]) : fmax(v, part[b * 6 + q]);
    for (int o = 16; o > 0; o >>= 1) {
        const double w = __shfl_xor_sync(0xffffffffu, v, o);
        v = q < 3 ? fmin(v, w) : fmax(v, w);
    }
    if (lane == 0) out[q] = v;
}

__global__ void k_gather_vol(const double4 *__restrict__ p, const uint32_t *__restrict__ order, int64_t n,
                             double4 *__restrict__ out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    out[i] = p[order[i]];
}

__global__ void k_gather_u32(const uint32_t *__restrict__ src, const uint32_t *__restrict__ idx, int64_t n,
                             uint32_t *__restrict__ out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    out[i] = src[idx[i]];
}

__global__ void k_scatter_d(const double *__restrict__ d, const uint32_t *__restrict__ orig, int64_t n,
                            double *__restrict__ out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    out[orig[i]] = d[i];
}

__global__ void k_scatter_out(const double4 *__restrict__ acc, const uint32_t *__restrict__ orig, int64_t n,
                              int dim, int f64, void *__restrict__ out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double4 a = acc[i];
    int64_t o = orig[i];
    if (f64) {
        double *q = static_cast<double *>(out) + o * dim;
        q[0] = a.x;
        q[1] = a.y;
        if (dim == 3) q[2] = a.z;
    } else {
        float *q = static_cast<float *>(out) + o * dim;
        q[0] = (float)a.x;
        q[1] = (float)a.y;
        if (dim == 3) q[2] = (float)a.z;
    }
}

__device__ __forceinline__ uint32_t blk_excl_scan(uint32_t v, uint32_t *sw, uint32_t *total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sw[w] = x;
    __syncthreads();
    if (w == 0) {
        uint32_t t = lane < nw ? sw[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < nw) sw[lane] = t;
    }
    __syncthreads();
    uint32_t before = (w > 0 ? sw[w - 1] : 0u) + x - v;
    *total = sw[nw - 1];
    __syncthreads();
    return before;
}

struct VolArgs {
    int64_t n_list;
    const uint32_t *n_list_dev;  // if set: the list length in device memory (n_list is then an upper bound)
    const uint32_t *list;   // sorted positions of the points with d < D_l
    const double4 *vpos;    // sorted points (x, y, z, d)
    double4 *vacc;          // accumulated displacement per sorted point (FP32-input path: double-float)
    const double4 *cx, *alpha;
    const uint32_t *cell_start, *cell_ctrl;
    double3 g0;
    double h, R, Dl;
    int3 gd;
    float invR_hi, invR_lo;
    unsigned long long *pairs;
    // FP32-input path (mode 2): the same points as float4, the level's controls
    // and weights as double-float, the grid in FP32
    const float4 *vp4;
    const float4 *cdf;      // [2n]: coordinates hi, lo
    const float4 *adf;      // [2n]: (ax hi, ax lo, ay hi, ay lo), (az hi, az lo, -, -)
    float g0f[3], hf, Rf, invDlf;
    // if set: D_l and its FP32 inverse in device memory (they replace Dl, invDlf)
    const double *Dl_dev;
    const float *invDlf_dev;
    // FP32-input path: the level's control records in the grid's cell order
    // (4 float4 each), staged by bulk copies; err: set if a staging wait ran out
    const float4 *rec;
    unsigned *err;
};

// ---- bulk copies global -> shared completing on an mbarrier (the TMA
// engine's 1D form): a cell's controls are contiguous records, so one copy
// per (cell, tile) segment replaces a gather by every thread
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// bounded: false if the phase did not complete within `limit` polls
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity, unsigned limit) {
    for (unsigned i = 0; i < limit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, unsigned bytes, uint64_t *bar) {
    // the shared destination was read through the generic proxy before
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

constexpr unsigned kStagePolls = 1u << 22;  // polls of a staging wait (each may suspend briefly): seconds at most

template <int DIM, int BASIS, int MODE>
__global__ void __launch_bounds__(kThreads) k_vol_sweep(VolArgs a) {
    __shared__ double sb[6][kThreads / 32];
    __shared__ uint32_t s_start[kThreads], s_off[kThreads], sw[32];
    __shared__ double t64[6][kTile];
    __shared__ float t32[12][kTile];
    __shared__ unsigned char s_hits[4][kTile];
    const int tid = threadIdx.x;
    const int64_t n_list = a.n_list_dev ? (int64_t)*a.n_list_dev : a.n_list;
    if ((int64_t)blockIdx.x * kThreads >= n_list) return;  // (block-uniform)
    const int64_t i = (int64_t)blockIdx.x * kThreads + tid;
    const bool valid = i < n_list;
    const uint32_t s = valid ? a.list[i] : 0u;
    const double4 P = valid ? a.vpos[s] : make_double4(0, 0, 0, 0);
    // block bounding box
    double lo[3] = {valid ? P.x : INFINITY, valid ? P.y : INFINITY, valid ? P.z : INFINITY};
    double hi[3] = {valid ? P.x : -INFINITY, valid ? P.y : -INFINITY, valid ? P.z : -INFINITY};
    for (int o = 16; o > 0; o >>= 1)
        for (int k = 0; k < 3; ++k) {
            lo[k] = fmin(lo[k], __shfl_xor_sync(0xffffffffu, lo[k], o));
            hi[k] = fmax(hi[k], __shfl_xor_sync(0xffffffffu, hi[k], o));
        }
    if ((tid & 31) == 0)
        for (int k = 0; k < 3; ++k) {
            sb[k][tid >> 5] = lo[k];
            sb[3 + k][tid >> 5] = hi[k];
        }
    __syncthreads();
    for (int k = 0; k < 3; ++k) {
        lo[k] = sb[k][0];
        hi[k] = sb[3 + k][0];
        for (int q = 1; q < kThreads / 32; ++q) {
            lo[k] = fmin(lo[k], sb[k][q]);
            hi[k] = fmax(hi[k], sb[3 + k][q]);
        }
    }
    auto cidx = [&](double v, double g, int nmax) {
        double f = floor((v - g) / a.h);
        f = fmin(fmax(f, 0.0), (double)(nmax - 1));
        return (int)f;
    };
    const int ix0 = cidx(lo[0] - a.R, a.g0.x, a.gd.x), ix1 = cidx(hi[0] + a.R, a.g0.x, a.gd.x);
    const int iy0 = cidx(lo[1] - a.R, a.g0.y, a.gd.y), iy1 = cidx(hi[1] + a.R, a.g0.y, a.gd.y);
    const int iz0 = DIM == 3 ? cidx(lo[2] - a.R, a.g0.z, a.gd.z) : 0;
    const int iz1 = DIM == 3 ? cidx(hi[2] + a.R, a.g0.z, a.gd.z) : 0;
    const int nx = ix1 - ix0 + 1, ny = iy1 - iy0 + 1, nz = iz1 - iz0 + 1;
    const int ncr = nx * ny * nz;

    // point coordinates: FP64 absolute, or double-float relative to the box corner
    df qx{0, 0}, qy{0, 0}, qz{0, 0};
    if (MODE == 1) {
        qx = df_from_double(P.x - lo[0]);
        qy = df_from_double(P.y - lo[1]);
        qz = df_from_double(P.z - lo[2]);
    }
    const df invR = {a.invR_hi, a.invR_lo};
    double acc64[3] = {0, 0, 0};
    df acc[3] = {{0, 0}, {0, 0}, {0, 0}};
    unsigned useful = 0;
    unsigned long long visited = 0;
    float3 wlo, whi;
    if (MODE == 1) warp_box(valid, qx.hi, qy.hi, qz.hi, wlo, whi);
    const float R2m = (float)(1.002 * a.R) * (float)(1.002 * a.R);  // filter margin
    for (int cb = 0; cb < ncr; cb += kThreads) {
        const int c = cb + tid;
        uint32_t cnt = 0, st0 = 0;
        if (c < ncr) {
            int ix = ix0 + c % nx, iy = iy0 + (c / nx) % ny, iz = iz0 + c / (nx * ny);
            int cell = (iz * a.gd.y + iy) * a.gd.x + ix;
            st0 = a.cell_start[cell];
            cnt = a.cell_start[cell + 1] - st0;
        }
        uint32_t T;
        uint32_t off = blk_excl_scan(cnt, sw, &T);
        s_start[tid] = st0;
        s_off[tid] = off;
        __syncthreads();
        for (uint32_t w0 = 0; w0 < T; w0 += kTile) {
            const int m = (int)min((uint32_t)kTile, T - w0);
            if (tid < m) {
                uint32_t q = w0 + tid;
                int l = 0, r = kThreads;  // last k with s_off[k] <= q
                while (r - l > 1) {
                    int mid = (l + r) >> 1;
                    if (s_off[mid] <= q) l = mid;
                    else r = mid;
                }
                uint32_t j = a.cell_ctrl[s_start[l] + (q - s_off[l])];
                double4 cc = a.cx[j], al = a.alpha[j];
                if (MODE == 0) {
                    t64[0][tid] = cc.x; t64[1][tid] = cc.y; t64[2][tid] = cc.z;
                    t64[3][tid] = al.x; t64[4][tid] = al.y; t64[5][tid] = al.z;
                } else {
                    df rx = df_from_double(cc.x - lo[0]), ry = df_from_double(cc.y - lo[1]),
                       rz = df_from_double(cc.z - lo[2]);
                    df ax = df_from_double(al.x), ay = df_from_double(al.y), az = df_from_double(al.z);
                    t32[0][tid] = rx.hi; t32[1][tid] = rx.lo; t32[2][tid] = ry.hi; t32[3][tid] = ry.lo;
                    t32[4][tid] = rz.hi; t32[5][tid] = rz.lo; t32[6][tid] = ax.hi; t32[7][tid] = ax.lo;
                    t32[8][tid] = ay.hi; t32[9][tid] = ay.lo; t32[10][tid] = az.hi; t32[11][tid] = az.lo;
                }
            }
            __syncthreads();
            if (MODE == 0) {
                if (valid) {
                    visited += m;
                    for (int q = 0; q < m; ++q) {
                        double eta = __ddiv_rn(dist_f64<DIM>(P.x, P.y, P.z, t64[0][q], t64[1][q], t64[2][q]), a.R);
                        double f = phi_f64<BASIS>(eta);
                        useful += (eta < 1.0);
                        acc64[0] = __dadd_rn(acc64[0], __dmul_rn(t64[3][q], f));
                        acc64[1] = __dadd_rn(acc64[1], __dmul_rn(t64[4][q], f));
                        if (DIM == 3) acc64[2] = __dadd_rn(acc64[2], __dmul_rn(t64[5][q], f));
                    }
                }
            } else {
                // the whole warp takes part in the filter; lanes with a point accumulate
                const int nh = warp_hits<DIM>(t32, m, wlo, whi, R2m, s_hits[tid >> 5]);
                if (valid) {
                    visited += nh;
                    hits_accumulate_df<DIM, BASIS>(qx, qy, qz, t32, s_hits[tid >> 5], nh, invR, acc, useful);
                }
            }
            __syncthreads();
        }
    }
    if (MODE == 1) {
        acc64[0] = df_to_double(acc[0]);
        acc64[1] = df_to_double(acc[1]);
        acc64[2] = df_to_double(acc[2]);
    }
    if (valid) {
        const double Dl = a.Dl_dev ? *a.Dl_dev : a.Dl;
        const double w = __dsub_rn(1.0, __ddiv_rn(P.w, Dl));  // psi(d / D_l), d < D_l here
        double4 v = a.vacc[s];
        v.x = __dadd_rn(v.x, __dmul_rn(w, acc64[0]));
        v.y = __dadd_rn(v.y, __dmul_rn(w, acc64[1]));
        v.z = __dadd_rn(v.z, __dmul_rn(w, acc64[2]));
        a.vacc[s] = v;
    }
    unsigned u = useful;
    unsigned long long vv = visited;
    for (int o = 16; o > 0; o >>= 1) {
        u += __shfl_xor_sync(0xffffffffu, u, o);
        vv += __shfl_xor_sync(0xffffffffu, vv, o);
    }
    if ((tid & 31) == 0) {
        if (u) atomicAdd(&a.pairs[0], (unsigned long long)u);
        if (vv) atomicAdd(&a.pairs[1], vv);
    }
}

// The volume update for FP32 volume inputs in mixed precision: the same
// double-float pair evaluation as mode 1, with every per-point and per-tile
// step off the FP64 pipe (one FP64 warp instruction costs 64 cycles per SM
// sub-partition on this GPU): FP32 block box and cell range (one guard cell
// each side), block-relative coordinates by exact FP32 TwoSum, controls and
// weights pre-split per level, psi in FP32, double-float accumulator.
struct VolF32Smem {
    alignas(16) float4 rec[kTile][4];  // a tile of control records, as the bulk copies leave them
    uint64_t bar;                      // their mbarrier (one arrival with the tile's byte count)
    unsigned phase;                    // its current parity
    float sb[6][kThreads / 32];
    uint32_t s_start[kThreads], s_off[kThreads], sw[32];
    float t32[12][kTile];
    unsigned char s_hits[4][kTile];
};

// The block's mbarrier (once per launch, before its first tile).
__device__ __forceinline__ void vol_smem_init(VolF32Smem &sm) {
    if (threadIdx.x == 0) {
        mbar_init(&sm.bar, 1);
        sm.phase = 0;
    }
    __syncthreads();
}

// One block of 128 list entries (block index blk of the level's list).
// COHERENT: the accumulator is read through L2 (another block of the same
// launch may have written it: the work-list launch's earlier level).
template <int DIM, int BASIS, bool COHERENT>
__device__ __forceinline__ void vol_f32_block(const VolArgs &a, int64_t blk, VolF32Smem &sm) {
    auto &sb = sm.sb;
    auto &s_start = sm.s_start;
    auto &s_off = sm.s_off;
    auto &sw = sm.sw;
    auto &t32 = sm.t32;
    auto &s_hits = sm.s_hits;
    const int tid = threadIdx.x;
    const int64_t n_list = a.n_list_dev ? (int64_t)*a.n_list_dev : a.n_list;
    if (blk * kThreads >= n_list) return;  // (block-uniform)
    unsigned phase = sm.phase;  // the staging mbarrier's parity
    const int64_t i = blk * kThreads + tid;
    const bool valid = i < n_list;
    const uint32_t s = valid ? a.list[i] : 0u;
    const float4 P = valid ? a.vp4[s] : make_float4(0, 0, 0, 0);
    float lo[3] = {valid ? P.x : INFINITY, valid ? P.y : INFINITY, valid ? P.z : INFINITY};
    float hi[3] = {valid ? P.x : -INFINITY, valid ? P.y : -INFINITY, valid ? P.z : -INFINITY};
    for (int o = 16; o > 0; o >>= 1)
        for (int k = 0; k < 3; ++k) {
            lo[k] = fminf(lo[k], __shfl_xor_sync(0xffffffffu, lo[k], o));
            hi[k] = fmaxf(hi[k], __shfl_xor_sync(0xffffffffu, hi[k], o));
        }
    if ((tid & 31) == 0)
        for (int k = 0; k < 3; ++k) {
            sb[k][tid >> 5] = lo[k];
            sb[3 + k][tid >> 5] = hi[k];
        }
    __syncthreads();
    for (int k = 0; k < 3; ++k) {
        lo[k] = sb[k][0];
        hi[k] = sb[3 + k][0];
        for (int q = 1; q < kThreads / 32; ++q) {
            lo[k] = fminf(lo[k], sb[k][q]);
            hi[k] = fmaxf(hi[k], sb[3 + k][q]);
        }
    }
    // cell range of the box grown by R, one guard cell each side against FP32 rounding
    auto cidx = [&](float v, float g, int nmax, int guard) {
        float f = floorf((v - g) / a.hf) + (float)guard;
        f = fminf(fmaxf(f, 0.0f), (float)(nmax - 1));
        return (int)f;
    };
    const int ix0 = cidx(lo[0] - a.Rf, a.g0f[0], a.gd.x, -1), ix1 = cidx(hi[0] + a.Rf, a.g0f[0], a.gd.x, 1);
    const int iy0 = cidx(lo[1] - a.Rf, a.g0f[1], a.gd.y, -1), iy1 = cidx(hi[1] + a.Rf, a.g0f[1], a.gd.y, 1);
    const int iz0 = DIM == 3 ? cidx(lo[2] - a.Rf, a.g0f[2], a.gd.z, -1) : 0;
    const int iz1 = DIM == 3 ? cidx(hi[2] + a.Rf, a.g0f[2], a.gd.z, 1) : 0;
    const int nx = ix1 - ix0 + 1, ny = iy1 - iy0 + 1, nz = iz1 - iz0 + 1;
    const int ncr = nx * ny * nz;
    // point relative to the box corner: exact as a double-float (both are floats)
    const df qx = two_sum(P.x, -lo[0]), qy = two_sum(P.y, -lo[1]), qz = two_sum(P.z, -lo[2]);
    const df invR = {a.invR_hi, a.invR_lo};
    df acc[3] = {{0, 0}, {0, 0}, {0, 0}};
    unsigned useful = 0;
    unsigned long long visited = 0;
    float3 wlo, whi;
    warp_box(valid, qx.hi, qy.hi, qz.hi, wlo, whi);
    const float R2m = (1.002f * a.Rf) * (1.002f * a.Rf);  // filter margin
    for (int cb = 0; cb < ncr; cb += kThreads) {
        const int c = cb + tid;
        uint32_t cnt = 0, st0 = 0;
        if (c < ncr) {
            int ix = ix0 + c % nx, iy = iy0 + (c / nx) % ny, iz = iz0 + c / (nx * ny);
            int cell = (iz * a.gd.y + iy) * a.gd.x + ix;
            st0 = a.cell_start[cell];
            cnt = a.cell_start[cell + 1] - st0;
        }
        uint32_t T;
        uint32_t off = blk_excl_scan(cnt, sw, &T);
        s_start[tid] = st0;
        s_off[tid] = off;
        __syncthreads();
        for (uint32_t w0 = 0; w0 < T; w0 += kTile) {
            const int m = (int)min((uint32_t)kTile, T - w0);
            float4 ch, cl, a0, a1;
            if (a.rec) {
                // the tile's records by bulk copies, one per (cell, tile)
                // segment: a cell's controls are contiguous in the records
                if (tid == 0) mbar_arrive_expect_tx(&sm.bar, (unsigned)m * 64u);
                __syncthreads();
                const uint32_t s_lo = max(off, w0), s_hi = min(off + cnt, w0 + (uint32_t)m);
                if (s_hi > s_lo)
                    bulk_copy_g2s(&sm.rec[s_lo - w0][0], a.rec + 4 * (size_t)(st0 + (s_lo - off)), (s_hi - s_lo) * 64u,
                                  &sm.bar);
                const bool ok = mbar_wait(&sm.bar, phase, kStagePolls);
                if (!ok) {  // (not expected) record it, let the copies land, leave the block
                    atomicExch(a.err, 1u);
                    mbar_wait(&sm.bar, phase, kStagePolls);
                }
                if (__syncthreads_or(!ok)) return;  // the host reports RBFD_ETIMEOUT
                phase ^= 1u;
                if (tid < m) {
                    ch = sm.rec[tid][0];
                    cl = sm.rec[tid][1];
                    a0 = sm.rec[tid][2];
                    a1 = sm.rec[tid][3];
                }
            } else if (tid < m) {
                uint32_t q = w0 + tid;
                int l = 0, r = kThreads;  // last k with s_off[k] <= q
                while (r - l > 1) {
                    int mid = (l + r) >> 1;
                    if (s_off[mid] <= q) l = mid;
                    else r = mid;
                }
                const uint32_t j = a.cell_ctrl[s_start[l] + (q - s_off[l])];
                ch = a.cdf[2 * j];
                cl = a.cdf[2 * j + 1];
                a0 = a.adf[2 * j];
                a1 = a.adf[2 * j + 1];
            }
            if (tid < m) {
                const df rx = df_add({ch.x, cl.x}, {-lo[0], 0.f}), ry = df_add({ch.y, cl.y}, {-lo[1], 0.f}),
                         rz = df_add({ch.z, cl.z}, {-lo[2], 0.f});
                t32[0][tid] = rx.hi; t32[1][tid] = rx.lo; t32[2][tid] = ry.hi; t32[3][tid] = ry.lo;
                t32[4][tid] = rz.hi; t32[5][tid] = rz.lo; t32[6][tid] = a0.x; t32[7][tid] = a0.y;
                t32[8][tid] = a0.z; t32[9][tid] = a0.w; t32[10][tid] = a1.x; t32[11][tid] = a1.y;
            }
            __syncthreads();
            // the whole warp takes part in the filter; lanes with a point accumulate
            const int nh = warp_hits<DIM>(t32, m, wlo, whi, R2m, s_hits[tid >> 5]);
            if (valid) {
                visited += nh;
                hits_accumulate_df<DIM, BASIS>(qx, qy, qz, t32, s_hits[tid >> 5], nh, invR, acc, useful);
            }
            __syncthreads();
        }
    }
    if (valid) {
        const float w = 1.0f - P.w * (a.invDlf_dev ? *a.invDlf_dev : a.invDlf);  // psi(d / D_l), d < D_l here
        float4 *va = reinterpret_cast<float4 *>(a.vacc + s);
        const float4 v0 = COHERENT ? __ldcg(va) : va[0], v1 = COHERENT ? __ldcg(va + 1) : va[1];
        const df sx = df_add({v0.x, v0.y}, df_mul(acc[0], {w, 0.f}));
        const df sy = df_add({v0.z, v0.w}, df_mul(acc[1], {w, 0.f}));
        const df sz = df_add({v1.x, v1.y}, df_mul(acc[2], {w, 0.f}));
        va[0] = make_float4(sx.hi, sx.lo, sy.hi, sy.lo);
        va[1] = make_float4(sz.hi, sz.lo, 0.f, 0.f);
    }
    if (tid == 0) sm.phase = phase;  // (read by the block's next call after a block barrier)
    unsigned u = useful;
    unsigned long long vv = visited;
    for (int o = 16; o > 0; o >>= 1) {
        u += __shfl_xor_sync(0xffffffffu, u, o);
        vv += __shfl_xor_sync(0xffffffffu, vv, o);
    }
    if ((tid & 31) == 0) {
        if (u) atomicAdd(&a.pairs[0], (unsigned long long)u);
        if (vv) atomicAdd(&a.pairs[1], vv);
    }
}

template <int DIM, int BASIS>
__global__ void __launch_bounds__(kThreads, 8) k_vol_sweep_f32(VolArgs a) {
    __shared__ VolF32Smem sm;
    vol_smem_init(sm);
    vol_f32_block<DIM, BASIS, false>(a, (int64_t)blockIdx.x, sm);
}

// ------------------------------------------ work-list launch over meshes
//
// The volume sweeps of several meshes (and all their levels) in one
// persistent launch: entry e = (mesh, level), in level-major order; its work
// is the blocks of 128 entries of that level's list (the list length is read
// on the device).  Blocks take items of item_blocks consecutive blocks from a
// global counter as they come free, so small and large meshes share the SMs.
// A level of a mesh adds into the accumulator its previous level wrote: its
// items wait (bounded) until every block of the previous level is done.  The
// previous level's items have lower numbers, so they were taken earlier by
// blocks that are running: the wait always ends.
constexpr int kWLMax = 64;

struct WorkList {
    VolArgs e[kWLMax];
    int dep[kWLMax];             // the entry that must be complete first (-1: none)
    int n;                       // entries
    int item_blocks;             // list blocks per item
    unsigned int *ctl;           // [0] next item, [1] error (a wait ran out), [2 + e] blocks done of entry e
    unsigned int poll_limit;     // polls of a dependency before the launch gives up
};

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

template <int DIM, int BASIS>
__global__ void __launch_bounds__(kThreads, 8) k_vol_worklist(const __grid_constant__ WorkList w) {
    __shared__ VolF32Smem sm;
    __shared__ int s_pre[kWLMax + 1];
    __shared__ unsigned s_item;
    __shared__ int s_fail;
    vol_smem_init(sm);
    if (threadIdx.x == 0) {
        int acc = 0;
        for (int e = 0; e < w.n; ++e) {
            s_pre[e] = acc;
            const int64_t nl = w.e[e].n_list_dev ? (int64_t)*w.e[e].n_list_dev : w.e[e].n_list;
            acc += (int)((nl + kThreads - 1) / kThreads);
        }
        s_pre[w.n] = acc;
        s_fail = 0;
    }
    __syncthreads();
    const unsigned total = (unsigned)s_pre[w.n];
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(&w.ctl[0], (unsigned)w.item_blocks);
        __syncthreads();
        const unsigned it0 = s_item;
        __syncthreads();
        if (it0 >= total) break;
        const unsigned it1 = min(it0 + (unsigned)w.item_blocks, total);
        for (unsigned it = it0; it < it1; ++it) {
            int e = 0;
            while ((unsigned)s_pre[e + 1] <= it) ++e;
            const int dp = w.dep[e];
            if (dp >= 0 && threadIdx.x == 0) {
                const unsigned need = (unsigned)(s_pre[dp + 1] - s_pre[dp]);
                unsigned polls = 0;
                while (ld_acquire_u32(&w.ctl[2 + dp]) < need) {
                    if (++polls > w.poll_limit || ld_acquire_u32(&w.ctl[1])) {
                        atomicExch(&w.ctl[1], 1u);
                        s_fail = 1;
                        break;
                    }
                    __nanosleep(256);
                }
            }
            __syncthreads();
            if (s_fail) return;  // (block-uniform; the host reports the timeout)
            vol_f32_block<DIM, BASIS, true>(w.e[e], (int64_t)(it - (unsigned)s_pre[e]), sm);
            // every thread's accumulator stores before the block's count
            __threadfence();
            __syncthreads();
            if (threadIdx.x == 0) atomicAdd(&w.ctl[2 + e], 1u);
        }
    }
}

// Volume points taking part in a level, summed on the device (statistics).
__global__ void k_count_points(const uint32_t *__restrict__ n, unsigned long long *__restrict__ total) {
    if (threadIdx.x == 0) *total += *n;
}

// Sorted points as float4 for the FP32-input path.
__global__ void k_to_f4(const double4 *__restrict__ p, int64_t n, float4 *__restrict__ out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double4 q = p[i];
    out[i] = make_float4((float)q.x, (float)q.y, (float)q.z, (float)q.w);
}

// The double-float accumulator of the FP32-input path to the caller's order.
__global__ void k_scatter_out_df(const double4 *__restrict__ acc, const uint32_t *__restrict__ orig, int64_t n,
                                 int dim, float *__restrict__ out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float4 *va = reinterpret_cast<const float4 *>(acc + i);
    const float4 v0 = va[0], v1 = va[1];
    float *q = out + (int64_t)orig[i] * dim;
    q[0] = v0.x + v0.y;
    q[1] = v0.z + v0.w;
    if (dim == 3) q[2] = v1.x + v1.y;
}

template <int DIM, int BASIS>
void launch_vol_t(int mode, unsigned g, const VolArgs &a, cudaStream_t st) {
    if (mode == 0) k_vol_sweep<DIM, BASIS, 0><<<g, kThreads, 0, st>>>(a);
    else if (mode == 1) k_vol_sweep<DIM, BASIS, 1><<<g, kThreads, 0, st>>>(a);
    else k_vol_sweep_f32<DIM, BASIS><<<g, kThreads, 0, st>>>(a);
}

void launch_vol(int dim, int basis, int mode, unsigned g, const VolArgs &a, cudaStream_t st) {
    if (dim == 2) {
        switch (basis) {
        case 0: launch_vol_t<2, 0>(mode, g, a, st); break;
        case 4: launch_vol_t<2, 4>(mode, g, a, st); break;
        case 6: launch_vol_t<2, 6>(mode, g, a, st); break;
        default: launch_vol_t<2, 2>(mode, g, a, st); break;
        }
    } else {
        switch (basis) {
        case 0: launch_vol_t<3, 0>(mode, g, a, st); break;
        case 4: launch_vol_t<3, 4>(mode, g, a, st); break;
        case 6: launch_vol_t<3, 6>(mode, g, a, st); break;
        default: launch_vol_t<3, 2>(mode, g, a, st); break;
        }
    }
}

void reserve_volume(rbfd_mesh *m, size_t n) {
    if (n <= m->vol_cap) return;
    dfree(m->d_vin);
    dfree(m->d_vpos);
    dfree(m->d_vorig);
    dfree(m->d_vflag);
    dfree(m->d_vscan);
    dfree(m->d_vlist);
    dfree(m->d_vkeys);
    dfree(m->d_vacc);
    m->d_vin = nullptr;
    m->vol_cap = 0;
    m->d_vin = reinterpret_cast<float4 *>(dalloc<double4>(n, "volume points"));
    m->d_vpos = reinterpret_cast<float4 *>(dalloc<double4>(n, "sorted volume points"));
    m->d_vorig = dalloc<uint32_t>(n, "volume order");
    m->d_vflag = dalloc<uint32_t>(n, "volume flags");
    m->d_vscan = dalloc<uint32_t>(n, "volume scan");
    m->d_vlist = dalloc<uint32_t>(n, "volume list");
    m->d_vkeys = dalloc<uint32_t>(n, "volume keys");
    m->d_vacc = dalloc<double4>(n, "volume displacement");
    dfree(m->d_vpos4);
    m->d_vpos4 = nullptr;
    m->d_vpos4 = dalloc<float4>(n, "sorted volume points (FP32)");
    m->vol_cap = n;
}

// Morton order of n packed points vin: sorted copy into vsorted, caller
// index of each sorted point into orig.  Uses the mesh's key buffer.
void morton_order(rbfd_mesh *m, int64_t n, const double4 *vin, double4 *vsorted, uint32_t *orig,
                  cudaStream_t st, double *red, double *box, SortScratch &ss) {
    const int dim = m->dim;
    const int nbb = std::min<int>(cdiv(n, 256), 256);
    k_bbox_partial_v<<<nbb, 256, 0, st>>>(vin, n, red);
    k_bbox_reduce<<<1, 192, 0, st>>>(red, nbb, box);
    morton_keys_f64_dev(vin, n, dim, box, m->d_vkeys, orig, st, vol_key_shift(dim), true);  // (cubic cells)
    radix_sort_pairs(m->d_vkeys, orig, (size_t)n, kVolKeyBits, ss, st);
    k_gather_vol<<<cdiv(n, 256), 256, 0, st>>>(vin, orig, n, vsorted);
    RBFD_CUDA(cudaGetLastError());
    m->stats.launches += 4;
}

// Steps (3) and (4) of the volume update for nV Morton-sorted points vpos
// (caller indices vorig): per level, compaction to d < D_l and the fused
// evaluation into the accumulator; then the scatter into dout (caller order).
// The parts of steps (3) and (4) of the volume update for nV Morton-sorted
// points vpos (caller indices vorig), each on stream st: clear the
// accumulator (and make the float4 copy for the FP32-input sweep), then per
// level the compaction to d < D_l and the fused evaluation into the
// accumulator, then the scatter into dout (caller order).
bool deform_fast(const rbfd_mesh *m, bool f64) { return m->opt.precision != RBFD_FP64 && !f64 && m->d_vpos4; }

void deform_acc_init(rbfd_mesh *m, int64_t nV, const double4 *vpos, bool f64, cudaStream_t st) {
    RBFD_CUDA(cudaMemsetAsync(m->d_vacc, 0, sizeof(double4) * nV, st));
    if (deform_fast(m, f64)) {
        k_to_f4<<<cdiv(nV, 256), 256, 0, st>>>(vpos, nV, m->d_vpos4);
        m->stats.launches += 1;
    }
}

void deform_one_level(rbfd_mesh *m, int l, int64_t nV, const double4 *vpos, double Dl, bool f64, cudaStream_t st,
                      SortScratch &ss, const double *Dl_dev = nullptr, const float *invDlf_dev = nullptr) {
    const Level &Lv = m->levels[l];
    if (Lv.nc == 0 || (!Dl_dev && !(Dl > 0.0))) return;
    const bool fast = deform_fast(m, f64);
    const int mode = m->opt.precision == RBFD_FP64 ? 0 : (fast ? 2 : 1);
    // d < D_l, then the fused evaluation; the list length stays on the
    // device (the sweep reads it), so no level waits for the host
    k_flag_below<<<cdiv(nV, 256), 256, 0, st>>>(vpos, nullptr, nV, Dl, m->d_vflag, Dl_dev);
    exclusive_scan_u32(m->d_vflag, m->d_vscan, (size_t)nV, &m->d_misc[5], ss, st);
    k_compact<<<cdiv(nV, 256), 256, 0, st>>>(m->d_vflag, m->d_vscan, nV, m->d_vlist);
    k_count_points<<<1, 32, 0, st>>>(&m->d_misc[5], m->d_pairs + 7);
    VolArgs a{};
    a.n_list = nV;  // upper bound; the exact count is read on the device
    a.n_list_dev = &m->d_misc[5];
    a.list = m->d_vlist;
    a.vpos = vpos;
    a.vacc = m->d_vacc;
    a.cx = Lv.d_cx;
    a.alpha = Lv.d_alpha;
    a.cell_start = Lv.d_cell_start;
    a.cell_ctrl = Lv.d_cell_ctrl;
    a.g0 = Lv.g0;
    a.h = Lv.h;
    a.gd = Lv.gdim;
    a.R = Lv.R;
    a.Dl = Dl;
    double inv = 1.0 / Lv.R;
    a.invR_hi = (float)inv;
    a.invR_lo = (float)(inv - (double)a.invR_hi);
    a.pairs = m->d_pairs + 2;
    a.Dl_dev = Dl_dev;
    a.invDlf_dev = invDlf_dev;
    if (fast) {
        a.vp4 = m->d_vpos4;
        a.cdf = Lv.d_cdf;
        a.adf = Lv.d_adf;
        a.g0f[0] = (float)Lv.g0.x;
        a.g0f[1] = (float)Lv.g0.y;
        a.g0f[2] = (float)Lv.g0.z;
        a.hf = (float)Lv.h;
        a.Rf = (float)Lv.R;
        a.invDlf = Dl > 0.0 ? (float)(1.0 / Dl) : 0.f;
        a.rec = Lv.d_rec;
        a.err = &m->d_misc[12];
    }
    m->stats.launches += 4;  // flags, compaction, count (+ scan counted in the scan)
    cudaEvent_t e0 = m->prof.begin(st);
    launch_vol(m->dim, m->opt.basis, mode, cdiv(nV, kThreads), a, st);
    RBFD_CUDA(cudaGetLastError());
    m->prof.end(kProfVol, e0, st, 1);
    m->stats.launches += 1;
}

void deform_scatter(rbfd_mesh *m, int64_t nV, const uint32_t *vorig, void *dout, bool f64, cudaStream_t st) {
    if (deform_fast(m, f64))
        k_scatter_out_df<<<cdiv(nV, 256), 256, 0, st>>>(m->d_vacc, vorig, nV, m->dim, static_cast<float *>(dout));
    else
        k_scatter_out<<<cdiv(nV, 256), 256, 0, st>>>(m->d_vacc, vorig, nV, m->dim, f64 ? 1 : 0, dout);
    RBFD_CUDA(cudaGetLastError());
}

void deform_levels(rbfd_mesh *m, int64_t nV, const double4 *vpos, const uint32_t *vorig, const double *Dl, int L,
                   void *dout, bool f64) {
    deform_acc_init(m, nV, vpos, f64, m->stream);
    for (int l = 0; l < L; ++l) deform_one_level(m, l, nV, vpos, Dl[l], f64, m->stream, m->sort);
    deform_scatter(m, nV, vorig, dout, f64, m->stream);
}

}  // namespace

namespace {
// Staging streams, kept across meshes (creating one costs more than a launch).
std::mutex g_side_mu;
std::vector<std::pair<int, cudaStream_t>> g_side_free;

cudaStream_t side_acquire(int dev) {
    {
        std::lock_guard<std::mutex> lk(g_side_mu);
        for (size_t i = 0; i < g_side_free.size(); ++i)
            if (g_side_free[i].first == dev) {
                cudaStream_t s = g_side_free[i].second;
                g_side_free.erase(g_side_free.begin() + (std::ptrdiff_t)i);
                return s;
            }
    }
    // the lowest priority: the staged volume work fills the SMs the greedy leaves
    cudaStream_t s = nullptr;
    int lo = 0, hi = 0;
    RBFD_CUDA(cudaDeviceGetStreamPriorityRange(&lo, &hi));
    RBFD_CUDA(cudaStreamCreateWithPriority(&s, cudaStreamNonBlocking, lo));
    return s;
}

// The device copy of the volume inputs: the inputs themselves when they are
// device pointers, else the mesh's staging buffer filled on stream st.
struct VolumeIO {
    const void *x, *d;
    void *out;
};

VolumeIO volume_io(rbfd_mesh *m, int64_t n_v, const void *xyz_v, const void *d_v, void *out, bool f64,
                   cudaStream_t st, bool copy = true) {
    VolumeIO io{xyz_v, d_v, out};
    if (m->opt.inputs_on_device || n_v <= 0) return io;
    const int dim = m->dim;
    const size_t es = f64 ? sizeof(double) : sizeof(float);
    const size_t need = (size_t)n_v * dim * es * 2 + (size_t)n_v * es + 256;
    if (need > m->vio_bytes) {
        dfree(m->d_vio);
        m->d_vio = nullptr;
        m->vio_bytes = 0;
        m->d_vio = dmalloc(need, "volume staging");
        m->vio_bytes = need;
    }
    char *base = static_cast<char *>(m->d_vio);
    void *sx = base;
    void *sd = base + (size_t)n_v * dim * es;
    io.out = base + (size_t)n_v * dim * es + (((size_t)n_v * es + 255) / 256) * 256;
    if (copy) {
        RBFD_CUDA(cudaMemcpyAsync(sx, xyz_v, (size_t)n_v * dim * es, cudaMemcpyHostToDevice, st));
        if (d_v) RBFD_CUDA(cudaMemcpyAsync(sd, d_v, (size_t)n_v * es, cudaMemcpyHostToDevice, st));
    }
    io.x = sx;
    io.d = d_v ? sd : nullptr;
    return io;
}
}  // namespace

void volume_stage(rbfd_mesh *m, int64_t n_v, const void *xyz_v, const void *d_v, bool f64, double D, double k) {
    mesh_ready(m);  // (S0 gives D_0)
    volume_unstage(m);
    if (n_v <= 0 || !d_v) return;  // (wall distances on the device are capped by the levels' D_l)
    if (!m->vstream) m->vstream = side_acquire(m->device);
    if (!m->ev_vfork) RBFD_CUDA(cudaEventCreateWithFlags(&m->ev_vfork, cudaEventDisableTiming));
    if (!m->ev_vdone) RBFD_CUDA(cudaEventCreateWithFlags(&m->ev_vdone, cudaEventDisableTiming));
    if (!m->d_vred) m->d_vred = dalloc<double>(6 * 256, "volume box partials");
    if (!m->d_vbox) m->d_vbox = dalloc<double>(8, "volume box");
    if (!m->vsort.launches) m->vsort.launches = &m->stats.launches;
    reserve_volume(m, (size_t)n_v);
    // the staging stream starts from here (the inputs are ready in the
    // caller's order); its work is queued by volume_stage_enqueue, which the
    // greedy calls once its first launch is on its way
    RBFD_CUDA(cudaEventRecord(m->ev_vfork, m->stream));
    RBFD_CUDA(cudaStreamWaitEvent(m->vstream, m->ev_vfork, 0));
    const VolumeIO io = volume_io(m, n_v, xyz_v, d_v, nullptr, f64, m->vstream, false);
    m->vst_io_x = io.x;
    m->vst_io_d = io.d;
    m->vst_queued = false;
    // D_0 = k max|dS_0| (capped at D) is known now: max|dS_0| = S0
    double d0 = (k > 0.0) ? k * m->S0 : D;
    if (k > 0.0 && D > 0.0 && d0 > D) d0 = D;
    m->vst_D0 = d0;
    m->vst_l0 = false;
    m->vst_ok = true;
    m->vst_n = n_v;
    m->vst_x = xyz_v;
    m->vst_d = d_v;
    m->vst_f64 = f64;
    m->vst_dout = io.out;  // (null for device outputs: the caller's array)
}

void volume_stage_enqueue(rbfd_mesh *m) {
    if (!m->vst_ok || m->vst_queued) return;
    cudaStream_t vs = m->vstream;
    const int64_t n_v = m->vst_n;
    const bool f64 = m->vst_f64;
    if (!m->opt.inputs_on_device) {  // host inputs: into the staging buffer
        const size_t es = f64 ? sizeof(double) : sizeof(float);
        RBFD_CUDA(cudaMemcpyAsync(const_cast<void *>(m->vst_io_x), m->vst_x, (size_t)n_v * m->dim * es,
                                  cudaMemcpyHostToDevice, vs));
        RBFD_CUDA(cudaMemcpyAsync(const_cast<void *>(m->vst_io_d), m->vst_d, (size_t)n_v * es, cudaMemcpyHostToDevice,
                                  vs));
    }
    double4 *vin = reinterpret_cast<double4 *>(m->d_vin);
    double4 *vpos = reinterpret_cast<double4 *>(m->d_vpos);
    k_vol_pack<<<cdiv(n_v, 256), 256, 0, vs>>>(m->vst_io_x, m->vst_io_d, n_v, m->dim, f64 ? 1 : 0, vin);
    morton_order(m, n_v, vin, vpos, m->d_vorig, vs, m->d_vred, m->d_vbox, m->vsort);
    deform_acc_init(m, n_v, vpos, f64, vs);
    RBFD_CUDA(cudaEventRecord(m->ev_vdone, vs));
    RBFD_CUDA(cudaGetLastError());
    m->stats.launches += 1;
    m->vst_queued = true;
}

void volume_level_early(rbfd_mesh *m, int l) {
    volume_stage_enqueue(m);
    if (!m->vst_ok || l != 0 || m->vst_l0 || m->levels.empty() || !(m->vst_D0 > 0.0)) return;
    // the level's controls, weights and cell grid are queued on the mesh's stream
    RBFD_CUDA(cudaEventRecord(m->ev_vfork, m->stream));
    RBFD_CUDA(cudaStreamWaitEvent(m->vstream, m->ev_vfork, 0));
    deform_one_level(m, 0, m->vst_n, reinterpret_cast<const double4 *>(m->d_vpos), m->vst_D0, m->vst_f64, m->vstream,
                     m->vsort);
    RBFD_CUDA(cudaEventRecord(m->ev_vdone, m->vstream));
    m->vst_l0 = true;
}

void volume_unstage(rbfd_mesh *m) {
    if (!m->vst_ok) return;
    m->vst_ok = false;
    // its buffers are reused after this (nothing was queued: the fork is all)
    if (m->vst_queued) RBFD_CUDA(cudaStreamWaitEvent(m->stream, m->ev_vdone, 0));
}

void volume_stage_release(rbfd_mesh *m) {
    if (m->vstream) {
        cudaStreamSynchronize(m->vstream);
        std::lock_guard<std::mutex> lk(g_side_mu);
        g_side_free.push_back({m->device, m->vstream});
        m->vstream = nullptr;
    }
    if (m->ev_vfork) cudaEventDestroy(m->ev_vfork);
    if (m->ev_vdone) cudaEventDestroy(m->ev_vdone);
    m->ev_vfork = m->ev_vdone = nullptr;
    m->vsort.release();
    dfree(m->d_vred);
    dfree(m->d_vbox);
    m->d_vred = m->d_vbox = nullptr;
    m->vst_ok = false;
}

namespace {
// A staging wait of the FP32-input sweep that ran out (the sweep set the
// mesh's error word): reported as RBFD_ETIMEOUT (the stream is synchronised).
void vol_staging_check(rbfd_mesh *m) {
    uint32_t err = 0;
    RBFD_CUDA(cudaMemcpy(&err, &m->d_misc[12], sizeof(err), cudaMemcpyDeviceToHost));
    if (err) {
        RBFD_CUDA(cudaMemset(&m->d_misc[12], 0, sizeof(err)));
        fail(RBFD_ETIMEOUT, "volume update: a staging wait exceeded its bound");
    }
}
}  // namespace

void deform_run_impl(rbfd_mesh *m, int64_t n_v, const void *xyz_v, const void *d_v, bool f64, double D, double k,
                     void *out);

void deform_run(rbfd_mesh *m, int64_t n_v, const void *xyz_v, const void *d_v, bool f64, double D, double k,
                void *out) {
    NvtxRange nvtx("rbfd volume update");
    deform_run_impl(m, n_v, xyz_v, d_v, f64, D, k, out);
    vol_staging_check(m);
}

void deform_run_impl(rbfd_mesh *m, int64_t n_v, const void *xyz_v, const void *d_v, bool f64, double D, double k,
                     void *out) {
    cudaStream_t st = m->stream;
    const int dim = m->dim;
    const size_t es = f64 ? sizeof(double) : sizeof(float);
    RBFD_CUDA(cudaEventRecord(m->ev0, st));
    const int L = (int)m->levels.size();
    std::vector<double> Dl(L, 0.0);  // (filled once the levels' scalars are on the host)
    double Dmax = 0.0;
    const bool host = !m->opt.inputs_on_device;
    if (m->vst_ok && m->vst_n == n_v && m->vst_x == xyz_v && m->vst_d == d_v && m->vst_f64 == f64) {
        volume_stage_enqueue(m);
        // staged ahead: every point packed and Morton-sorted; the levels'
        // reductions d < D_l run over all of them (points beyond every D_l
        // stay 0)
        m->vst_ok = false;
        RBFD_CUDA(cudaStreamWaitEvent(st, m->ev_vdone, 0));
        void *dout = host ? m->vst_dout : out;
        const double4 *vs_pos = reinterpret_cast<const double4 *>(m->d_vpos);
        // level 0 may have run on the staging stream during the greedy (with
        // D_0 from S0; the same value as from the level, checked here)
        bool l0 = m->vst_l0;
        m->vst_l0 = false;
        if (m->greedy_pending && L > 0) {
            // the greedy's last wait has not happened (its work is queued
            // ahead on this stream): D_l from the levels' scalars on the
            // device, and no host wait between the greedy and this update
            RBFD_CUDA(cudaMemsetAsync(&m->d_misc[9], 0, sizeof(uint32_t), st));
            k_level_D<<<1, (unsigned)cdiv(L, 32) * 32, 0, st>>>(m->d_lvl_hist, L, k, D, m->d_Dl, m->d_invDlf,
                                                               m->vst_D0, l0 ? &m->d_misc[9] : nullptr);
            for (int l = l0 ? 1 : 0; l < L; ++l)
                deform_one_level(m, l, n_v, vs_pos, 0.0, f64, st, m->sort, m->d_Dl + l, m->d_invDlf + l);
            deform_scatter(m, n_v, m->d_vorig, dout, f64, st);
            RBFD_CUDA(cudaMemcpyAsync(m->h_prep, &m->d_misc[9], sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
            m->stats.launches += 1;
            if (host) RBFD_CUDA(cudaMemcpyAsync(out, dout, (size_t)n_v * dim * es, cudaMemcpyDeviceToHost, st));
            RBFD_CUDA(cudaEventRecord(m->ev1, st));
            RBFD_CUDA(cudaEventSynchronize(m->ev1));
            greedy_finish(m);
            unsigned mismatch = 0;
            std::memcpy(&mismatch, m->h_prep, sizeof(mismatch));
            if (mismatch) {  // (not expected: D_0 from S0 and from level 0 agree) the update again, host D_l
                for (int l = 0; l < L; ++l) {
                    double v = (k > 0.0) ? k * m->levels[l].smax : D;
                    if (k > 0.0 && D > 0.0 && v > D) v = D;
                    Dl[l] = (m->levels[l].nc > 0) ? v : 0.0;
                }
                deform_acc_init(m, n_v, vs_pos, f64, st);
                for (int l = 0; l < L; ++l) deform_one_level(m, l, n_v, vs_pos, Dl[l], f64, st, m->sort);
                deform_scatter(m, n_v, m->d_vorig, dout, f64, st);
                if (host) RBFD_CUDA(cudaMemcpyAsync(out, dout, (size_t)n_v * dim * es, cudaMemcpyDeviceToHost, st));
                RBFD_CUDA(cudaEventRecord(m->ev1, st));
                RBFD_CUDA(cudaEventSynchronize(m->ev1));
            }
            float ms = 0;
            RBFD_CUDA(cudaEventElapsedTime(&ms, m->ev0, m->ev1));
            m->stats.deform_ms = ms;
            m->prof.flush();
            return;
        }
        greedy_finish(m);
        for (int l = 0; l < L; ++l) {  // (the levels' D_l, now that their scalars are on the host)
            double v = (k > 0.0) ? k * m->levels[l].smax : D;
            if (k > 0.0 && D > 0.0 && v > D) v = D;
            Dl[l] = (m->levels[l].nc > 0) ? v : 0.0;
            Dmax = std::max(Dmax, Dl[l]);
        }
        if (l0 && !(L > 0 && Dl[0] == m->vst_D0)) {
            deform_acc_init(m, n_v, vs_pos, f64, st);
            l0 = false;
        }
        if (Dmax > 0.0) {
            for (int l = l0 ? 1 : 0; l < L; ++l) deform_one_level(m, l, n_v, vs_pos, Dl[l], f64, st, m->sort);
            deform_scatter(m, n_v, m->d_vorig, dout, f64, st);
        } else {
            RBFD_CUDA(cudaMemsetAsync(dout, 0, (size_t)n_v * dim * es, st));
        }
        if (host) RBFD_CUDA(cudaMemcpyAsync(out, dout, (size_t)n_v * dim * es, cudaMemcpyDeviceToHost, st));
        RBFD_CUDA(cudaEventRecord(m->ev1, st));
        RBFD_CUDA(cudaEventSynchronize(m->ev1));
        float ms = 0;
        RBFD_CUDA(cudaEventElapsedTime(&ms, m->ev0, m->ev1));
        m->stats.deform_ms = ms;
        m->prof.flush();
        return;
    }
    volume_unstage(m);
    greedy_finish(m);
    for (int l = 0; l < L; ++l) {  // (the levels' D_l, now that their scalars are on the host)
        double v = (k > 0.0) ? k * m->levels[l].smax : D;
        if (k > 0.0 && D > 0.0 && v > D) v = D;
        Dl[l] = (m->levels[l].nc > 0) ? v : 0.0;
        Dmax = std::max(Dmax, Dl[l]);
    }
    void *dout = out;
    const void *dx = xyz_v, *dd = d_v;
    if (n_v > 0) {
        reserve_volume(m, (size_t)n_v);
        const size_t need = (size_t)n_v * dim * es * 2 + (size_t)n_v * es + 256;
        if (host) {
            if (need > m->vio_bytes) {
                dfree(m->d_vio);
                m->d_vio = nullptr;
                m->vio_bytes = 0;
                m->d_vio = dmalloc(need, "volume staging");
                m->vio_bytes = need;
            }
            char *base = static_cast<char *>(m->d_vio);
            void *sx = base;
            void *sd = base + (size_t)n_v * dim * es;
            dout = base + (size_t)n_v * dim * es + (((size_t)n_v * es + 255) / 256) * 256;
            RBFD_CUDA(cudaMemcpyAsync(sx, xyz_v, (size_t)n_v * dim * es, cudaMemcpyHostToDevice, st));
            if (d_v) RBFD_CUDA(cudaMemcpyAsync(sd, d_v, (size_t)n_v * es, cudaMemcpyHostToDevice, st));
            dx = sx;
            dd = d_v ? sd : nullptr;
        }
        RBFD_CUDA(cudaMemsetAsync(dout, 0, (size_t)n_v * dim * es, st));
    }
    double4 *vin = reinterpret_cast<double4 *>(m->d_vin);
    double4 *vpos = reinterpret_cast<double4 *>(m->d_vpos);
    if (n_v > 0 && Dmax > 0.0 && !dd) {
        // No wall distances given: Morton-sort every point, compute d(r) on
        // the device (needed only below max_l D_l, so capped there), then
        // keep d < max_l D_l in Morton order (steps (1) and (2) in one).
        k_vol_pack<<<cdiv(n_v, 256), 256, 0, st>>>(dx, nullptr, n_v, dim, f64 ? 1 : 0, vin);
        morton_order(m, n_v, vin, vpos, m->d_vorig, st, m->d_red, m->d_bbox, m->sort);
        wall_distance_sorted(m, n_v, vpos, Dmax, nullptr);
        k_flag_below<<<cdiv(n_v, 256), 256, 0, st>>>(vpos, nullptr, n_v, Dmax, m->d_vflag);
        exclusive_scan_u32(m->d_vflag, m->d_vscan, (size_t)n_v, &m->d_misc[4], m->sort, st);
        k_compact<<<cdiv(n_v, 256), 256, 0, st>>>(m->d_vflag, m->d_vscan, n_v, m->d_vlist);
        uint32_t cnt = 0;
        RBFD_CUDA(cudaMemcpyAsync(&cnt, &m->d_misc[4], sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
        RBFD_CUDA(cudaStreamSynchronize(st));
        const int64_t nk = cnt;
        if (nk > 0) {
            k_gather_vol<<<cdiv(nk, 256), 256, 0, st>>>(vpos, m->d_vlist, nk, vin);  // kept points, sorted
            k_gather_u32<<<cdiv(nk, 256), 256, 0, st>>>(m->d_vorig, m->d_vlist, nk, m->d_vflag);
            RBFD_CUDA(cudaMemcpyAsync(m->d_vorig, m->d_vflag, sizeof(uint32_t) * nk, cudaMemcpyDeviceToDevice, st));
            deform_levels(m, nk, vin, m->d_vorig, Dl.data(), L, dout, f64);
        }
        m->stats.launches += 6;  // pack, flags, compaction, gathers x2, scatter
    } else if (n_v > 0 && Dmax > 0.0) {
        // every point packed and Morton-sorted (what a staged volume does
        // ahead of the greedy), then the levels' reductions d < D_l over all
        // of them: the same points in the same blocks either way, so both
        // give the same results bit for bit
        k_vol_pack<<<cdiv(n_v, 256), 256, 0, st>>>(dx, dd, n_v, dim, f64 ? 1 : 0, vin);
        morton_order(m, n_v, vin, vpos, m->d_vorig, st, m->d_red, m->d_bbox, m->sort);
        deform_levels(m, n_v, vpos, m->d_vorig, Dl.data(), L, dout, f64);
        m->stats.launches += 1;
    }
    if (host && n_v > 0)
        RBFD_CUDA(cudaMemcpyAsync(out, dout, (size_t)n_v * dim * es, cudaMemcpyDeviceToHost, st));
    RBFD_CUDA(cudaEventRecord(m->ev1, st));
    RBFD_CUDA(cudaEventSynchronize(m->ev1));
    float ms = 0;
    RBFD_CUDA(cudaEventElapsedTime(&ms, m->ev0, m->ev1));
    m->stats.deform_ms = ms;
    m->prof.flush();
}

// Register a volume mesh for repeated updates (rbfd_set_volume): its points
// are packed and Morton-sorted once; deform_registered then runs only the
// per-level compaction, evaluation and scatter for each new displacement.
// ------------------------------------------------ work-list volume update

namespace {

// Tuned settings per batch shape (meshes, their volume sizes, levels).
struct WLCached {
    std::vector<int64_t> key;
    rbfd_worklist_tune t;
};
std::mutex g_wl_mu;
std::vector<WLCached> g_wl_cache;

// The level's FP32-input sweep arguments (mode 2) for list l of mesh m,
// on the level's grid of cell size R_l / cell_div.
VolArgs wl_args(rbfd_mesh *m, int l, int64_t n_v, double Dl, int cell_div) {
    const Level &Lv = m->levels[l];
    VolArgs a{};
    a.n_list = n_v;  // upper bound; the length is read on the device
    a.n_list_dev = &m->d_wl_cnt[l];
    a.list = m->d_wl_list + (size_t)l * m->wl_cap;
    a.vpos = reinterpret_cast<const double4 *>(m->d_vpos);
    a.vacc = m->d_vacc;
    a.cx = Lv.d_cx;
    a.alpha = Lv.d_alpha;
    const bool fine = cell_div == 2 && Lv.f_cell_start;
    a.cell_start = fine ? Lv.f_cell_start : Lv.d_cell_start;
    a.cell_ctrl = fine ? Lv.f_cell_ctrl : Lv.d_cell_ctrl;
    a.g0 = fine ? Lv.f_g0 : Lv.g0;
    a.h = fine ? Lv.f_h : Lv.h;
    a.gd = fine ? Lv.f_gdim : Lv.gdim;
    a.R = Lv.R;
    a.Dl = Dl;
    const double inv = 1.0 / Lv.R;
    a.invR_hi = (float)inv;
    a.invR_lo = (float)(inv - (double)a.invR_hi);
    a.pairs = m->d_pairs + 2;
    a.vp4 = m->d_vpos4;
    a.cdf = Lv.d_cdf;
    a.adf = Lv.d_adf;
    a.g0f[0] = (float)a.g0.x;
    a.g0f[1] = (float)a.g0.y;
    a.g0f[2] = (float)a.g0.z;
    a.hf = (float)a.h;
    a.Rf = (float)Lv.R;
    a.invDlf = Dl > 0.0 ? (float)(1.0 / Dl) : 0.f;
    a.rec = fine ? Lv.f_rec : Lv.d_rec;
    a.err = &m->d_misc[12];
    return a;
}

void launch_worklist(int dim, int basis, unsigned grid, const WorkList &w, cudaStream_t st) {
    if (dim == 2) {
        switch (basis) {
        case 0: k_vol_worklist<2, 0><<<grid, kThreads, 0, st>>>(w); break;
        case 4: k_vol_worklist<2, 4><<<grid, kThreads, 0, st>>>(w); break;
        case 6: k_vol_worklist<2, 6><<<grid, kThreads, 0, st>>>(w); break;
        default: k_vol_worklist<2, 2><<<grid, kThreads, 0, st>>>(w); break;
        }
    } else {
        switch (basis) {
        case 0: k_vol_worklist<3, 0><<<grid, kThreads, 0, st>>>(w); break;
        case 4: k_vol_worklist<3, 4><<<grid, kThreads, 0, st>>>(w); break;
        case 6: k_vol_worklist<3, 6><<<grid, kThreads, 0, st>>>(w); break;
        default: k_vol_worklist<3, 2><<<grid, kThreads, 0, st>>>(w); break;
        }
    }
    RBFD_CUDA(cudaGetLastError());
}

int worklist_max_ctas_per_sm(int dim, int basis) {
    int b = 1;
    const void *fn = nullptr;
    if (dim == 2) fn = basis == 0 ? (const void *)k_vol_worklist<2, 0> : basis == 4 ? (const void *)k_vol_worklist<2, 4>
                     : basis == 6 ? (const void *)k_vol_worklist<2, 6> : (const void *)k_vol_worklist<2, 2>;
    else fn = basis == 0 ? (const void *)k_vol_worklist<3, 0> : basis == 4 ? (const void *)k_vol_worklist<3, 4>
              : basis == 6 ? (const void *)k_vol_worklist<3, 6> : (const void *)k_vol_worklist<3, 2>;
    RBFD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, fn, kThreads, 0));
    return std::max(1, b);
}

}  // namespace

void deform_worklist(rbfd_mesh **ms, int n, const int64_t *n_v_in, const float *const *xyz_v,
                     const float *const *d_v, const double *D, const double *k, float *const *out,
                     rbfd_worklist_tune *tune, bool registered) {
    NvtxRange nvtx("rbfd work-list volume update");
    // registered volumes (rbfd_set_volume): already packed and Morton-sorted
    std::vector<int64_t> n_v_reg;
    if (registered) {
        for (int i = 0; i < n; ++i) n_v_reg.push_back(ms[i]->vreg_n);
        n_v_in = n_v_reg.data();
    }
    const int64_t *n_v = n_v_in;
    if (n < 1 || n > 16) fail(RBFD_EINVAL, "rbfd_deform_worklist: 1 to 16 meshes");
    const int dim = ms[0]->dim, basis = ms[0]->opt.basis, dev = ms[0]->device;
    int n_entries = 0;
    for (int i = 0; i < n; ++i) {
        rbfd_mesh *m = ms[i];
        if (!m->greedy_done) fail(RBFD_ESTATE, "rbfd_deform_worklist: mesh " + std::to_string(i) + " has no greedy");
        if (m->opt.precision == RBFD_FP64 || m->dim != dim || m->opt.basis != basis || m->device != dev)
            fail(RBFD_EINVAL, "rbfd_deform_worklist: the meshes must all be mixed precision, of one dimension, "
                              "basis and device (mesh " + std::to_string(i) + " is not)");
        if (n_v[i] < 0 || n_v[i] >= (int64_t)1 << 31 || (n_v[i] > 0 && ((!registered && !xyz_v[i]) || !out[i])))
            fail(RBFD_EINVAL, "rbfd_deform_worklist: bad volume arrays of mesh " + std::to_string(i));
        if (!(D[i] >= 0.0) || !(k[i] >= 0.0) || (D[i] == 0.0 && k[i] == 0.0))
            fail(RBFD_EINVAL, "rbfd_deform_worklist: D and k must be >= 0 and not both 0");
        n_entries += (int)m->levels.size();
    }
    if (n_entries > kWLMax) fail(RBFD_EINVAL, "rbfd_deform_worklist: more than 64 (mesh, level) pairs");
    RBFD_CUDA(cudaSetDevice(dev));
    cudaStream_t st0 = ms[0]->stream;

    // ---- per mesh, on its own stream: inputs, packing, Morton order, wall
    // distances if not given, accumulator, the lists d < D_l of every level
    std::vector<std::vector<double>> Dl(n);
    std::vector<void *> dout(n, nullptr);
    std::vector<cudaEvent_t> ev(n, nullptr);
    for (int i = 0; i < n; ++i) {
        rbfd_mesh *m = ms[i];
        cudaStream_t st = m->stream;
        volume_unstage(m);
        greedy_finish(m);
        const int L = (int)m->levels.size();
        Dl[i].assign(L, 0.0);
        double Dmax = 0.0;
        for (int l = 0; l < L; ++l) {
            double v = (k[i] > 0.0) ? k[i] * m->levels[l].smax : D[i];
            if (k[i] > 0.0 && D[i] > 0.0 && v > D[i]) v = D[i];
            Dl[i][l] = (m->levels[l].nc > 0) ? v : 0.0;
            Dmax = std::max(Dmax, Dl[i][l]);
        }
        RBFD_CUDA(cudaEventRecord(m->ev0, st));
        VolumeIO io{nullptr, nullptr, out[i]};
        if (registered) {
            if (!m->opt.inputs_on_device && n_v[i] > 0) {  // the output through the staging buffer
                const size_t need = sizeof(float) * (size_t)n_v[i] * dim;
                if (need > m->vio_bytes) {
                    dfree(m->d_vio);
                    m->d_vio = nullptr;
                    m->vio_bytes = 0;
                    m->d_vio = dmalloc(need, "volume output staging");
                    m->vio_bytes = need;
                }
                io.out = m->d_vio;
            }
        } else {
            io = volume_io(m, n_v[i], xyz_v[i], d_v ? d_v[i] : nullptr, out[i], false, st);
        }
        dout[i] = io.out;
        const int64_t nv = n_v[i];
        if (nv > 0) {
            reserve_volume(m, (size_t)nv);
            if (m->wl_cap < (size_t)nv || m->wl_levels < L) {
                dfree(m->d_wl_list);
                m->d_wl_list = nullptr;
                m->wl_cap = 0;
                m->d_wl_list = dalloc<uint32_t>((size_t)std::max(L, 1) * (size_t)nv, "work-list level lists");
                m->wl_cap = (size_t)nv;
                m->wl_levels = std::max(L, 1);
            }
            if (!m->d_wl_cnt) m->d_wl_cnt = dalloc<uint32_t>(kWLMax, "work-list list lengths");
            RBFD_CUDA(cudaMemsetAsync(m->d_wl_cnt, 0, sizeof(uint32_t) * kWLMax, st));
            double4 *vin = reinterpret_cast<double4 *>(m->d_vin);
            double4 *vpos = registered ? m->d_vreg : reinterpret_cast<double4 *>(m->d_vpos);
            if (!registered) {
                k_vol_pack<<<cdiv(nv, 256), 256, 0, st>>>(io.x, io.d, nv, dim, 0, vin);
                morton_order(m, nv, vin, vpos, m->d_vorig, st, m->d_red, m->d_bbox, m->sort);
                if (!io.d && Dmax > 0.0) wall_distance_sorted(m, nv, vpos, Dmax, nullptr);
            }
            deform_acc_init(m, nv, vpos, false, st);
            for (int l = 0; l < L; ++l) {
                if (!(Dl[i][l] > 0.0)) continue;
                k_flag_below<<<cdiv(nv, 256), 256, 0, st>>>(vpos, nullptr, nv, Dl[i][l], m->d_vflag);
                exclusive_scan_u32(m->d_vflag, m->d_vscan, (size_t)nv, &m->d_wl_cnt[l], m->sort, st);
                k_compact<<<cdiv(nv, 256), 256, 0, st>>>(m->d_vflag, m->d_vscan, nv,
                                                         m->d_wl_list + (size_t)l * m->wl_cap);
                k_count_points<<<1, 32, 0, st>>>(&m->d_wl_cnt[l], m->d_pairs + 7);
                m->stats.launches += 4;
            }
            if (tune == nullptr || tune->autotune || tune->cell_div[i] == 2)
                for (auto &Lv : m->levels) level_fine_grid(m, Lv);
            m->stats.launches += 2;
        }
        RBFD_CUDA(cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming));
        RBFD_CUDA(cudaEventRecord(ev[i], st));
        RBFD_CUDA(cudaStreamWaitEvent(st0, ev[i], 0));
        RBFD_CUDA(cudaGetLastError());
    }

    // ---- the work list: (mesh, level) entries, level-major
    rbfd_worklist_tune t{};
    t.autotune = tune ? tune->autotune : 1;
    t.ctas_per_sm = 2;
    t.item_blocks = 1;
    for (int i = 0; i < 16; ++i) t.cell_div[i] = 1;
    if (tune && !tune->autotune) {
        t.ctas_per_sm = tune->ctas_per_sm;
        t.item_blocks = tune->item_blocks;
        for (int i = 0; i < n; ++i) t.cell_div[i] = tune->cell_div[i];
    }
    const int occ = worklist_max_ctas_per_sm(dim, basis);
    int sms = 0;
    RBFD_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    auto sanitize = [&](rbfd_worklist_tune &x) {
        x.ctas_per_sm = std::max(1, std::min(x.ctas_per_sm, std::min(occ, 8)));
        x.item_blocks = x.item_blocks >= 4 ? 4 : x.item_blocks >= 2 ? 2 : 1;
        for (int i = 0; i < n; ++i) x.cell_div[i] = x.cell_div[i] == 2 ? 2 : 1;
    };
    sanitize(t);
    auto build = [&](const rbfd_worklist_tune &x, unsigned int *ctl, unsigned long long *pairs_scratch) {
        WorkList w{};
        std::vector<int> prev(n, -1);
        int Lmax = 0;
        for (int i = 0; i < n; ++i) Lmax = std::max(Lmax, (int)ms[i]->levels.size());
        for (int l = 0; l < Lmax; ++l)
            for (int i = 0; i < n; ++i) {
                rbfd_mesh *m = ms[i];
                if (l >= (int)m->levels.size() || n_v[i] == 0 || m->levels[l].nc == 0 || !(Dl[i][l] > 0.0)) continue;
                const int e = w.n++;
                w.e[e] = wl_args(m, l, n_v[i], Dl[i][l], x.cell_div[i]);
                w.e[e].err = ctl + 1;  // (a staging wait that ran out fails the launch like a level wait)
                if (pairs_scratch) w.e[e].pairs = pairs_scratch;
                w.dep[e] = prev[i];
                prev[i] = e;
            }
        w.item_blocks = x.item_blocks;
        w.ctl = ctl;
        w.poll_limit = 1u << 24;  // about 5 s of polls: far beyond any level's sweep
        return w;
    };
    // control words + scratch pair counters for the timed candidates
    const size_t ctl_words = 2 + kWLMax;
    void *blk = dmalloc(sizeof(unsigned int) * 128 + sizeof(unsigned long long) * 4, "work-list control");
    unsigned int *ctl = static_cast<unsigned int *>(blk);
    unsigned long long *scratch = reinterpret_cast<unsigned long long *>(ctl + 128);
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    RBFD_CUDA(cudaEventCreate(&t0));
    RBFD_CUDA(cudaEventCreate(&t1));
    auto run = [&](const rbfd_worklist_tune &x, bool trial) {
        const WorkList w = build(x, ctl, trial ? scratch : nullptr);
        RBFD_CUDA(cudaMemsetAsync(ctl, 0, sizeof(unsigned int) * ctl_words, st0));
        RBFD_CUDA(cudaEventRecord(t0, st0));
        if (w.n > 0) launch_worklist(dim, basis, (unsigned)(x.ctas_per_sm * sms), w, st0);
        RBFD_CUDA(cudaEventRecord(t1, st0));
        unsigned int err = 0;
        RBFD_CUDA(cudaMemcpyAsync(&err, ctl + 1, sizeof(err), cudaMemcpyDeviceToHost, st0));
        RBFD_CUDA(cudaStreamSynchronize(st0));
        if (err) fail(RBFD_ETIMEOUT, "rbfd_deform_worklist: a level's wait for the previous level ran out");
        float ms_ = 0.f;
        RBFD_CUDA(cudaEventElapsedTime(&ms_, t0, t1));
        return (double)ms_;
    };
    auto reset_acc = [&]() {
        for (int i = 0; i < n; ++i)
            if (n_v[i] > 0) RBFD_CUDA(cudaMemsetAsync(ms[i]->d_vacc, 0, sizeof(double4) * n_v[i], st0));
    };
    // ---- the settings: given, cached for this batch shape, or tuned here
    std::vector<int64_t> key{(int64_t)n, (int64_t)dim, (int64_t)basis};
    for (int i = 0; i < n; ++i) {
        key.push_back(n_v[i]);
        key.push_back((int64_t)ms[i]->levels.size());
    }
    int trials = 0, cached = 0;
    if (t.autotune) {
        bool hit = false;
        {
            std::lock_guard<std::mutex> lk(g_wl_mu);
            for (auto &c : g_wl_cache)
                if (c.key == key) {
                    t = c.t;
                    hit = true;
                }
        }
        if (hit) {
            cached = 1;
        } else {
            // coordinate descent on this call's own work (results discarded,
            // the accumulators cleared after): each mesh's cell size, then
            // blocks per SM, then list blocks per item
            double best = run(t, true);
            ++trials;
            reset_acc();
            for (int i = 0; i < n; ++i) {
                if (n_v[i] == 0) continue;
                rbfd_worklist_tune c = t;
                c.cell_div[i] = 2;
                const double v = run(c, true);
                ++trials;
                reset_acc();
                if (v < best) {
                    best = v;
                    t = c;
                }
            }
            for (int cps : {1, 2, 3, 4, 6, 8}) {
                if (cps > std::min(occ, 8) || cps == t.ctas_per_sm) continue;
                rbfd_worklist_tune c = t;
                c.ctas_per_sm = cps;
                const double v = run(c, true);
                ++trials;
                reset_acc();
                if (v < best) {
                    best = v;
                    t = c;
                }
            }
            for (int ib : {2, 4}) {
                rbfd_worklist_tune c = t;
                c.item_blocks = ib;
                const double v = run(c, true);
                ++trials;
                reset_acc();
                if (v < best) {
                    best = v;
                    t = c;
                }
            }
            std::lock_guard<std::mutex> lk(g_wl_mu);
            g_wl_cache.push_back({key, t});
        }
    }
    // ---- the launch, then each mesh's scatter to the caller's order
    const double launch_ms = run(t, false);
    int64_t items = 0;
    {
        const WorkList w = build(t, ctl, nullptr);
        std::vector<unsigned int> done(ctl_words, 0u);
        RBFD_CUDA(cudaMemcpy(done.data(), ctl, sizeof(unsigned int) * ctl_words, cudaMemcpyDeviceToHost));
        for (int e = 0; e < w.n; ++e) items += done[2 + e];
    }
    RBFD_CUDA(cudaEventRecord(t1, st0));
    for (int i = 0; i < n; ++i) {
        rbfd_mesh *m = ms[i];
        cudaStream_t st = m->stream;
        RBFD_CUDA(cudaStreamWaitEvent(st, t1, 0));
        const int64_t nv = n_v[i];
        if (nv > 0) {
            k_scatter_out_df<<<cdiv(nv, 256), 256, 0, st>>>(m->d_vacc, registered ? m->d_vreg_orig : m->d_vorig,
                                                           nv, dim, static_cast<float *>(dout[i]));
            RBFD_CUDA(cudaGetLastError());
            m->stats.launches += 1;
            if (!m->opt.inputs_on_device)
                RBFD_CUDA(cudaMemcpyAsync(out[i], dout[i], sizeof(float) * nv * dim, cudaMemcpyDeviceToHost, st));
        }
        RBFD_CUDA(cudaEventRecord(m->ev1, st));
    }
    for (int i = 0; i < n; ++i) {
        rbfd_mesh *m = ms[i];
        RBFD_CUDA(cudaEventSynchronize(m->ev1));
        float ms_ = 0.f;
        RBFD_CUDA(cudaEventElapsedTime(&ms_, m->ev0, m->ev1));
        m->stats.deform_ms = ms_;
        if (m->prof.on) {  // (the shared launch, split evenly over the meshes' counters)
            m->prof.ms[kProfVol] += launch_ms / n;
            m->prof.launches[kProfVol] += 1;
        }
        cudaEventDestroy(ev[i]);
    }
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    dfree(blk);
    ms[0]->stats.launches += 1 + trials;
    if (tune) {
        *tune = t;
        tune->autotune = t.autotune;
        tune->cached = cached;
        tune->trials = trials;
        tune->launch_ms = launch_ms;
        tune->items = items;
    }
}

void volume_register(rbfd_mesh *m, int64_t n_v, const float *xyz_v, const float *d_v) {
    cudaStream_t st = m->stream;
    const int dim = m->dim;
    dfree(m->d_vreg);
    dfree(m->d_vreg_orig);
    m->d_vreg = nullptr;
    m->d_vreg_orig = nullptr;
    m->vreg_n = 0;
    if (n_v == 0) return;
    reserve_volume(m, (size_t)n_v);
    const void *dx = xyz_v, *dd = d_v;
    float *stage = nullptr;
    if (!m->opt.inputs_on_device) {
        stage = dalloc<float>((size_t)n_v * (dim + 1), "volume staging");
        RBFD_CUDA(cudaMemcpyAsync(stage, xyz_v, sizeof(float) * n_v * dim, cudaMemcpyHostToDevice, st));
        if (d_v)
            RBFD_CUDA(cudaMemcpyAsync(stage + (size_t)n_v * dim, d_v, sizeof(float) * n_v, cudaMemcpyHostToDevice,
                                      st));
        dx = stage;
        dd = d_v ? stage + (size_t)n_v * dim : nullptr;
    }
    double4 *vin = reinterpret_cast<double4 *>(m->d_vin);
    k_vol_pack<<<cdiv(n_v, 256), 256, 0, st>>>(dx, dd, n_v, dim, 0, vin);
    m->d_vreg = dalloc<double4>((size_t)n_v, "registered volume");
    m->d_vreg_orig = dalloc<uint32_t>((size_t)n_v, "registered volume order");
    morton_order(m, n_v, vin, m->d_vreg, m->d_vreg_orig, st, m->d_red, m->d_bbox, m->sort);
    // no wall distances given: d(r) of every point, computed once (later
    // displacements may need any D_l)
    if (!dd) wall_distance_sorted(m, n_v, m->d_vreg, INFINITY, nullptr);
    RBFD_CUDA(cudaStreamSynchronize(st));
    dfree(stage);
    m->vreg_n = n_v;
    m->stats.launches += 1;
}

// rbfd_wall_distance: pack, Morton-sort, query, scatter back to the caller's order.
void wall_distance_run(rbfd_mesh *m, int64_t n_v, const void *xyz_v, bool f64, double *out) {
    cudaStream_t st = m->stream;
    const int dim = m->dim;
    if (n_v == 0) return;
    RBFD_CUDA(cudaEventRecord(m->ev0, st));
    reserve_volume(m, (size_t)n_v);
    const size_t es = f64 ? sizeof(double) : sizeof(float);
    const void *dx = xyz_v;
    double *dout = out;
    void *stage = nullptr;
    if (!m->opt.inputs_on_device) {
        const size_t xb = ((size_t)n_v * dim * es + 255) / 256 * 256;
        stage = dmalloc(xb + sizeof(double) * (size_t)n_v, "wall distance staging");
        RBFD_CUDA(cudaMemcpyAsync(stage, xyz_v, (size_t)n_v * dim * es, cudaMemcpyHostToDevice, st));
        dx = stage;
        dout = reinterpret_cast<double *>(static_cast<char *>(stage) + xb);
    }
    double4 *vin = reinterpret_cast<double4 *>(m->d_vin);
    double4 *vpos = reinterpret_cast<double4 *>(m->d_vpos);
    k_vol_pack<<<cdiv(n_v, 256), 256, 0, st>>>(dx, nullptr, n_v, dim, f64 ? 1 : 0, vin);
    morton_order(m, n_v, vin, vpos, m->d_vorig, st, m->d_red, m->d_bbox, m->sort);
    double *dsorted = reinterpret_cast<double *>(m->d_vacc);
    wall_distance_sorted(m, n_v, vpos, INFINITY, dsorted);
    k_scatter_d<<<cdiv(n_v, 256), 256, 0, st>>>(dsorted, m->d_vorig, n_v, dout);
    RBFD_CUDA(cudaGetLastError());
    m->stats.launches += 2;
    if (dout != out) RBFD_CUDA(cudaMemcpyAsync(out, dout, sizeof(double) * n_v, cudaMemcpyDeviceToHost, st));
    RBFD_CUDA(cudaEventRecord(m->ev1, st));
    RBFD_CUDA(cudaEventSynchronize(m->ev1));
    dfree(stage);
    m->prof.flush();
}

void deform_registered(rbfd_mesh *m, double D, double k, float *out) {
    cudaStream_t st = m->stream;
    const int dim = m->dim;
    const int64_t n_v = m->vreg_n;
    RBFD_CUDA(cudaEventRecord(m->ev0, st));
    const int L = (int)m->levels.size();
    std::vector<double> Dl(L, 0.0);
    for (int l = 0; l < L; ++l) {
        double v = (k > 0.0) ? k * m->levels[l].smax : D;
        if (k > 0.0 && D > 0.0 && v > D) v = D;
        Dl[l] = (m->levels[l].nc > 0) ? v : 0.0;
    }
    float *dout = out;
    if (!m->opt.inputs_on_device && n_v > 0) {
        const size_t need = sizeof(float) * (size_t)n_v * dim;
        if (need > m->vio_bytes) {
            dfree(m->d_vio);
            m->d_vio = nullptr;
            m->vio_bytes = 0;
            m->d_vio = dmalloc(need, "volume output staging");
            m->vio_bytes = need;
        }
        dout = static_cast<float *>(m->d_vio);
    }
    if (n_v > 0) {
        RBFD_CUDA(cudaMemsetAsync(dout, 0, sizeof(float) * n_v * dim, st));
        deform_levels(m, n_v, m->d_vreg, m->d_vreg_orig, Dl.data(), L, dout, false);
        if (dout != out) RBFD_CUDA(cudaMemcpyAsync(out, dout, sizeof(float) * n_v * dim, cudaMemcpyDeviceToHost, st));
    }
    RBFD_CUDA(cudaEventRecord(m->ev1, st));
    RBFD_CUDA(cudaEventSynchronize(m->ev1));
    float ms = 0;
    RBFD_CUDA(cudaEventElapsedTime(&ms, m->ev0, m->ev1));
    m->stats.deform_ms = ms;
    m->prof.flush();
    vol_staging_check(m);
}

}  // namespace rbfd

// ==================================================== allocation-free variant
//
// rbfd_deform_noalloc: the volume update above for callers that must not
// allocate device memory during the call -- code running between the
// iterations of a solver whose device memory is fully reserved up front, or
// hosts that forbid cudaMalloc/cudaFree on their hot path because those calls
// synchronise the device and can fail mid-run.  Every per-call buffer (packed,
// compacted and sorted points, lists, Morton keys, sort scratch, accumulators)
// lives in one file-scope device array of fixed size, so the call allocates
// nothing; it is limited to kNoAllocMaxPoints volume points.
namespace rbfd {
namespace {

constexpr int64_t kNoAllocMaxPoints = 1 << 17;  // 131,072 volume points per call
constexpr size_t al256(size_t b) { return (b + 255) / 256 * 256; }
constexpr size_t kNaD4 = al256(sizeof(double4) * (size_t)kNoAllocMaxPoints);
constexpr size_t kNaU32 = al256(sizeof(uint32_t) * (size_t)kNoAllocMaxPoints);
// the sort and scan scratch at their largest (SortScratch::reserve's own
// formulas): reserve() then never allocates for a call of up to
// kNoAllocMaxPoints points
constexpr size_t kNaHistN = sort_hist_need((size_t)kNoAllocMaxPoints);
constexpr size_t kNaSumsN = sort_sums_need((size_t)kNoAllocMaxPoints);
static_assert(kNaHistN >= sort_hist_need(1) && kNaSumsN >= sort_sums_need(1), "scratch sizes grow with n");
constexpr size_t kNaBytes = 3 * kNaD4 + 7 * kNaU32 + al256(sizeof(uint32_t) * kNaHistN) +
                            al256(sizeof(uint32_t) * kNaSumsN);

// Shared by every call in the process on a given device (about 16 MB).
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaBytes];

constexpr int kMaxDevices = 64;
std::mutex g_na_mutex;
unsigned char *g_na_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once
// per device (host code must not use the symbol itself as an address).
unsigned char *noalloc_scratch() {
    int dev = 0;
    RBFD_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) fail(RBFD_EINVAL, "rbfd_deform_noalloc: device index out of range");
    std::lock_guard<std::mutex> lk(g_na_mutex);
    if (!g_na_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            fail(RBFD_ECUDA, std::string("rbfd_deform_noalloc: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e));
        }
        g_na_addr[dev] = static_cast<unsigned char *>(p);
    }
    return g_na_addr[dev];
}

void deform_noalloc_run(rbfd_mesh *m, int64_t n_v, const float *xyz_v, const float *d_v, double D, double k,
                        float *out) {
    cudaStream_t st = m->stream;
    const int dim = m->dim;
    unsigned char *base = noalloc_scratch();
    double4 *vin = reinterpret_cast<double4 *>(base);
    double4 *vpos = reinterpret_cast<double4 *>(base + kNaD4);
    double4 *vacc = reinterpret_cast<double4 *>(base + 2 * kNaD4);
    unsigned char *u = base + 3 * kNaD4;
    uint32_t *vorig = reinterpret_cast<uint32_t *>(u + 0 * kNaU32);
    uint32_t *vflag = reinterpret_cast<uint32_t *>(u + 1 * kNaU32);
    uint32_t *vscan = reinterpret_cast<uint32_t *>(u + 2 * kNaU32);
    uint32_t *vlist = reinterpret_cast<uint32_t *>(u + 3 * kNaU32);
    uint32_t *vkeys = reinterpret_cast<uint32_t *>(u + 4 * kNaU32);
    SortScratch ss;  // a view into the static array with its capacities: reserve() never allocates
    ss.launches = &m->stats.launches;
    ss.keys_alt = reinterpret_cast<uint32_t *>(u + 5 * kNaU32);
    ss.vals_alt = reinterpret_cast<uint32_t *>(u + 6 * kNaU32);
    ss.hist = reinterpret_cast<uint32_t *>(u + 7 * kNaU32);
    ss.block_sums = reinterpret_cast<uint32_t *>(u + 7 * kNaU32 + al256(sizeof(uint32_t) * kNaHistN));
    ss.cap_items = (size_t)kNoAllocMaxPoints;
    ss.cap_hist = kNaHistN;
    ss.cap_sums = kNaSumsN;

    RBFD_CUDA(cudaEventRecord(m->ev0, st));
    const int L = (int)m->levels.size();
    double Dl[64] = {0};
    double Dmax = 0.0;
    for (int l = 0; l < L; ++l) {
        double v = (k > 0.0) ? k * m->levels[l].smax : D;
        if (k > 0.0 && D > 0.0 && v > D) v = D;
        Dl[l] = (m->levels[l].nc > 0) ? v : 0.0;
        Dmax = std::max(Dmax, Dl[l]);
    }
    if (n_v > 0) RBFD_CUDA(cudaMemsetAsync(out, 0, (size_t)n_v * dim * sizeof(float), st));
    int64_t nV = 0;
    if (n_v > 0 && Dmax > 0.0) {
        k_vol_pack<<<cdiv(n_v, 256), 256, 0, st>>>(xyz_v, d_v, n_v, dim, 0, vin);
        k_flag_below<<<cdiv(n_v, 256), 256, 0, st>>>(vin, nullptr, n_v, Dmax, vflag);
        exclusive_scan_u32(vflag, vscan, (size_t)n_v, &m->d_misc[6], ss, st);
        k_compact<<<cdiv(n_v, 256), 256, 0, st>>>(vflag, vscan, n_v, vlist);
        uint32_t cnt = 0;
        RBFD_CUDA(cudaMemcpyAsync(&cnt, &m->d_misc[6], sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
        RBFD_CUDA(cudaStreamSynchronize(st));
        nV = cnt;
    }
    if (nV > 0) {
        const int nbb = std::min<int>(cdiv(nV, 256), 256);
        k_bbox_idx<<<nbb, 256, 0, st>>>(vin, vlist, nV, m->d_red);
        k_bbox_reduce<<<1, 192, 0, st>>>(m->d_red, nbb, m->d_bbox);
        k_gather_vol<<<cdiv(nV, 256), 256, 0, st>>>(vin, vlist, nV, vpos);
        morton_keys_f64_dev(vpos, nV, dim, m->d_bbox, vkeys, vorig, st, vol_key_shift(dim), true);
        radix_sort_pairs(vkeys, vorig, (size_t)nV, kVolKeyBits, ss, st);
        k_gather_vol<<<cdiv(nV, 256), 256, 0, st>>>(vpos, vorig, nV, vin);  // vin := sorted points
        k_gather_u32<<<cdiv(nV, 256), 256, 0, st>>>(vlist, vorig, nV, vflag);
        RBFD_CUDA(cudaMemcpyAsync(vorig, vflag, sizeof(uint32_t) * nV, cudaMemcpyDeviceToDevice, st));
        RBFD_CUDA(cudaMemsetAsync(vacc, 0, sizeof(double4) * nV, st));  // the array keeps the last call's data
        const int mode = m->opt.precision == RBFD_FP64 ? 0 : 1;
        for (int l = 0; l < L; ++l) {
            const Level &Lv = m->levels[l];
            if (Lv.nc == 0 || !(Dl[l] > 0.0)) continue;
            k_flag_below<<<cdiv(nV, 256), 256, 0, st>>>(vin, nullptr, nV, Dl[l], vflag);
            exclusive_scan_u32(vflag, vscan, (size_t)nV, &m->d_misc[7], ss, st);
            k_compact<<<cdiv(nV, 256), 256, 0, st>>>(vflag, vscan, nV, vlist);
            // the level's list length stays on the device (the sweep reads
            // it, nV is its upper bound): no host wait per level
            VolArgs a{};
            a.n_list = nV;
            a.n_list_dev = &m->d_misc[7];
            a.list = vlist;
            a.vpos = vin;
            a.vacc = vacc;
            a.cx = Lv.d_cx;
            a.alpha = Lv.d_alpha;
            a.cell_start = Lv.d_cell_start;
            a.cell_ctrl = Lv.d_cell_ctrl;
            a.g0 = Lv.g0;
            a.h = Lv.h;
            a.gd = Lv.gdim;
            a.R = Lv.R;
            a.Dl = Dl[l];
            double inv = 1.0 / Lv.R;
            a.invR_hi = (float)inv;
            a.invR_lo = (float)(inv - (double)a.invR_hi);
            a.pairs = m->d_pairs + 2;
            launch_vol(dim, m->opt.basis, mode, cdiv(nV, kThreads), a, st);
            RBFD_CUDA(cudaGetLastError());
            m->stats.launches += 4;
        }
        k_scatter_out<<<cdiv(nV, 256), 256, 0, st>>>(vacc, vorig, nV, dim, 0, out);
        RBFD_CUDA(cudaGetLastError());
        m->stats.launches += 9;
    }
    RBFD_CUDA(cudaEventRecord(m->ev1, st));
    RBFD_CUDA(cudaEventSynchronize(m->ev1));
    float ms = 0;
    RBFD_CUDA(cudaEventElapsedTime(&ms, m->ev0, m->ev1));
    m->stats.deform_ms = ms;
}

// p is device (or managed) memory of GPU `device`
bool na_is_device_ptr(const void *p, int device) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) && at.device == device;
}

}  // namespace
}  // namespace rbfd

extern "C" int rbfd_deform_noalloc(rbfd_mesh *m, int64_t n_v, const float *xyz_v, const float *d_v, double D,
                                   double k, float *out) {
    try {
        if (!m) rbfd::fail(RBFD_EINVAL, "rbfd_deform_noalloc: NULL mesh");
        if (n_v < 0 || n_v > rbfd::kNoAllocMaxPoints)
            rbfd::fail(RBFD_EINVAL, "rbfd_deform_noalloc: n_v = " + std::to_string(n_v) +
                                        " is outside [0, 131072], the size of the fixed scratch array");
        if (n_v > 0 && (!xyz_v || !d_v || !out)) rbfd::fail(RBFD_EINVAL, "rbfd_deform_noalloc: NULL array");
        if (!(D >= 0.0) || !(k >= 0.0) || !std::isfinite(D) || !std::isfinite(k))
            rbfd::fail(RBFD_EINVAL, "rbfd_deform_noalloc: D and k must be finite and >= 0");
        if (D == 0.0 && k == 0.0) rbfd::fail(RBFD_EINVAL, "rbfd_deform_noalloc: D and k cannot both be 0");
        if (!m->greedy_done) rbfd::fail(RBFD_ESTATE, "rbfd_deform_noalloc: run rbfd_greedy first");
        if ((int)m->levels.size() > 64) rbfd::fail(RBFD_EINVAL, "rbfd_deform_noalloc: more than 64 levels");
        RBFD_CUDA(cudaSetDevice(m->device));
        if (n_v > 0 && (!rbfd::na_is_device_ptr(xyz_v, m->device) || !rbfd::na_is_device_ptr(d_v, m->device) ||
                        !rbfd::na_is_device_ptr(out, m->device)))
            rbfd::fail(RBFD_EINVAL, "rbfd_deform_noalloc: xyz_v, d_v and out must be device memory of the mesh's GPU");
        rbfd::deform_noalloc_run(m, n_v, xyz_v, d_v, D, k, out);
        rbfd::set_last_error("");
        return RBFD_OK;
    } catch (const rbfd::Error &e) {
        rbfd::set_last_error(e.msg);
        return e.status;
    } catch (...) {
        rbfd::set_last_error("rbfd_deform_noalloc: unexpected internal error");
        return RBFD_ECUDA;
    }
}
