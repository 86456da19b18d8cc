// quality.cu -- mesh quality of a deformed structured grid: the orthogonality
// angle by which the paper judges its deformations (Section 5).
//
// The grid grows off the surface: node layer j = 0 is the wall (surface point
// (k, i) plus its displacement), layers j >= 1 are volume points (k, i, j - 1)
// plus theirs; i runs round the section (optionally closing on itself), k
// along the span (3D), j away from the wall.  The orthogonality angle of a
// cell is the smallest angle between two grid lines meeting at one of its
// corners, folded into [0, 90] degrees (90 = orthogonal); a cell whose corners
// disagree in orientation (a fold or an inversion) is counted as tangled.
//
// One thread per cell (wall-normal index fastest, so neighbouring threads
// read neighbouring nodes).  Node coordinates and edge vectors are formed in
// FP64 exactly as a plain FP64 evaluation forms them; the angles are compared
// and evaluated in FP32 on unit edge vectors (one atan2 per cell, for the
// smallest corner); the orientation signs are taken in FP32 where the margin
// certifies them and recomputed in FP64 otherwise, so every tangled decision
// equals the FP64 one.  Per-block partials (min, argmin, sum, tangled,
// 10-degree histogram) are reduced by a second kernel in a fixed order, so
// the summary is deterministic.
#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "internal.h"

namespace rbfd {

namespace {

constexpr int kThreads = 256;
constexpr int kBins = 9;

struct QPart {
    double min_deg;
    long long argmin;
    double sum;
    long long tangled;
    long long hist[kBins];
};

struct QualArgs {
    int64_t n_i, n_k, n_layers, n_ci, cells;
    const double *wall, *wall_disp;
    const float *vol, *vol_disp;
    float *theta;
    QPart *part;
};

template <int DIM>
__device__ __forceinline__ double3 node(const QualArgs &a, int64_t i, int64_t k, int64_t j) {
    double p[3] = {0.0, 0.0, 0.0};
    if (j == 0) {
        const int64_t q = (k * a.n_i + i) * DIM;
#pragma unroll
        for (int c = 0; c < DIM; ++c) p[c] = __dadd_rn(a.wall[q + c], a.wall_disp ? a.wall_disp[q + c] : 0.0);
    } else {
        const int64_t q = ((k * a.n_i + i) * a.n_layers + (j - 1)) * DIM;
#pragma unroll
        for (int c = 0; c < DIM; ++c)
            p[c] = __dadd_rn((double)a.vol[q + c], a.vol_disp ? (double)a.vol_disp[q + c] : 0.0);
    }
    return make_double3(p[0], p[1], p[2]);
}

__device__ __forceinline__ double3 dsub3(double3 a, double3 b) {
    return make_double3(__dsub_rn(a.x, b.x), __dsub_rn(a.y, b.y), __dsub_rn(a.z, b.z));
}

// Unit vector of an FP64 edge, in FP32 (zero stays zero).
__device__ __forceinline__ float3 unit_f(double3 e) {
    float3 f = make_float3((float)e.x, (float)e.y, (float)e.z);
    const float n2 = fmaf(f.x, f.x, fmaf(f.y, f.y, f.z * f.z));
    const float s = n2 > 0.f ? rsqrtf(n2) : 0.f;
    return make_float3(f.x * s, f.y * s, f.z * s);
}

// Smallest folded corner angle so far as (S, C) = (|a x b|, |a . b|), compared
// by cross-multiplication (tan = S / C); a corner with S = C = 0 (an empty
// edge) has angle 0.
struct MinAngle {
    float S = 1.f, C = 0.f;  // 90 degrees
    __device__ __forceinline__ void offer(float s, float c) {
        if (s == 0.f && c == 0.f) c = 1.f;
        if (s * C < S * c) {
            S = s;
            C = c;
        }
    }
};

__device__ __forceinline__ void pair_2d(float3 a, float3 b, MinAngle &m) {
    m.offer(fabsf(a.x * b.y - a.y * b.x), fabsf(fmaf(a.x, b.x, a.y * b.y)));
}

__device__ __forceinline__ float3 cross_f(float3 a, float3 b) {
    return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}

__device__ __forceinline__ void pair_3d(float3 a, float3 b, MinAngle &m) {
    const float3 x = cross_f(a, b);
    m.offer(sqrtf(fmaf(x.x, x.x, fmaf(x.y, x.y, x.z * x.z))), fabsf(fmaf(a.x, b.x, fmaf(a.y, b.y, a.z * b.z))));
}

// FP64 triple product Ei . (Ek x Ej) in the plain evaluation order.
__device__ __forceinline__ double triple_f64(double3 ei, double3 ek, double3 ej) {
    const double x0 = __dsub_rn(__dmul_rn(ek.y, ej.z), __dmul_rn(ek.z, ej.y));
    const double x1 = __dsub_rn(__dmul_rn(ek.z, ej.x), __dmul_rn(ek.x, ej.z));
    const double x2 = __dsub_rn(__dmul_rn(ek.x, ej.y), __dmul_rn(ek.y, ej.x));
    return __dadd_rn(__dadd_rn(__dmul_rn(ei.x, x0), __dmul_rn(ei.y, x1)), __dmul_rn(ei.z, x2));
}

// Orientation of corner (di, dk, dj) of 3D cell (k, i, j) in FP64, from the nodes.
__device__ __noinline__ double corner_triple_f64(const QualArgs &a, int64_t i, int64_t i1, int64_t k, int64_t j,
                                                 int di, int dk, int dj) {
    const int64_t ic = di ? i1 : i;
    const double3 ei = dsub3(node<3>(a, i1, k + dk, j + dj), node<3>(a, i, k + dk, j + dj));
    const double3 ek = dsub3(node<3>(a, ic, k + 1, j + dj), node<3>(a, ic, k, j + dj));
    const double3 ej = dsub3(node<3>(a, ic, k + dk, j + 1), node<3>(a, ic, k + dk, j));
    return triple_f64(ei, ek, ej);
}

// Orthogonality angle (degrees) and tangled flag of one cell.
template <int DIM>
__device__ __forceinline__ float cell_quality(const QualArgs &a, int64_t idx, bool &tangled) {
    int64_t j, i, k;
    if (a.cells < (int64_t(1) << 31)) {  // 32-bit division where it fits
        const uint32_t u = (uint32_t)idx, nl = (uint32_t)a.n_layers, nc = (uint32_t)a.n_ci;
        const uint32_t r = u / nl;
        j = u - r * nl;
        k = r / nc;
        i = r - (uint32_t)k * nc;
    } else {
        const int64_t r = idx / a.n_layers;
        j = idx - r * a.n_layers;
        k = r / a.n_ci;
        i = r - k * a.n_ci;
    }
    const int64_t i1 = (i + 1 == a.n_i) ? 0 : i + 1;
    MinAngle m;
    bool pos = false, neg = false;
    if (DIM == 2) {
        // corners round the cell; E[q] = P[q+1] - P[q]
        double3 P[4] = {node<2>(a, i, 0, j), node<2>(a, i1, 0, j), node<2>(a, i1, 0, j + 1), node<2>(a, i, 0, j + 1)};
        double3 E[4];
        float3 U[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            E[q] = dsub3(P[(q + 1) & 3], P[q]);
            U[q] = unit_f(E[q]);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            // corner q: edges to the next corner (E[q]) and to the previous one (-E[q-1])
            const double3 e0 = E[q], e1 = make_double3(-E[(q + 3) & 3].x, -E[(q + 3) & 3].y, 0.0);
            const float3 u1 = make_float3(-U[(q + 3) & 3].x, -U[(q + 3) & 3].y, 0.f);
            pair_2d(U[q], u1, m);
            const double o = __dsub_rn(__dmul_rn(e0.x, e1.y), __dmul_rn(e0.y, e1.x));
            pos |= o > 0.0;
            neg |= o < 0.0;
        }
    } else {
        float3 Ui[2][2], Uk[2][2], Uj[2][2];  // unit edges in the +i [dk][dj], +k [di][dj], +j [di][dk] directions
        {
            double3 P[2][2][2];  // [di][dk][dj]
#pragma unroll
            for (int di = 0; di < 2; ++di)
#pragma unroll
                for (int dk = 0; dk < 2; ++dk)
#pragma unroll
                    for (int dj = 0; dj < 2; ++dj) P[di][dk][dj] = node<3>(a, di ? i1 : i, k + dk, j + dj);
#pragma unroll
            for (int s = 0; s < 2; ++s)
#pragma unroll
                for (int t = 0; t < 2; ++t) {
                    Ui[s][t] = unit_f(dsub3(P[1][s][t], P[0][s][t]));
                    Uk[s][t] = unit_f(dsub3(P[s][1][t], P[s][0][t]));
                    Uj[s][t] = unit_f(dsub3(P[s][t][1], P[s][t][0]));
                }
        }
#pragma unroll
        for (int di = 0; di < 2; ++di)
#pragma unroll
            for (int dk = 0; dk < 2; ++dk)
#pragma unroll
                for (int dj = 0; dj < 2; ++dj) {
                    // folded angles do not depend on the edge directions' signs
                    const float3 ui = Ui[dk][dj], uk = Uk[di][dj], uj = Uj[di][dk];
                    pair_3d(ui, uk, m);
                    pair_3d(ui, uj, m);
                    pair_3d(uk, uj, m);
                    // orientation: with the corner's edges pointing into the
                    // cell and the parity correction, the sign is that of
                    // Ei . (Ek x Ej) at the corner
                    const float3 x = cross_f(uk, uj);
                    const float t = fmaf(ui.x, x.x, fmaf(ui.y, x.y, ui.z * x.z));
                    double o = (double)t;
                    // unit vectors carry an FP32 error below 1e-6: closer than
                    // 1e-5 to zero, redo the corner in FP64 from the nodes
                    if (!(fabsf(t) > 1e-5f)) o = corner_triple_f64(a, i, i1, k, j, di, dk, dj);
                    pos |= o > 0.0;
                    neg |= o < 0.0;
                }
    }
    tangled = pos && neg;
    return atan2f(m.S, m.C) * 57.29577951308232f;
}

template <int DIM>
__global__ void __launch_bounds__(kThreads, 2) k_quality(QualArgs a) {
    float mn = INFINITY;
    long long amin = -1;
    double sum = 0.0;
    unsigned tang = 0;
    unsigned hist[kBins];  // per thread: far below 2^32
#pragma unroll
    for (int b = 0; b < kBins; ++b) hist[b] = 0;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < a.cells;
         idx += (int64_t)gridDim.x * blockDim.x) {
        bool t = false;
        const float th = cell_quality<DIM>(a, idx, t);
        if (a.theta) a.theta[idx] = th;
        if (th < mn) {  // indices increase along the loop: the first minimum stays
            mn = th;
            amin = idx;
        }
        sum += (double)th;
        tang += t ? 1u : 0u;
        const int b = min(kBins - 1, max(0, (int)(th * 0.1f)));
#pragma unroll
        for (int q = 0; q < kBins; ++q) hist[q] += (b == q) ? 1u : 0u;  // stays in registers
    }
    // block reduction in a fixed order
    __shared__ float s_mn[kThreads];
    __shared__ long long s_am[kThreads];
    __shared__ double s_sum[kThreads];
    __shared__ long long s_cnt[kThreads];
    const int tid = threadIdx.x;
    s_mn[tid] = mn;
    s_am[tid] = amin;
    s_sum[tid] = sum;
    __syncthreads();
    for (int s = kThreads / 2; s > 0; s >>= 1) {
        if (tid < s) {
            const float om = s_mn[tid + s];
            const long long oa = s_am[tid + s];
            if (om < s_mn[tid] || (om == s_mn[tid] && oa >= 0 && (s_am[tid] < 0 || oa < s_am[tid]))) {
                s_mn[tid] = om;
                s_am[tid] = oa;
            }
            s_sum[tid] += s_sum[tid + s];
        }
        __syncthreads();
    }
    QPart *p = a.part + blockIdx.x;
    if (tid == 0) {
        p->min_deg = s_mn[0];
        p->argmin = s_am[0];
        p->sum = s_sum[0];
    }
    // integer counts: order does not matter
#pragma unroll
    for (int b = -1; b < kBins; ++b) {
        __syncthreads();
        s_cnt[tid] = b < 0 ? (long long)tang : (long long)hist[b];
        __syncthreads();
        for (int s = kThreads / 2; s > 0; s >>= 1) {
            if (tid < s) s_cnt[tid] += s_cnt[tid + s];
            __syncthreads();
        }
        if (tid == 0) {
            if (b < 0)
                p->tangled = s_cnt[0];
            else
                p->hist[b] = s_cnt[0];
        }
    }
}

// Combine two partials: smaller minimum (lower index on ties), sums, counts.
__device__ __forceinline__ void qmerge(QPart &r, const QPart &p) {
    if (p.min_deg < r.min_deg || (p.min_deg == r.min_deg && p.argmin >= 0 && (r.argmin < 0 || p.argmin < r.argmin))) {
        r.min_deg = p.min_deg;
        r.argmin = p.argmin;
    }
    r.sum += p.sum;
    r.tangled += p.tangled;
#pragma unroll
    for (int q = 0; q < kBins; ++q) r.hist[q] += p.hist[q];
}

// One block: thread t folds partials t, t + 256, ... in order, then a fixed
// tree; the result does not depend on timing.
__global__ void __launch_bounds__(kThreads) k_quality_reduce(const QPart *__restrict__ part, int nb,
                                                             QPart *__restrict__ out) {
    __shared__ QPart s[kThreads];
    const int t = threadIdx.x;
    QPart r;
    r.min_deg = INFINITY;
    r.argmin = -1;
    r.sum = 0.0;
    r.tangled = 0;
#pragma unroll
    for (int q = 0; q < kBins; ++q) r.hist[q] = 0;
    for (int b = t; b < nb; b += kThreads) qmerge(r, part[b]);
    s[t] = r;
    __syncthreads();
    for (int w = kThreads / 2; w > 0; w >>= 1) {
        if (t < w) {
            QPart x = s[t];
            qmerge(x, s[t + w]);
            s[t] = x;
        }
        __syncthreads();
    }
    if (t == 0) *out = s[0];
}

}  // namespace

void orthogonality_run(int dim, int64_t n_i, int64_t n_k, int64_t n_layers, int periodic_i, const double *wall,
                       const double *wall_disp, const float *vol, const float *vol_disp, bool on_device,
                       cudaStream_t st, float *theta, rbfd_quality *q) {
    if (dim == 2) n_k = 1;
    const int64_t n_ci = periodic_i ? n_i : n_i - 1;
    const int64_t n_ck = dim == 3 ? n_k - 1 : 1;
    const int64_t cells = n_ck * n_ci * n_layers;
    const size_t nw = (size_t)(n_k * n_i * dim), nv = (size_t)(n_k * n_i * n_layers * dim);
    QualArgs a{};
    a.n_i = n_i;
    a.n_k = n_k;
    a.n_layers = n_layers;
    a.n_ci = n_ci;
    a.cells = cells;
    std::vector<void *> owned;
    auto stage = [&](const void *src, size_t bytes) -> void * {
        if (!src) return nullptr;
        if (on_device) return const_cast<void *>(src);
        void *d = dmalloc(bytes, "quality staging");
        owned.push_back(d);
        RBFD_CUDA(cudaMemcpyAsync(d, src, bytes, cudaMemcpyHostToDevice, st));
        return d;
    };
    try {
        a.wall = static_cast<const double *>(stage(wall, sizeof(double) * nw));
        a.wall_disp = static_cast<const double *>(stage(wall_disp, sizeof(double) * nw));
        a.vol = static_cast<const float *>(stage(vol, sizeof(float) * nv));
        a.vol_disp = static_cast<const float *>(stage(vol_disp, sizeof(float) * nv));
        float *dtheta = theta;
        if (theta && !on_device) {
            dtheta = dalloc<float>((size_t)cells, "quality angles");
            owned.push_back(dtheta);
        }
        a.theta = dtheta;
        int dev = 0;
        RBFD_CUDA(cudaGetDevice(&dev));
        int sms = 0;
        RBFD_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        const int nb = (int)std::max<int64_t>(1, std::min<int64_t>((cells + kThreads - 1) / kThreads, 8LL * sms));
        QPart *part = dalloc<QPart>((size_t)nb + 1, "quality partials");
        owned.push_back(part);
        a.part = part;
        if (dim == 2)
            k_quality<2><<<nb, kThreads, 0, st>>>(a);
        else
            k_quality<3><<<nb, kThreads, 0, st>>>(a);
        RBFD_CUDA(cudaGetLastError());
        k_quality_reduce<<<1, kThreads, 0, st>>>(part, nb, part + nb);
        RBFD_CUDA(cudaGetLastError());
        QPart r{};
        RBFD_CUDA(cudaMemcpyAsync(&r, part + nb, sizeof(QPart), cudaMemcpyDeviceToHost, st));
        if (theta && !on_device)
            RBFD_CUDA(cudaMemcpyAsync(theta, dtheta, sizeof(float) * cells, cudaMemcpyDeviceToHost, st));
        RBFD_CUDA(cudaStreamSynchronize(st));
        if (q) {
            q->min_deg = r.min_deg;
            q->mean_deg = cells ? r.sum / (double)cells : 0.0;
            q->argmin = r.argmin;
            q->cells = cells;
            q->tangled = r.tangled;
            for (int b = 0; b < kBins; ++b) q->hist[b] = r.hist[b];
        }
    } catch (...) {
        cudaStreamSynchronize(st);
        for (void *p : owned) dfree(p);
        throw;
    }
    for (void *p : owned) dfree(p);
}

}  // namespace rbfd
