// greedy.cu -- multi-level greedy surface point selection (Section 3) on the
// device, plus the per-mesh preparation of the surface.
//
// One greedy step, with n controls C = (c_0 .. c_{n-1}) selected so far:
//
//   sweep      E_i = dS_l,i - sum_{j in list(block(i))} alpha_j phi(|r_i - r_cj| / R)   (Eq. 12)
//              for every surface point i; the controls a point block can reach
//              (those within R of the block's bounding box) are kept in a
//              per-block list that grows by at most one entry per step.  The
//              same launch reduces max |E_i|^2 over the unselected points to
//              the next control (last-block-done reductions, no spin waits)
//              and applies the stop test max|E| / max|dS| < tau_l in FP64.
//   grow       append c_n to Phi_cc = L L^T through the INVERSE factor
//              G = L^{-1}: y = G phi(C, c_n), l = sqrt(phi(0) - y.y),
//              G row n = [-(y^T G) / l, 1 / l], w_n = (dS_l(c_n) - y.w) / l,
//              alpha += w_n * (G row n).  In exact arithmetic this is the
//              bordered Cholesky solve of Eq. 9 on the control set; every
//              product is a matrix-vector product (no sequential substitution),
//              and alpha is updated in O(n) instead of re-solved.
//
// Level close: FP64 iterative refinement of alpha against the matrix-free
// FP64 residual dS_c - Phi_cc alpha (preconditioned by G^T G), an FP64 confirm
// sweep that stores E (the next level's target, dS_{l+1} = E), and the
// per-level uniform cell grid of the controls for the volume update.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstdio>
#include <cstring>

#include "internal.h"

namespace rbfd {

namespace {

constexpr int kThreads = 128;
constexpr int kJT = 256;       // rows per tile of the column-sum kernels
constexpr int kYWarps = 8;     // warps per block of the G*phi kernel
constexpr int kTargetCTAs = 152 * 4;

inline unsigned cdiv(size_t a, size_t b) { return (unsigned)((a + b - 1) / b); }

// ------------------------------------------------------------- prep kernels

__global__ void k_unpack(const double *__restrict__ xyz, const double *__restrict__ dS, int64_t n, int dim,
                         double4 *__restrict__ x4, double4 *__restrict__ d4) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double *p = xyz + i * dim, *q = dS + i * dim;
    x4[i] = make_double4(p[0], p[1], dim == 3 ? p[2] : 0.0, 0.0);
    d4[i] = make_double4(q[0], q[1], dim == 3 ? q[2] : 0.0, 0.0);
}

// Two-pass bounding box of double4 points: per-block partials, then one block.
__global__ void k_bbox_partial(const double4 *__restrict__ p, int64_t n, double *__restrict__ part) {
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

// Final box from nb per-block partials [nb][6]: one warp per coordinate bound.
__global__ void k_bbox_final(const double *__restrict__ part, int nb, double *__restrict__ out) {
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

__global__ void k_gather_sorted(const uint32_t *__restrict__ perm, int64_t n, const double4 *__restrict__ x4,
                                const double4 *__restrict__ d4, double4 *__restrict__ xs, double4 *__restrict__ ds,
                                uint32_t *__restrict__ inv) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t o = perm[i];
    xs[i] = x4[o];
    ds[i] = d4[o];
    inv[o] = (uint32_t)i;
}

// Point blocks of kPB consecutive Morton-ordered points: bounding box, origin
// (the box's low corner) and the points' coordinates relative to it as
// double-float (hi, lo) pairs for the mixed-precision sweep.
__global__ void k_point_blocks(const double4 *__restrict__ xs, int64_t n, double4 *__restrict__ lo_out,
                               double4 *__restrict__ hi_out, double4 *__restrict__ org_out,
                               float4 *__restrict__ xhi, float4 *__restrict__ xlo, float4 *__restrict__ wbox) {
    __shared__ double s[6][kPB / 32];
    int64_t i = (int64_t)blockIdx.x * kPB + threadIdx.x;
    bool valid = i < n;
    double4 q = valid ? xs[i] : make_double4(0, 0, 0, 0);
    double lo[3] = {valid ? q.x : INFINITY, valid ? q.y : INFINITY, valid ? q.z : INFINITY};
    double hi[3] = {valid ? q.x : -INFINITY, valid ? q.y : -INFINITY, valid ? q.z : -INFINITY};
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
    if (wbox && lane == 0) {  // each warp's box in FP32, rounded outward (empty for a warp with no point)
        const size_t ww = (size_t)blockIdx.x * (kPB / 32) + w;
        wbox[2 * ww] = make_float4(__double2float_rd(lo[0]), __double2float_rd(lo[1]), __double2float_rd(lo[2]), 0.f);
        wbox[2 * ww + 1] = make_float4(__double2float_ru(hi[0]), __double2float_ru(hi[1]), __double2float_ru(hi[2]), 0.f);
    }
    __syncthreads();
    for (int k = 0; k < 3; ++k) {
        lo[k] = s[k][0];
        hi[k] = s[3 + k][0];
        for (int j = 1; j < kPB / 32; ++j) {
            lo[k] = fmin(lo[k], s[k][j]);
            hi[k] = fmax(hi[k], s[3 + k][j]);
        }
    }
    if (threadIdx.x == 0) {
        lo_out[blockIdx.x] = make_double4(lo[0], lo[1], lo[2], 0);
        hi_out[blockIdx.x] = make_double4(hi[0], hi[1], hi[2], 0);
        org_out[blockIdx.x] = make_double4(lo[0], lo[1], lo[2], 0);
    }
    if (valid) {
        double r[3] = {q.x - lo[0], q.y - lo[1], q.z - lo[2]};
        float h[3], l[3];
        for (int k = 0; k < 3; ++k) {
            h[k] = __double2float_rn(r[k]);
            l[k] = __double2float_rn(r[k] - (double)h[k]);
        }
        xhi[i] = make_float4(h[0], h[1], h[2], 0.f);
        xlo[i] = make_float4(l[0], l[1], l[2], 0.f);
    }
}

// max_i |v_i|^2 (each square summed in coordinate order) and its argmax
// (lowest original index on ties) over n points; last-block-done reduction.
// out[0] = key, ((int*)(out + 1))[0] = original index of the argmax.
__global__ void k_maxnorm(const double4 *__restrict__ v, const uint32_t *__restrict__ perm, int64_t n, int dim,
                          double *__restrict__ bkey, int *__restrict__ bidx, unsigned int *done,
                          double *__restrict__ out) {
    __shared__ double sk[32];
    __shared__ int si[32];
    __shared__ bool last;
    double k = -1.0;
    int id = -1;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double4 q = v[i];
        double key = __dmul_rn(q.x, q.x);
        key = __dadd_rn(key, __dmul_rn(q.y, q.y));
        if (dim == 3) key = __dadd_rn(key, __dmul_rn(q.z, q.z));
        int o = (int)perm[i];
        if (better(key, o, k, id)) {
            k = key;
            id = o;
        }
    }
    block_argmax(k, id, sk, si);
    if (threadIdx.x == 0) {
        bkey[blockIdx.x] = k;
        bidx[blockIdx.x] = id;
        __threadfence();
        last = atomicAdd(done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    k = -1.0;
    id = -1;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
        double kb = __ldcg(&bkey[b]);
        int ib = __ldcg(&bidx[b]);
        if (better(kb, ib, k, id)) {
            k = kb;
            id = ib;
        }
    }
    block_argmax(k, id, sk, si);
    if (threadIdx.x == 0) {
        out[0] = k;
        reinterpret_cast<int *>(out + 1)[0] = id;
        *done = 0;
    }
}

// ---------------------------------------------------------------- sweep

struct SweepArgs {
    int64_t n_s;
    int n_pb, cap, n, chunk_len;
    const double4 *xs;
    const float4 *xs_hi, *xs_lo;
    const double4 *pb_org;
    const double4 *cur;
    const unsigned char *sel;
    const uint32_t *perm;
    const uint32_t *nb_cnt, *nb_list;
    const double4 *cx, *alpha;
    double R, S0, tau, invR;
    float invR_hi, invR_lo;
    double4 *part;
    double4 *E_out;  // non-null: store E (confirm sweep)
    double *pb_key;
    int *pb_idx;
    unsigned int *pb_done;
    GreedyState *st;
    unsigned long long *pairs;
    int is_step;  // 1: greedy step (argmax over unselected + stop test); 0: confirm (max over all)
    int dim;
    // confirm: n from this state when given (no sweep if its launch handed
    // the level on); the lists are cut into min(ceil(n / 8), chunk_cap)
    // chunks of equal length, the launch's other chunk blocks are idle
    const GreedyState *n_from;
    int chunk_cap;
    // point blocks pb_lo .. pb_lo + pb_n - 1 only (grid.x = pb_n): a rank's
    // Morton range in the surface split; local_only: the tail records the
    // range's argmax and leaves the stop decision to the caller
    int pb_lo, pb_n, local_only;
};

template <int DIM, int BASIS, int MODE>
__global__ void __launch_bounds__(kThreads) k_sweep(SweepArgs a) {
    __shared__ double sk[32];
    __shared__ int si[32];
    __shared__ bool s_last;
    // control tile: FP64 coordinates + weights (MODE 0) or double-float relative
    // coordinates + weights (MODE 1)
    __shared__ double t64[6][kTile];
    __shared__ float t32[12][kTile];
    __shared__ unsigned char s_hits[4][kTile];
    if (a.is_step && a.st->stop) return;
    int n_c = a.n, nch = gridDim.y, chunk_len = a.chunk_len;
    if (!a.is_step) {
        if (a.n_from) {
            if (a.n_from->handoff) return;
            n_c = a.n_from->n;
        }
        nch = max(1, min((n_c + 7) / 8, a.chunk_cap));
        chunk_len = (n_c + nch - 1) / nch;
    }

    const int pb = a.pb_lo + (int)blockIdx.x, ch = blockIdx.y, tid = threadIdx.x;
    const int64_t p = (int64_t)pb * kPB + tid;
    const bool valid = p < a.n_s;
    const uint32_t cnt = a.nb_cnt[pb];
    const int lo = ch < nch ? ch * chunk_len : 0;
    const int hi = ch < nch ? min((int)cnt, lo + chunk_len) : 0;
    const double4 org = a.pb_org[pb];

    double acc64[3] = {0.0, 0.0, 0.0};
    df acc[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
    double px = 0, py = 0, pz = 0;
    df qx{0, 0}, qy{0, 0}, qz{0, 0};
    if (valid) {
        if (MODE == 0) {
            double4 q = a.xs[p];
            px = q.x; py = q.y; pz = q.z;
        } else {
            float4 h = a.xs_hi[p], l = a.xs_lo[p];
            qx = {h.x, l.x}; qy = {h.y, l.y}; qz = {h.z, l.z};
        }
    }
    const df invR = {a.invR_hi, a.invR_lo};
    unsigned useful = 0;
    float3 wlo, whi;
    if (MODE == 1) warp_box(valid, qx.hi, qy.hi, qz.hi, wlo, whi);
    const float R2m = (float)(1.002 * a.R) * (float)(1.002 * a.R);  // filter margin
    for (int t0 = lo; t0 < hi; t0 += kTile) {
        const int m = min(kTile, hi - t0);
        if (tid < m) {
            uint32_t j = a.nb_list[(size_t)pb * a.cap + t0 + tid];
            double4 c = a.cx[j], al = a.alpha[j];
            if (MODE == 0) {
                t64[0][tid] = c.x; t64[1][tid] = c.y; t64[2][tid] = c.z;
                t64[3][tid] = al.x; t64[4][tid] = al.y; t64[5][tid] = al.z;
            } else {
                df rx = df_from_double(c.x - org.x), ry = df_from_double(c.y - org.y), rz = df_from_double(c.z - org.z);
                df ax = df_from_double(al.x), ay = df_from_double(al.y), az = df_from_double(al.z);
                t32[0][tid] = rx.hi; t32[1][tid] = rx.lo; t32[2][tid] = ry.hi; t32[3][tid] = ry.lo;
                t32[4][tid] = rz.hi; t32[5][tid] = rz.lo; t32[6][tid] = ax.hi; t32[7][tid] = ax.lo;
                t32[8][tid] = ay.hi; t32[9][tid] = ay.lo; t32[10][tid] = az.hi; t32[11][tid] = az.lo;
            }
        }
        __syncthreads();
        if (MODE == 0) {
            // A warp skips a control farther than R from all its points: there
            // eta = |r - r_c| / R rounds to at least 1 and phi is exactly 0,
            // so the sums do not change.  (FP64 issues at one warp
            // instruction per 64 cycles per SM sub-partition, and the root,
            // the division and phi are most of a pair's instructions.)
            const double R2hi = __dmul_rn(__dmul_rn(a.R, a.R), 1.0 + 1e-12);
            for (int q = 0; q < m; ++q) {
                const double s2 = dist2_f64<DIM>(px, py, pz, t64[0][q], t64[1][q], t64[2][q]);
                if (!__any_sync(0xffffffffu, valid && s2 <= R2hi)) continue;
                if (valid) {
                    // a greedy step divides by R like the persistent engine's
                    // sweep (the engines agree bit for bit); the confirm sweep
                    // multiplies by 1/R (one rounding more in eta, a tenth of
                    // the FP64 instructions of the division)
                    const double d = __dsqrt_rn(s2);
                    double eta = a.is_step ? __ddiv_rn(d, a.R) : __dmul_rn(d, a.invR);
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
            if (valid) hits_accumulate_df<DIM, BASIS>(qx, qy, qz, t32, s_hits[tid >> 5], nh, invR, acc, useful);
        }
        __syncthreads();
    }
    if (MODE == 1) {
        acc64[0] = df_to_double(acc[0]);
        acc64[1] = df_to_double(acc[1]);
        acc64[2] = df_to_double(acc[2]);
    }
    if (valid) a.part[(size_t)ch * a.n_s + p] = make_double4(acc64[0], acc64[1], acc64[2], 0.0);
    // pair counters (one atomic per block)
    {
        unsigned u = useful;
        for (int o = 16; o > 0; o >>= 1) u += __shfl_xor_sync(0xffffffffu, u, o);
        if ((tid & 31) == 0 && u) atomicAdd(&a.pairs[0], (unsigned long long)u);
        if (tid == 0 && hi > lo) {
            unsigned long long nv = (unsigned long long)min((int64_t)kPB, a.n_s - (int64_t)pb * kPB);
            atomicAdd(&a.pairs[1], nv * (unsigned long long)(hi - lo));
        }
    }
    // last chunk-block of this point block reduces the partial sums in chunk order
    __threadfence();
    __syncthreads();
    if (tid == 0) s_last = atomicAdd(&a.pb_done[pb], 1u) == gridDim.y - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    double key = -1.0;
    int orig = -1;
    if (valid) {
        double s0 = 0.0, s1 = 0.0, s2 = 0.0;
        for (int c = 0; c < nch; ++c) {
            double4 v = ldcg_d4(&a.part[(size_t)c * a.n_s + p]);
            s0 = __dadd_rn(s0, v.x);
            s1 = __dadd_rn(s1, v.y);
            s2 = __dadd_rn(s2, v.z);
        }
        double4 cu = a.cur[p];
        double e0 = __dsub_rn(cu.x, s0), e1 = __dsub_rn(cu.y, s1), e2 = (DIM == 3) ? __dsub_rn(cu.z, s2) : 0.0;
        if (a.E_out) a.E_out[p] = make_double4(e0, e1, e2, 0.0);
        double k2 = __dmul_rn(e0, e0);
        k2 = __dadd_rn(k2, __dmul_rn(e1, e1));
        if (DIM == 3) k2 = __dadd_rn(k2, __dmul_rn(e2, e2));
        if (!a.is_step || !a.sel[p]) {
            key = k2;
            orig = (int)a.perm[p];
        }
    }
    block_argmax(key, orig, sk, si);
    if (tid == 0) {
        a.pb_key[pb] = key;
        a.pb_idx[pb] = orig;
        a.pb_done[pb] = 0;
        __threadfence();
        s_last = atomicAdd(&a.st->pb_done, 1u) == (unsigned)(a.pb_n - 1);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    key = -1.0;
    orig = -1;
    for (int b = a.pb_lo + tid; b < a.pb_lo + a.pb_n; b += kThreads) {
        double kb = __ldcg(&a.pb_key[b]);
        int ib = __ldcg(&a.pb_idx[b]);
        if (better(kb, ib, key, orig)) {
            key = kb;
            orig = ib;
        }
    }
    block_argmax(key, orig, sk, si);
    if (tid == 0) {
        GreedyState *st = a.st;
        st->pb_done = 0;
        st->best_orig = orig;
        st->best_key = key;
        double e = orig >= 0 ? __ddiv_rn(__dsqrt_rn(key), a.S0) : 0.0;
        st->emax = e;
        if (a.is_step && !a.local_only) {
            if (orig < 0 || e < a.tau) {
                st->stop = 1;
            } else if (a.n >= a.cap) {
                st->stop = 1;
                st->status = RBFD_ENOTCONV;
            }
        }
    }
}

// The step decision of the surface split, from the argmax over every rank's
// range (the caller's all-reduce-maxloc): the same stop test as k_sweep's tail.
__global__ void k_split_decide(GreedyState *st, double key, int orig, double S0, double tau, int n, int cap) {
    st->best_orig = orig;
    st->best_key = key;
    const double e = orig >= 0 ? __ddiv_rn(__dsqrt_rn(key), S0) : 0.0;
    st->emax = e;
    if (orig < 0 || e < tau) {
        st->stop = 1;
    } else if (n >= cap) {
        st->stop = 1;
        st->status = RBFD_ENOTCONV;
    }
}

// ----------------------------------------------------------------- growth

struct GrowArgs {
    int n, cap, n_pb, dim;
    double R, R2;
    const uint32_t *inv;
    const double4 *xs;
    const double4 *pb_lo, *pb_hi;
    unsigned char *sel;
    double4 *cx;
    uint32_t *cid;
    double *phi;
    uint32_t *nb_cnt, *nb_list;
    const double *G;
    double *Gw;
    double *Gt;
    double *y;
    double *red;  // [blocks][4]: y.y, y.w (3)
    int n_red;
    double *gpart;
    double4 *w, *alpha;
    const double4 *cur;
    GreedyState *st;
};

// phi(|r_cn - r_ck| / R) for k < n; list the new control in every point block
// within R of it; record it as control n.
template <int DIM, int BASIS>
__global__ void k_grow_phi(GrowArgs a) {
    if (a.st->stop) return;
    const uint32_t c = a.inv[a.st->best_orig];
    const double4 x = a.xs[c];
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < a.n) {
        double4 ck = a.cx[t];
        a.phi[t] = phi_f64<BASIS>(__ddiv_rn(dist_f64<DIM>(x.x, x.y, x.z, ck.x, ck.y, ck.z), a.R));
    }
    if (t < a.n_pb) {
        double4 l = a.pb_lo[t], h = a.pb_hi[t];
        double dx = fmax(fmax(l.x - x.x, x.x - h.x), 0.0);
        double dy = fmax(fmax(l.y - x.y, x.y - h.y), 0.0);
        double dz = DIM == 3 ? fmax(fmax(l.z - x.z, x.z - h.z), 0.0) : 0.0;
        if (dx * dx + dy * dy + dz * dz < a.R2 * (1.0 + 1e-9)) {
            uint32_t k = a.nb_cnt[t];
            a.nb_list[(size_t)t * a.cap + k] = (uint32_t)a.n;
            a.nb_cnt[t] = k + 1;
        }
    }
    if (t == 0) {
        a.sel[c] = 1;
        a.cx[a.n] = x;
        a.cid[a.n] = c;
    }
}

// y_j = sum_{k <= j} G_jk phi_k, one warp per row; per-block partial sums of
// y_j^2 and y_j w_j (3 components) in fixed order.
__global__ void k_grow_y(GrowArgs a) {
    if (a.st->stop) return;
    __shared__ double s[kYWarps][4];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int j = blockIdx.x * kYWarps + w;
    double yy = 0, yw0 = 0, yw1 = 0, yw2 = 0;
    if (j < a.n) {
        const double *row = a.G + (size_t)j * a.cap;
        double acc = 0.0;
        for (int k = lane; k <= j; k += 32) acc = fma(row[k], a.phi[k], acc);
        acc = warp_sum_d(acc);
        if (lane == 0) a.y[j] = acc;
        double4 wj = a.w[j];
        yy = acc * acc;
        yw0 = acc * wj.x;
        yw1 = acc * wj.y;
        yw2 = acc * wj.z;
    }
    if (lane == 0) {
        s[w][0] = yy; s[w][1] = yw0; s[w][2] = yw1; s[w][3] = yw2;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        double v = 0;
        for (int q = 0; q < kYWarps; ++q) v += s[q][threadIdx.x];
        a.red[blockIdx.x * 4 + threadIdx.x] = v;
    }
}

// Partial column sums of y^T G over a tile of kJT rows: gpart[jt][k].
__global__ void k_colsum(int n, int cap, const double *__restrict__ G, const double *__restrict__ y,
                         double *__restrict__ gpart, const GreedyState *st) {
    if (st && st->stop) return;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int jt = blockIdx.y;
    if (k >= n) return;
    int j0 = max(jt * kJT, k), j1 = min(n, (jt + 1) * kJT);
    double s = 0.0;
    for (int j = j0; j < j1; ++j) s = fma(y[j], G[(size_t)j * cap + k], s);
    gpart[(size_t)jt * cap + k] = s;
}

// Finish the row append: l, w_n, G row n and alpha += w_n * G row n.
__global__ void k_grow_finish(GrowArgs a, int n_jt) {
    if (a.st->stop) return;
    __shared__ double sh[4];
    if (threadIdx.x < 4) {
        double v = 0;
        for (int b = 0; b < a.n_red; ++b) v += a.red[b * 4 + threadIdx.x];
        sh[threadIdx.x] = v;
    }
    __syncthreads();
    const double l2 = 1.0 - sh[0];  // phi(0) = 1 for every Wendland function
    // 1 - y.y carries an absolute rounding error of about n u: a pivot below
    // a few times that is numerically zero (coincident controls)
    if (!(l2 > 8.0 * (a.n + 1) * 1.1102230246251565e-16)) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            a.st->status = RBFD_ESINGULAR;
            a.st->stop = 1;
        }
        return;
    }
    const double l = sqrt(l2);
    const uint32_t c = a.cid[a.n];
    const double4 b = a.cur[c];
    const double4 wn = make_double4((b.x - sh[1]) / l, (b.y - sh[2]) / l, (b.z - sh[3]) / l, 0.0);
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    double *Grow = a.Gw + (size_t)a.n * a.cap;
    if (k < a.n) {
        double s = 0.0;
        for (int jt = 0; jt < n_jt; ++jt) s += a.gpart[(size_t)jt * a.cap + k];
        double g = -s / l;
        Grow[k] = g;
        a.Gt[(size_t)k * a.cap + a.n] = g;
        double4 al = a.alpha[k];
        al.x = fma(wn.x, g, al.x);
        al.y = fma(wn.y, g, al.y);
        al.z = fma(wn.z, g, al.z);
        a.alpha[k] = al;
    } else if (k == a.n) {
        Grow[k] = 1.0 / l;
        a.Gt[(size_t)k * a.cap + k] = 1.0 / l;
        a.w[k] = wn;
        a.alpha[k] = make_double4(wn.x / l, wn.y / l, wn.z / l, 0.0);
        a.st->n = a.n + 1;
    }
}

// Start a level: control 0, G = [1], w_0 = alpha_0 = dS_l(c_0); list it.
__global__ void k_level_init(int first_orig_from_state, int first_orig, const uint32_t *inv, const double4 *xs,
                             const double4 *cur, int n_pb, int cap, int dim, double R2, const double4 *pb_lo,
                             const double4 *pb_hi, unsigned char *sel, double4 *cx, float4 *cdf, uint32_t *cid,
                             double *G,
                             double *Gt, double4 *w, double4 *alpha, uint32_t *nb_cnt, uint32_t *nb_list,
                             const double *red_out, GreedyState *st) {
    int o = first_orig_from_state ? reinterpret_cast<const int *>(red_out + 1)[0] : first_orig;
    const uint32_t c = inv[o];
    const double4 x = xs[c];
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n_pb) {
        double4 l = pb_lo[t], h = pb_hi[t];
        double dx = fmax(fmax(l.x - x.x, x.x - h.x), 0.0);
        double dy = fmax(fmax(l.y - x.y, x.y - h.y), 0.0);
        double dz = dim == 3 ? fmax(fmax(l.z - x.z, x.z - h.z), 0.0) : 0.0;
        bool in = dx * dx + dy * dy + dz * dz < R2 * (1.0 + 1e-9);
        nb_cnt[t] = in ? 1u : 0u;
        if (in) nb_list[(size_t)t * cap] = 0u;
    }
    if (t == 0) {
        sel[c] = 1;
        cx[0] = x;
        const float hx = __double2float_rn(x.x), hy = __double2float_rn(x.y), hz = __double2float_rn(x.z);
        cdf[0] = make_float4(hx, hy, hz, 0.f);
        cdf[cap + 1] = make_float4(__double2float_rn(x.x - (double)hx), __double2float_rn(x.y - (double)hy),
                                   __double2float_rn(x.z - (double)hz), 0.f);
        cid[0] = c;
        G[0] = 1.0;
        Gt[0] = 1.0;
        double4 b = cur[c];
        w[0] = b;
        alpha[0] = b;
        st->n = 1;
        st->stop = 0;
        st->status = RBFD_OK;
        st->best = -1;
        st->best_orig = -1;
        st->best_key = 0;
        st->second_key = 0;
        st->min_gap = 1.0;
        st->emax = 0;
        st->pb_done = 0;
        st->red_done = 0;
        st->max_cnt = 1;
        st->nnz = 0;
    }
}

// ------------------------------------------------------------ refinement

// r_i = dS_l(c_i) - sum_j alpha_j phi(|r_ci - r_cj| / R), FP64, one warp per
// control i; the sum runs over the controls listed for the point block that
// holds c_i (every control within R of it is listed, so the omitted ones
// contribute exactly 0).  Per block, max |r| and whether any residual is above
// its rounding level to red[2 block], red[2 block + 1]; the last block to
// finish (a counter in cnt, reset by that block) tests them on the device:
// once the largest residual is at most tol, or every residual is at the
// rounding level of its evaluation, lvl[2] is set and the rest of this level
// close does nothing; lvl[3] counts the corrections.
// The level-close kernels take n from nfrom when it is given (a close queued
// behind the greedy launch before the host has read n) and then do nothing
// if that launch handed the level on; warps stride over the rows.
__device__ __forceinline__ bool close_rows(const GreedyState *nfrom, int &n) {
    if (!nfrom) return true;
    if (nfrom->handoff) return false;
    n = nfrom->n;
    return true;
}

template <int DIM, int BASIS>
__global__ void __launch_bounds__(kThreads) k_resid(int n, const GreedyState *__restrict__ nfrom, double R, int cap,
                                                    const double4 *__restrict__ cx,
                                                    const double4 *__restrict__ alpha,
                                                    const uint32_t *__restrict__ cid,
                                                    const uint32_t *__restrict__ nb_cnt,
                                                    const uint32_t *__restrict__ nb_list,
                                                    const double4 *__restrict__ cur, double4 *__restrict__ r,
                                                    double *__restrict__ red, double tol, double *__restrict__ lvl,
                                                    unsigned *__restrict__ cnt) {
    if (lvl[2] != 0.0 || !close_rows(nfrom, n)) return;  // converged, or no close for this launch
    const double invR = 1.0 / R;
    __shared__ double sm[kThreads / 32], sb[kThreads / 32];
    __shared__ bool sa[kThreads / 32];
    __shared__ bool s_last;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    double mx = 0.0;
    bool above = false;
    for (int i = blockIdx.x * (kThreads / 32) + w; i < n; i += gridDim.x * (kThreads / 32)) {
        const uint32_t ci = cid[i];
        const double4 xi = cx[i];
        const int pb = (int)(ci / kPB);
        const int cnt = (int)nb_cnt[pb];
        const uint32_t *list = nb_list + (size_t)pb * cap;
        double a0 = 0, a1 = 0, a2 = 0, b0 = 0, b1 = 0, b2 = 0;
        for (int q = lane; q < cnt; q += 32) {
            const uint32_t j = list[q];
            const double4 c = cx[j], al = alpha[j];
            const double f = phi_f64<BASIS>(__dmul_rn(dist_f64<DIM>(xi.x, xi.y, xi.z, c.x, c.y, c.z), invR));
            a0 = fma(al.x, f, a0);
            a1 = fma(al.y, f, a1);
            a2 = fma(al.z, f, a2);
            b0 = fma(fabs(al.x), f, b0);  // (f >= 0)
            b1 = fma(fabs(al.y), f, b1);
            b2 = fma(fabs(al.z), f, b2);
        }
        a0 = warp_sum_d(a0);
        a1 = warp_sum_d(a1);
        a2 = warp_sum_d(a2);
        b0 = warp_sum_d(b0);
        b1 = warp_sum_d(b1);
        b2 = warp_sum_d(b2);
        if (lane == 0) {
            const double4 b = cur[ci];
            const double4 ri = make_double4(b.x - a0, b.y - a1, DIM == 3 ? b.z - a2 : 0.0, 0.0);
            r[i] = ri;
            mx = fmax(mx, fmax(fabs(ri.x), fmax(fabs(ri.y), fabs(ri.z))));
            // at the rounding level of its own evaluation: 32 u (|b| + sum |alpha phi|)
            const double u32 = 32.0 * 1.1102230246251565e-16;
            above |= fabs(ri.x) > u32 * (fabs(b.x) + b0) || fabs(ri.y) > u32 * (fabs(b.y) + b1) ||
                     (DIM == 3 && fabs(ri.z) > u32 * (fabs(b.z) + b2));
        }
    }
    if (lane == 0) {
        sm[w] = mx;
        sa[w] = above;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double v = sm[0];
        bool ab = sa[0];
        for (int q = 1; q < kThreads / 32; ++q) {
            v = fmax(v, sm[q]);
            ab = ab || sa[q];
        }
        red[2 * blockIdx.x] = v;
        red[2 * blockIdx.x + 1] = ab ? 1.0 : 0.0;
        __threadfence();
        s_last = atomicAdd(cnt, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    double v = 0.0, ab = 0.0;
    for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x) {
        v = fmax(v, __ldcg(&red[2 * b]));
        ab = fmax(ab, __ldcg(&red[2 * b + 1]));
    }
    for (int o = 16; o > 0; o >>= 1) {
        v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
        ab = fmax(ab, __shfl_xor_sync(0xffffffffu, ab, o));
    }
    __syncthreads();
    if (lane == 0) {
        sm[w] = v;
        sb[w] = ab;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int q = 1; q < kThreads / 32; ++q) {
            v = fmax(v, sm[q]);
            ab = fmax(ab, sb[q]);
        }
        // converged: below tol, or every residual at its rounding level
        // (further corrections cannot lower it)
        if (v <= tol || ab == 0.0) lvl[2] = 1.0;
        else lvl[3] += 1.0;
        *cnt = 0;
    }
}

// z_j = sum_{k <= j} G_jk r_k (3 right-hand sides), one warp per row.
__global__ void k_lower_mv3(int n, const GreedyState *__restrict__ nfrom, int cap, const double *__restrict__ G,
                            const double4 *__restrict__ r, double4 *__restrict__ z, const double *__restrict__ done) {
    if (*done != 0.0 || !close_rows(nfrom, n)) return;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int j = blockIdx.x * (blockDim.x >> 5) + w; j < n; j += gridDim.x * (blockDim.x >> 5)) {
    const double *row = G + (size_t)j * cap;
    double s0 = 0, s1 = 0, s2 = 0;
    for (int k = lane; k <= j; k += 32) {
        double g = row[k];
        double4 v = r[k];
        s0 = fma(g, v.x, s0);
        s1 = fma(g, v.y, s1);
        s2 = fma(g, v.z, s2);
    }
    s0 = warp_sum_d(s0);
    s1 = warp_sum_d(s1);
    s2 = warp_sum_d(s2);
    if (lane == 0) z[j] = make_double4(s0, s1, s2, 0.0);
    }
}

// alpha_k += sum_{j >= k} G_jk z_j (3 right-hand sides), one warp per k over
// row k of the transposed copy G^T (contiguous).
__global__ void k_upper_mv3_add(int n, const GreedyState *__restrict__ nfrom, int cap, const double *__restrict__ Gt,
                                const double4 *__restrict__ z, double4 *__restrict__ alpha,
                                const double *__restrict__ done) {
    if (*done != 0.0 || !close_rows(nfrom, n)) return;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int k = blockIdx.x * (blockDim.x >> 5) + w; k < n; k += gridDim.x * (blockDim.x >> 5)) {
    const double *row = Gt + (size_t)k * cap;
    double s0 = 0, s1 = 0, s2 = 0;
    for (int j = k + lane; j < n; j += 32) {
        const double g = row[j];
        const double4 v = z[j];
        s0 = fma(g, v.x, s0);
        s1 = fma(g, v.y, s1);
        s2 = fma(g, v.z, s2);
    }
    s0 = warp_sum_d(s0);
    s1 = warp_sum_d(s1);
    s2 = warp_sum_d(s2);
    if (lane == 0) {
        const double4 a = alpha[k];
        alpha[k] = make_double4(a.x + s0, a.y + s1, a.z + s2, 0.0);
    }
    }
}

// ------------------------------------------------------------ control grid

__global__ void k_orig_of_controls(const uint32_t *__restrict__ perm, const uint32_t *__restrict__ cid, int n,
                                   uint32_t *__restrict__ out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = perm[cid[i]];
}

__global__ void k_cell_keys(const double4 *__restrict__ cx, int n, double3 g0, double inv_h, int3 gd,
                            uint32_t *keys, uint32_t *vals) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double4 c = cx[i];
    int ix = min(max((int)floor((c.x - g0.x) * inv_h), 0), gd.x - 1);
    int iy = min(max((int)floor((c.y - g0.y) * inv_h), 0), gd.y - 1);
    int iz = min(max((int)floor((c.z - g0.z) * inv_h), 0), gd.z - 1);
    keys[i] = (uint32_t)((iz * gd.y + iy) * gd.x + ix);
    vals[i] = (uint32_t)i;
}

// cell_start[c] = first position whose key >= c (binary search in sorted keys)
__global__ void k_cell_start(const uint32_t *__restrict__ keys, int n, int ncell, uint32_t *__restrict__ start) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c > ncell) return;
    int lo = 0, hi = n;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (keys[mid] < (uint32_t)c) lo = mid + 1;
        else hi = mid;
    }
    start[c] = (uint32_t)lo;
}

// ---------------------------------------------------------- dispatch helpers

template <int DIM, int BASIS>
void launch_sweep_t(int mode, dim3 grid, const SweepArgs &a, cudaStream_t st) {
    if (mode == 0) k_sweep<DIM, BASIS, 0><<<grid, kThreads, 0, st>>>(a);
    else k_sweep<DIM, BASIS, 1><<<grid, kThreads, 0, st>>>(a);
}

template <int DIM>
void launch_sweep_d(int basis, int mode, dim3 grid, const SweepArgs &a, cudaStream_t st) {
    switch (basis) {
    case 0: launch_sweep_t<DIM, 0>(mode, grid, a, st); break;
    case 4: launch_sweep_t<DIM, 4>(mode, grid, a, st); break;
    case 6: launch_sweep_t<DIM, 6>(mode, grid, a, st); break;
    default: launch_sweep_t<DIM, 2>(mode, grid, a, st); break;
    }
}

void launch_sweep(int dim, int basis, int mode, dim3 grid, const SweepArgs &a, cudaStream_t st) {
    if (dim == 2) launch_sweep_d<2>(basis, mode, grid, a, st);
    else launch_sweep_d<3>(basis, mode, grid, a, st);
}

template <int DIM>
void launch_phi_d(int basis, unsigned g, const GrowArgs &a, cudaStream_t st) {
    switch (basis) {
    case 0: k_grow_phi<DIM, 0><<<g, kThreads, 0, st>>>(a); break;
    case 4: k_grow_phi<DIM, 4><<<g, kThreads, 0, st>>>(a); break;
    case 6: k_grow_phi<DIM, 6><<<g, kThreads, 0, st>>>(a); break;
    default: k_grow_phi<DIM, 2><<<g, kThreads, 0, st>>>(a); break;
    }
}

template <int DIM>
void launch_resid_d(int basis, unsigned g, int n, const GreedyState *nfrom, double R, rbfd_mesh *m,
                    cudaStream_t st) {
#define RBFD_RESID(B)                                                                                           \
    k_resid<DIM, B><<<g, kThreads, 0, st>>>(n, nfrom, R, m->cap, m->d_cx, m->d_alpha, m->d_cid, m->d_nb_cnt,    \
                                            m->d_nb_list, m->d_cur, m->d_vec, m->d_red, 1e-15 * m->S0, m->d_lvl, \
                                            &m->d_misc[8])
    switch (basis) {
    case 0: RBFD_RESID(0); break;
    case 4: RBFD_RESID(4); break;
    case 6: RBFD_RESID(6); break;
    default: RBFD_RESID(2); break;
    }
#undef RBFD_RESID
}

// ------------------------------------------------------------ warm start

// A level restarted from a previous run's n controls (sorted positions cid):
// coordinates (FP64 and double-float split), selected flags, the greedy
// state as after n - 1 steps; alpha cleared (re-solved by the caller).
__global__ void k_warm_restore(int n, int cap, const uint32_t *__restrict__ cid_in, const double4 *__restrict__ xs,
                               unsigned char *__restrict__ sel, double4 *__restrict__ cx, float4 *__restrict__ cdf,
                               uint32_t *__restrict__ cid, double4 *__restrict__ alpha, GreedyState *st) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) {
        const uint32_t c = cid_in[k];
        const double4 x = xs[c];
        sel[c] = 1;
        cx[k] = x;
        cid[k] = c;
        const float hx = __double2float_rn(x.x), hy = __double2float_rn(x.y), hz = __double2float_rn(x.z);
        cdf[k] = make_float4(hx, hy, hz, 0.f);
        cdf[cap + 1 + k] = make_float4(__double2float_rn(x.x - (double)hx), __double2float_rn(x.y - (double)hy),
                                       __double2float_rn(x.z - (double)hz), 0.f);
        alpha[k] = make_double4(0.0, 0.0, 0.0, 0.0);
    }
    if (k == 0) {
        st->n = n;
        st->stop = 0;
        st->status = RBFD_OK;
        st->best = -1;
        st->best_orig = -1;
        st->best_key = 0;
        st->second_key = 0;
        st->min_gap = 1.0;
        st->emax = 0;
        st->pb_done = 0;
        st->red_done = 0;
        st->max_cnt = 1;
        st->nnz = 0;
        st->handoff = 0;
    }
}

// The per-block control lists of the restored controls, in control order:
// the same test as a greedy step's listing (box distance below R).
__global__ void k_warm_lists(int n, int n_pb, int cap, int dim, double R2, const double4 *__restrict__ cx,
                             const double4 *__restrict__ pb_lo, const double4 *__restrict__ pb_hi,
                             uint32_t *__restrict__ nb_cnt, uint32_t *__restrict__ nb_list) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_pb) return;
    const double4 l = pb_lo[t], h = pb_hi[t];
    uint32_t cnt = 0;
    for (int k = 0; k < n; ++k) {
        const double4 x = cx[k];
        const double dx = fmax(fmax(l.x - x.x, x.x - h.x), 0.0);
        const double dy = fmax(fmax(l.y - x.y, x.y - h.y), 0.0);
        const double dz = dim == 3 ? fmax(fmax(l.z - x.z, x.z - h.z), 0.0) : 0.0;
        if (dx * dx + dy * dy + dz * dz < R2 * (1.0 + 1e-9)) nb_list[(size_t)t * cap + cnt++] = (uint32_t)k;
    }
    nb_cnt[t] = cnt;
}

// v_k = dS_l at control k (the right-hand sides of Eq. 9).
__global__ void k_gather_ctrl(int n, const uint32_t *__restrict__ cid, const double4 *__restrict__ cur,
                              double4 *__restrict__ v) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) v[k] = cur[cid[k]];
}

int n_chunks_for(const rbfd_mesh *m, int n) {
    int want = (kTargetCTAs + m->n_pb - 1) / m->n_pb;
    int by_len = (n + 31) / 32;
    return std::max(1, std::min(std::min(want, by_len), m->n_chunk_max));
}

SweepArgs base_sweep_args(rbfd_mesh *m, double R, double tau) {
    SweepArgs a{};
    a.n_s = m->n_s;
    a.n_pb = m->n_pb;
    a.cap = m->cap;
    a.xs = m->d_xs;
    a.xs_hi = m->d_xs_hi;
    a.xs_lo = m->d_xs_lo;
    a.pb_org = m->d_pb_org;
    a.cur = m->d_cur;
    a.sel = m->d_sel;
    a.perm = m->d_perm;
    a.nb_cnt = m->d_nb_cnt;
    a.nb_list = m->d_nb_list;
    a.cx = m->d_cx;
    a.alpha = m->d_alpha;
    a.R = R;
    a.S0 = m->S0;
    a.tau = tau;
    double inv = 1.0 / R;
    a.invR = inv;
    a.invR_hi = (float)inv;
    a.invR_lo = (float)(inv - (double)a.invR_hi);
    a.part = m->d_part;
    a.pb_key = m->d_pb_key;
    a.pb_idx = m->d_pb_idx;
    a.pb_done = m->d_pb_done;
    a.st = m->d_st;
    a.pairs = m->d_pairs;
    a.dim = m->dim;
    a.pb_lo = 0;
    a.pb_n = m->n_pb;
    a.local_only = 0;
    return a;
}

void read_state(rbfd_mesh *m) {
    RBFD_CUDA(cudaMemcpyAsync(m->h_st, m->d_st, sizeof(GreedyState), cudaMemcpyDeviceToHost, m->stream));
    RBFD_CUDA(cudaStreamSynchronize(m->stream));
}

// The state and the grid barrier after a persistent launch, in one round trip.
void read_state_bar(rbfd_mesh *m) {
    RBFD_CUDA(cudaMemcpyAsync(m->h_st, m->d_st, sizeof(GreedyState), cudaMemcpyDeviceToHost, m->stream));
    RBFD_CUDA(cudaMemcpyAsync(m->h_bar, m->d_bar, sizeof(GridBarrier), cudaMemcpyDeviceToHost, m->stream));
    RBFD_CUDA(cudaStreamSynchronize(m->stream));
}

// max_i |v_i|^2 and its argmax (original index, as int bits in out[1]) into
// out on the device, without waiting for it.
void maxnorm_async(rbfd_mesh *m, const double4 *v, double *out) {
    const int nb = std::min<int>(cdiv(m->n_s, 256), 1024);
    k_maxnorm<<<nb, 256, 0, m->stream>>>(v, m->d_perm, m->n_s, m->dim, m->d_pb_key, m->d_pb_idx, &m->d_misc[0], out);
    RBFD_CUDA(cudaGetLastError());
}

// max_i |v_i|^2 and its argmax over the sorted surface (FP64, exact order of
// each squared norm); returns the key, writes the argmax's original index.
// The result goes to slots 6, 7 of the box array; with box given, the box
// in slots 0-5 comes back in the same copy.
double maxnorm(rbfd_mesh *m, const double4 *v, int *arg, double *box = nullptr) {
    const int nb = std::min<int>(cdiv(m->n_s, 256), 1024);
    k_maxnorm<<<nb, 256, 0, m->stream>>>(v, m->d_perm, m->n_s, m->dim, m->d_pb_key, m->d_pb_idx,
                                         &m->d_misc[0], m->d_bbox + 6);
    RBFD_CUDA(cudaGetLastError());
    double h[8];
    RBFD_CUDA(cudaMemcpyAsync(h, m->d_bbox, sizeof(h), cudaMemcpyDeviceToHost, m->stream));
    RBFD_CUDA(cudaStreamSynchronize(m->stream));
    if (arg) std::memcpy(arg, &h[7], sizeof(int));
    if (box) std::memcpy(box, h, 6 * sizeof(double));
    return h[6];
}

// A level's controls and weights as double-float pairs (FP32-input volume sweep).
__global__ void k_level_split(const double4 *__restrict__ cx, const double4 *__restrict__ al, int n,
                              float4 *__restrict__ cdf, float4 *__restrict__ adf) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const double4 c = cx[j], a = al[j];
    const df x = df_from_double(c.x), y = df_from_double(c.y), z = df_from_double(c.z);
    const df ax = df_from_double(a.x), ay = df_from_double(a.y), az = df_from_double(a.z);
    cdf[2 * j] = make_float4(x.hi, y.hi, z.hi, 0.f);
    cdf[2 * j + 1] = make_float4(x.lo, y.lo, z.lo, 0.f);
    adf[2 * j] = make_float4(ax.hi, ax.lo, ay.hi, ay.lo);
    adf[2 * j + 1] = make_float4(az.hi, az.lo, 0.f, 0.f);
}

// The level's control records in the cell order of a grid: for position p
// of cell_ctrl, record p = (coordinates hi, lo, weights hi/lo) of control
// cell_ctrl[p], four float4.
__global__ void k_level_records(int n, const uint32_t *__restrict__ cell_ctrl, const float4 *__restrict__ cdf,
                                const float4 *__restrict__ adf, float4 *__restrict__ rec) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const uint32_t j = cell_ctrl[p];
    rec[4 * (size_t)p + 0] = cdf[2 * (size_t)j];
    rec[4 * (size_t)p + 1] = cdf[2 * (size_t)j + 1];
    rec[4 * (size_t)p + 2] = adf[2 * (size_t)j];
    rec[4 * (size_t)p + 3] = adf[2 * (size_t)j + 1];
}

// Uniform grid of cell size h0 (grown while the cell table would exceed 4M
// cells) over the level's controls, for the volume sweep; bb = the box the
// controls lie in (lo xyz, hi xyz), known on the host.
void grid_over_controls(rbfd_mesh *m, const Level &L, const double *bb, double h0, double3 &g0_out,
                        double &h_out, int3 &gd_out, uint32_t *&start, uint32_t *&ctrl) {
    const int n = (int)L.nc;
    double h = h0;
    auto dims = [&](double hh) {
        int nx = std::max(1, (int)std::floor((bb[3] - bb[0]) / hh) + 1);
        int ny = std::max(1, (int)std::floor((bb[4] - bb[1]) / hh) + 1);
        int nz = m->dim == 3 ? std::max(1, (int)std::floor((bb[5] - bb[2]) / hh) + 1) : 1;
        return make_int3(nx, ny, nz);
    };
    int3 gd = dims(h);
    while ((double)gd.x * gd.y * gd.z > 4.0e6) {  // keep the cell table small
        h *= 2.0;
        gd = dims(h);
    }
    h_out = h;
    g0_out = make_double3(bb[0], bb[1], m->dim == 3 ? bb[2] : 0.0);
    gd_out = gd;
    const int ncell = gd.x * gd.y * gd.z;
    start = dalloc<uint32_t>((size_t)ncell + 1, "control cell starts");
    ctrl = dalloc<uint32_t>((size_t)n, "control cell list");
    if (!m->d_ckeys) m->d_ckeys = dalloc<uint32_t>((size_t)m->cap + 1, "control cell keys");
    uint32_t *keys = m->d_ckeys;
    k_cell_keys<<<cdiv(n, 256), 256, 0, m->stream>>>(L.d_cx, n, g0_out, 1.0 / h, gd, keys, ctrl);
    int bits = 1;
    while ((1u << bits) < (unsigned)ncell && bits < 32) ++bits;
    radix_sort_pairs(keys, ctrl, (size_t)n, bits, m->sort, m->stream);
    k_cell_start<<<cdiv((size_t)ncell + 1, 256), 256, 0, m->stream>>>(keys, n, ncell, start);
    m->stats.launches += 2;
    RBFD_CUDA(cudaGetLastError());
}

void build_control_grid(rbfd_mesh *m, Level &L, const double *bb) {
    grid_over_controls(m, L, bb, L.R, L.g0, L.h, L.gdim, L.d_cell_start, L.d_cell_ctrl);
    L.ncell = L.gdim.x * L.gdim.y * L.gdim.z;
    const int n = (int)L.nc;
    L.d_rec = dalloc<float4>((size_t)4 * std::max(n, 1), "level control records");
    k_level_records<<<cdiv(std::max(n, 1), 256), 256, 0, m->stream>>>(n, L.d_cell_ctrl, L.d_cdf, L.d_adf, L.d_rec);
    RBFD_CUDA(cudaGetLastError());
    m->stats.launches += 1;
}

}  // namespace

// ====================================================================== API

namespace {
// Buffers carved out of one device block: one pool call instead of one per
// buffer (each 256-byte aligned).
struct Carver {
    struct Item {
        void **dst;
        size_t bytes;
    };
    std::vector<Item> items;
    template <typename T>
    void add(T *&p, size_t n) {
        items.push_back({reinterpret_cast<void **>(&p), sizeof(T) * std::max<size_t>(n, 1)});
    }
    size_t total() const {
        size_t t = 0;
        for (const Item &i : items) t += (i.bytes + 255) / 256 * 256;
        return t;
    }
    void assign(char *base) const {
        size_t off = 0;
        for (const Item &i : items) {
            *i.dst = base + off;
            off += (i.bytes + 255) / 256 * 256;
        }
    }
};
}  // namespace

void mesh_prepare(rbfd_mesh *m, const double *xyz_s, const double *dS) {
    const int64_t n = m->n_s;
    cudaStream_t st = m->stream;
    m->n_pb = (int)cdiv(n, kPB);
    int64_t cap = m->opt.nc_cap > 0 ? m->opt.nc_cap : 32768;
    cap = std::min<int64_t>(cap, n);
    m->cap = (int)cap;
    const int n_red = (int)cdiv(cap + 1, kYWarps) + 8;
    const int n_jt = (int)cdiv(cap + 1, kJT);
    m->n_chunk_max = std::max(128, (kTargetCTAs + m->n_pb - 1) / m->n_pb);
    // the mesh's fixed buffers in one block: first the words that start at
    // zero (one memset), then the rest; the two factors G and G^T apart
    Carver zero, rest;
    zero.add(m->d_misc, 16);
    zero.add(m->d_pairs, 16);
    zero.add(m->d_st, 1);
    zero.add(m->d_bar, 1);
    zero.add(m->d_phase_ns, 8);
    zero.add(m->d_lvl, 8);
    zero.add(m->d_pb_done, m->n_pb);
    zero.add(m->d_grp_done, (size_t)m->n_pb * ((m->n_chunk_max + 15) / 16));
    rest.add(m->d_bbox, 8);
    rest.add(m->d_perm, n);
    rest.add(m->d_inv, n);
    rest.add(m->d_xs, n);
    rest.add(m->d_dS, n);
    rest.add(m->d_cur, n);
    rest.add(m->d_E, n);
    rest.add(m->d_pb_lo, m->n_pb);
    rest.add(m->d_pb_hi, m->n_pb);
    rest.add(m->d_pb_org, m->n_pb);
    rest.add(m->d_xs_hi, n);
    rest.add(m->d_xs_lo, n);
    rest.add(m->d_sel, n);
    rest.add(m->d_w, cap + 1);
    rest.add(m->d_alpha, cap + 1);
    rest.add(m->d_cx, cap + 1);
    rest.add(m->d_cdf, 2 * (cap + 1));
    rest.add(m->d_cid, cap + 1);
    rest.add(m->d_phi, cap + 1);
    rest.add(m->d_y, cap + 1);
    rest.add(m->d_red, (size_t)4 * n_red + 6 * 256);
    rest.add(m->d_gpart, (size_t)n_jt * cap + cap);
    rest.add(m->d_vec, cap + 1);
    rest.add(m->d_vec2, cap + 1);
    rest.add(m->d_nb_cnt, m->n_pb);
    rest.add(m->d_nb_list, (size_t)m->n_pb * cap);
    rest.add(m->d_part, (size_t)m->n_chunk_max * n);
    rest.add(m->d_gpart4, (size_t)((m->n_chunk_max + 15) / 16) * n);
    rest.add(m->d_pb_key, std::max(m->n_pb, 1024));
    rest.add(m->d_pb_idx, std::max(m->n_pb, 1024));
    if (m->opt.prune && m->n_pb <= kPfxMax) {
        rest.add(m->d_bnd, (size_t)2 * 4 * m->n_pb);
        rest.add(m->d_bacc, (size_t)2 * 4 * m->n_pb);
        rest.add(m->d_wbox, (size_t)2 * 4 * m->n_pb);
        rest.add(m->d_rev, (size_t)(cap + 1) * m->n_pb);
        rest.add(m->d_rev_cnt, cap + 1);
    }
    rest.add(m->d_pred, (size_t)4 * kMaxPersistCTAs + 8);
    rest.add(m->d_nz_k, cap + 1);
    rest.add(m->d_nz_v, cap + 1);
    rest.add(m->d_lvl_hist, m->n_levels_req);
    rest.add(m->d_Dl, m->n_levels_req);
    rest.add(m->d_invDlf, m->n_levels_req);
    const size_t zbytes = zero.total();
    char *arena = static_cast<char *>(dmalloc(zbytes + rest.total(), "mesh state"));
    m->d_arena = arena;
    zero.assign(arena);
    rest.assign(arena + zbytes);
    RBFD_CUDA(cudaMemsetAsync(arena, 0, zbytes, st));
    m->d_G = dalloc<double>((size_t)cap * cap, "inverse factor");
    m->d_Gt = dalloc<double>((size_t)cap * cap, "inverse factor, transposed");
    m->h_st = static_cast<GreedyState *>(pinned_alloc(sizeof(GreedyState)));
    m->h_bar = static_cast<GridBarrier *>(pinned_alloc(sizeof(GridBarrier)));
    m->h_lvl = static_cast<double *>(pinned_alloc(8 * sizeof(double)));

    // temporaries (one block, back to the pool after the one synchronisation below)
    Carver tmp;
    double *dx = nullptr, *dd = nullptr, *part = nullptr;
    double4 *x4 = nullptr, *d4 = nullptr;
    uint32_t *keys = nullptr;
    if (!m->opt.inputs_on_device) {
        tmp.add(dx, (size_t)n * m->dim);
        tmp.add(dd, (size_t)n * m->dim);
    }
    tmp.add(x4, n);
    tmp.add(d4, n);
    tmp.add(part, 6 * 256);
    tmp.add(keys, n);
    void *temps = dmalloc(tmp.total(), "set-up temporaries");
    tmp.assign(static_cast<char *>(temps));
    // inputs to device (one copy each when they are host buffers)
    const size_t bytes = sizeof(double) * (size_t)n * m->dim;
    if (m->opt.inputs_on_device) {
        dx = const_cast<double *>(xyz_s);
        dd = const_cast<double *>(dS);
    } else {
        RBFD_CUDA(cudaMemcpyAsync(dx, xyz_s, bytes, cudaMemcpyHostToDevice, st));
        RBFD_CUDA(cudaMemcpyAsync(dd, dS, bytes, cudaMemcpyHostToDevice, st));
    }
    k_unpack<<<cdiv(n, 256), 256, 0, st>>>(dx, dd, n, m->dim, x4, d4);
    RBFD_CUDA(cudaGetLastError());
    // bounding box -> Morton keys -> stable sort -> permutation
    const int nbb = std::min<int>(cdiv(n, 256), 256);
    k_bbox_partial<<<nbb, 256, 0, st>>>(x4, n, part);
    k_bbox_final<<<1, 192, 0, st>>>(part, nbb, m->d_bbox);
    // (cubic cells: the wing's surface box is 3.5 x 0.12 x 3 chords, and
    // per-axis cells made the 128-point blocks' boxes 1.6x as wide)
    morton_keys_f64_dev(x4, n, m->dim, m->d_bbox, keys, m->d_perm, st, 0, true);
    radix_sort_pairs(keys, m->d_perm, n, m->dim == 2 ? 32 : 30, m->sort, st);
    k_gather_sorted<<<cdiv(n, 256), 256, 0, st>>>(m->d_perm, n, x4, d4, m->d_xs, m->d_dS, m->d_inv);
    RBFD_CUDA(cudaGetLastError());
    // point blocks
    k_point_blocks<<<m->n_pb, kPB, 0, st>>>(m->d_xs, n, m->d_pb_lo, m->d_pb_hi, m->d_pb_org, m->d_xs_hi, m->d_xs_lo,
                                            m->d_wbox);
    RBFD_CUDA(cudaGetLastError());

    m->stats.launches += 6;  // unpack, bbox x2, morton, gather, point blocks
    // S0 = max_i |dS_i| and the surface box reach the host with the first
    // call that needs them (mesh_ready): the set-up does not wait here
    const int nbm = std::min<int>(cdiv(m->n_s, 256), 1024);
    k_maxnorm<<<nbm, 256, 0, st>>>(m->d_dS, m->d_perm, m->n_s, m->dim, m->d_pb_key, m->d_pb_idx, &m->d_misc[0],
                                   m->d_bbox + 6);
    RBFD_CUDA(cudaGetLastError());
    m->stats.launches += 1;
    m->h_prep = static_cast<double *>(pinned_alloc(8 * sizeof(double)));
    RBFD_CUDA(cudaMemcpyAsync(m->h_prep, m->d_bbox, 8 * sizeof(double), cudaMemcpyDeviceToHost, st));
    RBFD_CUDA(cudaEventRecord(m->ev1, st));
    m->prep_temps = temps;  // (back to the pool once the set-up has run)
    m->prep_pending = true;
}

void mesh_ready(rbfd_mesh *m) {
    if (!m->prep_pending) return;
    RBFD_CUDA(cudaEventSynchronize(m->ev1));
    m->S0 = std::sqrt(m->h_prep[6]);
    std::memcpy(m->h_sbox, m->h_prep, 6 * sizeof(double));
    dfree(m->prep_temps);
    m->prep_temps = nullptr;
    m->prep_pending = false;
}

namespace {
__global__ void k_gather_disp(const double *__restrict__ dS, const uint32_t *__restrict__ perm, int64_t n, int dim,
                              double4 *__restrict__ out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double *q = dS + (int64_t)perm[i] * dim;
    out[i] = make_double4(q[0], q[1], dim == 3 ? q[2] : 0.0, 0.0);
}
}  // namespace

// New surface displacement on a prepared mesh: the Morton order, point blocks
// and workspace are kept; the greedy results of the previous displacement are
// dropped.
void mesh_set_displacement(rbfd_mesh *m, const double *dS) {
    mesh_ready(m);
    greedy_finish(m);
    cudaStream_t st = m->stream;
    const int64_t n = m->n_s;
    const double *dd = dS;
    double *tmp = nullptr;
    if (!m->opt.inputs_on_device) {
        tmp = dalloc<double>((size_t)n * m->dim, "surface displacements");
        RBFD_CUDA(cudaMemcpyAsync(tmp, dS, sizeof(double) * n * m->dim, cudaMemcpyHostToDevice, st));
        dd = tmp;
    }
    k_gather_disp<<<cdiv(n, 256), 256, 0, st>>>(dd, m->d_perm, n, m->dim, m->d_dS);
    RBFD_CUDA(cudaGetLastError());
    m->stats.launches += 1;
    m->S0 = std::sqrt(maxnorm(m, m->d_dS, nullptr));  // synchronises the stream
    m->stats.launches += 1;
    dfree(tmp);
    for (auto &L : m->warm_prev) level_free(L);
    m->warm_prev.clear();
    if (m->keep_factors) {
        m->warm_prev.swap(m->levels);  // (a warm greedy starts from them)
    } else {
        for (auto &L : m->levels) level_free(L);
        m->levels.clear();
    }
    m->greedy_done = false;
}

// RBFD_NEWTON=0 in the environment turns the Newton-basis start of a level off.
static bool newton_enabled() {
    const char *v = std::getenv("RBFD_NEWTON");
    return !(v && v[0] == '0');
}

void level_fine_grid(rbfd_mesh *m, Level &L) {
    if (L.f_cell_start || L.nc == 0) return;
    grid_over_controls(m, L, m->h_sbox, 0.5 * L.R, L.f_g0, L.f_h, L.f_gdim, L.f_cell_start, L.f_cell_ctrl);
    const int n = (int)L.nc;
    L.f_rec = dalloc<float4>((size_t)4 * n, "level control records (fine grid)");
    k_level_records<<<cdiv(n, 256), 256, 0, m->stream>>>(n, L.f_cell_ctrl, L.d_cdf, L.d_adf, L.f_rec);
    RBFD_CUDA(cudaGetLastError());
    m->stats.launches += 1;
}

void level_free(Level &L) {
    dfree(L.d_cx);
    dfree(L.d_alpha);
    dfree(L.d_cdf);
    dfree(L.d_adf);
    dfree(L.d_orig);
    dfree(L.d_cell_start);
    dfree(L.d_cell_ctrl);
    dfree(L.f_cell_start);
    dfree(L.f_cell_ctrl);
    L.f_cell_start = L.f_cell_ctrl = nullptr;
    dfree(L.d_rec);
    dfree(L.f_rec);
    L.d_rec = L.f_rec = nullptr;
    dfree(L.d_Gs);
    dfree(L.d_Gts);
    dfree(L.d_cids);
    L.d_Gs = L.d_Gts = nullptr;
    L.d_cids = nullptr;
    pinned_free(L.h_scal);
    L.d_cx = L.d_alpha = nullptr;
    L.d_cdf = L.d_adf = nullptr;
    L.d_orig = L.d_cell_start = L.d_cell_ctrl = nullptr;
    L.h_scal = nullptr;
}

void level_fetch(rbfd_mesh *m, Level &L) {
    if (L.fetched) return;
    const int64_t n = L.nc;
    std::vector<uint32_t> orig((size_t)n);
    std::vector<double4> al((size_t)n);
    if (n > 0) {
        RBFD_CUDA(cudaMemcpyAsync(orig.data(), L.d_orig, sizeof(uint32_t) * n, cudaMemcpyDeviceToHost, m->stream));
        RBFD_CUDA(cudaMemcpyAsync(al.data(), L.d_alpha, sizeof(double4) * n, cudaMemcpyDeviceToHost, m->stream));
        RBFD_CUDA(cudaStreamSynchronize(m->stream));
    }
    L.idx.resize((size_t)n);
    L.alpha.resize((size_t)n * m->dim);
    for (int64_t j = 0; j < n; ++j) {
        L.idx[j] = orig[j];
        L.alpha[(size_t)j * m->dim + 0] = al[j].x;
        L.alpha[(size_t)j * m->dim + 1] = al[j].y;
        if (m->dim == 3) L.alpha[(size_t)j * m->dim + 2] = al[j].z;
    }
    L.fetched = true;
}

void greedy_finish(rbfd_mesh *m) {
    if (!m->greedy_pending) return;
    m->greedy_pending = false;
    RBFD_CUDA(cudaEventSynchronize(m->ev_g1));
    for (auto &L : m->levels) {
        L.smax = std::sqrt(L.h_scal[0]);
        m->stats.refine_sweeps += (int64_t)L.h_scal[3];
    }
    float ms = 0;
    RBFD_CUDA(cudaEventElapsedTime(&ms, m->ev_g0, m->ev_g1));
    m->stats.greedy_ms = ms;
    m->prof.flush();
}

void greedy_run(rbfd_mesh *m, bool wait, bool warm) {
    mesh_ready(m);
    greedy_finish(m);  // (a previous run's)
    cudaStream_t st = m->stream;
    // the previous run's levels: their factors start a warm run's levels;
    // they are returned to the pools once this run's work is queued
    std::vector<Level> prev;
    prev.swap(m->levels);
    if (prev.empty()) prev.swap(m->warm_prev);
    for (auto &L : m->warm_prev) level_free(L);
    m->warm_prev.clear();
    struct FreePrev {
        std::vector<Level> &p;
        cudaStream_t s;
        ~FreePrev() {
            if (!p.empty()) cudaStreamSynchronize(s);
            for (auto &L : p) level_free(L);
        }
    } free_prev{prev, st};
    warm = warm && m->split_world == 1 && (int)prev.size() == m->n_levels_req;
    for (size_t l = 0; warm && l < prev.size(); ++l)
        warm = prev[l].d_Gs != nullptr && prev[l].R == m->R[l] && prev[l].nc >= 1;
    m->greedy_done = false;
    m->stats.greedy_steps = 0;
    // host wall time by part of the level (rbfd_stats.greedy_host_ms)
    for (double &v : m->stats.greedy_host_ms) v = 0.0;
    auto t_host = std::chrono::steady_clock::now();
    auto host_mark = [&](int part) {
        const auto t = std::chrono::steady_clock::now();
        m->stats.greedy_host_ms[part] += std::chrono::duration<double, std::milli>(t - t_host).count();
        t_host = t;
    };
    m->stats.newton_steps = 0;
    m->stats.persist_grow_fma = 0;
    m->stats.refine_sweeps = 0;
    m->stats.confirm_resumes = 0;
    RBFD_CUDA(cudaEventRecord(m->ev_g0, st));
    if (m->S0 == 0.0) {  // nothing moves: zero levels
        RBFD_CUDA(cudaEventRecord(m->ev_g1, st));
        RBFD_CUDA(cudaEventSynchronize(m->ev_g1));
        m->stats.greedy_ms = 0;
        m->greedy_done = true;
        return;
    }
    RBFD_CUDA(cudaMemcpyAsync(m->d_cur, m->d_dS, sizeof(double4) * m->n_s, cudaMemcpyDeviceToDevice, st));
    const int Lreq = m->n_levels_req;
    const double eps_rel = m->opt.eps_absolute ? m->eps / m->S0 : m->eps;
    const int mode = m->opt.precision == RBFD_FP64 ? 0 : 1;
    int final_status = RBFD_OK;
    for (int l = 0; l < Lreq; ++l) {
        host_mark(3);  // (the set-up before the first level counts with the saves)
        char level_name[48];
        std::snprintf(level_name, sizeof(level_name), "rbfd greedy level %d%s", l, warm ? " (warm)" : "");
        NvtxRange nvtx_level(level_name);
        Level L;
        L.R = m->R[l];
        L.tau = std::pow(eps_rel, (double)(l + 1) / (double)Lreq);
        // max |dS_l| (read with the level's results; the first-point rule reads it on the device)
        RBFD_CUDA(cudaMemsetAsync(m->d_lvl, 0, 8 * sizeof(double), st));
        maxnorm_async(m, m->d_cur, m->d_lvl);
        const double R2 = L.R * L.R;
        RBFD_CUDA(cudaMemsetAsync(m->d_sel, 0, m->n_s, st));
        // a warm level restarts from the previous run's controls of this level
        const int n_warm = warm ? (int)std::min<int64_t>(prev[l].nc, m->cap) : 0;
        if (n_warm > 0) {
            const Level &P = prev[l];
            const size_t pitch = sizeof(double) * (size_t)m->cap, row = sizeof(double) * (size_t)n_warm;
            RBFD_CUDA(cudaMemcpy2DAsync(m->d_G, pitch, P.d_Gs, sizeof(double) * (size_t)P.nc, row, n_warm,
                                        cudaMemcpyDeviceToDevice, st));
            RBFD_CUDA(cudaMemcpy2DAsync(m->d_Gt, pitch, P.d_Gts, sizeof(double) * (size_t)P.nc, row, n_warm,
                                        cudaMemcpyDeviceToDevice, st));
            k_warm_restore<<<cdiv(n_warm, 256), 256, 0, st>>>(n_warm, m->cap, P.d_cids, m->d_xs, m->d_sel, m->d_cx,
                                                            m->d_cdf, m->d_cid, m->d_alpha, m->d_st);
            k_warm_lists<<<cdiv(std::max(m->n_pb, 1), kThreads), kThreads, 0, st>>>(
                n_warm, m->n_pb, m->cap, m->dim, R2, m->d_cx, m->d_pb_lo, m->d_pb_hi, m->d_nb_cnt, m->d_nb_list);
            // Eq. 9 for the current target on the kept factor: w = G dS_l(C),
            // alpha = G^T w (the level close refines it)
            const unsigned nb8 = (unsigned)std::min<int64_t>(cdiv(n_warm, 8), 4 * 152);
            RBFD_CUDA(cudaMemsetAsync(m->d_lvl + 2, 0, sizeof(double), st));
            k_gather_ctrl<<<cdiv(n_warm, 256), 256, 0, st>>>(n_warm, m->d_cid, m->d_cur, m->d_vec);
            k_lower_mv3<<<nb8, 256, 0, st>>>(n_warm, nullptr, m->cap, m->d_G, m->d_vec, m->d_w, m->d_lvl + 2);
            k_upper_mv3_add<<<nb8, 256, 0, st>>>(n_warm, nullptr, m->cap, m->d_Gt, m->d_w, m->d_alpha,
                                                 m->d_lvl + 2);
            RBFD_CUDA(cudaGetLastError());
            m->stats.launches += 7;
        } else {
            k_level_init<<<cdiv(std::max(m->n_pb, 1), kThreads), kThreads, 0, st>>>(
                m->opt.first_point == 1 ? 1 : 0, 0, m->d_inv, m->d_xs, m->d_cur, m->n_pb, m->cap, m->dim, R2,
                m->d_pb_lo, m->d_pb_hi, m->d_sel, m->d_cx, m->d_cdf, m->d_cid, m->d_G, m->d_Gt, m->d_w, m->d_alpha,
                m->d_nb_cnt, m->d_nb_list, m->d_lvl, m->d_st);
            RBFD_CUDA(cudaGetLastError());
            m->stats.launches += 2;  // maxnorm + level init
        }

        GrowArgs g{};
        g.cap = m->cap;
        g.n_pb = m->n_pb;
        g.dim = m->dim;
        g.R = L.R;
        g.R2 = R2;
        g.inv = m->d_inv;
        g.xs = m->d_xs;
        g.pb_lo = m->d_pb_lo;
        g.pb_hi = m->d_pb_hi;
        g.sel = m->d_sel;
        g.cx = m->d_cx;
        g.cid = m->d_cid;
        g.phi = m->d_phi;
        g.nb_cnt = m->d_nb_cnt;
        g.nb_list = m->d_nb_list;
        g.G = m->d_G;
        g.Gw = m->d_G;
        g.Gt = m->d_Gt;
        g.y = m->d_y;
        g.red = m->d_red;
        g.gpart = m->d_gpart;
        g.w = m->d_w;
        g.alpha = m->d_alpha;
        g.cur = m->d_cur;
        g.st = m->d_st;

        int n = n_warm > 0 ? n_warm : 1;
        int resumes = 0;
        // a warm level's first pass only closes the restored control set
        // (refinement and confirm sweep); if that misses tau the greedy
        // continues from it like a resumed level
        bool warm_close = n_warm > 0;
        // ---- level close: FP64 iterative refinement of alpha, alpha +=
        // G^T G (dS_l - Phi_cc alpha) at the controls, then the FP64 confirm
        // sweep E = dS_l - Phi_sc alpha.  The convergence test of the
        // refinement runs on the device (in k_resid), so the sweeps after
        // convergence are launched but do nothing.  With from_state the
        // kernels read n from the greedy state (a close queued behind the
        // greedy launch before the host has read it, n_max bounding it) and
        // do nothing if that launch handed the level on.
        auto enqueue_close = [&](int n_max, bool from_state) {
            NvtxRange nvtx_close("rbfd level close");
            const GreedyState *nfrom = from_state ? m->d_st : nullptr;
            RBFD_CUDA(cudaMemsetAsync(m->d_lvl + 2, 0, sizeof(double), st));
            RBFD_CUDA(cudaMemsetAsync(&m->d_misc[8], 0, sizeof(uint32_t), st));  // k_resid's block counter
            // one warp per control (strided over a grid of at most 4 blocks per SM)
            const unsigned nb = (unsigned)std::min<int64_t>(cdiv(n_max, kThreads / 32), 4 * 152);
            const unsigned nb8 = (unsigned)std::min<int64_t>(cdiv(n_max, 8), 4 * 152);
            for (int it = 0; it < std::max(0, m->opt.refine_iters); ++it) {
                if (m->dim == 2) launch_resid_d<2>(m->opt.basis, nb, n_max, nfrom, L.R, m, st);
                else launch_resid_d<3>(m->opt.basis, nb, n_max, nfrom, L.R, m, st);
                k_lower_mv3<<<nb8, 256, 0, st>>>(n_max, nfrom, m->cap, m->d_G, m->d_vec, m->d_vec2, m->d_lvl + 2);
                k_upper_mv3_add<<<nb8, 256, 0, st>>>(n_max, nfrom, m->cap, m->d_Gt, m->d_vec2, m->d_alpha,
                                                     m->d_lvl + 2);
                RBFD_CUDA(cudaGetLastError());
                m->stats.launches += 3;
            }
            // Each confirm pair costs about 40 FP64 instructions, which issue
            // at one warp instruction per 64 cycles per SM sub-partition: the
            // lists are cut into chunks of 8 controls or more, so that the
            // blocks cover the SMs several times over
            SweepArgs a = base_sweep_args(m, L.R, L.tau);
            a.n = n_max;
            a.n_from = nfrom;
            a.chunk_cap = std::max(1, std::min((4 * kTargetCTAs + m->n_pb - 1) / m->n_pb, m->n_chunk_max));
            const int nch = std::max(1, std::min((n_max + 7) / 8, a.chunk_cap));
            a.chunk_len = 0;  // (from n in the kernel)
            a.is_step = 0;
            a.E_out = m->d_E;
            launch_sweep(m->dim, m->opt.basis, 0, dim3(m->n_pb, nch), a, st);
            RBFD_CUDA(cudaGetLastError());
            m->stats.launches += 1;
        };
        host_mark(0);
        for (;;) {
            bool closed = false;
            // ---- greedy steps: one persistent cooperative launch (engine 0) ...
            bool stopped = warm_close;
            // a level starts in the Newton basis (engine 0) while that pays; the
            // list sweep below takes over where it hands the level on
            const bool split = m->split_world > 1;
            if (m->opt.engine == 0 && resumes == 0 && newton_enabled() && !split && !stopped) {
                newton_reserve(m);
                // one block per 32 surface points, as far as they fit (newton_shape)
                int ctas = m->opt.grid_ctas > 0 ? m->opt.grid_ctas : kMaxPersistCTAs;
                if (m->batch_ctas_cap > 0) ctas = std::min(ctas, m->batch_ctas_cap);
                ctas = std::max(1, ctas);
                if (m->newton_cols >= 2 && newton_fits(m, ctas)) {
                    RBFD_CUDA(cudaMemsetAsync(&m->d_st->handoff, 0, sizeof(int), st));
                    RBFD_CUDA(cudaMemsetAsync(&m->d_st->nnz_tot, 0, sizeof(unsigned long long), st));
                    RBFD_CUDA(cudaMemsetAsync(m->d_bar, 0, sizeof(GridBarrier), st));
                    NvtxRange nvtx_newton("rbfd Newton-basis launch");
                    cudaEvent_t e0 = m->prof.begin(st);
                    newton_run_level(m, L.R, L.tau, ctas);
                    m->prof.end(kProfNewton, e0, st, 1);
                    enqueue_close(std::min(m->newton_cols, m->cap), true);
                    volume_stage_enqueue(m);  // (a staged volume: while this level runs)
                    read_state_bar(m);
                    m->prof.flush();
                    if (m->h_bar->err) fail(RBFD_ETIMEOUT, "Newton greedy: a grid barrier exceeded its wait bound");
                    if (m->h_st->status == RBFD_ESINGULAR)
                        fail(RBFD_ESINGULAR, "Phi_cc is not positive definite at level " + std::to_string(l) +
                                                 " (coincident or near-coincident controls)");
                    if (!m->h_st->stop) fail(RBFD_ECUDA, "Newton greedy ended without a stop decision");
                    n = m->h_st->n;
                    m->stats.newton_steps += n - 1;
                    if (m->h_st->handoff) {
                        RBFD_CUDA(cudaMemsetAsync(&m->d_st->stop, 0, sizeof(int), st));
                        RBFD_CUDA(cudaMemsetAsync(&m->d_st->handoff, 0, sizeof(int), st));
                    } else {
                        stopped = true;
                        closed = true;  // (the state read above follows the close)
                    }
                }
            }
            for (bool yielded = true; yielded && !stopped && !split && (m->opt.engine == 0 || m->opt.engine == 2);) {
                const int maxc = std::min(persist_max_ctas(m), kMaxPersistCTAs);
                if (maxc < 1) fail(RBFD_ECUDA, "persistent greedy kernel cannot be resident on this device");
                // small meshes: few blocks keep the barriers cheap; large ones fill the GPU
                int ctas = m->opt.grid_ctas > 0 ? m->opt.grid_ctas
                                                : (m->n_pb <= 128 ? std::min(std::max(64, 4 * m->n_pb), 2 * 152)
                                                                  : std::min(4 * m->n_pb, 8 * 152));
                // a batch's meshes share the blocks; once some have finished,
                // the others' next launches take the freed share (their
                // launches then yield every kYieldSteps steps to pick it up)
                int max_steps = 0;
                if (m->batch_active) {
                    const int act = std::max(1, m->batch_active->load());
                    ctas = std::min(ctas, std::max(1, m->batch_total / act));
                    if (act > 1) max_steps = kYieldSteps;
                    // (test hook: a shorter step limit, to exercise the relaunches)
                    if (const char *v = std::getenv("RBFD_TEST_YIELD_STEPS"); v && act > 1)
                        max_steps = std::max(1, std::atoi(v));
                } else if (m->batch_ctas_cap > 0) {
                    ctas = std::min(ctas, m->batch_ctas_cap);
                }
                ctas = std::max(1, std::min(ctas, maxc));
                RBFD_CUDA(cudaMemsetAsync(m->d_bar, 0, sizeof(GridBarrier), st));
                NvtxRange nvtx_persist("rbfd persistent list sweep");
                cudaEvent_t e0 = m->prof.begin(st);
                persist_run_level(m, L.R, L.tau, ctas, max_steps);
                m->prof.end(kProfPersist, e0, st, 1);
                volume_stage_enqueue(m);  // (a staged volume: while this level runs)
                m->stats.persist_ctas = ctas;
                read_state_bar(m);
                m->prof.flush();
                if (m->h_bar->err) fail(RBFD_ETIMEOUT, "persistent greedy: a grid barrier exceeded its wait bound");
                if (m->h_st->status == RBFD_ESINGULAR)
                    fail(RBFD_ESINGULAR, "Phi_cc is not positive definite at level " + std::to_string(l) +
                                             " (coincident or near-coincident controls)");
                if (!m->h_st->stop) fail(RBFD_ECUDA, "persistent greedy ended without a stop decision");
                {
                    // the launch's FP64 multiply-adds for the rows of G: a step
                    // that adds control k forms k (k + 1) / 2 of them
                    auto tri = [](int64_t q) { return q > 0 ? (q - 1) * q * (q + 1) / 6 : 0; };
                    m->stats.persist_grow_fma += tri(m->h_st->n) - tri(n);
                }
                n = m->h_st->n;
                yielded = m->h_st->handoff != 0;  // (stopped at the step limit: relaunch)
                if (yielded) {
                    RBFD_CUDA(cudaMemsetAsync(&m->d_st->stop, 0, sizeof(int), st));
                    RBFD_CUDA(cudaMemsetAsync(&m->d_st->handoff, 0, sizeof(int), st));
                } else {
                    stopped = true;
                }
            }
            // ... or separate launches per step, in batches (engine 1).  In
            // the surface split every step sweeps this rank's range of point
            // blocks, waits for the range's argmax, combines it with the other
            // ranks' through the caller's all-reduce-maxloc and takes the
            // step's decision from the combined argmax: one step per batch
            const int kBatch = split ? 1 : 16;
            const int pb_lo = split ? (int)((int64_t)m->n_pb * m->split_rank / m->split_world) : 0;
            const int pb_hi = split ? (int)((int64_t)m->n_pb * (m->split_rank + 1) / m->split_world) : m->n_pb;
            while (!stopped) {
                for (int s = 0; s < kBatch; ++s) {
                    NvtxRange nvtx_step("rbfd greedy step");
                    SweepArgs a = base_sweep_args(m, L.R, L.tau);
                    a.n = n;
                    int nch = n_chunks_for(m, n);
                    a.chunk_len = (n + nch - 1) / nch;
                    a.is_step = 1;
                    a.E_out = nullptr;
                    cudaEvent_t e0 = m->prof.begin(st);
                    if (split) {
                        a.pb_lo = pb_lo;
                        a.pb_n = pb_hi - pb_lo;
                        a.local_only = 1;
                        double key = -1.0;
                        int64_t orig = -1;
                        if (a.pb_n > 0) {  // (a rank may own no block of a tiny surface)
                            launch_sweep(m->dim, m->opt.basis, mode, dim3(a.pb_n, nch), a, st);
                            m->stats.launches += 1;
                            read_state(m);
                            key = m->h_st->best_key;
                            orig = m->h_st->best_orig;
                        }
                        if (m->split_maxloc(m->split_user, &key, &orig) != 0)
                            fail(RBFD_ECOMM, "rbfd_greedy_split: the all-reduce-maxloc callback failed");
                        if (orig < -1 || orig >= m->n_s)
                            fail(RBFD_ECOMM, "rbfd_greedy_split: the all-reduce-maxloc returned index " +
                                                 std::to_string(orig));
                        k_split_decide<<<1, 1, 0, st>>>(m->d_st, key, (int)orig, m->S0, L.tau, n, m->cap);
                        m->stats.launches += 1;
                    } else {
                        launch_sweep(m->dim, m->opt.basis, mode, dim3(m->n_pb, nch), a, st);
                        m->stats.launches += 1;
                    }
                    m->prof.end(kProfSweep, e0, st, 1);
                    if (n >= m->cap) break;  // the sweep above stops the level
                    cudaEvent_t e1 = m->prof.begin(st);
                    g.n = n;
                    const unsigned gp = cdiv(std::max(n, m->n_pb), kThreads);
                    if (m->dim == 2) launch_phi_d<2>(m->opt.basis, gp, g, st);
                    else launch_phi_d<3>(m->opt.basis, gp, g, st);
                    const int nyb = (int)cdiv(n, kYWarps);
                    g.n_red = nyb;
                    k_grow_y<<<nyb, kYWarps * 32, 0, st>>>(g);
                    const int n_jt = (int)cdiv(n, kJT);
                    k_colsum<<<dim3(cdiv(n, kThreads), n_jt), kThreads, 0, st>>>(n, m->cap, m->d_G, m->d_y,
                                                                                 m->d_gpart, m->d_st);
                    k_grow_finish<<<cdiv(n + 1, kThreads), kThreads, 0, st>>>(g, n_jt);
                    RBFD_CUDA(cudaGetLastError());
                    m->prof.end(kProfGrow, e1, st, 4);
                    m->stats.launches += 4;
                    ++n;
                }
                read_state(m);
                m->prof.flush();
                stopped = m->h_st->stop != 0 || n >= m->cap;
                if (m->h_st->status == RBFD_ESINGULAR)
                    fail(RBFD_ESINGULAR, "Phi_cc is not positive definite at level " + std::to_string(l) +
                                             " (coincident or near-coincident controls)");
            }
            if (!warm_close) n = m->h_st->n;
            host_mark(1);
            if (!closed) {
                enqueue_close(n, false);
                read_state(m);
            }
            host_mark(2);
            const double emax = m->h_st->emax;
            // a level stops early only if its confirmed error is below tau
            if (emax < L.tau || n >= m->cap || resumes >= 4 || n >= m->n_s) {
                L.emax = emax;
                L.status = (emax < L.tau) ? RBFD_OK : RBFD_ENOTCONV;
                break;
            }
            // the mixed-precision selection stopped a little early, or a warm
            // level's restored controls do not reach tau for this target: resume
            if (!warm_close) {
                ++resumes;
                m->stats.confirm_resumes++;
            }
            warm_close = false;
            RBFD_CUDA(cudaMemsetAsync(&m->d_st->stop, 0, sizeof(int), st));
        }
        L.nc = n;
        m->stats.greedy_steps += n - std::max(1, n_warm);
        // save the level
        L.d_cx = dalloc<double4>(n, "level controls");
        L.d_alpha = dalloc<double4>(n, "level weights");
        RBFD_CUDA(cudaMemcpyAsync(L.d_cx, m->d_cx, sizeof(double4) * n, cudaMemcpyDeviceToDevice, st));
        RBFD_CUDA(cudaMemcpyAsync(L.d_alpha, m->d_alpha, sizeof(double4) * n, cudaMemcpyDeviceToDevice, st));
        L.d_cdf = dalloc<float4>((size_t)2 * n, "level controls (double-float)");
        L.d_adf = dalloc<float4>((size_t)2 * n, "level weights (double-float)");
        k_level_split<<<cdiv(n, 256), 256, 0, st>>>(m->d_cx, m->d_alpha, n, L.d_cdf, L.d_adf);
        L.d_orig = dalloc<uint32_t>(n, "level control indices");
        k_orig_of_controls<<<cdiv(n, 256), 256, 0, st>>>(m->d_perm, m->d_cid, n, L.d_orig);
        m->stats.launches += 2;
        if (m->keep_factors) {  // the factor for a warm start of the next time step
            const size_t pitch = sizeof(double) * (size_t)m->cap, row = sizeof(double) * (size_t)n;
            L.d_Gs = dalloc<double>((size_t)n * n, "kept inverse factor");
            L.d_Gts = dalloc<double>((size_t)n * n, "kept inverse factor (transposed)");
            L.d_cids = dalloc<uint32_t>(n, "kept control positions");
            RBFD_CUDA(cudaMemcpy2DAsync(L.d_Gs, row, m->d_G, pitch, row, n, cudaMemcpyDeviceToDevice, st));
            RBFD_CUDA(cudaMemcpy2DAsync(L.d_Gts, row, m->d_Gt, pitch, row, n, cudaMemcpyDeviceToDevice, st));
            RBFD_CUDA(cudaMemcpyAsync(L.d_cids, m->d_cid, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, st));
        }
        // the level's scalars reach the host with the final wait of the
        // greedy; indices and weights are copied only when asked for
        L.h_scal = static_cast<double *>(pinned_alloc(4 * sizeof(double)));
        RBFD_CUDA(cudaMemcpyAsync(L.h_scal, m->d_lvl, 4 * sizeof(double), cudaMemcpyDeviceToHost, st));
        RBFD_CUDA(cudaMemcpyAsync(m->d_lvl_hist + l, m->d_lvl, sizeof(double), cudaMemcpyDeviceToDevice, st));
        build_control_grid(m, L, m->h_sbox);
        if (L.status != RBFD_OK) final_status = RBFD_ENOTCONV;
        m->levels.push_back(std::move(L));
        volume_level_early(m, l);  // (a staged volume's sweep of this level, if it can start now)
        // multi-level subspace: the next level interpolates this level's error
        RBFD_CUDA(cudaMemcpyAsync(m->d_cur, m->d_E, sizeof(double4) * m->n_s, cudaMemcpyDeviceToDevice, st));
    }
    RBFD_CUDA(cudaEventRecord(m->ev_g1, st));
    m->greedy_pending = true;
    m->greedy_done = true;
    if (wait) greedy_finish(m);
    host_mark(3);
    if (!m->levels.empty() && !(m->levels.back().emax < eps_rel)) final_status = RBFD_ENOTCONV;
    if (final_status != RBFD_OK) fail(final_status, "greedy selection did not reach eps before the control cap");
}

}  // namespace rbfd
