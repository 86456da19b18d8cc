// newton.cu -- the greedy selection of one level (Section 3) in the Newton
// basis of the selected controls, as one cooperative launch with one grid
// barrier per greedy step.
//
// With Phi_cc = L L^T and G = L^{-1} (the inverse factor the growth keeps),
// the functions v_k(x) = sum_m G_km phi(|x - r_cm| / R) form the Newton basis
// of the interpolation space, and the interpolant of the level target dS_l on
// n controls is sum_{k<n} w_k v_k with w = G dS_l(c).  Adding control c_j
// changes the error of Eq. 12 by one term:
//
//     E <- E - w_j v_j,     v_j(x) = (phi(|x - r_cj| / R) - sum_{k<j} y_k v_k(x)) / l_j,
//     y_k = v_k(r_cj),      l_j^2 = 1 - sum_{k<j} y_k^2,   w_j = E(r_cj) / l_j
//
// (phi(0) = 1 for every Wendland function; E(r_cj) here is the error before
// c_j joins, so w_j = (dS_l(c_j) - y.w) / l_j).  A step thus needs the values
// v_k(x_i) of the earlier basis functions at the surface points, kept as
// V[k][i], one FP64 dot product of length j per point and ONE evaluation of
// phi per point, instead of a sweep over every control within R of every
// point.  It pays while the supports overlap most of the controls (large R
// relative to the surface, early in a level); the host hands the level to the
// list sweep (persist.cu) once the lists get much shorter than the control
// count or V is full.  In mixed precision the per-point work (dot product,
// phi, E, s2) runs in double-float on the FP32 pipe and the inverse-factor
// rows in FP64; in FP64 mode everything is FP64.
//
// Each block owns fixed groups of 32 surface points and keeps their state in
// shared memory across steps: the first cs columns of V, E, coordinates, the
// running sum s2 = sum_k v_k(x)^2 and the selected flags.  Every candidate
// point therefore knows l^2 = 1 - s2 and w = E / l of its own, and a block
// publishes a 16-byte head (key, index, longest list), a record of its best
// candidate (position, coordinates, l^2, E) and that candidate's column
// y = V[.][candidate].  Per pass, for the control c_j decided in the previous
// pass (y = the winner's published column, loaded during that decision):
//   c_j appended to the control lists of the point blocks within R;
//   (a) v_j at the block's points: warp 0 evaluates phi while seven warps
//       compute the dot product in slices; then V[j][i], E_i -= w_j v_j(x_i),
//       s2_i += v_j^2 and the block's argmax of |E_i|^2 over the unselected
//       points -> its head, record and column;
//   -- the last warp arrives at the grid barrier and polls it, while --
//   (b) the other seven grow the inverse factor for c_j on the rows this
//       block owns (row j of G, column j of G^T: g_k = -(sum_m G_mk y_m) / l_j,
//       alpha_k += w_j g_k): no other block reads them during the launch;
//   -- the barrier has passed --
//   every block reads the P heads and takes the same decision: global
//   argmax, stop test |E|max / S0 < tau_l in FP64 (on the keys outside a
//   narrow bracket), pivot test, the next control; block 0 records it.  One
//   warp fetches the winner's record and computes the step's scalars while
//   the others load the winner's column.
#include <algorithm>
#include <cfloat>
#include <climits>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>

#include "internal.h"

namespace rbfd {

namespace {

constexpr int kNT = 256;  // threads per block (8 warps)
constexpr int kNW = kNT / 32;
constexpr int kRound = 2;     // point groups per round of (a)
constexpr int kDotW = kNW - 1;  // warps computing the dot of (a) (warp 0 evaluates phi)
constexpr int kRowChunk = 8;  // entries per lane of a row of (b) loaded together

// Keys of the argmax as unsigned 64-bit integers in the order of the values:
// FP64 mode, the bit pattern of the non-negative double plus one; mixed mode,
// the high float's bits above an order-preserving image of the low float.
// 0 means "no candidate".  Comparisons then run on the integer pipes.
__device__ __forceinline__ unsigned long long key_of_double(double k) {
    return (unsigned long long)__double_as_longlong(k) + 1ull;
}
__device__ __forceinline__ unsigned float_order(float x) {
    const unsigned u = __float_as_uint(x);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float float_unorder(unsigned u) {
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}
__device__ __forceinline__ unsigned long long key_of_df(df k) {  // k.hi >= 0
    return ((unsigned long long)__float_as_uint(k.hi) << 32) | float_order(k.lo);
}
template <int MODE>
__device__ __forceinline__ double key_value(unsigned long long k) {
    if (MODE == 0) return __longlong_as_double((long long)(k - 1ull));
    return (double)__uint_as_float((unsigned)(k >> 32)) + (double)float_unorder((unsigned)k);
}

__device__ __forceinline__ bool better_key(unsigned long long ka, int ia, unsigned long long kb, int ib) {
    return (ka > kb) || (ka == kb && ia < ib && ia >= 0) || (ib < 0 && ia >= 0);
}

// acc += y * v in double-float (TwoProduct by FMA, TwoSum on the high
// parts, low parts summed plainly; renormalised once at the end).
__device__ __forceinline__ void df_fma_acc(float &ah, float &al, float yh, float yl, float vh, float vl) {
    const float p = __fmul_rn(yh, vh);
    float pe = __fmaf_rn(yh, vh, -p);
    pe = __fmaf_rn(yh, vl, __fmaf_rn(yl, vh, pe));
    const float s = __fadd_rn(ah, p);
    const float bb = __fsub_rn(s, ah);
    const float e = __fadd_rn(__fsub_rn(ah, __fsub_rn(s, bb)), __fsub_rn(p, bb));
    ah = s;
    al = __fadd_rn(al, __fadd_rn(pe, e));
}

// 1 / sqrt(x) of a positive double-float: FP32 estimate, two Newton steps.
__device__ __forceinline__ df df_rsqrt(df x) {
    df y = {rsqrtf(x.hi), 0.0f};
#pragma unroll
    for (int it = 0; it < 2; ++it) {
        const df h = df_mul(x, df_sqr(y));                       // ~ 1
        const df r = df_add({1.5f, 0.0f}, df_mul({-0.5f, 0.0f}, h));
        y = df_mul(y, r);
    }
    return y;
}

struct NewtonArgs {
    int64_t n_s;
    int n_pb, cap, cn;  // cn: columns of V (controls the launch may reach)
    int ppb, cs;        // points per block (32 per group), columns of V held in shared memory
    double R, invR, R2, S0, tau, piv_tol_per_n, piv_tol_df_per_n, switch_ratio, switch_work;
    // the stop test's bracket as argmax keys: key < key_lo is below the
    // threshold, key >= key_hi above it, keys between are tested exactly
    unsigned long long key_lo, key_hi;
    float invR_hi, invR_lo;
    float Rlist;  // R (1 + 1e-9), rounded up to FP32: the list test's radius
    const double4 *xs, *pb_lo, *pb_hi;
    const uint32_t *perm;
    const double4 *E0;  // E at the start of the level (= dS_l)
    unsigned char *sel;
    uint32_t *nb_cnt, *nb_list;
    double4 *cx, *alpha, *w;
    float4 *wdf;  // mixed mode: w of each control in double-float ([2] float4 per control)
    float4 *cdf;
    uint32_t *cid;
    double *G, *Gt, *V;  // V: FP64, or hi/lo float pairs in mixed mode
    double4 *rec;  // [2][P][3] per block: integers (key, original index, longest list, position), coordinates + l^2, E
    ulonglong2 *head;  // [2][P] per block: key, original index | longest list << 32 (what every block reads)
    double *ycol;  // [2][P][cn + 1] per block: V[.][candidate] (mixed mode: hi/lo float pairs)
    // (two copies, by the parity of the step: a block writes the next step's
    // record while a slower block may still read this step's)
    GridBarrier *bar;
    unsigned long long spin_limit;
    GreedyState *st;
    unsigned long long *pairs;
    unsigned long long *phase_ns;
    int test_skip_arrival;  // tests only: block 0 leaves before its first barrier arrival
};

// Dynamic shared memory of one block (8-byte words): y [cn], V slice
// [cs][ppb], E [3][ppb], coordinates [3][ppb], s2 [ppb]; then original
// indices [ppb] and selected flags [ppb].  Mixed mode keeps y as (hi, lo)
// float pairs and each other 8-byte value as a hi float array followed by a
// lo float array.
inline size_t newton_smem_bytes(int cn, int cs, int ppb) {
    return 8 * ((size_t)cn + (size_t)cs * ppb + 7 * (size_t)ppb) + 4 * (size_t)ppb + (size_t)ppb;
}

template <int DIM, int BASIS, int MODE>
__global__ void __launch_bounds__(kNT, 1) k_greedy_newton(NewtonArgs a) {
    extern __shared__ double dsm[];
    const int ppb = a.ppb, n_grp = ppb / 32;
    double *s_y = dsm;                        // y [cn] (mixed: as FP64 only during (b))
    float2 *s_y2 = reinterpret_cast<float2 *>(dsm);  // mixed: y as (hi, lo) pairs in the same words
    double *s_V = dsm + a.cn;                 // FP64: V[k][slot], k < cs
    float *s_Vh = reinterpret_cast<float *>(s_V), *s_Vl = s_Vh + (size_t)a.cs * ppb;
    double *s_E = s_V + (size_t)a.cs * ppb;   // E of the block's points (x, y, z rows)
    float *s_Eh = reinterpret_cast<float *>(s_E), *s_El = s_Eh + 3 * ppb;
    double *s_X = s_E + 3 * ppb;              // their coordinates
    float *s_Xh = reinterpret_cast<float *>(s_X), *s_Xl = s_Xh + 3 * ppb;
    double *s_S2 = s_X + 3 * ppb;             // sum_k v_k(x)^2
    float *s_S2h = reinterpret_cast<float *>(s_S2), *s_S2l = s_S2h + ppb;
    int *s_orig = reinterpret_cast<int *>(s_S2 + ppb);  // original surface index
    unsigned char *s_sel = reinterpret_cast<unsigned char *>(s_orig + ppb);
    // partial dots of the two groups of a round of (a), [group][warp][lane]
    // (FP64; mixed: hi [8][32] then lo [8][32] per group)
    __shared__ double s_part[kRound][kNW][32];
    __shared__ double s_phi[kRound][32];  // phi at the round's points (mixed: hi [32] then lo [32] as floats)
    __shared__ unsigned long long sk[32];
    __shared__ int si[32], sbw[32];
    // the step's scalars, computed by one warp: [2] 1 / l_j (mixed: its
    // double-float bits), [3] 1 / l_j and [4..6] w_j in FP64 for (b)
    __shared__ double s_dec[8];
    __shared__ int s_flags, s_mc, s_bar_ok;
    __shared__ unsigned s_nz[kNW], s_lm[kNW];
    __shared__ double4 s_wrec[3];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned P = gridDim.x;
    const size_t ycl = (size_t)a.cn + 1;
    // slot s of this block is surface point (blockIdx + (s / 32) P) * 32 + s % 32
    auto point_of = [&](int slot) -> int64_t {
        return ((int64_t)blockIdx.x + (int64_t)(slot / 32) * P) * 32 + slot % 32;
    };
    for (int sl = tid; sl < ppb; sl += kNT) {
        const int64_t i = point_of(sl);
        const bool valid = i < a.n_s;
        const double4 x = valid ? a.xs[i] : make_double4(0, 0, 0, 0);
        const double4 e = valid ? a.E0[i] : make_double4(0, 0, 0, 0);
        const double xv[3] = {x.x, x.y, x.z}, ev[3] = {e.x, e.y, e.z};
        for (int c = 0; c < 3; ++c) {
            if (MODE) {
                const df xd = df_from_double(xv[c]), ed = df_from_double(ev[c]);
                s_Xh[c * ppb + sl] = xd.hi;
                s_Xl[c * ppb + sl] = xd.lo;
                s_Eh[c * ppb + sl] = ed.hi;
                s_El[c * ppb + sl] = ed.lo;
            } else {
                s_X[c * ppb + sl] = xv[c];
                s_E[c * ppb + sl] = ev[c];
            }
        }
        if (MODE) {
            s_S2h[sl] = 0.f;
            s_S2l[sl] = 0.f;
        } else {
            s_S2[sl] = 0.0;
        }
        s_orig[sl] = valid ? (int)a.perm[i] : -1;
        s_sel[sl] = valid ? __ldcg(a.sel + i) : 1;
    }
    // control lists: point block t is kept by thread t / P of block t % P
    // (box and count in registers: appends never read back)
    const int t_own = (int)blockIdx.x + tid * (int)P;
    const bool own_list = t_own < a.n_pb;
    // the block box rounded outward to FP32: the list test below runs in
    // FP32 with a radius that covers its rounding, so it keeps every control
    // within R of the box (and a few just beyond it, which add zero terms)
    float3 own_lo = make_float3(0.f, 0.f, 0.f), own_hi = own_lo;
    uint32_t own_cnt = 0;
    if (own_list) {
        const double4 lo = a.pb_lo[t_own], hi = a.pb_hi[t_own];
        own_lo = make_float3(__double2float_rd(lo.x), __double2float_rd(lo.y), __double2float_rd(lo.z));
        own_hi = make_float3(__double2float_ru(hi.x), __double2float_ru(hi.y), __double2float_ru(hi.z));
        own_cnt = __ldcg(&a.nb_cnt[t_own]);
    }
    // the launch starts a level: control 0 placed, nothing propagated yet
    int n = __ldcg(&a.st->n);
    uint32_t cj = __ldcg(&a.cid[0]);
    // c_j: coordinates (FP64; mixed: double-float), 1 / l_j and w_j
    double4 xcj = ldcg_d4(&a.cx[0]);
    df xcd[3] = {df_from_double(xcj.x), df_from_double(xcj.y), df_from_double(xcj.z)};
    double ilj = 1.0;
    df ild = {1.0f, 0.0f};
    double4 wj = ldcg_d4(&a.w[0]);
    df wd[3] = {df_from_double(wj.x), df_from_double(wj.y), df_from_double(wj.z)};
    if (tid == 0) {  // (b) of control 0: l_0 = 1
        s_dec[3] = 1.0;
        s_dec[4] = wj.x;
        s_dec[5] = wj.y;
        s_dec[6] = wj.z;
    }
    // counts kept per block and added once at the end: nonzeros of Phi_sc in
    // this block's points so far, and the pairs a list sweep of each step
    // would have evaluated there
    unsigned long long nz_cum = 0, pairs_useful = 0;
    uint32_t list_max = own_list ? own_cnt : 0;  // longest list this block keeps
    // rows of the inverse factor: row k belongs to warp (k / P) % 7 of block
    // k % P (the last warp arrives at and waits for the grid barrier meanwhile)
    constexpr int kRowWarps = kNW - 1;
    const int k_first = warp < kRowWarps ? (int)blockIdx.x + warp * (int)P : INT_MAX;
    const df invRd = {a.invR_hi, a.invR_lo};
    // profile mode, block 0: [0] marking c_j, [1] (a), [2] lists + record, [3] (b),
    // [4] barrier wait, [5] reading the records, [6] their argmax, [7] scalars
    // and the next y
    const bool timing = a.phase_ns && blockIdx.x == 0 && tid == 0;
    unsigned long long acc_ns[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    unsigned long long t_mark = timing ? gtimer() : 0ull;
#define RBFD_TMARK(SLOT)                        \
    if (timing) {                               \
        const unsigned long long t_ = gtimer(); \
        acc_ns[SLOT] += t_ - t_mark;            \
        t_mark = t_;                            \
    }
#define RBFD_NEXIT()                                                                  \
    {                                                                                 \
        if (timing)                                                                   \
            for (int q_ = 0; q_ < 8; ++q_) atomicAdd(&a.phase_ns[q_], acc_ns[q_]);    \
        return;                                                                       \
    }
    if (n != 1) {  // (only ever launched at the start of a level)
        if (blockIdx.x == 0 && tid == 0) {
            a.st->handoff = 1;
            a.st->stop = 1;
        }
        RBFD_NEXIT()
    }

    __syncthreads();  // the block's state is in shared memory
    // Block barriers per pass: two per group of (a), two in the record, one
    // after the grid barrier's arrival (mixed mode), one in the wait, three in
    // the decision.  The first of (a) orders the marking below and the
    // previous decision's shared writes before their readers.
    for (int guard = 0; guard <= a.cap; ++guard) {
        const int j = n - 1;  // the control this pass propagates
        // (y of c_j was loaded by the previous pass's decision)
        {  // the owner marks c_j as selected
            const int64_t item = (int64_t)cj / 32;
            if (tid == 0 && item % P == blockIdx.x) s_sel[(int)(item / P) * 32 + (int)(cj % 32)] = 1;
        }
        // this warp's first row of the inverse factor for (b): its entries
        // before column j are final (this warp wrote them), so the loads
        // start now and arrive during (a)
        double gpre[kRowChunk];
        double4 apre = make_double4(0, 0, 0, 0);
        if (k_first < j) {
            const double *trow = a.Gt + (size_t)k_first * a.cap;
#pragma unroll
            for (int q = 0; q < kRowChunk; ++q) {
                const int m = k_first + lane + 32 * q;
                gpre[q] = m < j ? __ldcg(trow + m) : 0.0;
            }
            if (lane == 0) apre = ldcg_d4(&a.alpha[k_first]);
        }
        RBFD_TMARK(0)

        // ---- (a) v_j at the block's points, E update, argmax
        unsigned long long bkey = 0;
        int bidx = -1, bslot = -1;
        unsigned nz = 0;
        const int kcs = min(j, a.cs);
        // rounds of up to kRound groups of 32 points: warp 0 evaluates
        // phi(|x_i - c_j| / R) at the round's points while the other seven
        // warps compute the dot sum_k y_k V[k][i] in seven slices (columns
        // k = w - 1 mod 7); then warp g of the block finishes group g.  The
        // per-point arithmetic does not depend on the number of groups.
        for (int g0 = 0; g0 < n_grp; g0 += kRound) {
            const int ng = min(kRound, n_grp - g0);
            if (warp == 0) {
                for (int gg = 0; gg < ng; ++gg) {
                    const int sl = (g0 + gg) * 32 + lane;
                    if (point_of(sl) >= a.n_s) continue;
                    if (MODE) {
                        df r2 = {0.f, 0.f};
#pragma unroll
                        for (int c = 0; c < DIM; ++c) {
                            const df d = df_add({s_Xh[c * ppb + sl], s_Xl[c * ppb + sl]}, df_neg(xcd[c]));
                            r2 = df_add(r2, df_sqr(d));
                        }
                        const df f = phi_df<BASIS>(df_mul(df_sqrt(r2), invRd));
                        nz += (f.hi != 0.f);
                        float *fh = reinterpret_cast<float *>(&s_phi[gg][0]);
                        fh[lane] = f.hi;
                        fh[32 + lane] = f.lo;
                    } else {
                        const double f = phi_f64<BASIS>(
                            dist_f64<DIM>(s_X[sl], s_X[ppb + sl], s_X[2 * ppb + sl], xcj.x, xcj.y, xcj.z) * a.invR);
                        nz += (f != 0.0);
                        s_phi[gg][lane] = f;
                    }
                }
            } else {
                const int ks = warp - 1;  // this warp's slice
                for (int gg = 0; gg < ng; ++gg) {
                    const int g = g0 + gg;
                    const int sl = g * 32 + lane;
                    const int64_t i = point_of(sl);
                    const bool valid = i < a.n_s;
                    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
                    float h0 = 0.f, l0 = 0.f, h1 = 0.f, l1 = 0.f;
                    if (valid) {
                        int k = ks;
                        if (MODE) {
                            // double-float on the FP32 pipe (FP64 issues at a small
                            // fraction of the FP32 rate on this GPU)
                            const float *Vh = s_Vh + sl, *Vl = s_Vl + sl;
                            for (; k + kDotW < kcs; k += 2 * kDotW) {
                                const float2 y0 = s_y2[k], y1 = s_y2[k + kDotW];
                                df_fma_acc(h0, l0, y0.x, y0.y, Vh[(size_t)k * ppb], Vl[(size_t)k * ppb]);
                                df_fma_acc(h1, l1, y1.x, y1.y, Vh[(size_t)(k + kDotW) * ppb],
                                           Vl[(size_t)(k + kDotW) * ppb]);
                            }
                            for (; k < kcs; k += kDotW) {
                                const float2 y0 = s_y2[k];
                                df_fma_acc(h0, l0, y0.x, y0.y, Vh[(size_t)k * ppb], Vl[(size_t)k * ppb]);
                            }
                            // columns beyond the shared slice: hi/lo pairs from global memory
                            const float2 *Vi = reinterpret_cast<const float2 *>(a.V) + i;
                            for (; k + kDotW < j; k += 2 * kDotW) {
                                const float2 v0 = __ldcg(Vi + (size_t)k * a.n_s),
                                             v1 = __ldcg(Vi + (size_t)(k + kDotW) * a.n_s);
                                const float2 y0 = s_y2[k], y1 = s_y2[k + kDotW];
                                df_fma_acc(h0, l0, y0.x, y0.y, v0.x, v0.y);
                                df_fma_acc(h1, l1, y1.x, y1.y, v1.x, v1.y);
                            }
                            for (; k < j; k += kDotW) {
                                const float2 v = __ldcg(Vi + (size_t)k * a.n_s), y0 = s_y2[k];
                                df_fma_acc(h0, l0, y0.x, y0.y, v.x, v.y);
                            }
                        } else {
                            const double *Vs = s_V + sl;
                            for (; k + 3 * kDotW < kcs; k += 4 * kDotW) {
                                s0 = fma(s_y[k], Vs[(size_t)k * ppb], s0);
                                s1 = fma(s_y[k + kDotW], Vs[(size_t)(k + kDotW) * ppb], s1);
                                s2 = fma(s_y[k + 2 * kDotW], Vs[(size_t)(k + 2 * kDotW) * ppb], s2);
                                s3 = fma(s_y[k + 3 * kDotW], Vs[(size_t)(k + 3 * kDotW) * ppb], s3);
                            }
                            for (; k < kcs; k += kDotW) s0 = fma(s_y[k], Vs[(size_t)k * ppb], s0);
                            const double *Vi = a.V + i;
                            const size_t ld = (size_t)a.n_s;
                            for (; k + 3 * kDotW < j; k += 4 * kDotW) {
                                const double v0 = __ldcg(Vi + (size_t)k * ld), v1 = __ldcg(Vi + (size_t)(k + kDotW) * ld),
                                             v2 = __ldcg(Vi + (size_t)(k + 2 * kDotW) * ld),
                                             v3 = __ldcg(Vi + (size_t)(k + 3 * kDotW) * ld);
                                s0 = fma(s_y[k], v0, s0);
                                s1 = fma(s_y[k + kDotW], v1, s1);
                                s2 = fma(s_y[k + 2 * kDotW], v2, s2);
                                s3 = fma(s_y[k + 3 * kDotW], v3, s3);
                            }
                            for (; k < j; k += kDotW) s0 = fma(s_y[k], __ldcg(Vi + (size_t)k * ld), s0);
                        }
                    }
                    if (MODE) {
                        const df t = df_add({h0, l0}, {h1, l1});
                        float *ph = reinterpret_cast<float *>(&s_part[gg][0][0]);
                        ph[ks * 32 + lane] = t.hi;
                        ph[kNW * 32 + ks * 32 + lane] = t.lo;
                    } else {
                        s_part[gg][ks][lane] = (s0 + s1) + (s2 + s3);
                    }
                }
            }
            __syncthreads();
            if (warp < ng) {
                const int g = g0 + warp;
                const int sl = g * 32 + lane;
                const int64_t i = point_of(sl);
                if (i < a.n_s) {
                    unsigned long long key;
                    if (MODE) {
                        // the seven partial sums as a tree
                        const float *ph = reinterpret_cast<const float *>(&s_part[warp][0][0]);
                        const float *pl = ph + kNW * 32;
                        auto part = [&](int q) { return df{ph[q * 32 + lane], pl[q * 32 + lane]}; };
                        const df sum = df_add(df_add(df_add(part(0), part(1)), df_add(part(2), part(3))),
                                              df_add(df_add(part(4), part(5)), part(6)));
                        const float *fh = reinterpret_cast<const float *>(&s_phi[warp][0]);
                        const df f = {fh[lane], fh[32 + lane]};
                        const df v = df_mul(df_add(f, df_neg(sum)), ild);
                        if (j < a.cs) {
                            s_Vh[(size_t)j * ppb + sl] = v.hi;
                            s_Vl[(size_t)j * ppb + sl] = v.lo;
                        } else {
                            reinterpret_cast<float2 *>(a.V)[(size_t)j * a.n_s + i] = make_float2(v.hi, v.lo);
                        }
                        df k2 = {0.f, 0.f};
#pragma unroll
                        for (int c = 0; c < DIM; ++c) {
                            df e = {s_Eh[c * ppb + sl], s_El[c * ppb + sl]};
                            e = df_add(e, df_neg(df_mul(wd[c], v)));
                            s_Eh[c * ppb + sl] = e.hi;
                            s_El[c * ppb + sl] = e.lo;
                            k2 = df_add(k2, df_sqr(e));
                        }
                        const df s2n = df_add({s_S2h[sl], s_S2l[sl]}, df_sqr(v));
                        s_S2h[sl] = s2n.hi;
                        s_S2l[sl] = s2n.lo;
                        key = key_of_df(k2);
                    } else {
                        auto part = [&](int q) { return s_part[warp][q][lane]; };
                        const double sum = ((part(0) + part(1)) + (part(2) + part(3))) + ((part(4) + part(5)) + part(6));
                        const double f = s_phi[warp][lane];
                        const double v = (f - sum) * ilj;
                        if (j < a.cs) s_V[(size_t)j * ppb + sl] = v;
                        else a.V[(size_t)j * a.n_s + i] = v;
                        const double e0 = fma(-wj.x, v, s_E[sl]);
                        const double e1 = fma(-wj.y, v, s_E[ppb + sl]);
                        const double e2 = DIM == 3 ? fma(-wj.z, v, s_E[2 * ppb + sl]) : 0.0;
                        s_E[sl] = e0;
                        s_E[ppb + sl] = e1;
                        s_E[2 * ppb + sl] = e2;
                        s_S2[sl] = fma(v, v, s_S2[sl]);
                        double k2 = __dmul_rn(e0, e0);
                        k2 = __dadd_rn(k2, __dmul_rn(e1, e1));
                        if (DIM == 3) k2 = __dadd_rn(k2, __dmul_rn(e2, e2));
                        key = key_of_double(k2);
                    }
                    if (!s_sel[sl]) {
                        const int o = s_orig[sl];
                        if (better_key(key, o, bkey, bidx)) {
                            bkey = key;
                            bidx = o;
                            bslot = sl;
                        }
                    }
                }
            }
            __syncthreads();
        }
        RBFD_TMARK(1)

        // ---- lists (control 0: listed at level start), nonzero count, the block's record
        if (j > 0 && own_list) {
            // c_j rounded to FP32 (u = 2^-24 relative); with the box rounded
            // outward each gap exceeds the exact one by at most u |c| (1 + u)
            // and the sum of squares carries (1 + u)^5, which the radius
            // (R (1 + 1e-9) + 2.5 u max|c|)^2 (1 + 2^-21), rounded up, covers
            float xf, yf, zf;
            if (MODE) {
                xf = xcd[0].hi;
                yf = xcd[1].hi;
                zf = xcd[2].hi;
            } else {
                xf = __double2float_rn(xcj.x);
                yf = __double2float_rn(xcj.y);
                zf = __double2float_rn(xcj.z);
            }
            const float mx = fmaxf(fmaxf(fabsf(xf), fabsf(yf)), DIM == 3 ? fabsf(zf) : 0.f);
            const float rr = __fadd_ru(a.Rlist, __fmul_ru(mx, 1.4901161193847656e-7f));
            const float r2 = __fmul_ru(__fmul_ru(rr, rr), 1.0f + 4.76837158203125e-7f);
            const float dx = fmaxf(fmaxf(own_lo.x - xf, xf - own_hi.x), 0.f);
            const float dy = fmaxf(fmaxf(own_lo.y - yf, yf - own_hi.y), 0.f);
            const float dz = DIM == 3 ? fmaxf(fmaxf(own_lo.z - zf, zf - own_hi.z), 0.f) : 0.f;
            if (dx * dx + dy * dy + dz * dz < r2) {
                a.nb_list[(size_t)t_own * a.cap + own_cnt] = (uint32_t)j;
                ++own_cnt;
                a.nb_cnt[t_own] = own_cnt;
            }
        }
        {
            // the block's best candidate, its nonzero count and longest list:
            // per warp by shuffles, then every thread reduces the warps'
            // entries itself (one block barrier)
            unsigned long long kk = bkey;
            int ii = bidx, ws = bslot;
            unsigned u = nz, lm = own_list ? own_cnt : 0u;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const unsigned long long k2 = __shfl_xor_sync(0xffffffffu, kk, o);
                const int i2 = __shfl_xor_sync(0xffffffffu, ii, o), w2 = __shfl_xor_sync(0xffffffffu, ws, o);
                if (better_key(k2, i2, kk, ii)) {
                    kk = k2;
                    ii = i2;
                    ws = w2;
                }
                u += __shfl_xor_sync(0xffffffffu, u, o);
                lm = max(lm, __shfl_xor_sync(0xffffffffu, lm, o));
            }
            if (lane == 0) {
                sk[warp] = kk;
                si[warp] = ii;
                sbw[warp] = ws;
                s_nz[warp] = u;
                s_lm[warp] = lm;
            }
            __syncthreads();
            kk = sk[0];
            ii = si[0];
            ws = sbw[0];
#pragma unroll
            for (int w8 = 1; w8 < kNW; ++w8)
                if (better_key(sk[w8], si[w8], kk, ii)) {
                    kk = sk[w8];
                    ii = si[w8];
                    ws = sbw[w8];
                }
            if (ii < 0) ws = -1;
            if (tid == 0) {
                unsigned bnz = 0;
                for (int w8 = 0; w8 < kNW; ++w8) {
                    bnz += s_nz[w8];
                    list_max = max(list_max, s_lm[w8]);
                }
                nz_cum += bnz;
                pairs_useful += nz_cum;  // the list sweep of this step would evaluate these pairs
                a.head[(size_t)(j & 1) * P + blockIdx.x] =
                    make_ulonglong2(ws >= 0 ? kk : 0ull, (unsigned long long)(unsigned)(ws >= 0 ? ii : -1) |
                                                             ((unsigned long long)list_max << 32));
                double4 *r = a.rec + 3 * ((size_t)(j & 1) * P + blockIdx.x);
                ulonglong2 *ri = reinterpret_cast<ulonglong2 *>(r);
                if (ws >= 0) {
                    ri[0] = make_ulonglong2(kk, (unsigned long long)(long long)ii);
                    ri[1] = make_ulonglong2((unsigned long long)list_max, (unsigned long long)point_of(ws));
                    if (MODE) {
                        float4 *rf = reinterpret_cast<float4 *>(r + 1);
                        const df l2 = df_add({1.0f, 0.0f}, df_neg({s_S2h[ws], s_S2l[ws]}));
                        rf[0] = make_float4(s_Xh[ws], s_Xl[ws], s_Xh[ppb + ws], s_Xl[ppb + ws]);
                        rf[1] = make_float4(s_Xh[2 * ppb + ws], s_Xl[2 * ppb + ws], l2.hi, l2.lo);
                        rf[2] = make_float4(s_Eh[ws], s_El[ws], s_Eh[ppb + ws], s_El[ppb + ws]);
                        rf[3] = make_float4(s_Eh[2 * ppb + ws], s_El[2 * ppb + ws], 0.f, 0.f);
                    } else {
                        r[1] = make_double4(s_X[ws], s_X[ppb + ws], s_X[2 * ppb + ws], 1.0 - s_S2[ws]);
                        r[2] = make_double4(s_E[ws], s_E[ppb + ws], s_E[2 * ppb + ws], 0.0);
                    }
                } else {
                    ri[0] = make_ulonglong2(0ull, ~0ull);  // key 0, index -1
                    ri[1] = make_ulonglong2((unsigned long long)list_max, ~0ull);
                }
            }
            if (ws >= 0) {  // the candidate's column: y of the next control if it wins
                const int64_t pw = point_of(ws);
                double *yc = a.ycol + ((size_t)(j & 1) * P + blockIdx.x) * ycl;
                if (MODE) {
                    float2 *yf = reinterpret_cast<float2 *>(yc);
                    for (int k = tid; k <= j; k += kNT) {
                        float2 v;
                        if (k < a.cs)
                            v = make_float2(s_Vh[(size_t)k * ppb + ws], s_Vl[(size_t)k * ppb + ws]);
                        else
                            v = __ldcg(reinterpret_cast<const float2 *>(a.V) + (size_t)k * a.n_s + pw);
                        yf[k] = v;
                    }
                } else {
                    for (int k = tid; k <= j; k += kNT)
                        yc[k] = k < a.cs ? s_V[(size_t)k * ppb + ws] : __ldcg(a.V + (size_t)k * a.n_s + pw);
                }
            }
        }
        RBFD_TMARK(2)
        if (a.test_skip_arrival && blockIdx.x == 0) return;  // the others' waits run out
        __syncthreads();  // the block's record and candidate column are written
        if (warp == kRowWarps) {
            // the last warp arrives at the grid barrier and waits for it
            if (lane == 0) {
                grid_arrive_mono_one(a.bar);
                s_bar_ok = grid_poll_mono_one(a.bar, (unsigned)(guard + 1) * P, a.spin_limit);
            }
        } else {
            // ---- (b) row j of the inverse factor on this block's rows, alpha (FP64)
            if (MODE) {  // y to FP64 once per block, in place (each pair becomes its double)
                for (int m = tid; m < j; m += kRowWarps * 32) {
                    const float2 v = s_y2[m];
                    s_y[m] = (double)v.x + (double)v.y;
                }
                asm volatile("bar.sync 1, %0;" ::"n"(kRowWarps * 32) : "memory");  // the row warps only
            }
            const double ilj64 = s_dec[3];
            const double4 wj64 = make_double4(s_dec[4], s_dec[5], s_dec[6], 0.0);
            for (int k = k_first; k <= j; k += (int)P * kRowWarps) {
                if (k == j) {  // the diagonal and alpha_j
                    if (lane == 0) {
                        a.G[(size_t)j * a.cap + j] = ilj64;
                        a.Gt[(size_t)j * a.cap + j] = ilj64;
                        a.alpha[j] = make_double4(wj64.x * ilj64, wj64.y * ilj64, wj64.z * ilj64, 0.0);
                    }
                    break;
                }
                const double *trow = a.Gt + (size_t)k * a.cap;
                double4 al = make_double4(0, 0, 0, 0);
                // t0 sums the entries m = k + lane + 64 i, t1 those 32 further on,
                // in chunks of 32 kRowChunk entries whose loads are issued together
                double t0 = 0.0, t1 = 0.0;
                int m0 = k + lane;
                if (k == k_first) {  // (loaded at the start of the pass)
                    al = apre;
#pragma unroll
                    for (int q = 0; q < kRowChunk; ++q) {
                        const int m = m0 + 32 * q;
                        if (m < j) {
                            if (q & 1) t1 = fma(gpre[q], s_y[m], t1);
                            else t0 = fma(gpre[q], s_y[m], t0);
                        }
                    }
                    m0 += 32 * kRowChunk;
                } else if (lane == 0) {
                    al = ldcg_d4(&a.alpha[k]);
                }
                for (; m0 < j; m0 += 32 * kRowChunk) {
                    double g[kRowChunk];
#pragma unroll
                    for (int q = 0; q < kRowChunk; ++q) {
                        const int m = m0 + 32 * q;
                        g[q] = m < j ? __ldcg(trow + m) : 0.0;
                    }
#pragma unroll
                    for (int q = 0; q < kRowChunk; ++q) {
                        const int m = m0 + 32 * q;
                        if (m < j) {
                            if (q & 1) t1 = fma(g[q], s_y[m], t1);
                            else t0 = fma(g[q], s_y[m], t0);
                        }
                    }
                }
                const double t = warp_sum_d(t0 + t1);
                if (lane == 0) {
                    const double gk = -t * ilj64;
                    a.G[(size_t)j * a.cap + k] = gk;
                    a.Gt[(size_t)k * a.cap + j] = gk;
                    al.x = fma(wj64.x, gk, al.x);
                    al.y = fma(wj64.y, gk, al.y);
                    al.z = fma(wj64.z, gk, al.z);
                    a.alpha[k] = al;
                }
            }
        }
        RBFD_TMARK(3)
        __syncthreads();  // the grid barrier has passed (or failed: s_bar_ok)
        if (!s_bar_ok) RBFD_NEXIT()
        RBFD_TMARK(4)

        // ---- the step's decision: every block from the same records
        // every block reads the P heads (16 bytes each), takes the argmax per
        // warp and then over the warps' entries (one block barrier); the
        // winner's full record is read by one warp afterwards
        unsigned long long K = 0;
        int I = -1, Bw = -1;
        unsigned lmax = 0;
        const ulonglong2 *hj = a.head + (size_t)(j & 1) * P;
        for (unsigned b = tid; b < P; b += kNT) {
            const ulonglong2 h = __ldcg(&hj[b]);
            lmax = max(lmax, (unsigned)(h.y >> 32));
            const int ib = (int)(unsigned)h.y;
            if (better_key(h.x, ib, K, I)) {
                K = h.x;
                I = ib;
                Bw = (int)b;
            }
        }
        RBFD_TMARK(5)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long k2 = __shfl_xor_sync(0xffffffffu, K, o);
            const int i2 = __shfl_xor_sync(0xffffffffu, I, o), b2 = __shfl_xor_sync(0xffffffffu, Bw, o);
            if (better_key(k2, i2, K, I)) {
                K = k2;
                I = i2;
                Bw = b2;
            }
            lmax = max(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
        }
        if (lane == 0) {
            sk[warp] = K;
            si[warp] = I;
            sbw[warp] = Bw;
            s_lm[warp] = lmax;
        }
        __syncthreads();
        K = sk[0];
        I = si[0];
        Bw = sbw[0];
#pragma unroll
        for (int w8 = 1; w8 < kNW; ++w8)
            if (better_key(sk[w8], si[w8], K, I)) {
                K = sk[w8];
                I = si[w8];
                Bw = sbw[w8];
            }
        RBFD_TMARK(6)
        const int nn = n;  // index the next control takes
        if (warp == 0) {  // the step's scalars, on one warp
            if (I >= 0) {  // the winner's record: 96 bytes, 16 per lane
                if (lane < 6)
                    reinterpret_cast<ulonglong2 *>(s_wrec)[lane] =
                        __ldcg(reinterpret_cast<const ulonglong2 *>(a.rec + 3 * ((size_t)(j & 1) * P + Bw)) + lane);
                __syncwarp();
            }
            int mc = 1;
            for (int w8 = 0; w8 < kNW; ++w8) mc = max(mc, (int)s_lm[w8]);
            // e = sqrt(K) / S0 < tau, the same rounded test as the other
            // engines; the square root and the division only near the threshold
            bool below;
            if (I < 0) below = true;
            else if (K < a.key_lo) below = true;
            else if (K >= a.key_hi) below = false;
            else below = __ddiv_rn(__dsqrt_rn(key_value<MODE>(K)), a.S0) < a.tau;
            const bool stop = I < 0 || below || nn >= a.cap;
            // hand over to the list sweep when V is full, or when the Newton
            // update (n_s * n multiply-adds) is large and the lists are much
            // shorter than the control count
            const bool hand = !stop && (nn >= a.cn || ((double)a.n_s * nn > a.switch_work &&
                                                       (double)nn > a.switch_ratio * (double)mc));
            bool singular = false, weak = false;
            if (!stop && !hand) {
                // 1 / l_j, and w_j = E(c_j) / l_j in FP64 for (b): lanes 0-2
                // take w_j's components, lane 3 takes 1 / l_j
                if (MODE) {
                    const float4 *rf = reinterpret_cast<const float4 *>(&s_wrec[1]);
                    const df l2 = {rf[1].z, rf[1].w};
                    // 1 - s2 in double-float carries an error of about
                    // n 2^-47: a pivot within 8 times that cannot be told from
                    // zero here, and the level goes on in the list sweep,
                    // whose FP64 growth tests it (ESINGULAR only there)
                    weak = !(l2.hi > (float)(a.piv_tol_df_per_n * (nn + 1)));
                    if (!weak) {
                        const df il = df_rsqrt(l2);
                        const float *ef = reinterpret_cast<const float *>(&s_wrec[2]);
                        const df q = lane < 3 ? df_mul({ef[2 * lane], ef[2 * lane + 1]}, il) : il;
                        if (lane < 4) s_dec[lane < 3 ? 4 + lane : 3] = (double)q.hi + (double)q.lo;
                        if (lane == 0)
                            s_dec[2] = __longlong_as_double(
                                (long long)(((unsigned long long)__float_as_uint(il.hi) << 32) | __float_as_uint(il.lo)));
                    }
                } else {
                    const double l2 = s_wrec[1].w;
                    singular = !(l2 > a.piv_tol_per_n * (nn + 1));
                    if (!singular) {
                        // 1 / sqrt(l2): FP32 estimate and two Newton steps in FP64
                        double il = (double)rsqrtf((float)l2);
                        il = il * fma(-0.5 * l2 * il, il, 1.5);
                        il = il * fma(-0.5 * l2 * il, il, 1.5);
                        const double *er = reinterpret_cast<const double *>(&s_wrec[2]);
                        if (lane < 3) s_dec[4 + lane] = er[lane] * il;
                        if (lane == 3) s_dec[3] = il;
                    }
                }
            }
            if (lane == 0) {
                s_flags = (stop ? 1 : 0) | ((hand || weak) ? 2 : 0) | (singular ? 4 : 0);
                s_mc = mc;
            }
        } else if (I >= 0) {
            // meanwhile the other warps load the winner's column, y of the
            // next pass (written before this step's barrier, parity j & 1;
            // unused if the level stops here)
            const double *yb = a.ycol + ((size_t)(j & 1) * P + Bw) * ycl;
            if (MODE) {
                const float2 *yf = reinterpret_cast<const float2 *>(yb);
                for (int k = tid - 32; k < nn; k += kNT - 32) s_y2[k] = __ldcg(&yf[k]);
            } else {
                for (int k = tid - 32; k < nn; k += kNT - 32) s_y[k] = __ldcg(&yb[k]);
            }
        }
        __syncthreads();
        const int flags = s_flags;
        const bool writer = blockIdx.x == 0 && tid == 0;
        if (flags) {
            if (tid == 0) {
                // pairs evaluated here (phi of each step's control at this
                // block's points within R), and the Eq. 12 nonzeros a list
                // sweep of every step would have evaluated instead
                atomicAdd(&a.pairs[8], nz_cum);
                atomicAdd(&a.pairs[10], pairs_useful);
            }
            if (blockIdx.x == 0) {
                if (MODE)  // the controls' records in FP64 for what follows the launch
                    for (int k = 1 + tid; k < nn; k += kNT) {
                        const double4 x = a.xs[__ldcg(&a.cid[k])];
                        const float hx = __double2float_rn(x.x), hy = __double2float_rn(x.y),
                                    hz = __double2float_rn(x.z);
                        a.cx[k] = x;
                        a.cdf[k] = make_float4(hx, hy, hz, 0.f);
                        a.cdf[a.cap + 1 + k] = make_float4(__double2float_rn(x.x - (double)hx),
                                                           __double2float_rn(x.y - (double)hy),
                                                           __double2float_rn(x.z - (double)hz), 0.f);
                        const float4 w0 = __ldcg(&a.wdf[2 * k]), w1 = __ldcg(&a.wdf[2 * k + 1]);
                        a.w[k] = make_double4((double)w0.x + (double)w0.y, (double)w0.z + (double)w0.w,
                                              (double)w1.x + (double)w1.y, 0.0);
                    }
                if (writer) {
                    const bool stop = flags & 1, hand = flags & 2, singular = flags & 4;
                    const double e = I >= 0 ? __ddiv_rn(__dsqrt_rn(key_value<MODE>(K)), a.S0) : 0.0;
                    // per step, the basis update touches n_s x (controls so far) values of V
                    const unsigned long long terms =
                        (unsigned long long)a.n_s * (unsigned long long)(nn) * (unsigned long long)(nn + 1) / 2;
                    a.pairs[6] += terms;
                    // phi values formed by the basis update: every point, every step
                    a.pairs[9] += (unsigned long long)a.n_s * (unsigned long long)nn;
                    a.st->best_orig = I;
                    a.st->best_key = I >= 0 ? key_value<MODE>(K) : -1.0;
                    a.st->emax = e;
                    a.st->max_cnt = s_mc;
                    a.st->n = nn;
                    if (singular) a.st->status = RBFD_ESINGULAR;
                    else if (stop && !(I < 0 || e < a.tau)) a.st->status = RBFD_ENOTCONV;
                    a.st->handoff = hand ? 1 : 0;
                    a.st->stop = 1;
                }
            }
            RBFD_TMARK(7)
            RBFD_NEXIT()
        }
        cj = (uint32_t)reinterpret_cast<const ulonglong2 *>(&s_wrec[0])[1].y;
        if (MODE) {
            const float4 *rf = reinterpret_cast<const float4 *>(&s_wrec[1]);
            xcd[0] = {rf[0].x, rf[0].y};
            xcd[1] = {rf[0].z, rf[0].w};
            xcd[2] = {rf[1].x, rf[1].y};
            const unsigned long long ib = (unsigned long long)__double_as_longlong(s_dec[2]);
            ild = {__uint_as_float((unsigned)(ib >> 32)), __uint_as_float((unsigned)ib)};
            const float4 *ef = reinterpret_cast<const float4 *>(&s_wrec[2]);
            wd[0] = df_mul({ef[0].x, ef[0].y}, ild);
            wd[1] = df_mul({ef[0].z, ef[0].w}, ild);
            wd[2] = df_mul({ef[1].x, ef[1].y}, ild);
            if (writer) {
                a.sel[cj] = 1;
                a.cid[nn] = cj;
                a.wdf[2 * nn] = make_float4(wd[0].hi, wd[0].lo, wd[1].hi, wd[1].lo);
                a.wdf[2 * nn + 1] = make_float4(wd[2].hi, wd[2].lo, 0.f, 0.f);
            }
        } else {
            ilj = s_dec[3];
            const double4 wr1 = s_wrec[1];
            xcj = make_double4(wr1.x, wr1.y, wr1.z, 0.0);
            wj = make_double4(s_dec[4], s_dec[5], s_dec[6], 0.0);
            if (writer) {
                const float hx = __double2float_rn(xcj.x), hy = __double2float_rn(xcj.y),
                            hz = __double2float_rn(xcj.z);
                a.sel[cj] = 1;
                a.cx[nn] = xcj;
                a.cdf[nn] = make_float4(hx, hy, hz, 0.f);
                a.cdf[a.cap + 1 + nn] = make_float4(__double2float_rn(xcj.x - (double)hx),
                                                    __double2float_rn(xcj.y - (double)hy),
                                                    __double2float_rn(xcj.z - (double)hz), 0.f);
                a.cid[nn] = cj;
                a.w[nn] = wj;
            }
        }
        ++n;
        RBFD_TMARK(7)
    }
    RBFD_NEXIT()
#undef RBFD_NEXIT
#undef RBFD_TMARK
}

template <int DIM, int BASIS>
const void *newton_ptr(int mode) {
    return mode ? reinterpret_cast<const void *>(&k_greedy_newton<DIM, BASIS, 1>)
                : reinterpret_cast<const void *>(&k_greedy_newton<DIM, BASIS, 0>);
}

const void *select_newton(int dim, int basis, int mode) {
#define RBFD_SEL(D, B) \
    if (dim == D && basis == B) return newton_ptr<D, B>(mode);
    RBFD_SEL(2, 0) RBFD_SEL(2, 2) RBFD_SEL(2, 4) RBFD_SEL(2, 6)
    RBFD_SEL(3, 0) RBFD_SEL(3, 2) RBFD_SEL(3, 4) RBFD_SEL(3, 6)
#undef RBFD_SEL
    return nullptr;
}

}  // namespace

// The argmax keys that bracket the stop threshold (the keys order the
// values of |E|^2).  FP64 keys are the bit pattern plus one: key < bits(K_lo)
// + 1 is exactly value < K_lo, key >= bits(K_hi) + 2 exactly value > K_hi.
// Mixed-mode keys put the high float's bits above the low float's: with
// h the largest float <= K_lo, a key below (bits(h) << 32) has hi < h and so
// a value below h <= K_lo; with h' the smallest float >= K_hi, a key from
// (bits(next(next(h'))) << 32) on has a value above next(h') - ulp / 2 >= h'.
unsigned long long stop_key(double K, bool mixed, bool upper) {
    if (!mixed) {
        unsigned long long b;
        std::memcpy(&b, &K, sizeof(b));
        return b + (upper ? 2ull : 1ull);
    }
    if (!upper) {
        if (!(K > 0.0)) return 0ull;
        float h = K >= (double)FLT_MAX ? FLT_MAX : (float)K;
        if ((double)h > K) h = std::nextafter(h, 0.0f);
        unsigned u;
        std::memcpy(&u, &h, sizeof(u));
        return (unsigned long long)u << 32;
    }
    if (!(K < (double)FLT_MAX)) return ~0ull;
    float h = K > 0.0 ? (float)K : 0.0f;
    if ((double)h < K) h = std::nextafter(h, HUGE_VALF);
    h = std::nextafter(std::nextafter(h, HUGE_VALF), HUGE_VALF);
    if (std::isinf(h)) return ~0ull;
    unsigned u;
    std::memcpy(&u, &h, sizeof(u));
    return (unsigned long long)u << 32;
}

int newton_columns(rbfd_mesh *m) {
    // V holds n_s doubles per column; at most kNewtonCols columns, at most
    // RBFD_NEWTON_MB (default 1024) MB; RBFD_NEWTON_COLS caps the columns (tests)
    size_t budget = (size_t)1024 << 20;
    if (const char *v = std::getenv("RBFD_NEWTON_MB")) budget = (size_t)std::strtoull(v, nullptr, 10) << 20;
    size_t cols = budget / (sizeof(double) * (size_t)std::max<int64_t>(1, m->n_s));
    if (const char *v = std::getenv("RBFD_NEWTON_COLS")) cols = std::min<size_t>(cols, std::strtoull(v, nullptr, 10));
    return (int)std::min<size_t>({cols, (size_t)kNewtonCols, (size_t)m->cap});
}

void newton_reserve(rbfd_mesh *m) {
    if (m->d_V) return;
    const int cn = newton_columns(m);
    m->newton_cols = cn;
    if (cn < 2) return;
    m->d_V = dalloc<double>((size_t)cn * (size_t)m->n_s, "Newton basis values");
    m->d_nwdf = dalloc<float4>((size_t)2 * (m->cap + 1), "Newton weights (double-float)");
}

// Blocks and shared-memory layout of a launch on this mesh: ppb points per
// block, cs columns of V in shared memory (the rest is read from HBM).
struct NewtonShape {
    int ctas = 0, ppb = 0, cs = 0;
    size_t smem = 0;
};

NewtonShape newton_shape(rbfd_mesh *m, int want_ctas) {
    const int mode = m->opt.precision == RBFD_FP64 ? 0 : 1;
    const void *k = select_newton(m->dim, m->opt.basis, mode);
    static const size_t kSmemMax = 220 * 1024;   // dynamic shared memory per block (of 227 KB)
    static const size_t kSmemPerSM = 228 * 1024;  // shared memory of one SM
    static const size_t kPerBlockReserve = 7 * 1024;  // static shared memory (5.2 KB) and the system's 1 KB
    NewtonShape s;
    int sms = 0;
    RBFD_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, m->device));
    const int64_t items = (m->n_s + 31) / 32;
    const int share = std::max(1, m->batch_share);
    int ctas = (int)std::max<int64_t>(1, std::min<int64_t>(want_ctas, items));
    // meshes running side by side (batch calls, server slots) share the SMs:
    // their blocks should fit on the GPU together
    ctas = std::min(ctas, std::max(1, 2 * sms / share));
    // one value for every launch: the attribute belongs to the kernel, and
    // meshes on other host threads launch it concurrently
    RBFD_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemMax));
    for (;;) {
        const int ppb = (int)(32 * ((items + ctas - 1) / ctas));
        // blocks each SM must hold when every sharing mesh runs this shape
        const int per_sm = (int)std::max<int64_t>(1, ((int64_t)ctas * share + sms - 1) / sms);
        const size_t budget = std::min(kSmemMax, kSmemPerSM / per_sm - kPerBlockReserve);
        const size_t fixed = newton_smem_bytes(m->newton_cols, 0, ppb);
        if (fixed + 8 * 32 * (size_t)ppb <= budget) {  // at least 32 columns in shared memory
            const int cs = (int)std::min<size_t>((size_t)m->newton_cols, (budget - fixed) / (sizeof(double) * ppb));
            const size_t smem = newton_smem_bytes(m->newton_cols, cs, ppb);
            int occ = 0;
            RBFD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, kNT, smem));
            if (occ >= per_sm && ctas <= std::min(occ * sms, kMaxPersistCTAs)) {
                s.ctas = ctas;
                s.ppb = ppb;
                s.cs = cs;
                s.smem = smem;
                return s;
            }
        }
        // the block state does not fit even on the whole GPU's share of this
        // mesh: no Newton launch (the level runs in the list sweep)
        if (ctas == 1) return s;
        ctas = std::max(1, ctas * 3 / 4);  // fewer blocks, more points each
    }
}

// The launch shape for `ctas` blocks asked (cached per mesh size and kind);
// false if the Newton launch does not fit on this mesh's share of the GPU.
bool newton_fits(rbfd_mesh *m, int ctas) {
    // the shape depends on the mesh, the request and the co-running meshes only
    const int key = ctas * 64 + std::min(m->batch_share, 63);
    if (m->newton_shape_key != key) {
        // shapes are shared by meshes of the same size and kind (the queries behind them are host calls)
        static std::mutex mu;
        static std::map<std::tuple<int, int, int, int, int64_t, int, int, int>, NewtonShape> cache;
        const auto ck = std::make_tuple(m->device, m->dim, m->opt.basis, m->opt.precision, m->n_s, m->newton_cols,
                                        ctas, m->batch_share);
        NewtonShape s;
        {
            std::lock_guard<std::mutex> lk(mu);
            auto it = cache.find(ck);
            if (it != cache.end()) s = it->second;
        }
        if (s.ctas == 0) {
            s = newton_shape(m, ctas);
            std::lock_guard<std::mutex> lk(mu);
            cache[ck] = s;
        }
        m->newton_shape_key = key;
        m->newton_ctas = s.ctas;
        m->newton_ppb = s.ppb;
        m->newton_cs = s.cs;
        m->newton_smem = s.smem;
    }
    return m->newton_ctas > 0;
}

void newton_run_level(rbfd_mesh *m, double R, double tau, int ctas) {
    if (!newton_fits(m, ctas)) fail(RBFD_ENOMEM, "Newton greedy: block state exceeds shared memory");
    NewtonShape sh;
    sh.ctas = m->newton_ctas;
    sh.ppb = m->newton_ppb;
    sh.cs = m->newton_cs;
    sh.smem = m->newton_smem;
    NewtonArgs a{};
    a.n_s = m->n_s;
    a.n_pb = m->n_pb;
    a.cap = m->cap;
    a.cn = m->newton_cols;
    a.ppb = sh.ppb;
    a.cs = sh.cs;
    a.R = R;
    a.invR = 1.0 / R;
    a.invR_hi = (float)a.invR;
    a.invR_lo = (float)(a.invR - (double)a.invR_hi);
    a.R2 = R * R;
    a.S0 = m->S0;
    a.tau = tau;
    {
        float rl = (float)(R * (1.0 + 1e-9));
        if ((double)rl < R * (1.0 + 1e-9)) rl = std::nextafter(rl, HUGE_VALF);
        a.Rlist = rl;
        const bool mixed = m->opt.precision != RBFD_FP64;
        const double K_lo = (tau * m->S0) * (tau * m->S0) * (1.0 - 1e-12);
        const double K_hi = (tau * m->S0) * (tau * m->S0) * (1.0 + 1e-12);
        a.key_lo = stop_key(K_lo, mixed, false);
        a.key_hi = stop_key(K_hi, mixed, true);
    }
    a.piv_tol_per_n = 8.0 * 1.1102230246251565e-16;
    a.piv_tol_df_per_n = 5.684341886080802e-14;  // 2^-44
    // (the pruned list sweep made the hand-over pay earlier: on the 60k wing
    // ratios 1.25 to 2 gave 10.46 s against 10.70 s at 3, and below 1.25
    // level 0 left the Newton basis too, 10.72 s)
    a.switch_ratio = 2.0;
    a.switch_work = 2e7;  // ~30 us of FP64 multiply-adds per step
    if (const char *v = std::getenv("RBFD_NEWTON_SWITCH")) a.switch_ratio = std::strtod(v, nullptr);
    a.xs = m->d_xs;
    a.pb_lo = m->d_pb_lo;
    a.pb_hi = m->d_pb_hi;
    a.perm = m->d_perm;
    a.E0 = m->d_cur;
    a.sel = m->d_sel;
    a.nb_cnt = m->d_nb_cnt;
    a.nb_list = m->d_nb_list;
    a.cx = m->d_cx;
    a.alpha = m->d_alpha;
    a.w = m->d_w;
    a.wdf = m->d_nwdf;
    a.cdf = m->d_cdf;
    a.cid = m->d_cid;
    a.G = m->d_G;
    a.Gt = m->d_Gt;
    a.V = m->d_V;
    // per-block records and candidate columns for this grid
    if (m->newton_rec_rows < sh.ctas) {
        dfree(m->d_nrec);
        dfree(m->d_nycol);
        m->d_nrec = nullptr;
        m->d_nycol = nullptr;
        m->newton_rec_rows = 0;
        // records [2][P][3], then the heads [2][P] (16 bytes each: P double4)
        m->d_nrec = dalloc<double4>((size_t)2 * 3 * sh.ctas + sh.ctas, "Newton block records");
        m->d_nycol = dalloc<double>((size_t)2 * sh.ctas * ((size_t)m->newton_cols + 1), "Newton candidate columns");
        m->newton_rec_rows = sh.ctas;
    }
    a.rec = m->d_nrec;
    a.head = reinterpret_cast<ulonglong2 *>(m->d_nrec + (size_t)2 * 3 * m->newton_rec_rows);
    a.ycol = m->d_nycol;
    a.bar = m->d_bar;
    a.spin_limit = 1ull << 24;
    if (const char *v = std::getenv("RBFD_TEST_BARRIER_POLLS")) a.spin_limit = std::strtoull(v, nullptr, 10);
    if (const char *v = std::getenv("RBFD_TEST_SKIP_ARRIVAL")) a.test_skip_arrival = std::atoi(v) != 0;
    a.st = m->d_st;
    a.pairs = m->d_pairs;
    a.phase_ns = m->prof.on ? m->d_phase_ns : nullptr;
    const void *k = select_newton(m->dim, m->opt.basis, m->opt.precision == RBFD_FP64 ? 0 : 1);
    void *args[] = {&a};
    RBFD_CUDA(cudaLaunchCooperativeKernel(k, dim3(sh.ctas), dim3(kNT), args, sh.smem, m->stream));
    m->stats.launches += 1;
    m->stats.persist_ctas = sh.ctas;
}

}  // namespace rbfd
