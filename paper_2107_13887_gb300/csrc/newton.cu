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
// count or V is full.  Everything runs in FP64.
//
// Each block owns fixed groups of 32 surface points and keeps their state in
// shared memory across steps: the first cs columns of V, E, coordinates, the
// running sum s2 = sum_k v_k(x)^2 and the selected flags.  Every candidate
// point therefore knows l^2 = 1 - s2 and w = E / l of its own, and a block
// publishes a complete record of its best candidate (key, position,
// coordinates, l^2, E) plus its column y = V[.][candidate].  Per pass, for the
// control c_j decided in the previous pass:
//   y <- the winner's published column;
//   (a) v_j at the block's points: V[j][i], E_i -= w_j v_j(x_i), s2_i += v_j^2,
//       the block's argmax of |E_i|^2 over unselected points -> its record;
//       c_j appended to the control lists of the point blocks within R;
//   -- arrive at the grid barrier --
//   (b) the growth of the inverse factor for c_j on the rows this block owns
//       (row j of G, column j of G^T: g_k = -(sum_m G_mk y_m) / l_j,
//       alpha_k += w_j g_k): no other block reads them during the launch, so
//       this work overlaps the barrier wait;
//   -- wait --
//   every block reads the P records and takes the same decision: global
//   argmax, stop test |E|max / S0 < tau_l in FP64, pivot test, the next
//   control; block 0 records it.
#include <algorithm>
#include <cmath>
#include <cstdlib>

#include "internal.h"

namespace rbfd {

namespace {

constexpr int kNT = 256;  // threads per block (8 warps)
constexpr int kNW = kNT / 32;

// Argmax by (key, index) with the keys compared as the bit patterns of
// non-negative doubles (same order as the values; -1 marks "none"), so that no
// comparison runs on the narrow FP64 pipe.
__device__ __forceinline__ bool better_bits(long long ka, int ia, long long kb, int ib) {
    return (ka > kb) || (ka == kb && ia < ib && ia >= 0) || (ib < 0 && ia >= 0);
}

__device__ __forceinline__ void block_argmax_bits(long long &k, int &i, long long *sk, int *si) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const long long k2 = __shfl_xor_sync(0xffffffffu, k, o);
        const int i2 = __shfl_xor_sync(0xffffffffu, i, o);
        if (better_bits(k2, i2, k, i)) {
            k = k2;
            i = i2;
        }
    }
    __syncthreads();
    if (lane == 0) {
        sk[w] = k;
        si[w] = i;
    }
    __syncthreads();
    if (w == 0) {
        k = lane < nw ? sk[lane] : (long long)0x8000000000000000ll;
        i = lane < nw ? si[lane] : -1;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const long long k2 = __shfl_xor_sync(0xffffffffu, k, o);
            const int i2 = __shfl_xor_sync(0xffffffffu, i, o);
            if (better_bits(k2, i2, k, i)) {
                k = k2;
                i = i2;
            }
        }
        if (lane == 0) {
            sk[0] = k;
            si[0] = i;
        }
    }
    __syncthreads();
    k = sk[0];
    i = si[0];
}

struct NewtonArgs {
    int64_t n_s;
    int n_pb, cap, cn;  // cn: columns of V (controls the launch may reach)
    int ppb, cs;        // points per block (32 per group), columns of V held in shared memory
    double R, invR, R2, S0, tau, piv_tol_per_n, switch_ratio, switch_work;
    const double4 *xs, *pb_lo, *pb_hi;
    const uint32_t *perm;
    const double4 *E0;  // E at the start of the level (= dS_l)
    unsigned char *sel;
    uint32_t *nb_cnt, *nb_list;
    double4 *cx, *alpha, *w;
    float4 *cdf;
    uint32_t *cid;
    double *G, *Gt, *V;
    double4 *rec;  // [2][P][3] per block: (key, original index, longest list, position), (coordinates, l^2), E
    double *ycol;  // [2][P][cn + 1] per block: V[.][candidate]
    // (two copies, by the parity of the step: a block writes the next step's
    // record while a slower block may still read this step's)
    GridBarrier *bar;
    unsigned long long spin_limit;
    GreedyState *st;
    unsigned long long *pairs;
    unsigned long long *phase_ns;
    int test_skip_arrival;  // tests only: block 0 leaves before its first barrier arrival
};

// Dynamic shared memory of one block: y [cn], V slice [cs][ppb], E [3][ppb],
// coordinates [3][ppb], s2 [ppb], selected flags [ppb].
inline size_t newton_smem_bytes(int cn, int cs, int ppb) {
    return sizeof(double) * ((size_t)cn + (size_t)cs * ppb + 7 * (size_t)ppb) + (size_t)ppb;
}

template <int DIM, int BASIS>
__global__ void __launch_bounds__(kNT) k_greedy_newton(NewtonArgs a) {
    extern __shared__ double dsm[];
    double *s_y = dsm;                         // y of the control being propagated
    double *s_V = s_y + a.cn;                  // V[k][slot], k < cs
    double *s_E = s_V + (size_t)a.cs * a.ppb;  // E of the block's points (x, y, z rows)
    double *s_X = s_E + 3 * a.ppb;             // their coordinates
    double *s_S2 = s_X + 3 * a.ppb;            // sum_k v_k(x)^2
    unsigned char *s_sel = reinterpret_cast<unsigned char *>(s_S2 + a.ppb);
    __shared__ double s_part[kNW][32];
    __shared__ long long sk[32];
    __shared__ int si[32];
    __shared__ double s_dec[8];  // the step's scalars, computed by one warp
    __shared__ int s_flags;
    __shared__ unsigned s_nz[kNW], s_lm[kNW];
    __shared__ int s_win;
    __shared__ double4 s_wrec[3];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned P = gridDim.x;
    const int ppb = a.ppb, n_grp = ppb / 32;
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
        s_X[sl] = x.x;
        s_X[ppb + sl] = x.y;
        s_X[2 * ppb + sl] = x.z;
        s_E[sl] = e.x;
        s_E[ppb + sl] = e.y;
        s_E[2 * ppb + sl] = e.z;
        s_S2[sl] = 0.0;
        s_sel[sl] = valid ? __ldcg(a.sel + i) : 1;
    }
    // control lists: point block t is kept by thread t / P of block t % P
    // (box and count in registers: appends never read back)
    const int t_own = (int)blockIdx.x + tid * (int)P;
    const bool own_list = t_own < a.n_pb;
    double4 own_lo = make_double4(0, 0, 0, 0), own_hi = own_lo;
    uint32_t own_cnt = 0;
    if (own_list) {
        own_lo = a.pb_lo[t_own];
        own_hi = a.pb_hi[t_own];
        own_cnt = __ldcg(&a.nb_cnt[t_own]);
    }
    // the launch starts a level: control 0 placed, nothing propagated yet
    int n = __ldcg(&a.st->n);
    uint32_t cj = __ldcg(&a.cid[0]);
    double4 xcj = ldcg_d4(&a.cx[0]);
    double lj = 1.0, ilj = 1.0;
    double4 wj = ldcg_d4(&a.w[0]);
    int B = -1;  // block whose column is y of c_j
    // counts kept per block and added once at the end: nonzeros of Phi_sc in
    // this block's points so far, and the pairs a list sweep of each step
    // would have evaluated there
    unsigned long long nz_cum = 0, pairs_useful = 0;
    uint32_t list_max = own_list ? own_cnt : 0;  // longest list this block keeps
    // rows of the inverse factor: row k belongs to warp (k / P) % 8 of block k % P
    const int k_first = (int)blockIdx.x + warp * (int)P;
    // profile mode, block 0: [0] y, [1] (a), [2] lists + record, [3] (b),
    // [4] barrier wait, [5] reading the records, [6] their argmax, [7] the rest
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

    for (int guard = 0; guard <= a.cap; ++guard) {
        const int j = n - 1;  // the control this pass propagates
        if (B >= 0) {  // written in the previous pass, parity (j - 1) & 1
            const double *yb = a.ycol + ((size_t)((j - 1) & 1) * P + B) * ycl;
            for (int k = tid; k < j; k += kNT) s_y[k] = __ldcg(&yb[k]);
        }
        {  // the owner marks c_j as selected
            const int64_t item = (int64_t)cj / 32;
            if (tid == 0 && item % P == blockIdx.x) s_sel[(int)(item / P) * 32 + (int)(cj % 32)] = 1;
        }
        __syncthreads();
        RBFD_TMARK(0)

        // ---- (a) v_j at the block's points, E update, argmax
        long long bkey = __double_as_longlong(-1.0);
        int bidx = -1, bslot = -1;
        unsigned nz = 0;
        const int kcs = min(j, a.cs);
        for (int g = 0; g < n_grp; ++g) {
            const int sl = g * 32 + lane;
            const int64_t i = point_of(sl);
            const bool valid = i < a.n_s;
            double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
            if (valid) {
                const double *Vs = s_V + sl;
                int k = warp;
                for (; k + 3 * kNW < kcs; k += 4 * kNW) {
                    s0 = fma(s_y[k], Vs[(size_t)k * ppb], s0);
                    s1 = fma(s_y[k + kNW], Vs[(size_t)(k + kNW) * ppb], s1);
                    s2 = fma(s_y[k + 2 * kNW], Vs[(size_t)(k + 2 * kNW) * ppb], s2);
                    s3 = fma(s_y[k + 3 * kNW], Vs[(size_t)(k + 3 * kNW) * ppb], s3);
                }
                for (; k < kcs; k += kNW) s0 = fma(s_y[k], Vs[(size_t)k * ppb], s0);
                // columns beyond the shared slice come from global memory
                const double *Vi = a.V + i;
                const size_t ld = (size_t)a.n_s;
                for (; k + 3 * kNW < j; k += 4 * kNW) {
                    const double v0 = __ldcg(Vi + (size_t)k * ld), v1 = __ldcg(Vi + (size_t)(k + kNW) * ld),
                                 v2 = __ldcg(Vi + (size_t)(k + 2 * kNW) * ld),
                                 v3 = __ldcg(Vi + (size_t)(k + 3 * kNW) * ld);
                    s0 = fma(s_y[k], v0, s0);
                    s1 = fma(s_y[k + kNW], v1, s1);
                    s2 = fma(s_y[k + 2 * kNW], v2, s2);
                    s3 = fma(s_y[k + 3 * kNW], v3, s3);
                }
                for (; k < j; k += kNW) s0 = fma(s_y[k], __ldcg(Vi + (size_t)k * ld), s0);
            }
            s_part[warp][lane] = (s0 + s1) + (s2 + s3);
            __syncthreads();
            if (warp == 0 && valid) {
                double sum = s_part[0][lane];
#pragma unroll
                for (int w8 = 1; w8 < kNW; ++w8) sum += s_part[w8][lane];
                const double f = phi_f64<BASIS>(
                    dist_f64<DIM>(s_X[sl], s_X[ppb + sl], s_X[2 * ppb + sl], xcj.x, xcj.y, xcj.z) * a.invR);
                nz += (f != 0.0);
                const double v = (f - sum) * ilj;
                if (j < a.cs) s_V[(size_t)j * ppb + sl] = v;
                a.V[(size_t)j * a.n_s + i] = v;
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
                if (!s_sel[sl]) {
                    const int o = (int)a.perm[i];
                    const long long kb = __double_as_longlong(k2);
                    if (better_bits(kb, o, bkey, bidx)) {
                        bkey = kb;
                        bidx = o;
                        bslot = sl;
                    }
                }
            }
            __syncthreads();
        }
        RBFD_TMARK(1)

        // ---- lists (control 0: listed at level start), nonzero count, the block's record
        if (j > 0 && own_list) {
            const double dx = fmax(fmax(own_lo.x - xcj.x, xcj.x - own_hi.x), 0.0);
            const double dy = fmax(fmax(own_lo.y - xcj.y, xcj.y - own_hi.y), 0.0);
            const double dz = DIM == 3 ? fmax(fmax(own_lo.z - xcj.z, xcj.z - own_hi.z), 0.0) : 0.0;
            if (dx * dx + dy * dy + dz * dz < a.R2 * (1.0 + 1e-9)) {
                a.nb_list[(size_t)t_own * a.cap + own_cnt] = (uint32_t)j;
                ++own_cnt;
                a.nb_cnt[t_own] = own_cnt;
            }
        }
        {
            long long kk = bkey;
            int ii = bidx;
            block_argmax_bits(kk, ii, sk, si);  // (ends with __syncthreads)
            if (ii >= 0 && bidx == ii) s_win = bslot;  // the one thread holding it
            unsigned u = nz;
            for (int o = 16; o > 0; o >>= 1) u += __shfl_xor_sync(0xffffffffu, u, o);
            unsigned lm = own_list ? own_cnt : 0u;
            for (int o = 16; o > 0; o >>= 1) lm = max(lm, __shfl_xor_sync(0xffffffffu, lm, o));
            if (lane == 0) {
                s_nz[warp] = u;
                s_lm[warp] = lm;
            }
            __syncthreads();
            const int ws = ii >= 0 ? s_win : -1;
            if (tid == 0) {
                unsigned bnz = 0;
                for (int w8 = 0; w8 < kNW; ++w8) {
                    bnz += s_nz[w8];
                    list_max = max(list_max, s_lm[w8]);
                }
                nz_cum += bnz;
                pairs_useful += nz_cum;  // the list sweep of this step would evaluate these pairs
                double4 *r = a.rec + 3 * ((size_t)(j & 1) * P + blockIdx.x);
                if (ws >= 0) {
                    r[0] = make_double4(__longlong_as_double(kk), (double)ii, (double)list_max, (double)point_of(ws));
                    r[1] = make_double4(s_X[ws], s_X[ppb + ws], s_X[2 * ppb + ws], 1.0 - s_S2[ws]);
                    r[2] = make_double4(s_E[ws], s_E[ppb + ws], s_E[2 * ppb + ws], 0.0);
                } else {
                    r[0] = make_double4(-1.0, -1.0, (double)list_max, -1.0);
                }
            }
            if (ws >= 0) {  // the candidate's column: y of the next control if it wins
                const int64_t pw = point_of(ws);
                double *yc = a.ycol + ((size_t)(j & 1) * P + blockIdx.x) * ycl;
                for (int k = tid; k <= j; k += kNT)
                    yc[k] = k < a.cs ? s_V[(size_t)k * ppb + ws] : __ldcg(a.V + (size_t)k * a.n_s + pw);
            }
        }
        RBFD_TMARK(2)
        if (a.test_skip_arrival && blockIdx.x == 0) return;  // the others' waits run out
        const unsigned gen = grid_arrive(a.bar, P);

        // ---- (b) row j of the inverse factor on this block's rows, alpha
        for (int k = k_first; k <= j; k += (int)P * kNW) {
            if (k == j) {  // the diagonal and alpha_j
                if (lane == 0) {
                    a.G[(size_t)j * a.cap + j] = ilj;
                    a.Gt[(size_t)j * a.cap + j] = ilj;
                    a.alpha[j] = make_double4(wj.x * ilj, wj.y * ilj, wj.z * ilj, 0.0);
                }
                break;
            }
            const double *trow = a.Gt + (size_t)k * a.cap;
            double4 al = make_double4(0, 0, 0, 0);
            if (lane == 0) al = ldcg_d4(&a.alpha[k]);
            double t0 = 0.0, t1 = 0.0, t2 = 0.0, t3 = 0.0;
            int m = k + lane;
            for (; m + 96 < j; m += 128) {
                t0 = fma(__ldcg(trow + m), s_y[m], t0);
                t1 = fma(__ldcg(trow + m + 32), s_y[m + 32], t1);
                t2 = fma(__ldcg(trow + m + 64), s_y[m + 64], t2);
                t3 = fma(__ldcg(trow + m + 96), s_y[m + 96], t3);
            }
            for (; m < j; m += 32) t0 = fma(__ldcg(trow + m), s_y[m], t0);
            const double t = warp_sum_d((t0 + t1) + (t2 + t3));
            if (lane == 0) {
                const double gk = -t * ilj;
                a.G[(size_t)j * a.cap + k] = gk;
                a.Gt[(size_t)k * a.cap + j] = gk;
                al.x = fma(wj.x, gk, al.x);
                al.y = fma(wj.y, gk, al.y);
                al.z = fma(wj.z, gk, al.z);
                a.alpha[k] = al;
            }
        }
        RBFD_TMARK(3)
        if (!grid_wait(a.bar, gen, a.spin_limit)) RBFD_NEXIT()
        RBFD_TMARK(4)

        // ---- the step's decision: every block from the same records
        long long K = __double_as_longlong(-1.0);
        int I = -1, Bw = -1;
        unsigned lmax = 0;
        double4 r0 = make_double4(0, 0, 0, 0), r1 = r0, r2 = r0;
        const double4 *rj = a.rec + 3 * (size_t)(j & 1) * P;
        for (unsigned b = tid; b < P; b += kNT) {
            const double4 q0 = ldcg_d4(&rj[3 * (size_t)b]);
            const double4 q1 = ldcg_d4(&rj[3 * (size_t)b + 1]);
            const double4 q2 = ldcg_d4(&rj[3 * (size_t)b + 2]);
            lmax = max(lmax, (unsigned)q0.z);
            const int ib = (int)q0.y;
            const long long kb = __double_as_longlong(q0.x);
            if (better_bits(kb, ib, K, I)) {
                K = kb;
                I = ib;
                Bw = (int)b;
                r0 = q0;
                r1 = q1;
                r2 = q2;
            }
        }
        for (int o = 16; o > 0; o >>= 1) lmax = max(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
        if (lane == 0) s_lm[warp] = lmax;
        RBFD_TMARK(5)
        {
            const long long kk = K;
            const int ii = I;
            block_argmax_bits(K, I, sk, si);  // (its barriers also publish s_lm)
            if (I >= 0 && ii == I && kk == K) {
                s_win = Bw;
                s_wrec[0] = r0;
                s_wrec[1] = r1;
                s_wrec[2] = r2;
            }
            __syncthreads();
        }
        RBFD_TMARK(6)
        // the step's scalars in FP64, on one warp
        const int nn = n;  // index the next control takes
        if (warp == 0) {
            int mc = 1;
            for (int w8 = 0; w8 < kNW; ++w8) mc = max(mc, (int)s_lm[w8]);
            const double Kd = __longlong_as_double(K);
            const double e = I >= 0 ? __ddiv_rn(__dsqrt_rn(Kd), a.S0) : 0.0;
            const bool stop = I < 0 || e < a.tau || nn >= a.cap;
            // hand over to the list sweep when V is full, or when the Newton
            // update (n_s * n multiply-adds) is large and the lists are much
            // shorter than the control count
            const bool hand = !stop && (nn >= a.cn || ((double)a.n_s * nn > a.switch_work &&
                                                       (double)nn > a.switch_ratio * (double)mc));
            const double l2 = stop ? 1.0 : s_wrec[1].w;
            const bool singular = !stop && !hand && !(l2 > a.piv_tol_per_n * (nn + 1));
            if (lane == 0) {
                s_flags = (stop ? 1 : 0) | (hand ? 2 : 0) | (singular ? 4 : 0);
                s_dec[0] = e;
                s_dec[1] = (double)mc;
                if (!(stop || hand || singular)) {
                    const double l = sqrt(l2), il = 1.0 / l;
                    s_dec[2] = l;
                    s_dec[3] = il;
                    s_dec[4] = s_wrec[2].x * il;
                    s_dec[5] = s_wrec[2].y * il;
                    s_dec[6] = s_wrec[2].z * il;
                }
            }
        }
        __syncthreads();
        const int flags = s_flags;
        const bool writer = blockIdx.x == 0 && tid == 0;
        if (flags) {
            if (tid == 0) {
                atomicAdd(&a.pairs[0], pairs_useful);
                if (writer) {
                    const bool stop = flags & 1, hand = flags & 2, singular = flags & 4;
                    const double e = s_dec[0];
                    // a list sweep visits n_s x (controls so far) pairs per step
                    a.pairs[1] += (unsigned long long)a.n_s * (unsigned long long)(nn) * (unsigned long long)(nn + 1) / 2;
                    a.st->best_orig = I;
                    a.st->best_key = __longlong_as_double(K);
                    a.st->emax = e;
                    a.st->max_cnt = (int)s_dec[1];
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
        const double4 wr0 = s_wrec[0], wr1 = s_wrec[1], wr2 = s_wrec[2];
        B = s_win;
        xcj = make_double4(wr1.x, wr1.y, wr1.z, 0.0);
        cj = (uint32_t)wr0.w;
        lj = s_dec[2];
        ilj = s_dec[3];
        wj = make_double4(s_dec[4], s_dec[5], s_dec[6], 0.0);
        (void)wr2;
        if (writer) {
            const float hx = __double2float_rn(xcj.x), hy = __double2float_rn(xcj.y), hz = __double2float_rn(xcj.z);
            a.sel[cj] = 1;
            a.cx[nn] = xcj;
            a.cdf[nn] = make_float4(hx, hy, hz, 0.f);
            a.cdf[a.cap + 1 + nn] = make_float4(__double2float_rn(xcj.x - (double)hx),
                                                __double2float_rn(xcj.y - (double)hy),
                                                __double2float_rn(xcj.z - (double)hz), 0.f);
            a.cid[nn] = cj;
            a.w[nn] = wj;
        }
        ++n;
        RBFD_TMARK(7)
        __syncthreads();  // shared scratch is reused
    }
    RBFD_NEXIT()
#undef RBFD_NEXIT
#undef RBFD_TMARK
}

template <int DIM, int BASIS>
const void *newton_ptr() {
    return reinterpret_cast<const void *>(&k_greedy_newton<DIM, BASIS>);
}

const void *select_newton(int dim, int basis) {
#define RBFD_SEL(D, B) \
    if (dim == D && basis == B) return newton_ptr<D, B>();
    RBFD_SEL(2, 0) RBFD_SEL(2, 2) RBFD_SEL(2, 4) RBFD_SEL(2, 6)
    RBFD_SEL(3, 0) RBFD_SEL(3, 2) RBFD_SEL(3, 4) RBFD_SEL(3, 6)
#undef RBFD_SEL
    return nullptr;
}

}  // namespace

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
}

// Blocks and shared-memory layout of a launch on this mesh: ppb points per
// block, cs columns of V in shared memory (the rest is read from HBM).
struct NewtonShape {
    int ctas = 0, ppb = 0, cs = 0;
    size_t smem = 0;
};

NewtonShape newton_shape(rbfd_mesh *m, int want_ctas) {
    const void *k = select_newton(m->dim, m->opt.basis);
    static const size_t kSmemMax = 220 * 1024;  // dynamic shared memory per block (of 227 KB)
    NewtonShape s;
    int sms = 0;
    RBFD_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, m->device));
    const int64_t items = (m->n_s + 31) / 32;
    int ctas = (int)std::max<int64_t>(1, std::min<int64_t>(want_ctas, items));
    // meshes running side by side (batch calls, server slots) share the SMs:
    // one block per SM each, so that their launches stay resident together
    if (m->batch_share > 1) ctas = std::min(ctas, std::max(1, sms / m->batch_share));
    // one value for every launch: the attribute belongs to the kernel, and
    // meshes on other host threads launch it concurrently
    RBFD_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemMax));
    for (;;) {
        const int ppb = (int)(32 * ((items + ctas - 1) / ctas));
        const size_t fixed = newton_smem_bytes(m->newton_cols, 0, ppb);
        if (fixed > kSmemMax) fail(RBFD_ENOMEM, "Newton greedy: block state exceeds shared memory");
        const int cs = (int)std::min<size_t>((size_t)m->newton_cols, (kSmemMax - fixed) / (sizeof(double) * ppb));
        const size_t smem = newton_smem_bytes(m->newton_cols, cs, ppb);
        int occ = 0;
        RBFD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, kNT, smem));
        const int maxc = std::min(occ * sms, kMaxPersistCTAs);
        if (maxc < 1) fail(RBFD_ECUDA, "Newton greedy kernel cannot be resident on this device");
        if (ctas <= maxc) {
            s.ctas = ctas;
            s.ppb = ppb;
            s.cs = cs;
            s.smem = smem;
            return s;
        }
        ctas = maxc;  // fewer blocks, more points each
    }
}

void newton_run_level(rbfd_mesh *m, double R, double tau, int ctas) {
    const NewtonShape sh = newton_shape(m, ctas);
    NewtonArgs a{};
    a.n_s = m->n_s;
    a.n_pb = m->n_pb;
    a.cap = m->cap;
    a.cn = m->newton_cols;
    a.ppb = sh.ppb;
    a.cs = sh.cs;
    a.R = R;
    a.invR = 1.0 / R;
    a.R2 = R * R;
    a.S0 = m->S0;
    a.tau = tau;
    a.piv_tol_per_n = 8.0 * 1.1102230246251565e-16;
    a.switch_ratio = 3.0;
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
        m->d_nrec = dalloc<double4>((size_t)2 * 3 * sh.ctas, "Newton block records");
        m->d_nycol = dalloc<double>((size_t)2 * sh.ctas * ((size_t)m->newton_cols + 1), "Newton candidate columns");
        m->newton_rec_rows = sh.ctas;
    }
    a.rec = m->d_nrec;
    a.ycol = m->d_nycol;
    a.bar = m->d_bar;
    a.spin_limit = 1ull << 24;
    if (const char *v = std::getenv("RBFD_TEST_BARRIER_POLLS")) a.spin_limit = std::strtoull(v, nullptr, 10);
    if (const char *v = std::getenv("RBFD_TEST_SKIP_ARRIVAL")) a.test_skip_arrival = std::atoi(v) != 0;
    a.st = m->d_st;
    a.pairs = m->d_pairs;
    a.phase_ns = m->prof.on ? m->d_phase_ns : nullptr;
    const void *k = select_newton(m->dim, m->opt.basis);
    void *args[] = {&a};
    RBFD_CUDA(cudaLaunchCooperativeKernel(k, dim3(sh.ctas), dim3(kNT), args, sh.smem, m->stream));
    m->stats.launches += 1;
    m->stats.persist_ctas = sh.ctas;
}

}  // namespace rbfd
