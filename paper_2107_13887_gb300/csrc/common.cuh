// common.cuh -- device helpers shared by the rbfd CUDA kernels (sm_103a).
//
// Contents:
//   * status codes mirrored from include/rbfd.h;
//   * IEEE double evaluation of the Wendland basis (Table 1, Eq. 2) with every
//     product and sum separately rounded (no FMA contraction), so FP64 mode
//     evaluates eta and phi exactly as the textbook formula is written;
//   * double-float ("df") arithmetic: an unevaluated sum hi + lo of two
//     floats carrying ~44-48 significant bits, built from the classical
//     error-free transformations (Knuth's TwoSum, Dekker's Fast2Sum and the
//     FMA-based TwoProduct).  It runs on the FP32 pipe, which on GB300 issues
//     ~64x more operations per clock than the FP64 pipe;
//   * warp / block reduction helpers and the (key, index) argmax order used
//     by the greedy selection (largest key, then lowest surface index).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/rbfd.h"

namespace rbfd {

constexpr int kPB = 128;      // surface / volume points per block (one per thread)
constexpr int kTile = 128;    // controls staged in shared memory per tile
constexpr int kMaxBasis = 6;

// ------------------------------------------------------------------ FP64 path

// phi(eta) of Table 1 in IEEE double, each operation rounded on its own.
template <int BASIS>
__device__ __forceinline__ double phi_f64(double eta) {
    if (eta >= 1.0) return 0.0;
    double t = __dsub_rn(1.0, eta);
    double t2 = __dmul_rn(t, t);
    if (BASIS == 0) return t2;
    double t4 = __dmul_rn(t2, t2);
    if (BASIS == 2) return __dmul_rn(t4, __dadd_rn(__dmul_rn(4.0, eta), 1.0));
    if (BASIS == 4) {
        double t6 = __dmul_rn(t4, t2);
        double q = __dadd_rn(__dadd_rn(__dmul_rn(__dmul_rn(35.0 / 3.0, eta), eta), __dmul_rn(6.0, eta)), 1.0);
        return __dmul_rn(t6, q);
    }
    double t8 = __dmul_rn(t4, t4);
    double e2 = __dmul_rn(eta, eta);
    double q = __dadd_rn(__dadd_rn(__dadd_rn(__dmul_rn(__dmul_rn(32.0, e2), eta), __dmul_rn(25.0, e2)),
                                   __dmul_rn(8.0, eta)),
                         1.0);
    return __dmul_rn(t8, q);
}

// |a - b|_2^2 summed in coordinate order, no contraction.
template <int DIM>
__device__ __forceinline__ double dist2_f64(double ax, double ay, double az, double bx, double by, double bz) {
    double dx = __dsub_rn(ax, bx);
    double s = __dmul_rn(dx, dx);
    double dy = __dsub_rn(ay, by);
    s = __dadd_rn(s, __dmul_rn(dy, dy));
    if (DIM == 3) {
        double dz = __dsub_rn(az, bz);
        s = __dadd_rn(s, __dmul_rn(dz, dz));
    }
    return s;
}

// |a - b|_2 (the square root of dist2_f64).
template <int DIM>
__device__ __forceinline__ double dist_f64(double ax, double ay, double az, double bx, double by, double bz) {
    return __dsqrt_rn(dist2_f64<DIM>(ax, ay, az, bx, by, bz));
}

// ------------------------------------------------------------ double-float

struct df {
    float hi, lo;
};

// Knuth TwoSum: s + e == a + b exactly.
__device__ __forceinline__ df two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

// Dekker Fast2Sum (requires |a| >= |b| or a == 0).
__device__ __forceinline__ df fast_two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float e = __fsub_rn(b, __fsub_rn(s, a));
    return {s, e};
}

// TwoProduct with one fused multiply-add: p + e == a * b exactly.
__device__ __forceinline__ df two_prod(float a, float b) {
    float p = __fmul_rn(a, b);
    float e = __fmaf_rn(a, b, -p);
    return {p, e};
}

__device__ __forceinline__ df df_add(df a, df b) {
    df s = two_sum(a.hi, b.hi);
    df t = two_sum(a.lo, b.lo);
    float lo = __fadd_rn(s.lo, t.hi);
    s = fast_two_sum(s.hi, lo);
    lo = __fadd_rn(s.lo, t.lo);
    return fast_two_sum(s.hi, lo);
}

__device__ __forceinline__ df df_neg(df a) { return {-a.hi, -a.lo}; }

__device__ __forceinline__ df df_mul(df a, df b) {
    df p = two_prod(a.hi, b.hi);
    float lo = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, p.lo));
    return fast_two_sum(p.hi, lo);
}

__device__ __forceinline__ df df_sqr(df a) {
    df p = two_prod(a.hi, a.hi);
    float lo = __fmaf_rn(__fmul_rn(2.0f, a.hi), a.lo, p.lo);
    return fast_two_sum(p.hi, lo);
}

// sqrt of a double-float: a single-precision estimate s = a.hi * rsqrt(a.hi),
// then one Newton correction s + (a - s^2) / (2 s) with the residual formed
// exactly through TwoProduct.
__device__ __forceinline__ df df_sqrt(df a) {
    if (!(a.hi > 0.0f)) return {0.0f, 0.0f};
    float y = rsqrtf(a.hi);
    float s = __fmul_rn(a.hi, y);
    df p = two_prod(s, s);
    float r = __fadd_rn(__fsub_rn(__fsub_rn(a.hi, p.hi), p.lo), a.lo);
    float c = __fmul_rn(r, __fmul_rn(0.5f, y));
    return fast_two_sum(s, c);
}

__device__ __forceinline__ df df_from_double(double x) {
    float hi = __double2float_rn(x);
    float lo = __double2float_rn(x - (double)hi);
    return {hi, lo};
}

__device__ __forceinline__ double df_to_double(df a) { return (double)a.hi + (double)a.lo; }

// phi(eta) of Table 1 in double-float; eta >= 1 gives exactly 0.
template <int BASIS>
__device__ __forceinline__ df phi_df(df eta) {
    if (!(eta.hi < 1.0f)) return {0.0f, 0.0f};
    df t = df_add({1.0f, 0.0f}, df_neg(eta));
    df t2 = df_sqr(t);
    if (BASIS == 0) return t2;
    df t4 = df_sqr(t2);
    if (BASIS == 2) {
        df q = df_add({__fmul_rn(4.0f, eta.hi), __fmul_rn(4.0f, eta.lo)}, {1.0f, 0.0f});
        return df_mul(t4, q);
    }
    if (BASIS == 4) {
        df t6 = df_mul(t4, t2);
        df e2 = df_sqr(eta);
        const df c35_3 = {11.666666984558105f, -3.1789145e-07f};  // 35/3 as hi + lo
        df q = df_add(df_add(df_mul(c35_3, e2), {__fmul_rn(6.0f, eta.hi), __fmul_rn(6.0f, eta.lo)}), {1.0f, 0.0f});
        return df_mul(t6, q);
    }
    df t8 = df_sqr(t4);
    df e2 = df_sqr(eta);
    df e3 = df_mul(e2, eta);
    df q = df_add(df_add(df_add({__fmul_rn(32.0f, e3.hi), __fmul_rn(32.0f, e3.lo)},
                                df_mul({25.0f, 0.0f}, e2)),
                         {__fmul_rn(8.0f, eta.hi), __fmul_rn(8.0f, eta.lo)}),
                  {1.0f, 0.0f});
    return df_mul(t8, q);
}

// An upper bound on phi(eta) of Table 1 from FP32 arithmetic: eta is taken
// 2^-20 smaller (phi decreases on [0, 1]) and the value 2^-18 larger, more
// than the rounding of the dozen FP32 operations (each within 2^-24).
template <int BASIS>
__device__ __forceinline__ float phi_f32_upper(float eta) {
    eta = fmaxf(eta * (1.0f - 0x1p-20f), 0.0f);
    if (!(eta < 1.0f)) return 0.0f;
    const float t = 1.0f - eta, t2 = t * t;
    float v;
    if (BASIS == 0) {
        v = t2;
    } else if (BASIS == 2) {
        v = (t2 * t2) * (4.0f * eta + 1.0f);
    } else if (BASIS == 4) {
        v = (t2 * t2 * t2) * ((35.0f / 3.0f) * eta * eta + 6.0f * eta + 1.0f);
    } else {
        const float t4 = t2 * t2;
        v = (t4 * t4) * (((32.0f * eta + 25.0f) * eta + 8.0f) * eta + 1.0f);
    }
    return fminf(v * (1.0f + 0x1p-18f), 1.0f);
}

// One pair of the double-float evaluation: phi(|q - c| / R) for a point q and
// a control c, both given relative to the same origin as (hi, lo) floats.
// t32 holds the staged controls: rows 0..5 = x hi, x lo, y hi, y lo, z hi, z lo.
template <int DIM, int BASIS>
__device__ __forceinline__ df pair_phi_df(df qx, df qy, df qz, const float (*t32)[kTile], int q, df invR,
                                          unsigned &useful) {
    df dx = df_add(qx, {-t32[0][q], -t32[1][q]});
    df dy = df_add(qy, {-t32[2][q], -t32[3][q]});
    df r2 = df_add(df_sqr(dx), df_sqr(dy));
    if (DIM == 3) {
        df dz = df_add(qz, {-t32[4][q], -t32[5][q]});
        r2 = df_add(r2, df_sqr(dz));
    }
    df eta = df_mul(df_sqrt(r2), invR);
    useful += (eta.hi < 1.0f);
    return phi_df<BASIS>(eta);
}

// Accumulate sum_q alpha_q phi_q over the m staged controls of a tile, in
// order q = 0, 1, ..., two pairs per iteration so that the compiler can
// interleave their independent instruction chains (one warp per scheduler
// has nothing else to hide the FP32 latencies with).  Rows 6..11 of t32 are
// alpha x hi, lo, y hi, lo, z hi, lo.
template <int DIM, int BASIS>
__device__ __forceinline__ void tile_accumulate_df(df qx, df qy, df qz, const float (*t32)[kTile], int m,
                                                   df invR, df acc[3], unsigned &useful) {
    int q = 0;
    for (; q + 2 <= m; q += 2) {
        const df f0 = pair_phi_df<DIM, BASIS>(qx, qy, qz, t32, q, invR, useful);
        const df f1 = pair_phi_df<DIM, BASIS>(qx, qy, qz, t32, q + 1, invR, useful);
        acc[0] = df_add(acc[0], df_mul(f0, {t32[6][q], t32[7][q]}));
        acc[1] = df_add(acc[1], df_mul(f0, {t32[8][q], t32[9][q]}));
        if (DIM == 3) acc[2] = df_add(acc[2], df_mul(f0, {t32[10][q], t32[11][q]}));
        acc[0] = df_add(acc[0], df_mul(f1, {t32[6][q + 1], t32[7][q + 1]}));
        acc[1] = df_add(acc[1], df_mul(f1, {t32[8][q + 1], t32[9][q + 1]}));
        if (DIM == 3) acc[2] = df_add(acc[2], df_mul(f1, {t32[10][q + 1], t32[11][q + 1]}));
    }
    if (q < m) {
        const df f0 = pair_phi_df<DIM, BASIS>(qx, qy, qz, t32, q, invR, useful);
        acc[0] = df_add(acc[0], df_mul(f0, {t32[6][q], t32[7][q]}));
        acc[1] = df_add(acc[1], df_mul(f0, {t32[8][q], t32[9][q]}));
        if (DIM == 3) acc[2] = df_add(acc[2], df_mul(f0, {t32[10][q], t32[11][q]}));
    }
}

// Bounding box of the warp's valid points (coordinates relative to the block
// origin, hi parts), for the per-warp control filter below.
__device__ __forceinline__ void warp_box(bool valid, float x, float y, float z, float3 &lo, float3 &hi) {
    lo = valid ? make_float3(x, y, z) : make_float3(INFINITY, INFINITY, INFINITY);
    hi = valid ? make_float3(x, y, z) : make_float3(-INFINITY, -INFINITY, -INFINITY);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lo.x = fminf(lo.x, __shfl_xor_sync(0xffffffffu, lo.x, o));
        lo.y = fminf(lo.y, __shfl_xor_sync(0xffffffffu, lo.y, o));
        lo.z = fminf(lo.z, __shfl_xor_sync(0xffffffffu, lo.z, o));
        hi.x = fmaxf(hi.x, __shfl_xor_sync(0xffffffffu, hi.x, o));
        hi.y = fmaxf(hi.y, __shfl_xor_sync(0xffffffffu, hi.y, o));
        hi.z = fmaxf(hi.z, __shfl_xor_sync(0xffffffffu, hi.z, o));
    }
}

// Indices of the staged controls (of m) that lie within R of the warp's box
// (squared box distance below R2m, which carries a safety margin): a
// warp-uniform filter, so the warp skips controls none of its points can
// reach.  Writes them in order into hits[] and returns how many.
template <int DIM>
__device__ __forceinline__ int warp_hits(const float (*t32)[kTile], int m, float3 lo, float3 hi, float R2m,
                                         unsigned char *hits) {
    const int lane = threadIdx.x & 31;
    int cnt = 0;
    for (int base = 0; base < m; base += 32) {
        const int q = base + lane;
        bool in = false;
        if (q < m) {
            const float cx = t32[0][q], cy = t32[2][q];
            const float dx = fmaxf(fmaxf(lo.x - cx, cx - hi.x), 0.0f);
            const float dy = fmaxf(fmaxf(lo.y - cy, cy - hi.y), 0.0f);
            float d2 = dx * dx + dy * dy;
            if (DIM == 3) {
                const float cz = t32[4][q];
                const float dz = fmaxf(fmaxf(lo.z - cz, cz - hi.z), 0.0f);
                d2 += dz * dz;
            }
            in = d2 < R2m;
        }
        const unsigned b = __ballot_sync(0xffffffffu, in);
        if (in) hits[cnt + __popc(b & ((1u << lane) - 1u))] = (unsigned char)q;
        cnt += __popc(b);
    }
    __syncwarp();
    return cnt;
}

// tile_accumulate_df over the filtered controls hits[0..cnt) of a tile.
template <int DIM, int BASIS>
__device__ __forceinline__ void hits_accumulate_df(df qx, df qy, df qz, const float (*t32)[kTile],
                                                   const unsigned char *hits, int cnt, df invR, df acc[3],
                                                   unsigned &useful) {
    int i = 0;
    for (; i + 2 <= cnt; i += 2) {
        const int q0 = hits[i], q1 = hits[i + 1];
        const df f0 = pair_phi_df<DIM, BASIS>(qx, qy, qz, t32, q0, invR, useful);
        const df f1 = pair_phi_df<DIM, BASIS>(qx, qy, qz, t32, q1, invR, useful);
        acc[0] = df_add(acc[0], df_mul(f0, {t32[6][q0], t32[7][q0]}));
        acc[1] = df_add(acc[1], df_mul(f0, {t32[8][q0], t32[9][q0]}));
        if (DIM == 3) acc[2] = df_add(acc[2], df_mul(f0, {t32[10][q0], t32[11][q0]}));
        acc[0] = df_add(acc[0], df_mul(f1, {t32[6][q1], t32[7][q1]}));
        acc[1] = df_add(acc[1], df_mul(f1, {t32[8][q1], t32[9][q1]}));
        if (DIM == 3) acc[2] = df_add(acc[2], df_mul(f1, {t32[10][q1], t32[11][q1]}));
    }
    if (i < cnt) {
        const int q0 = hits[i];
        const df f0 = pair_phi_df<DIM, BASIS>(qx, qy, qz, t32, q0, invR, useful);
        acc[0] = df_add(acc[0], df_mul(f0, {t32[6][q0], t32[7][q0]}));
        acc[1] = df_add(acc[1], df_mul(f0, {t32[8][q0], t32[9][q0]}));
        if (DIM == 3) acc[2] = df_add(acc[2], df_mul(f0, {t32[10][q0], t32[11][q0]}));
    }
}

// hits_accumulate_df that also sums phi |alpha|_1 in FP32 (row 12 of t32:
// |alpha_x| + |alpha_y| + |alpha_z| rounded up), the scale of the sum's
// rounding that the pruned sweep's bounds need.
template <int DIM, int BASIS>
__device__ __forceinline__ void hits_accumulate_df_abs(df qx, df qy, df qz, const float (*t32)[kTile],
                                                       const unsigned char *hits, int cnt, df invR, df acc[3],
                                                       unsigned &useful, float &sabs) {
    int i = 0;
    for (; i + 2 <= cnt; i += 2) {
        const int q0 = hits[i], q1 = hits[i + 1];
        const df f0 = pair_phi_df<DIM, BASIS>(qx, qy, qz, t32, q0, invR, useful);
        const df f1 = pair_phi_df<DIM, BASIS>(qx, qy, qz, t32, q1, invR, useful);
        acc[0] = df_add(acc[0], df_mul(f0, {t32[6][q0], t32[7][q0]}));
        acc[1] = df_add(acc[1], df_mul(f0, {t32[8][q0], t32[9][q0]}));
        if (DIM == 3) acc[2] = df_add(acc[2], df_mul(f0, {t32[10][q0], t32[11][q0]}));
        acc[0] = df_add(acc[0], df_mul(f1, {t32[6][q1], t32[7][q1]}));
        acc[1] = df_add(acc[1], df_mul(f1, {t32[8][q1], t32[9][q1]}));
        if (DIM == 3) acc[2] = df_add(acc[2], df_mul(f1, {t32[10][q1], t32[11][q1]}));
        sabs = fmaf(f0.hi, t32[12][q0], sabs);
        sabs = fmaf(f1.hi, t32[12][q1], sabs);
    }
    if (i < cnt) {
        const int q0 = hits[i];
        const df f0 = pair_phi_df<DIM, BASIS>(qx, qy, qz, t32, q0, invR, useful);
        acc[0] = df_add(acc[0], df_mul(f0, {t32[6][q0], t32[7][q0]}));
        acc[1] = df_add(acc[1], df_mul(f0, {t32[8][q0], t32[9][q0]}));
        if (DIM == 3) acc[2] = df_add(acc[2], df_mul(f0, {t32[10][q0], t32[11][q0]}));
        sabs = fmaf(f0.hi, t32[12][q0], sabs);
    }
}

// L2-coherent load of a double4 written by another block of the same launch.
__device__ __forceinline__ double4 ldcg_d4(const double4 *p) {
    const double2 *q = reinterpret_cast<const double2 *>(p);
    double2 a = __ldcg(q), b = __ldcg(q + 1);
    return make_double4(a.x, a.y, b.x, b.y);
}

// ------------------------------------------------------------------ argmax

// Order of the greedy selection: larger key first, then lower surface index.
__device__ __forceinline__ bool better(double ka, int ia, double kb, int ib) {
    return (ka > kb) || (ka == kb && ia < ib && ia >= 0) || (ib < 0 && ia >= 0);
}

__device__ __forceinline__ void warp_argmax(double &k, int &i) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        double k2 = __shfl_xor_sync(0xffffffffu, k, o);
        int i2 = __shfl_xor_sync(0xffffffffu, i, o);
        if (better(k2, i2, k, i)) {
            k = k2;
            i = i2;
        }
    }
}

// Block-wide argmax over (key, idx); every thread gets the result.
// scratch must hold 2 * 32 entries.
__device__ __forceinline__ void block_argmax(double &k, int &i, double *sk, int *si) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    warp_argmax(k, i);
    __syncthreads();
    if (lane == 0) {
        sk[w] = k;
        si[w] = i;
    }
    __syncthreads();
    if (w == 0) {
        k = lane < nw ? sk[lane] : -1.0;
        i = lane < nw ? si[lane] : -1;
        warp_argmax(k, i);
        if (lane == 0) {
            sk[0] = k;
            si[0] = i;
        }
    }
    __syncthreads();
    k = sk[0];
    i = si[0];
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide exclusive scan of one unsigned per thread (blockDim a multiple
// of 32); *total receives the block sum.  sw: 32 words of shared scratch.
__device__ __forceinline__ unsigned block_excl_scan_u32(unsigned v, unsigned *sw, unsigned *total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    unsigned x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sw[w] = x;
    __syncthreads();
    if (w == 0) {
        unsigned t = lane < nw ? sw[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            unsigned y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < nw) sw[lane] = t;
    }
    __syncthreads();
    const unsigned before = (w > 0 ? sw[w - 1] : 0u) + x - v;
    *total = sw[nw - 1];
    __syncthreads();
    return before;
}

// ---------------------------------------------------------- greedy state

// Device-resident state of one greedy level (lives in device memory; a
// pinned host mirror is refreshed once per batch of steps).
struct GreedyState {
    int n;            // controls in the current level
    int stop;         // 1 once the level's stop test passed or a limit was hit
    int status;       // RBFD_OK, RBFD_ESINGULAR, RBFD_ENOTCONV
    int best;         // sorted position of the current argmax point (-1 if none)
    int best_orig;    // its original surface index
    int pad;
    double best_key;  // |E|^2 at the argmax
    double second_key;
    double min_gap;   // smallest (key1 - key2) / key1 seen this level
    double emax;      // sqrt(best_key) / S0 of the last sweep
    unsigned int pb_done;   // last-block-done counter of the sweep
    unsigned int red_done;  // last-block-done counter of reductions
    int max_cnt;            // longest per-block control list (persistent engine)
    int nnz;                // nonzeros of the phi column of the newest control
    int handoff;            // Newton-basis launch ended to let the list sweep go on
    int pad2;
    unsigned long long nnz_tot;  // nonzeros of Phi_sc for the level's controls so far (Newton launch)
};

// Counter + generation word of the bounded grid barrier of the persistent
// greedy launch; err is set by a block that waited too long.
struct alignas(16) GridBarrier {
    unsigned int count;
    unsigned int gen;
    int err;
    int pad;
};

// Global nanosecond timer (phase timing of the persistent launches).
__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid-wide barrier with a bounded wait.  Returns false (in every thread of
// the block) if the launch is failing: this block timed out or another one did.
__device__ __forceinline__ bool grid_sync(GridBarrier *b, unsigned nblk, unsigned long long limit) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *vgen = &b->gen;
        volatile int *verr = &b->err;
        const unsigned g = *vgen;
        __threadfence();
        const unsigned arrived = atomicAdd(&b->count, 1u);
        if (arrived == nblk - 1) {
            b->count = 0;
            __threadfence();
            atomicAdd(&b->gen, 1u);
        } else {
            unsigned long long it = 0;
            while (*vgen == g) {
                if (*verr) break;
                if (++it > limit) {
                    atomicExch(&b->err, 1);
                    break;
                }
                __nanosleep(8);
            }
        }
        __threadfence();
        s_ok = (*verr == 0);
    }
    __syncthreads();
    return s_ok != 0;
}

// A grid barrier in two halves on a monotone arrival counter (the word
// `count` of a GridBarrier zeroed before the launch): barrier number t (from
// 0) is passed once count reaches (t + 1) * nblk.  Arriving is a release
// fence and an atomic add whose result nobody waits for; between arriving
// and waiting a block can do work that no other block waits for.
__device__ __forceinline__ void grid_arrive_mono(GridBarrier *b) {
    __syncthreads();
    if (threadIdx.x == 0) {
        // release: the block's writes (ordered before this thread by the
        // block barrier) become visible to a block that observes the count
        asm volatile("fence.acq_rel.gpu;\n\tred.relaxed.gpu.global.add.u32 [%0], 1;" ::"l"(&b->count) : "memory");
    }
}

// The same two halves for one thread of the block: arrive (after a block
// barrier that ordered the block's writes before it), then poll until the
// count reaches target or the bound runs out (sets the error word); returns
// false on error.  The caller publishes the result to the block.
__device__ __forceinline__ void grid_arrive_mono_one(GridBarrier *b) {
    asm volatile("fence.acq_rel.gpu;\n\tred.relaxed.gpu.global.add.u32 [%0], 1;" ::"l"(&b->count) : "memory");
}

__device__ __forceinline__ bool grid_poll_mono_one(GridBarrier *b, unsigned target, unsigned long long limit) {
    unsigned long long it = 0;
    unsigned err = 0;
    for (;;) {
        uint4 v;  // count, generation, error word, pad
        asm volatile("ld.relaxed.gpu.global.v4.u32 {%0, %1, %2, %3}, [%4];"
                     : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                     : "l"(b)
                     : "memory");
        err = v.z;
        if (v.x >= target || err) break;
        if (++it > limit) {
            atomicExch(&b->err, 1);
            err = 1;
            break;
        }
        // (no sleep: one thread per block polls, and the barrier is on the critical path)
    }
    asm volatile("fence.acq_rel.gpu;" ::: "memory");  // acquire: pairs with the arrivals' release
    return err == 0;
}

__device__ __forceinline__ bool grid_wait_mono(GridBarrier *b, unsigned target, unsigned long long limit) {
    __shared__ int s_ok;
    if (threadIdx.x == 0) {
        // one 16-byte load per poll reads the count and the error word together
        unsigned long long it = 0;
        unsigned err = 0;
        for (;;) {
            uint4 v;  // count, generation, error word, pad
            asm volatile("ld.relaxed.gpu.global.v4.u32 {%0, %1, %2, %3}, [%4];"
                         : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                         : "l"(b)
                         : "memory");
            err = v.z;
            if (v.x >= target || err) break;
            if (++it > limit) {
                atomicExch(&b->err, 1);
                err = 1;
                break;
            }
            __nanosleep(8);
        }
        asm volatile("fence.acq_rel.gpu;" ::: "memory");  // acquire: pairs with the arrivals' release
        s_ok = (err == 0);
    }
    __syncthreads();
    return s_ok != 0;
}

}  // namespace rbfd
