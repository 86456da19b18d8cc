// persist.cu -- the greedy selection of one level (Section 3) as ONE
// cooperative launch: the grid stays resident and walks through the greedy
// steps itself, separated by a grid barrier, so no step waits for the host.
//
// Per step, with n controls selected so far (every block tracks n in lockstep):
//   phase 1  surface error sweep (Eq. 12): items (point block, chunk of its
//            control list), the chunk length set by the longest list so that
//            heavy blocks near the ice spread over many blocks; chunk partial
//            sums -> scratch; the chunk partials are reduced in FP64 in a
//            fixed order, in two levels (groups of 16 chunks, then the
//            groups; atomic counters find the last of each), and the last
//            forms E = dS_l - sum and the key |E|^2 and writes the block's
//            argmax;
//            the last point block to finish (second counter) takes the step's
//            decision: global argmax, stop test max|E|/S0 < tau_l in FP64,
//            and, if the level goes on, the nonzeros of phi(|r_cn - r_ck|/R)
//            (only controls on c_n's block list can be within R) and c_n.
//            With pruning, only the warps of 32 points whose bounds show
//            they may hold the argmax are swept (warp_bounds below); the
//            items go out heaviest first.
//   -- barrier --
//   phase 3  c_n listed in every point block within R of it (after the
//            barrier: no sweep reads the lists any more); y = G phi over the
//            nonzeros of phi (one warp per row of the inverse factor
//            G = L^{-1}); per-block partial sums of y.y, y.w, which the last
//            block sums into l = sqrt(1 - y.y) and w_n = (dS_l(c_n) - y.w) / l.
//   -- barrier --
//   phase 4  the new row g = -(y^T G) / l as one warp per column over the
//            rows of the transposed copy G^T (contiguous reads), the columns
//            dealt to the warps in snake order; G row n, G^T column n,
//            alpha += w_n g; with pruning, the move bound of every warp near
//            each updated control.
//   -- barrier --
//
// A batch mesh's launch may end between steps after a step limit (st->handoff)
// and be relaunched from st->n.
//
// The barrier is a counter plus generation word in global memory; a block
// that waits longer than a fixed number of polls sets an error word and
// returns, and every other block returns at its next barrier, so a failure
// ends the launch instead of hanging it.  Data written by another block of
// this launch is read with ld.global.cg (L2), never through L1.
#include <algorithm>
#include <cmath>
#include <cstdlib>

#include "internal.h"

namespace rbfd {

namespace {

constexpr int kT = 128;        // threads per block (4 warps)
constexpr int kRG = 16;        // chunk partial sums reduced per group (two-level reduction)


struct PersistArgs {
    int64_t n_s;
    int n_pb, cap, dim, n_chunk_max;
    double R, R2, S0, tau, piv_tol_per_n;
    float invR_hi, invR_lo;
    const double4 *xs, *pb_org, *pb_lo, *pb_hi, *cur;
    const float4 *xs_hi, *xs_lo;
    const uint32_t *perm, *inv;
    unsigned char *sel;
    uint32_t *nb_cnt, *nb_list;
    double4 *cx, *alpha, *w;
    float4 *cdf;  // control coordinates split hi [0, cap] / lo [cap + 1, 2 cap + 1] (double-float)
    uint32_t *cid;
    double *G, *Gt, *phi, *y, *red;
    uint32_t *nz_k;
    double *nz_v;
    double4 *part;
    double4 *gpart;          // group partial sums [max_grp][n_s]
    unsigned int *grp_done;  // [n_pb][max_grp] finished chunks per group (zero between steps)
    int max_grp;
    unsigned int *pb_done;
    double *pb_key;
    int *pb_idx;
    GridBarrier *bar;
    unsigned long long spin_limit;
    GreedyState *st;
    unsigned long long *pairs;
    int test_skip_arrival;  // tests only: block 0 leaves before its first barrier arrival
    unsigned long long *phase_ns;  // non-null: block 0 accumulates [work, wait] ns per phase (8 words)
    unsigned long long *item_ctr;  // the sweep's item counter (zero at launch)
    int pfx_max;                   // balanced sweep items up to this many point blocks (<= kPfxMax)
    int chunk_target;              // controls per sweep item the chunking aims at
    int max_steps;                 // > 0: end the launch after that many steps (st->handoff = 1)
    // pruned sweep (balanced items only), per warp of points w (32 points,
    // w = 4 pb + warp): bnd[parity * 4 n_pb + w] = {M rounded up, M rounded
    // down, unused, A} in FP32 (every block evaluates every warp's bounds each
    // step: in FP64 that arithmetic alone took 40 us per step on the FP64
    // pipe), with M the warp's max |E| over unselected points at its last
    // sweep and A the largest sum_c phi |alpha_c|_1 at its points then;
    // bacc[parity * 4 n_pb + w] = acc, the bound on how far any |E| of the
    // warp has moved since (a sum of atomic additions, in FP64); wbox[2 w], [2 w +
    // 1] the warp's box in FP32 rounded outward; rev[k * n_pb + i] the point
    // blocks whose list holds control k (rev_cnt[k] of them); err_u the
    // relative rounding of one operation of the sweep's arithmetic, with
    // margin; marg bounds the FP32 rounding of a control-to-box distance
    int prune;
    float err_u, S0f;
    float4 *bnd;
    double *bacc;
    const float4 *wbox;
    float marg;
    uint32_t *rev, *rev_cnt;
};

// Bounds on what a sweep of warp w would find now, from its state at its
// last sweep: hi >= the largest |E| it could compute for an unselected point,
// lo <= the largest it would compute.  acc bounds the move of the exact E of
// the stored weights since then; err bounds the rounding of the sweep then
// and now (at most cnt list terms and 2 nch chunk sums, each of relative
// error err_u on sums of at most A + 2 acc: the weights moved by at most
// sqrt(3) acc in phi-weighted 1-norm), plus the subtraction from dS_l
// (|dS_l| <= S0).
// (In FP32 with margins, but acc is summed in FP64 by atomic additions,
// each within 2^-53 of the running sum: over fewer than 2^40 additions that
// is within 2^-13, and acc is taken rounded up and raised by 2^-8; every
// other operation here is within 2^-24, covered by the 2^-20 factors.  In
// FP32 the sum itself would lose the small additions a far warp receives.)
__device__ __forceinline__ void warp_bounds(const PersistArgs &a, const float4 s, double accd, int cnt, int nch,
                                            float &lo, float &hi) {
    const float acc = __double2float_ru(accd) * (1.0f + 0x1p-8f);
    const float err = (float)(cnt + 2 * nch + 16) * a.err_u * (s.w + 2.0f * acc + a.S0f) * (1.0f + 0x1p-20f);
    const float mv = (acc + 2.0f * err) * (1.0f + 0x1p-20f);
    lo = s.y * (1.0f - 0x1p-20f) - mv;
    hi = (s.x + mv) * (1.0f + 0x1p-20f);
}

// A control at x (FP32, absolute) moved the weights by inc / |phi| times
// phi: add inc times an upper bound of phi(dist(x, box) / R) to the move
// bound of every warp of point block t within R of x (the distance shrunk by
// marg for the FP32 rounding).
template <int BASIS>
__device__ __forceinline__ void push_bound(const PersistArgs &a, double *acc, int t, float3 x, float inc,
                                           float invR) {
#pragma unroll
    for (int w4 = 0; w4 < 4; ++w4) {
        const int w = 4 * t + w4;
        const float4 lo = __ldg(&a.wbox[2 * w]), hi = __ldg(&a.wbox[2 * w + 1]);
        const float dx = fmaxf(fmaxf(lo.x - x.x, x.x - hi.x), 0.0f);
        const float dy = fmaxf(fmaxf(lo.y - x.y, x.y - hi.y), 0.0f);
        const float dz = fmaxf(fmaxf(lo.z - x.z, x.z - hi.z), 0.0f);
        const float d = fmaxf(sqrtf(dx * dx + dy * dy + dz * dz) - a.marg, 0.0f);
        const float f = phi_f32_upper<BASIS>(d * invR);
        if (f > 0.0f) atomicAdd(&acc[w], (double)(inc * f * (1.0f + 0x1p-20f)));
    }
}

// Adds the partial sums [c0, c1) of point p (stride apart) in order, eight
// loads in flight.
__device__ __forceinline__ void sum_parts(const double4 *base, size_t stride, int c0, int c1, double &s0,
                                          double &s1, double &s2, double &s3) {
    int c = c0;
    for (; c + 8 <= c1; c += 8) {
        double4 v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) v[q] = ldcg_d4(base + (size_t)(c + q) * stride);
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            s0 = __dadd_rn(s0, v[q].x);
            s1 = __dadd_rn(s1, v[q].y);
            s2 = __dadd_rn(s2, v[q].z);
            s3 += v[q].w;
        }
    }
    for (; c < c1; ++c) {
        const double4 v = ldcg_d4(base + (size_t)c * stride);
        s0 = __dadd_rn(s0, v.x);
        s1 = __dadd_rn(s1, v.y);
        s2 = __dadd_rn(s2, v.z);
        s3 += v.w;
    }
}

__device__ __forceinline__ uint32_t ldcg_u32(const uint32_t *p) { return __ldcg(p); }
__device__ __forceinline__ double ldcg_d(const double *p) { return __ldcg(p); }
__device__ __forceinline__ float4 ldcg_f4(const float4 *p) { return __ldcg(p); }

template <int DIM, int BASIS, int MODE>
__global__ void __launch_bounds__(kT, 5) k_greedy_persist(PersistArgs a) {
    __shared__ double t64[7][kTile];
    __shared__ float t32[13][kTile];
    __shared__ double sk[32];
    __shared__ int si[32];
    __shared__ double scol[4][32];
    __shared__ double sred[4][4];
    __shared__ bool s_last, s_lead, s_glast;
    __shared__ unsigned s_scan[32];
    __shared__ unsigned char s_hits[4][kTile];
    __shared__ unsigned s_pfx[kPfxMax + 1];
    __shared__ unsigned s_order[kPfxMax];  // pruned steps: point block | chunks << 16, in item order
    __shared__ unsigned s_act[kPfxMax / 8];  // pruned steps: one bit per warp of points, set if it is swept
    __shared__ int s_item;
    __shared__ unsigned s_nsw;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned P = gridDim.x;
    int n = __ldcg(&a.st->n);
    const df invR = {a.invR_hi, a.invR_lo};
    // phase timing (block 0, thread 0): work = phase start -> barrier entry,
    // wait = barrier entry -> exit
    const bool timing = a.phase_ns && blockIdx.x == 0 && tid == 0;
    unsigned long long acc_ns[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    unsigned long long t_mark = timing ? gtimer() : 0ull;
#define RBFD_SYNC(PH)                                                            \
    {                                                                            \
        unsigned long long t_in = timing ? gtimer() : 0ull;                      \
        bool ok_ = grid_sync(a.bar, P, a.spin_limit);                            \
        if (timing) {                                                            \
            unsigned long long t_out = gtimer();                                 \
            acc_ns[2 * (PH)] += t_in - t_mark;                                   \
            acc_ns[2 * (PH) + 1] += t_out - t_in;                                \
            t_mark = t_out;                                                      \
        }                                                                        \
        if (!ok_) {                                                              \
            if (timing)                                                          \
                for (int q = 0; q < 8; ++q) atomicAdd(&a.phase_ns[q], acc_ns[q]); \
            return;                                                              \
        }                                                                        \
    }
#define RBFD_EXIT()                                                              \
    {                                                                            \
        if (timing)                                                              \
            for (int q = 0; q < 8; ++q) atomicAdd(&a.phase_ns[q], acc_ns[q]);   \
        return;                                                                  \
    }

    // the sweep's items are handed out by one counter over the launch: a step
    // with N items takes N + P fetches (every block's last fetch finds none),
    // so every block knows the step's base
    unsigned long long item_base = 0;
    const bool keep_bounds = a.prune && a.n_pb <= a.pfx_max;
    if (keep_bounds) {
        // the point blocks listing each control the level already has (the
        // counts were zeroed before the launch); later controls are entered
        // as they are listed
        for (int t = blockIdx.x * 4 + warp; t < a.n_pb; t += P * 4) {
            const int cnt = (int)ldcg_u32(&a.nb_cnt[t]);
            for (int q = lane; q < cnt; q += 32) {
                const uint32_t j = ldcg_u32(&a.nb_list[(size_t)t * a.cap + q]);
                const uint32_t pos = atomicAdd(&a.rev_cnt[j], 1u);
                a.rev[(size_t)j * a.n_pb + pos] = (uint32_t)t;
            }
        }
        RBFD_SYNC(0)
    }
    for (int guard = 0; guard <= a.cap; ++guard) {
        // (a step limit ends the launch here, between steps, every block
        // alike; the host relaunches it from st->n)
        if (a.max_steps > 0 && guard >= a.max_steps) {
            if (blockIdx.x == 0 && tid == 0) {
                a.st->n = n;
                a.st->handoff = 1;
                a.st->stop = 1;
            }
            RBFD_EXIT()
        }
        // ------------------------------------------------ phase 1: sweep (+ the step's decision)
        // every block list is cut into chunks of at most cl controls, cl set by
        // the longest list, so that no point block holds the step back
        const int max_cnt = max(1, (int)__ldcg(&a.st->max_cnt));
        int nch = max((int)((P + a.n_pb - 1) / a.n_pb), (max_cnt + a.chunk_target - 1) / a.chunk_target);
        nch = max(1, min(nch, min(a.n_chunk_max, (max_cnt + 15) / 16)));
        const int cl = (max_cnt + nch - 1) / nch;
        // the items are the chunks the lists occupy (at least one per point
        // block, whose last chunk forms E): every block builds the same
        // prefix over the point blocks, to map an item to its (point block,
        // chunk).  (Beyond kPfxMax point blocks: every (point block, chunk)
        // pair is an item, the unoccupied ones skipped.)
        const bool balanced = a.n_pb <= a.pfx_max;
        // bounds of this step (written by the last) and of the next
        const int n_w = 4 * a.n_pb;
        const float4 *bcur = keep_bounds ? a.bnd + (size_t)(guard & 1) * n_w : nullptr;
        float4 *bnext = keep_bounds ? a.bnd + (size_t)((guard & 1) ^ 1) * n_w : nullptr;
        const double *acur = keep_bounds ? a.bacc + (size_t)(guard & 1) * n_w : nullptr;
        double *anext = keep_bounds ? a.bacc + (size_t)((guard & 1) ^ 1) * n_w : nullptr;
        const bool prune_now = keep_bounds && guard > 0;  // (the launch's first step sweeps every warp)
        int n_items = a.n_pb * nch;
        int n_swept = a.n_pb;
        // a warp of points is skipped if even its upper bound stays below the
        // largest lower bound: the warp attaining that is swept and finds at
        // least as much, so the argmax and the stop test are those of a full
        // sweep.  A point block is swept if one of its warps is.
        float LB = -INFINITY;
        if (balanced) {
            const int per = (a.n_pb + kT - 1) / kT;
            const int b0 = min(a.n_pb, tid * per), b1 = min(a.n_pb, b0 + per);
            unsigned long long skip_pairs = 0;
            unsigned skip_w = 0;
            if (prune_now) {
                // Two passes over the warps' states, consecutive lanes on
                // consecutive warps (coalesced: with a thread per point block
                // the loads took 11 us a pass, every block reading): LB, then
                // one bit per warp in s_act.  Block 0 carries a skipped warp's
                // state over to the next step.
                float lmax = -INFINITY;
                for (int w = tid; w < n_w; w += kT) {
                    float lo, hi;
                    warp_bounds(a, __ldcg(bcur + w), __ldcg(acur + w), (int)ldcg_u32(&a.nb_cnt[w >> 2]), nch, lo, hi);
                    lmax = fmaxf(lmax, lo);
                }
                for (int o = 16; o > 0; o >>= 1) lmax = fmaxf(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
                if (lane == 0) sk[warp] = lmax;
                if (tid == 0) s_nsw = 0;
                __syncthreads();
                LB = (float)fmax(fmax(sk[0], sk[1]), fmax(sk[2], sk[3]));
                __syncthreads();
                for (int w0 = warp * 32; w0 < n_w; w0 += kT) {
                    const int w = w0 + lane;
                    bool act = false;
                    if (w < n_w) {
                        const float4 s = __ldcg(bcur + w);
                        const double accd = __ldcg(acur + w);
                        const int cb = (int)ldcg_u32(&a.nb_cnt[w >> 2]);
                        float lo, hi;
                        warp_bounds(a, s, accd, cb, nch, lo, hi);
                        act = hi >= LB;
                        if (!act && blockIdx.x == 0) {
                            bnext[w] = s;
                            anext[w] = accd;
                            skip_pairs += (unsigned long long)max((int64_t)0, min((int64_t)32, a.n_s - (int64_t)w * 32)) *
                                          (unsigned long long)cb;
                            ++skip_w;
                        }
                    }
                    const unsigned bits = __ballot_sync(0xffffffffu, act);
                    if (lane == 0) s_act[w0 >> 5] = bits;
                }
                __syncthreads();
            }
            unsigned mine = 0, swept = 0;
            unsigned bc0 = 0, bc1 = 0, bc2 = 0, bc3 = 0;
            for (int b = b0; b < b1; ++b) {
                const int cb = (int)ldcg_u32(&a.nb_cnt[b]);
                unsigned ub = (unsigned)min(nch, max(1, (cb + cl - 1) / cl));
                if (prune_now) {
                    const int act = __popc((s_act[b >> 3] >> ((b & 7) * 4)) & 0xFu);
                    if (act == 0) ub = 0;
                    else ++swept;
                    // (bucket of the item order: 4 active warps first, then 3, 2, at most 1)
                    const int bk = act >= 2 ? 4 - act : 3;
                    bc0 += bk == 0;
                    bc1 += bk == 1;
                    bc2 += bk == 2;
                    bc3 += bk == 3;
                    ub |= (unsigned)bk << 16;
                }
                s_pfx[b] = ub;
                mine += ub & 0xFFFFu;
            }
            if (prune_now) {
                if (swept) atomicAdd(&s_nsw, swept);
                if (blockIdx.x == 0 && skip_w) {  // (counters of the skipped work)
                    atomicAdd(&a.pairs[11], skip_pairs);
                    atomicAdd(&a.pairs[12], (unsigned long long)skip_w);
                }
            }
            unsigned tot;
            if (prune_now) {
                // Items go out heaviest first: the point blocks with four
                // warps to sweep, then three, two, one (stable within each),
                // so that the step's last items are light ones.  Positions by
                // a counting sort (two scans of packed 16-bit counts), then
                // the chunk prefix over the sorted order.
                unsigned t01, t23;
                const unsigned e01 = block_excl_scan_u32(bc0 | (bc1 << 16), s_scan, &t01);
                const unsigned e23 = block_excl_scan_u32(bc2 | (bc3 << 16), s_scan, &t23);
                unsigned p0 = e01 & 0xFFFFu, p1 = (t01 & 0xFFFFu) + (e01 >> 16),
                         p2 = (t01 & 0xFFFFu) + (t01 >> 16) + (e23 & 0xFFFFu),
                         p3 = (t01 & 0xFFFFu) + (t01 >> 16) + (t23 & 0xFFFFu) + (e23 >> 16);
                for (int b = b0; b < b1; ++b) {
                    const unsigned v = s_pfx[b], k = v >> 16;
                    const unsigned at = k == 0 ? p0 : k == 1 ? p1 : k == 2 ? p2 : p3;
                    s_order[at] = (unsigned)b | ((v & 0xFFFFu) << 16);
                    p0 += k == 0;
                    p1 += k == 1;
                    p2 += k == 2;
                    p3 += k == 3;
                }
                __syncthreads();
                unsigned m2 = 0;
                for (int i = b0; i < b1; ++i) m2 += s_order[i] >> 16;
                unsigned run = block_excl_scan_u32(m2, s_scan, &tot);
                for (int i = b0; i < b1; ++i) {
                    s_pfx[i] = run;
                    run += s_order[i] >> 16;
                }
            } else {
                unsigned run = block_excl_scan_u32(mine, s_scan, &tot);
                for (int b = b0; b < b1; ++b) {
                    const unsigned ub = s_pfx[b];
                    s_pfx[b] = run;
                    run += ub;
                }
            }
            if (tid == 0) {
                s_pfx[a.n_pb] = tot;
                s_item = (int)(atomicAdd(a.item_ctr, 1ull) - item_base);
            }
            __syncthreads();
            n_items = (int)tot;
            if (prune_now) n_swept = (int)s_nsw;
        }
        // balanced: items taken from the counter as blocks come free (their
        // costs differ with the density of controls); the next index is
        // fetched when the current item is done, so that no block holds an
        // item back while others run out at the end of the step.  Otherwise
        // every P-th item.
        int item = balanced ? s_item : (int)blockIdx.x;
        for (; item < n_items; item = balanced ? s_item : item + (int)P) {
            int pb, ch, cnt, used;
            if (balanced) {
                int bl = 0, bh = a.n_pb;  // s_pfx[bl] <= item < s_pfx[bh] (item order)
                while (bh - bl > 1) {
                    const int mid = (bl + bh) >> 1;
                    if (s_pfx[mid] <= (unsigned)item) bl = mid; else bh = mid;
                }
                pb = prune_now ? (int)(s_order[bl] & 0xFFFFu) : bl;
                ch = item - (int)s_pfx[bl];
                used = (int)(s_pfx[bl + 1] - s_pfx[bl]);
                cnt = (int)ldcg_u32(&a.nb_cnt[pb]);
            } else {
                pb = item / nch;
                ch = item % nch;
                cnt = (int)ldcg_u32(&a.nb_cnt[pb]);
                used = min(nch, max(1, (cnt + cl - 1) / cl));  // chunks this block's list occupies
                if (ch >= used) continue;                     // same decision in every thread
            }
            const int64_t p = (int64_t)pb * kPB + tid;
            const bool valid = p < a.n_s;
            const int lo = ch * cl, hi = (ch == used - 1) ? cnt : min(cnt, lo + cl);  // the last takes the rest
            const double4 org = a.pb_org[pb];
            double acc64[3] = {0, 0, 0};
            df acc[3] = {{0, 0}, {0, 0}, {0, 0}};
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
            unsigned useful = 0;
            // this warp's points are evaluated unless its bound skips them
            // (the same decision as in the prefix above: same inputs)
            const int wsel = 4 * pb + warp;
            const bool wact = !prune_now || ((s_act[wsel >> 5] >> (wsel & 31)) & 1u);
            double sabs64 = 0.0;  // sum_c phi |alpha_c|_1 at this point (pruning bounds)
            float sabs = 0.0f;
            float3 wlo, whi;
            if (MODE == 1) warp_box(valid, qx.hi, qy.hi, qz.hi, wlo, whi);
            const float R2m = (float)(1.002 * a.R) * (float)(1.002 * a.R);  // filter margin
            for (int t0 = lo; t0 < hi; t0 += kTile) {
                const int m = min(kTile, hi - t0);
                if (tid < m) {
                    const uint32_t j = ldcg_u32(&a.nb_list[(size_t)pb * a.cap + t0 + tid]);
                    const double4 c = ldcg_d4(&a.cx[j]), al = ldcg_d4(&a.alpha[j]);
                    const double aabs = (fabs(al.x) + fabs(al.y)) + fabs(al.z);
                    if (MODE == 0) {
                        t64[0][tid] = c.x; t64[1][tid] = c.y; t64[2][tid] = c.z;
                        t64[3][tid] = al.x; t64[4][tid] = al.y; t64[5][tid] = al.z;
                        t64[6][tid] = aabs;
                    } else {
                        t32[12][tid] = __double2float_ru(aabs);
                        df rx = df_from_double(c.x - org.x), ry = df_from_double(c.y - org.y),
                           rz = df_from_double(c.z - org.z);
                        df ax = df_from_double(al.x), ay = df_from_double(al.y), az = df_from_double(al.z);
                        t32[0][tid] = rx.hi; t32[1][tid] = rx.lo; t32[2][tid] = ry.hi; t32[3][tid] = ry.lo;
                        t32[4][tid] = rz.hi; t32[5][tid] = rz.lo; t32[6][tid] = ax.hi; t32[7][tid] = ax.lo;
                        t32[8][tid] = ay.hi; t32[9][tid] = ay.lo; t32[10][tid] = az.hi; t32[11][tid] = az.lo;
                    }
                }
                __syncthreads();
                if (MODE == 0) {
                    // a warp skips a control farther than R from all its points
                    // (phi is exactly 0 there, the sums do not change)
                    const double R2hi = __dmul_rn(__dmul_rn(a.R, a.R), 1.0 + 1e-12);
                    for (int q = 0; wact && q < m; ++q) {
                        const double s2 = dist2_f64<DIM>(px, py, pz, t64[0][q], t64[1][q], t64[2][q]);
                        if (!__any_sync(0xffffffffu, valid && s2 <= R2hi)) continue;
                        if (valid) {
                            double eta = __ddiv_rn(__dsqrt_rn(s2), a.R);
                            double f = phi_f64<BASIS>(eta);
                            useful += (eta < 1.0);
                            acc64[0] = __dadd_rn(acc64[0], __dmul_rn(t64[3][q], f));
                            acc64[1] = __dadd_rn(acc64[1], __dmul_rn(t64[4][q], f));
                            if (DIM == 3) acc64[2] = __dadd_rn(acc64[2], __dmul_rn(t64[5][q], f));
                            if (keep_bounds) sabs64 = fma(f, t64[6][q], sabs64);
                        }
                    }
                } else if (wact) {
                    // every lane of the warp takes part in the filter, then only
                    // the lanes with a point accumulate
                    const int nh = warp_hits<DIM>(t32, m, wlo, whi, R2m, s_hits[warp]);
                    if (valid) {
                        if (keep_bounds)
                            hits_accumulate_df_abs<DIM, BASIS>(qx, qy, qz, t32, s_hits[warp], nh, invR, acc, useful,
                                                               sabs);
                        else
                            hits_accumulate_df<DIM, BASIS>(qx, qy, qz, t32, s_hits[warp], nh, invR, acc, useful);
                    }
                }
                __syncthreads();
            }
            if (MODE == 1) {
                acc64[0] = df_to_double(acc[0]);
                acc64[1] = df_to_double(acc[1]);
                acc64[2] = df_to_double(acc[2]);
            }
            // (w slot: this chunk's share of sum_c phi |alpha_c|_1 at the point)
            if (valid)
                a.part[(size_t)ch * a.n_s + p] =
                    make_double4(acc64[0], acc64[1], acc64[2], MODE == 0 ? sabs64 : (double)sabs);
            {
                unsigned u = useful;
                for (int o = 16; o > 0; o >>= 1) u += __shfl_xor_sync(0xffffffffu, u, o);
                if (lane == 0 && u) atomicAdd(&a.pairs[0], (unsigned long long)u);
                if (tid == 0 && hi > lo) {
                    unsigned long long nv = (unsigned long long)min((int64_t)kPB, a.n_s - (int64_t)pb * kPB);
                    atomicAdd(&a.pairs[1], nv * (unsigned long long)(hi - lo));
                }
            }
            // The chunks' partial sums are reduced in two levels, in a fixed
            // order: the last chunk of each group of kRG sums the group's,
            // the last group of the point block sums the groups' and forms E,
            // the key and the block argmax; the last point block to finish
            // then takes the step's decision
            __threadfence();
            __syncthreads();
            const int ng = (used + kRG - 1) / kRG, grp = ch / kRG;
            if (tid == 0) {
                const int gs = min(kRG, used - grp * kRG);
                const bool gl = ng == 1 ? atomicAdd(&a.pb_done[pb], 1u) == (unsigned)(used - 1)  // (used >= 1)
                                        : atomicAdd(&a.grp_done[(size_t)pb * a.max_grp + grp], 1u) ==
                                              (unsigned)(gs - 1);
                s_last = ng == 1 && gl;
                s_glast = ng > 1 && gl;
            }
            __syncthreads();
            if (s_glast) {
                __threadfence();
                if (valid && wact) {
                    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
                    sum_parts(a.part + p, (size_t)a.n_s, grp * kRG, min(used, (grp + 1) * kRG), s0, s1, s2, s3);
                    a.gpart[(size_t)grp * a.n_s + p] = make_double4(s0, s1, s2, s3);
                }
                __threadfence();
                __syncthreads();
                if (tid == 0) {
                    a.grp_done[(size_t)pb * a.max_grp + grp] = 0;
                    s_last = atomicAdd(&a.pb_done[pb], 1u) == (unsigned)(ng - 1);
                }
                __syncthreads();
            }
            if (s_last) {
                __threadfence();
                double key = -1.0;
                int orig = -1;
                double s3 = 0.0;  // sum_c phi |alpha_c|_1 at this point (pruning bounds)
                if (valid && wact) {  // (a skipped warp's points keep their last key: below the argmax)
                    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
                    if (ng == 1)
                        sum_parts(a.part + p, (size_t)a.n_s, 0, used, s0, s1, s2, s3);
                    else
                        sum_parts(a.gpart + p, (size_t)a.n_s, 0, ng, s0, s1, s2, s3);
                    const double4 cu = a.cur[p];
                    const double e0 = __dsub_rn(cu.x, s0), e1 = __dsub_rn(cu.y, s1);
                    const double e2 = (DIM == 3) ? __dsub_rn(cu.z, s2) : 0.0;
                    double k2 = __dmul_rn(e0, e0);
                    k2 = __dadd_rn(k2, __dmul_rn(e1, e1));
                    if (DIM == 3) k2 = __dadd_rn(k2, __dmul_rn(e2, e2));
                    if (!__ldcg(reinterpret_cast<const unsigned char *>(a.sel) + p)) {
                        key = k2;
                        orig = (int)a.perm[p];
                    }
                }
                if (keep_bounds && wact) {
                    // the warp's state for the next steps: its max |E| over the
                    // unselected points, no move yet, and the largest scale of
                    // the sums (the FP32 sums of phi |alpha| rounded up by a
                    // margin over their cnt terms)
                    double km = key, sm = s3;
                    for (int o = 16; o > 0; o >>= 1) {
                        km = fmax(km, __shfl_xor_sync(0xffffffffu, km, o));
                        sm = fmax(sm, __shfl_xor_sync(0xffffffffu, sm, o));
                    }
                    if (lane == 0) {
                        const double Mw = km > 0.0 ? sqrt(km) : 0.0;
                        anext[4 * pb + warp] = 0.0;
                        bnext[4 * pb + warp] = make_float4(__double2float_ru(Mw), __double2float_rd(Mw), 0.0f,
                                                           __double2float_ru(sm * (1.0 + (double)(cnt + 16) * 0x1p-22)));
                    }
                }
                block_argmax(key, orig, sk, si);
                if (tid == 0) {
                    a.pb_key[pb] = key;
                    a.pb_idx[pb] = orig;
                    a.pb_done[pb] = 0;
                    __threadfence();
                    s_lead = atomicAdd(&a.st->pb_done, 1u) == (unsigned)(n_swept - 1);
                }
                __syncthreads();
                if (s_lead) {
                    // ---- the step's decision (one block): argmax, stop test, phi column, lists
                    __threadfence();
                    double K = -1.0;
                    int I = -1;
                    for (int b = tid; b < a.n_pb; b += kT) {
                        const double kb = __ldcg(&a.pb_key[b]);
                        const int ib = __ldcg(&a.pb_idx[b]);
                        if (better(kb, ib, K, I)) {
                            K = kb;
                            I = ib;
                        }
                    }
                    block_argmax(K, I, sk, si);
                    const double e = I >= 0 ? __ddiv_rn(__dsqrt_rn(K), a.S0) : 0.0;
                    const bool stop = I < 0 || e < a.tau || n >= a.cap;
                    if (!stop) {
                        const uint32_t c = a.inv[I];
                        const double4 xc = a.xs[c];
                        const df xcx = df_from_double(xc.x), xcy = df_from_double(xc.y), xcz = df_from_double(xc.z);
                        // phi(|r_cn - r_ck| / R) is nonzero only for controls within R of
                        // c_n, all of which are on the list of c_n's point block; keep
                        // the nonzeros in list (= control) order
                        const int pbc = (int)(c / kPB);
                        const int cntc = (int)ldcg_u32(&a.nb_cnt[pbc]);
                        const uint32_t *lst = a.nb_list + (size_t)pbc * a.cap;
                        // each thread evaluates a contiguous stretch of the list (values
                        // parked in phi[]), then one block scan places the nonzeros in order
                        const int per = (cntc + kT - 1) / kT;
                        const int q0 = min(cntc, tid * per), q1 = min(cntc, q0 + per);
                        unsigned mine = 0;
                        if constexpr (MODE == 0) {
                            for (int q = q0; q < q1; ++q) {
                                const uint32_t k = ldcg_u32(lst + q);
                                const double4 ck = ldcg_d4(&a.cx[k]);
                                const double f = phi_f64<BASIS>(
                                    __ddiv_rn(dist_f64<DIM>(xc.x, xc.y, xc.z, ck.x, ck.y, ck.z), a.R));
                                a.phi[q] = f;
                                mine += (f != 0.0);
                            }
                        } else {
                            // double-float on the FP32 pipe from the split coordinates,
                            // four entries at a time (their loads issued together)
                            const float Rnear = (float)(1.002 * a.R) + a.marg, R2near = Rnear * Rnear;
                            for (int q = q0; q < q1; q += 4) {
                                uint32_t kk[4];
#pragma unroll
                                for (int u = 0; u < 4; ++u) kk[u] = q + u < q1 ? ldcg_u32(lst + q + u) : 0u;
                                float4 h[4], l[4];
#pragma unroll
                                for (int u = 0; u < 4; ++u) {
                                    h[u] = q + u < q1 ? ldcg_f4(&a.cdf[kk[u]]) : make_float4(0, 0, 0, 0);
                                    l[u] = q + u < q1 ? ldcg_f4(&a.cdf[a.cap + 1 + kk[u]]) : make_float4(0, 0, 0, 0);
                                }
                                // FP32 pre-filter on the hi parts: a control beyond
                                // (1.002 R + marg) has phi exactly 0 in double-float too
                                bool near[4];
#pragma unroll
                                for (int u = 0; u < 4; ++u) {
                                    const float fx = h[u].x - xcx.hi, fy = h[u].y - xcy.hi, fz = h[u].z - xcz.hi;
                                    near[u] = q + u < q1 && fx * fx + fy * fy + (DIM == 3 ? fz * fz : 0.0f) <= R2near;
                                }
#pragma unroll
                                for (int u = 0; u < 4; ++u) {
                                    if (q + u >= q1) break;
                                    double f = 0.0;
                                    if (near[u]) {
                                        const df dx = df_add({h[u].x, l[u].x}, df_neg(xcx)),
                                                 dy = df_add({h[u].y, l[u].y}, df_neg(xcy));
                                        df r2 = df_add(df_sqr(dx), df_sqr(dy));
                                        if (DIM == 3)
                                            r2 = df_add(r2, df_sqr(df_add({h[u].z, l[u].z}, df_neg(xcz))));
                                        f = df_to_double(phi_df<BASIS>(df_mul(df_sqrt(r2), invR)));
                                    }
                                    a.phi[q + u] = f;
                                    mine += (f != 0.0);
                                }
                            }
                        }
                        unsigned nnz;
                        unsigned pos = block_excl_scan_u32(mine, s_scan, &nnz);
                        for (int q = q0; q < q1; q += 4) {  // (loads of four entries issued together)
                            double ff[4];
                            uint32_t kk[4];
#pragma unroll
                            for (int u = 0; u < 4; ++u) {
                                ff[u] = q + u < q1 ? a.phi[q + u] : 0.0;  // written by this thread above
                                kk[u] = q + u < q1 ? ldcg_u32(lst + q + u) : 0u;
                            }
#pragma unroll
                            for (int u = 0; u < 4; ++u) {
                                if (ff[u] != 0.0) {
                                    a.nz_k[pos] = kk[u];
                                    a.nz_v[pos] = ff[u];
                                    ++pos;
                                }
                            }
                        }
                        // (the block lists get c_n after the barrier: other blocks may
                        // still be deciding their items of this step from the counts)
                        if (tid == 0) {
                            a.st->nnz = (int)nnz;
                            a.sel[c] = 1;
                            a.cx[n] = xc;
                            a.cdf[n] = make_float4(xcx.hi, xcy.hi, xcz.hi, 0.f);
                            a.cdf[a.cap + 1 + n] = make_float4(xcx.lo, xcy.lo, xcz.lo, 0.f);
                            a.cid[n] = c;
                            a.st->best = (int)c;
                        }
                    }
                    if (tid == 0) {
                        a.st->best_orig = I;
                        a.st->best_key = K;
                        a.st->emax = e;
                        a.st->pb_done = 0;
                        if (stop) {
                            a.st->n = n;
                            if (!(I < 0 || e < a.tau)) a.st->status = RBFD_ENOTCONV;
                            a.st->stop = 1;
                        }
                    }
                }
            }
            if (balanced) {
                // (every thread has read s_item: block barriers came after the read)
                if (tid == 0) s_item = (int)(atomicAdd(a.item_ctr, 1ull) - item_base);
                __syncthreads();
            }
        }
        if (balanced) item_base += (unsigned long long)n_items + P;
        if (a.test_skip_arrival && blockIdx.x == 0) return;  // the others' waits run out
        RBFD_SYNC(0)

        // ------------------------------------------------ every block: the decision
        if (__ldcg(&a.st->stop)) RBFD_EXIT()
        const uint32_t c = (uint32_t)__ldcg(&a.st->best);
        const bool first_block = blockIdx.x == 0 && tid == 0;
        const int nnz = __ldcg(&a.st->nnz);
        const int k0 = nnz > 0 ? (int)ldcg_u32(a.nz_k) : n;  // y_j = 0 for j < k0

        // ------------------------------------------------ phase 3: lists, y = G phi (phi sparse)
        {
            // list c_n in every point block within R of it; the next sweep
            // chunks the lists by the longest one
            const double4 xc = a.xs[c];
            for (int t = blockIdx.x * kT + tid; t < a.n_pb; t += P * kT) {
                const double4 l = a.pb_lo[t], h = a.pb_hi[t];
                const double dx = fmax(fmax(l.x - xc.x, xc.x - h.x), 0.0);
                const double dy = fmax(fmax(l.y - xc.y, xc.y - h.y), 0.0);
                const double dz = DIM == 3 ? fmax(fmax(l.z - xc.z, xc.z - h.z), 0.0) : 0.0;
                if (dx * dx + dy * dy + dz * dz < a.R2 * (1.0 + 1e-9)) {
                    const uint32_t k = ldcg_u32(&a.nb_cnt[t]);
                    a.nb_list[(size_t)t * a.cap + k] = (uint32_t)n;
                    a.nb_cnt[t] = k + 1;
                    atomicMax(&a.st->max_cnt, (int)(k + 1));
                    if (keep_bounds) {
                        const uint32_t pos = atomicAdd(&a.rev_cnt[n], 1u);
                        a.rev[(size_t)n * a.n_pb + pos] = (uint32_t)t;
                    }
                }
            }
            // c_n's own warp has lost the point its maximum was taken at: no
            // lower bound from it until it is swept again (which its infinite
            // bound forces)
            if (keep_bounds && first_block) anext[c / 32] = INFINITY;
        }
        double yy = 0, yw0 = 0, yw1 = 0, yw2 = 0;
        for (int j = blockIdx.x * 4 + warp; j < n; j += P * 4) {
            double s0 = 0.0, s1 = 0.0;
            if (j >= k0) {
                const double *row = a.G + (size_t)j * a.cap;
                int q = lane;
                for (; q + 32 < nnz; q += 64) {
                    const uint32_t ka = ldcg_u32(a.nz_k + q), kb = ldcg_u32(a.nz_k + q + 32);
                    const double va = ldcg_d(a.nz_v + q), vb = ldcg_d(a.nz_v + q + 32);
                    if ((int)ka <= j) s0 = fma(ldcg_d(row + ka), va, s0);
                    if ((int)kb <= j) s1 = fma(ldcg_d(row + kb), vb, s1);
                }
                for (; q < nnz; q += 32) {
                    const uint32_t ka = ldcg_u32(a.nz_k + q);
                    if ((int)ka <= j) s0 = fma(ldcg_d(row + ka), ldcg_d(a.nz_v + q), s0);
                }
            }
            const double s = warp_sum_d(s0 + s1);
            if (lane == 0) {
                a.y[j] = s;
                const double4 wj = ldcg_d4(&a.w[j]);
                yy += s * s;
                yw0 += s * wj.x;
                yw1 += s * wj.y;
                yw2 += s * wj.z;
            }
        }
        if (lane == 0) {
            sred[warp][0] = yy;
            sred[warp][1] = yw0;
            sred[warp][2] = yw1;
            sred[warp][3] = yw2;
        }
        __syncthreads();
        if (tid < 4) a.red[blockIdx.x * 4 + tid] = sred[0][tid] + sred[1][tid] + sred[2][tid] + sred[3][tid];
        // The last block here sums every block's partial y.y, y.w (in block
        // order: the same sums whichever block it is) and derives the pivot
        // and w_n once for the grid, in red[4 P ...]: on GB300's FP64 pipe
        // that reduction repeated in every block cost about 13 us per step.
        __threadfence();
        __syncthreads();
        if (tid == 0) s_glast = atomicAdd(&a.st->red_done, 1u) == P - 1;
        __syncthreads();
        if (s_glast) {
            __threadfence();
            double v0 = 0.0, v1 = 0.0, v2 = 0.0, v3 = 0.0;
            for (unsigned b = tid; b < P; b += kT) {
                v0 += ldcg_d(&a.red[b * 4 + 0]);
                v1 += ldcg_d(&a.red[b * 4 + 1]);
                v2 += ldcg_d(&a.red[b * 4 + 2]);
                v3 += ldcg_d(&a.red[b * 4 + 3]);
            }
            v0 = warp_sum_d(v0);
            v1 = warp_sum_d(v1);
            v2 = warp_sum_d(v2);
            v3 = warp_sum_d(v3);
            if (lane == 0) {
                scol[warp][0] = v0;
                scol[warp][1] = v1;
                scol[warp][2] = v2;
                scol[warp][3] = v3;
            }
            __syncthreads();
            if (tid == 0) {
                double r4[4];
                for (int q = 0; q < 4; ++q) r4[q] = ((scol[0][q] + scol[1][q]) + scol[2][q]) + scol[3][q];
                const double l2 = 1.0 - r4[0];  // phi(0) = 1 for every Wendland function
                const double l = sqrt(l2);
                const double4 bc = a.cur[c];
                double *out = a.red + 4 * (size_t)P;
                out[0] = l2;
                out[1] = l;
                out[2] = (bc.x - r4[1]) / l;
                out[3] = (bc.y - r4[2]) / l;
                out[4] = (bc.z - r4[3]) / l;
                a.st->red_done = 0;
            }
        }
        RBFD_SYNC(2)

        // ------------------------------------------------ phase 4: G row n (= G^T column n), alpha
        const double *piv = a.red + 4 * (size_t)P;
        const double l2 = ldcg_d(piv);
        if (!(l2 > a.piv_tol_per_n * (n + 1))) {
            if (first_block) {
                a.st->status = RBFD_ESINGULAR;
                a.st->stop = 1;
                a.st->n = n;
            }
            RBFD_EXIT()
        }
        const double l = ldcg_d(piv + 1), wn0 = ldcg_d(piv + 2), wn1 = ldcg_d(piv + 3), wn2 = ldcg_d(piv + 4);
        double *Grow = a.G + (size_t)n * a.cap;
        if (first_block) {
            Grow[n] = 1.0 / l;
            a.Gt[(size_t)n * a.cap + n] = 1.0 / l;
            a.w[n] = make_double4(wn0, wn1, wn2, 0.0);
            a.alpha[n] = make_double4(wn0 / l, wn1 / l, wn2 / l, 0.0);
        }
        // g_k = -(sum_{j >= k} y_j G_jk) / l, one warp per k over row k of G^T.
        // Pruning: alpha_k moves by w_n g_k, so |E| moves by at most
        // |w_n| |g_k| at the points within R of control k: that is added to
        // the bound of every block listing k (k = n too, g_n = 1 / l)
        // The k are dealt to the warps in rounds of P * 4, every other round
        // in reverse order, so that every warp's rows add up to about the
        // same length (row k has n - k entries)
        const double wnorm = keep_bounds ? sqrt(wn0 * wn0 + wn1 * wn1 + wn2 * wn2) * (1.0 + 1e-12) : 0.0;
        const int n_k = keep_bounds ? n + 1 : n, W = (int)P * 4, gw = blockIdx.x * 4 + warp;
        for (int r = 0; r * W < n_k; ++r) {
            const int k = r * W + ((r & 1) ? W - 1 - gw : gw);
            if (k >= n_k) continue;
            if (k == n) {  // (only with pruning)
                const float inc = __double2float_ru(wnorm / l);
                const int rc = (int)ldcg_u32(&a.rev_cnt[k]);
                const uint32_t *rv = a.rev + (size_t)k * a.n_pb;
                const float4 xk = ldcg_f4(&a.cdf[k]);
                for (int q = lane; q < rc; q += 32)
                    push_bound<BASIS>(a, anext, (int)ldcg_u32(rv + q), make_float3(xk.x, xk.y, xk.z), inc,
                                      invR.hi);
                continue;
            }
            const double *trow = a.Gt + (size_t)k * a.cap;
            // eight row entries in flight per lane: the rows stream from HBM
            // at the FP64 pipe's rate only with that many loads outstanding
            // (10% off this phase on the 60k wing, no extra registers)
            double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
            int j = max(k, k0) + lane;
            for (; j + 224 < n; j += 256) {
                double g[8], y[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) g[u] = ldcg_d(trow + j + 32 * u);
#pragma unroll
                for (int u = 0; u < 8; ++u) y[u] = ldcg_d(a.y + j + 32 * u);
                s0 = fma(g[0], y[0], s0);
                s1 = fma(g[1], y[1], s1);
                s2 = fma(g[2], y[2], s2);
                s3 = fma(g[3], y[3], s3);
                s0 = fma(g[4], y[4], s0);
                s1 = fma(g[5], y[5], s1);
                s2 = fma(g[6], y[6], s2);
                s3 = fma(g[7], y[7], s3);
            }
            for (; j + 96 < n; j += 128) {
                const double g0 = ldcg_d(trow + j), g1 = ldcg_d(trow + j + 32), g2 = ldcg_d(trow + j + 64),
                             g3 = ldcg_d(trow + j + 96);
                const double y0 = ldcg_d(a.y + j), y1 = ldcg_d(a.y + j + 32), y2 = ldcg_d(a.y + j + 64),
                             y3 = ldcg_d(a.y + j + 96);
                s0 = fma(g0, y0, s0);
                s1 = fma(g1, y1, s1);
                s2 = fma(g2, y2, s2);
                s3 = fma(g3, y3, s3);
            }
            for (; j < n; j += 32) s0 = fma(ldcg_d(trow + j), ldcg_d(a.y + j), s0);
            const double t = warp_sum_d((s0 + s1) + (s2 + s3));
            if (keep_bounds) {
                const float inc = __double2float_ru(wnorm * fabs(t / l));
                const int rc = (int)ldcg_u32(&a.rev_cnt[k]);
                const uint32_t *rv = a.rev + (size_t)k * a.n_pb;
                const float4 xk = ldcg_f4(&a.cdf[k]);
                for (int q = lane; q < rc; q += 32)
                    push_bound<BASIS>(a, anext, (int)ldcg_u32(rv + q), make_float3(xk.x, xk.y, xk.z), inc,
                                      invR.hi);
            }
            if (lane == 0) {
                const double g = -t / l;
                Grow[k] = g;
                a.Gt[(size_t)k * a.cap + n] = g;
                double4 al = ldcg_d4(&a.alpha[k]);
                al.x = fma(wn0, g, al.x);
                al.y = fma(wn1, g, al.y);
                al.z = fma(wn2, g, al.z);
                a.alpha[k] = al;
            }
        }
        if (first_block) a.st->n = n + 1;
        RBFD_SYNC(3)
        ++n;
    }
    RBFD_EXIT()
#undef RBFD_SYNC
#undef RBFD_EXIT
}

template <int DIM, int BASIS, int MODE>
const void *kernel_ptr() {
    return reinterpret_cast<const void *>(&k_greedy_persist<DIM, BASIS, MODE>);
}

const void *select_kernel(int dim, int basis, int mode) {
#define RBFD_SEL(D, B)                                                                  \
    if (dim == D && basis == B) return mode == 0 ? kernel_ptr<D, B, 0>() : kernel_ptr<D, B, 1>();
    RBFD_SEL(2, 0) RBFD_SEL(2, 2) RBFD_SEL(2, 4) RBFD_SEL(2, 6)
    RBFD_SEL(3, 0) RBFD_SEL(3, 2) RBFD_SEL(3, 4) RBFD_SEL(3, 6)
#undef RBFD_SEL
    return nullptr;
}

}  // namespace

int persist_max_ctas(rbfd_mesh *m) {
    const void *k = select_kernel(m->dim, m->opt.basis, m->opt.precision == RBFD_FP64 ? 0 : 1);
    int occ = 0, sms = 0;
    RBFD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, kT, 0));
    RBFD_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, m->device));
    return std::max(0, occ * sms);
}

void persist_run_level(rbfd_mesh *m, double R, double tau, int ctas, int max_steps) {
    PersistArgs a{};
    a.n_s = m->n_s;
    a.n_pb = m->n_pb;
    a.cap = m->cap;
    a.dim = m->dim;
    a.n_chunk_max = m->n_chunk_max;
    a.R = R;
    a.R2 = R * R;
    a.S0 = m->S0;
    a.tau = tau;
    a.piv_tol_per_n = 8.0 * 1.1102230246251565e-16;
    const double inv = 1.0 / R;
    a.invR_hi = (float)inv;
    a.invR_lo = (float)(inv - (double)a.invR_hi);
    a.xs = m->d_xs;
    a.pb_org = m->d_pb_org;
    a.pb_lo = m->d_pb_lo;
    a.pb_hi = m->d_pb_hi;
    a.cur = m->d_cur;
    a.xs_hi = m->d_xs_hi;
    a.xs_lo = m->d_xs_lo;
    a.perm = m->d_perm;
    a.inv = m->d_inv;
    a.sel = m->d_sel;
    a.nb_cnt = m->d_nb_cnt;
    a.nb_list = m->d_nb_list;
    a.cx = m->d_cx;
    a.cdf = m->d_cdf;
    a.alpha = m->d_alpha;
    a.w = m->d_w;
    a.cid = m->d_cid;
    a.G = m->d_G;
    a.Gt = m->d_Gt;
    a.phi = m->d_phi;
    a.y = m->d_y;
    a.red = m->d_pred;
    a.nz_k = m->d_nz_k;
    a.nz_v = m->d_nz_v;
    a.part = m->d_part;
    a.pb_done = m->d_pb_done;
    a.gpart = m->d_gpart4;
    a.grp_done = m->d_grp_done;
    a.max_grp = (m->n_chunk_max + kRG - 1) / kRG;
    // (the completion counters start at zero even after a launch that ended early)
    RBFD_CUDA(cudaMemsetAsync(a.pb_done, 0, sizeof(unsigned) * (size_t)m->n_pb, m->stream));
    RBFD_CUDA(cudaMemsetAsync(a.grp_done, 0, sizeof(unsigned) * (size_t)m->n_pb * a.max_grp, m->stream));
    RBFD_CUDA(cudaMemsetAsync(&m->d_st->red_done, 0, sizeof(unsigned), m->stream));
    a.pb_key = m->d_pb_key;
    a.pb_idx = m->d_pb_idx;
    a.bar = m->d_bar;
    a.spin_limit = 1ull << 24;  // polls of an L2 word (~0.1-0.5 us each): seconds at most
    // test hooks (environment, read per call): a short poll bound, and block 0
    // skipping its first barrier arrival so that the others' waits run out
    if (const char *v = std::getenv("RBFD_TEST_BARRIER_POLLS")) a.spin_limit = std::strtoull(v, nullptr, 10);
    if (const char *v = std::getenv("RBFD_TEST_SKIP_ARRIVAL")) a.test_skip_arrival = std::atoi(v) != 0;
    // (and the round-robin sweep items at any size, to check both assignments)
    a.pfx_max = kPfxMax;
    if (const char *v = std::getenv("RBFD_TEST_SWEEP_ROUND_ROBIN")) a.pfx_max = std::atoi(v) != 0 ? 0 : kPfxMax;
    // controls per sweep item: shorter items balance the step's tail, longer
    // ones cost fewer partial sums (RBFD_SWEEP_CHUNK sets it, 16 to 1024).
    // With the pruned sweep a step has few point blocks to sweep, so short
    // items win: the 60k wing's step took 9.96 / 10.10 / 10.42 / 10.75 s at
    // 32 / 64 / 96 / 128 controls.
    a.max_steps = max_steps;
    a.chunk_target = 32;
    if (const char *v = std::getenv("RBFD_SWEEP_CHUNK")) a.chunk_target = std::max(16, std::min(1024, std::atoi(v)));
    a.prune = (m->opt.prune && m->d_bnd && m->d_bacc && m->d_wbox && m->n_pb <= a.pfx_max) ? 1 : 0;
    // relative rounding per operation: FP64 2^-53, double-float about 2^-44;
    // a factor 16 of margin on each
    a.err_u = m->opt.precision == RBFD_FP64 ? 0x1p-49f : 0x1p-40f;
    a.S0f = (float)(m->S0 * (1.0 + 0x1p-20));
    a.bnd = m->d_bnd;
    a.bacc = m->d_bacc;
    a.wbox = m->d_wbox;
    {
        // FP32 rounding of a control-to-box distance: the control's hi part
        // (2^-24 relative per coordinate) and the arithmetic, with margin
        double xmax = R;
        for (int q = 0; q < 6; ++q) xmax = std::max(xmax, std::fabs(m->h_sbox[q]));
        a.marg = (float)(0x1p-19 * (xmax + R));
    }
    a.rev = m->d_rev;
    a.rev_cnt = m->d_rev_cnt;
    if (a.prune) RBFD_CUDA(cudaMemsetAsync(a.rev_cnt, 0, sizeof(uint32_t) * (size_t)(m->cap + 1), m->stream));
    a.phase_ns = m->prof.on ? m->d_phase_ns : nullptr;
    a.item_ctr = reinterpret_cast<unsigned long long *>(&m->d_misc[10]);  // (8-byte aligned)
    RBFD_CUDA(cudaMemsetAsync(a.item_ctr, 0, sizeof(unsigned long long), m->stream));
    a.st = m->d_st;
    a.pairs = m->d_pairs;
    const void *k = select_kernel(m->dim, m->opt.basis, m->opt.precision == RBFD_FP64 ? 0 : 1);
    if (!k) fail(RBFD_EINVAL, "persistent greedy: unsupported dim/basis");
    void *args[] = {&a};
    RBFD_CUDA(cudaLaunchCooperativeKernel(k, dim3(ctas), dim3(kT), args, 0, m->stream));
    m->stats.launches += 1;
}

}  // namespace rbfd
