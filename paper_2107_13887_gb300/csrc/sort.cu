// sort.cu -- spatial preparation primitives: Morton keys, a stable LSD radix
// sort of (key, value) pairs, and a device-wide exclusive scan (used for
// stream compaction of the volume points and for the sort's digit offsets).
//
// All of these are HBM-bound streaming kernels: coalesced loads of one tile
// per block, shared-memory histograms, and one write pass per radix digit.
#include <algorithm>

#include "internal.h"

namespace rbfd {

namespace {

constexpr int RS_THREADS = 256;
constexpr int RS_ITEMS = 8;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;
constexpr int SC_THREADS = 256;
constexpr int SC_ITEMS = 8;
constexpr int SC_TILE = SC_THREADS * SC_ITEMS;
static_assert(RS_TILE == kSortTile && SC_TILE == kScanTile, "tile sizes of internal.h");

__global__ void k_rs_hist(const uint32_t *__restrict__ keys, size_t n, int shift, uint32_t dmask,
                          uint32_t *__restrict__ hist, int nblk) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    size_t base = (size_t)blockIdx.x * RS_TILE;
#pragma unroll
    for (int r = 0; r < RS_ITEMS; ++r) {
        size_t i = base + (size_t)r * RS_THREADS + threadIdx.x;
        if (i < n) atomicAdd(&h[(keys[i] >> shift) & dmask], 1u);
    }
    __syncthreads();
    hist[(size_t)threadIdx.x * nblk + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter: items keep their input order among equal digits.  Each
// round ranks 256 consecutive items with warp match + per-warp digit counts.
__global__ void k_rs_scatter(const uint32_t *__restrict__ kin, const uint32_t *__restrict__ vin,
                             uint32_t *__restrict__ kout, uint32_t *__restrict__ vout, size_t n, int shift,
                             uint32_t dmask, const uint32_t *__restrict__ offs, int nblk) {
    __shared__ uint32_t base[256];
    __shared__ uint32_t wcnt[RS_THREADS / 32][256];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    base[tid] = offs[(size_t)tid * nblk + blockIdx.x];
    const unsigned lt = (1u << lane) - 1u;
    size_t tile = (size_t)blockIdx.x * RS_TILE;
    for (int r = 0; r < RS_ITEMS; ++r) {
        for (int q = tid; q < (RS_THREADS / 32) * 256; q += RS_THREADS) (&wcnt[0][0])[q] = 0;
        size_t i = tile + (size_t)r * RS_THREADS + tid;
        bool valid = i < n;
        uint32_t k = valid ? kin[i] : 0u;
        uint32_t v = valid ? vin[i] : 0u;
        uint32_t d = valid ? ((k >> shift) & dmask) : 256u;
        __syncthreads();
        unsigned peers = __match_any_sync(0xffffffffu, d);
        int lrank = __popc(peers & lt);
        if (valid && lrank == 0) wcnt[warp][d] = __popc(peers);
        __syncthreads();
        if (valid) {
            uint32_t pre = 0;
            for (int w = 0; w < warp; ++w) pre += wcnt[w][d];
            uint32_t pos = base[d] + pre + lrank;
            kout[pos] = k;
            vout[pos] = v;
        }
        __syncthreads();
        uint32_t tot = 0;
#pragma unroll
        for (int w = 0; w < RS_THREADS / 32; ++w) tot += wcnt[w][tid];
        base[tid] += tot;
        __syncthreads();
    }
}

// --- scan

__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t *sw, uint32_t *total) {
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
        if (lane < nw) sw[lane] = t;  // inclusive warp totals
    }
    __syncthreads();
    uint32_t before = (w > 0 ? sw[w - 1] : 0u) + x - v;
    if (total) *total = sw[nw - 1];
    __syncthreads();
    return before;
}

__global__ void k_scan_reduce(const uint32_t *__restrict__ in, size_t n, uint32_t *__restrict__ sums) {
    __shared__ uint32_t sw[32];
    size_t base = (size_t)blockIdx.x * SC_TILE + (size_t)threadIdx.x * SC_ITEMS;
    uint32_t s = 0;
#pragma unroll
    for (int r = 0; r < SC_ITEMS; ++r)
        if (base + r < n) s += in[base + r];
    uint32_t tot;
    block_excl_scan(s, sw, &tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

__global__ void k_scan_top(uint32_t *sums, int nb, uint32_t *total) {
    __shared__ uint32_t sw[32];
    __shared__ uint32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int b0 = 0; b0 < nb; b0 += blockDim.x) {
        int i = b0 + threadIdx.x;
        uint32_t v = i < nb ? sums[i] : 0u;
        uint32_t tot;
        uint32_t ex = block_excl_scan(v, sw, &tot);
        if (i < nb) sums[i] = carry + ex;
        __syncthreads();
        if (threadIdx.x == 0) carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0 && total) *total = carry;
}

__global__ void k_scan_down(const uint32_t *in, uint32_t *out, size_t n, const uint32_t *__restrict__ sums) {
    __shared__ uint32_t sw[32];
    size_t base = (size_t)blockIdx.x * SC_TILE + (size_t)threadIdx.x * SC_ITEMS;
    uint32_t v[SC_ITEMS];
    uint32_t s = 0;
#pragma unroll
    for (int r = 0; r < SC_ITEMS; ++r) {
        v[r] = (base + r < n) ? in[base + r] : 0u;
        s += v[r];
    }
    uint32_t ex = block_excl_scan(s, sw, nullptr) + sums[blockIdx.x];
#pragma unroll
    for (int r = 0; r < SC_ITEMS; ++r) {
        if (base + r < n) out[base + r] = ex;
        ex += v[r];
    }
}

// --- Morton

__device__ __forceinline__ uint32_t spread2(uint32_t x) {  // 16 bits -> even bits
    x &= 0xffffu;
    x = (x | (x << 8)) & 0x00ff00ffu;
    x = (x | (x << 4)) & 0x0f0f0f0fu;
    x = (x | (x << 2)) & 0x33333333u;
    x = (x | (x << 1)) & 0x55555555u;
    return x;
}

__device__ __forceinline__ uint32_t spread3(uint32_t x) {  // 10 bits -> every third bit
    x &= 0x3ffu;
    x = (x | (x << 16)) & 0x030000ffu;
    x = (x | (x << 8)) & 0x0300f00fu;
    x = (x | (x << 4)) & 0x030c30c3u;
    x = (x | (x << 2)) & 0x09249249u;
    return x;
}

__device__ __forceinline__ uint32_t quant(double v, double lo, double inv, uint32_t qmax) {
    double t = (v - lo) * inv;
    if (!(t > 0.0)) return 0u;
    if (t >= 1.0) return qmax;
    return (uint32_t)(t * (double)qmax);
}

__device__ __forceinline__ uint32_t morton(double x, double y, double z, int dim, double3 lo, double3 inv) {
    if (dim == 2) {
        return (spread2(quant(y, lo.y, inv.y, 0xffffu)) << 1) | spread2(quant(x, lo.x, inv.x, 0xffffu));
    }
    return (spread3(quant(z, lo.z, inv.z, 0x3ffu)) << 2) | (spread3(quant(y, lo.y, inv.y, 0x3ffu)) << 1) |
           spread3(quant(x, lo.x, inv.x, 0x3ffu));
}

// Morton keys with the box read from device memory (lo xyz, hi xyz), so that
// no host round trip separates the box reduction from the keys.  The three
// reciprocal extents are computed once per block (an FP64 division costs
// several times the rest of a key).  iso: every axis takes the box's longest
// extent (cubic cells; a thin box would otherwise get cells much finer
// across it than along it, and runs of consecutive keys long boxes).
__global__ void k_morton_f64_dev(const double4 *__restrict__ p, size_t n, int dim, const double *__restrict__ bb,
                                 int shift, int iso, uint32_t *keys, uint32_t *vals) {
    __shared__ double s_lo[3], s_inv[3];
    if (threadIdx.x < 3) {
        const int a = threadIdx.x;
        s_lo[a] = bb[a];
        double e = bb[a + 3] - bb[a];
        if (iso) {
            e = fmax(bb[3] - bb[0], bb[4] - bb[1]);
            if (dim == 3) e = fmax(e, bb[5] - bb[2]);
        }
        s_inv[a] = (e > 0.0) ? 1.0 / e : 0.0;
    }
    __syncthreads();
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double3 lo = make_double3(s_lo[0], s_lo[1], s_lo[2]);
    const double3 inv = make_double3(s_inv[0], s_inv[1], s_inv[2]);
    double4 q = p[i];
    keys[i] = morton(q.x, q.y, q.z, dim, lo, inv) >> shift;
    vals[i] = (uint32_t)i;
}

__global__ void k_morton_f32(const float4 *__restrict__ p, const uint32_t *__restrict__ idx, size_t n, int dim,
                             double3 lo, double3 inv, uint32_t *keys, uint32_t *vals) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t j = idx ? idx[i] : (uint32_t)i;
    float4 q = p[j];
    keys[i] = morton(q.x, q.y, q.z, dim, lo, inv);
    vals[i] = j;
}

double3 inv_extent(double3 lo, double3 hi) {
    auto f = [](double a, double b) { return (b > a) ? 1.0 / (b - a) : 0.0; };
    return make_double3(f(lo.x, hi.x), f(lo.y, hi.y), f(lo.z, hi.z));
}

inline unsigned grid1(size_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

void SortScratch::reserve(size_t n) {
    if (n > cap_items) {
        dfree(keys_alt);
        dfree(vals_alt);
        keys_alt = dalloc<uint32_t>(n, "sort keys");
        vals_alt = dalloc<uint32_t>(n, "sort values");
        cap_items = n;
    }
    const size_t nh = sort_hist_need(n);
    if (nh > cap_hist) {
        dfree(hist);
        hist = dalloc<uint32_t>(nh, "sort histogram");
        cap_hist = nh;
    }
    const size_t ns = sort_sums_need(n);
    if (ns > cap_sums) {
        dfree(block_sums);
        block_sums = dalloc<uint32_t>(ns, "scan block sums");
        cap_sums = ns;
    }
}

void SortScratch::release() {
    dfree(keys_alt);
    dfree(vals_alt);
    dfree(hist);
    dfree(block_sums);
    keys_alt = vals_alt = hist = block_sums = nullptr;
    cap_items = cap_hist = cap_sums = 0;
}

void exclusive_scan_u32(const uint32_t *in, uint32_t *out, size_t n, uint32_t *total_dev, SortScratch &s,
                        cudaStream_t st) {
    if (n == 0) {
        if (total_dev) RBFD_CUDA(cudaMemsetAsync(total_dev, 0, sizeof(uint32_t), st));
        return;
    }
    int nb = (int)((n + SC_TILE - 1) / SC_TILE);
    if ((size_t)nb + 2 > s.cap_sums) s.reserve(std::max(s.cap_items, n));
    k_scan_reduce<<<nb, SC_THREADS, 0, st>>>(in, n, s.block_sums);
    k_scan_top<<<1, 1024, 0, st>>>(s.block_sums, nb, total_dev);
    k_scan_down<<<nb, SC_THREADS, 0, st>>>(in, out, n, s.block_sums);
    RBFD_CUDA(cudaGetLastError());
    if (s.launches) *s.launches += 3;
}

// Small arrays in one block: a bitonic sort of the 64-bit values (low
// key_bits of the key) << 32 | position, which orders by key and keeps equal
// keys in input order (the same result as the stable radix sort), then keys
// and values are gathered by position.  One launch instead of five per 8-bit
// digit.  Thread t holds the E consecutive values E t .. E t + E - 1 in
// registers: compare-exchange partners closer than E are in the same thread,
// closer than 32 E in the same warp (shuffles), and only the farther ones go
// through shared memory (two block barriers per such stage; 15 of the 78
// stages of 4,096 values).
constexpr int kSmallSort = 8192;
constexpr int kSmallSortThreads = 1024;

// the kept value of a compare-exchange: the smaller one where the element
// sorts ascending and is the lower of the pair, or descending and the upper
__device__ __forceinline__ unsigned long long cx_keep(unsigned long long mine, unsigned long long other, bool asc,
                                                      bool lower) {
    const bool take_min = asc == lower;
    const unsigned long long lo = mine < other ? mine : other, hi = mine < other ? other : mine;
    return take_min ? lo : hi;
}

// partners J apart inside the thread (J < E)
template <int E, int J>
__device__ __forceinline__ void cx_in_thread(unsigned long long (&c)[E], int base, int k) {
#pragma unroll
    for (int r = 0; r < E; ++r) {
        if ((r & J) == 0) {
            const bool asc = ((base + r) & k) == 0;
            const unsigned long long a = c[r], b = c[r | J];
            if ((a > b) == asc) {
                c[r] = b;
                c[r | J] = a;
            }
        }
    }
}

// The bitonic network over the block's N values, E per thread in registers
// (element E t + r in c[r] of thread t); s_c: N values of shared memory.
template <int E>
__device__ __forceinline__ void bitonic_regs(unsigned long long (&c)[E], int N, unsigned long long *s_c) {
    const int base = E * (int)threadIdx.x;
    for (int k = 2; k <= N; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            if (j >= 32 * E) {  // partner in another warp
#pragma unroll
                for (int r = 0; r < E; ++r) s_c[base + r] = c[r];
                __syncthreads();
#pragma unroll
                for (int r = 0; r < E; ++r) {
                    const int i = base + r;
                    c[r] = cx_keep(c[r], s_c[i ^ j], (i & k) == 0, (i & j) == 0);
                }
                __syncthreads();
            } else if (j >= E) {  // partner in another lane of this warp, same register
#pragma unroll
                for (int r = 0; r < E; ++r) {
                    const int i = base + r;
                    const unsigned long long o = __shfl_xor_sync(0xffffffffu, c[r], j / E);
                    c[r] = cx_keep(c[r], o, (i & k) == 0, (i & j) == 0);
                }
            } else {  // same thread
                if constexpr (E > 4) { if (j == 4) cx_in_thread<E, 4>(c, base, k); }
                if constexpr (E > 2) { if (j == 2) cx_in_thread<E, 2>(c, base, k); }
                if constexpr (E > 1) { if (j == 1) cx_in_thread<E, 1>(c, base, k); }
            }
        }
    }
}

template <int E>
__global__ void __launch_bounds__(kSmallSortThreads) k_sort_small(uint32_t *keys, uint32_t *vals, int n, int N,
                                                                   uint32_t mask) {
    extern __shared__ unsigned long long s_c[];  // [N] values (far stages), then [n] (key, value) pairs
    uint2 *s_kv = reinterpret_cast<uint2 *>(s_c + N);
    const int base = E * (int)threadIdx.x;
    unsigned long long c[E];
#pragma unroll
    for (int r = 0; r < E; ++r) {
        const int i = base + r;
        if (i < n) {
            const uint32_t kk = keys[i];
            s_kv[i] = make_uint2(kk, vals[i]);
            c[r] = ((unsigned long long)(kk & mask) << 32) | (unsigned)i;
        } else {
            c[r] = ~0ull;  // padding sorts last
        }
    }
    bitonic_regs<E>(c, N, s_c);
#pragma unroll
    for (int r = 0; r < E; ++r) {
        const int i = base + r;
        if (i < n) {
            const uint2 kv = s_kv[(unsigned)c[r]];
            keys[i] = kv.x;
            vals[i] = kv.y;
        }
    }
}

void radix_sort_pairs(uint32_t *keys, uint32_t *vals, size_t n, int key_bits, SortScratch &s, cudaStream_t st) {
    if (n <= 1) return;
    if (n <= (size_t)kSmallSort) {
        // N = n rounded up to a power of two, at least a warp; T threads of E values each
        int N = 32;
        while (N < (int)n) N <<= 1;
        const int T = std::min(N, kSmallSortThreads), E = N / T;
        const size_t smem = (size_t)N * 8 + n * 8;
        const uint32_t mask = key_bits >= 32 ? 0xffffffffu : ((1u << key_bits) - 1u);
        auto launch = [&](auto kern) {
            // (one value for every launch and device: the attribute belongs to the kernel)
            if (smem > 48 * 1024)
                RBFD_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmallSort * 16));
            kern<<<1, T, smem, st>>>(keys, vals, (int)n, N, mask);
        };
        if (E == 1) launch(k_sort_small<1>);
        else if (E == 2) launch(k_sort_small<2>);
        else if (E == 4) launch(k_sort_small<4>);
        else launch(k_sort_small<8>);
        if (s.launches) *s.launches += 1;
        RBFD_CUDA(cudaGetLastError());
        return;
    }
    s.reserve(n);
    int nblk = (int)((n + RS_TILE - 1) / RS_TILE);
    uint32_t *ka = keys, *va = vals, *kb = s.keys_alt, *vb = s.vals_alt;
    int passes = (key_bits + 7) / 8;
    for (int p = 0; p < passes; ++p) {
        int shift = 8 * p;
        // (the last digit holds only the key bits that are left)
        const uint32_t dmask = (p == passes - 1 && key_bits % 8) ? (1u << (key_bits % 8)) - 1u : 255u;
        k_rs_hist<<<nblk, RS_THREADS, 0, st>>>(ka, n, shift, dmask, s.hist, nblk);
        exclusive_scan_u32(s.hist, s.hist, (size_t)256 * nblk, nullptr, s, st);
        k_rs_scatter<<<nblk, RS_THREADS, 0, st>>>(ka, va, kb, vb, n, shift, dmask, s.hist, nblk);
        if (s.launches) *s.launches += 2;
        std::swap(ka, kb);
        std::swap(va, vb);
    }
    if (ka != keys) {
        RBFD_CUDA(cudaMemcpyAsync(keys, ka, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, st));
        RBFD_CUDA(cudaMemcpyAsync(vals, va, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, st));
    }
    RBFD_CUDA(cudaGetLastError());
}

void morton_keys_f64_dev(const double4 *xyz, size_t n, int dim, const double *bbox, uint32_t *keys, uint32_t *vals,
                         cudaStream_t st, int shift, bool iso) {
    if (!n) return;
    k_morton_f64_dev<<<grid1(n, 256), 256, 0, st>>>(xyz, n, dim, bbox, shift, iso ? 1 : 0, keys, vals);
    RBFD_CUDA(cudaGetLastError());
}

void morton_keys_f32(const float4 *xyzd, const uint32_t *idx, size_t n, int dim, double3 lo, double3 hi,
                     uint32_t *keys, uint32_t *vals, cudaStream_t st) {
    if (!n) return;
    k_morton_f32<<<grid1(n, 256), 256, 0, st>>>(xyzd, idx, n, dim, lo, inv_extent(lo, hi), keys, vals);
    RBFD_CUDA(cudaGetLastError());
}

}  // namespace rbfd
