// api.cu -- the extern "C" boundary declared in include/rbfd.h.  Every entry
// point validates its arguments, converts internal errors into an
// rbfd_status, and records a thread-local message for rbfd_last_error().
#include <cmath>
#include <condition_variable>
#include <cstdlib>
#include <deque>
#include <functional>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>

#include "internal.h"

namespace rbfd {

static thread_local std::string g_last_error;

void set_last_error(const std::string &msg) { g_last_error = msg; }

void fail(int status, const std::string &msg) { throw Error{status, msg}; }

void check_cuda(cudaError_t e, const char *what) {
    if (e == cudaSuccess) return;
    cudaGetLastError();  // clear a sticky-free error so later calls can proceed
    if (e == cudaErrorMemoryAllocation) fail(RBFD_ENOMEM, std::string(what) + ": out of device memory");
    fail(RBFD_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// ------------------------------------------------------- device memory pool
//
// Meshes are created and destroyed per deformation request; the ~45 buffers a
// mesh owns would otherwise cost a cudaMalloc each and a device-synchronising
// cudaFree each.  Freed blocks are kept per device in a size-ordered free list
// and handed out again for requests of up to twice their size.  Every free in
// the library happens after the owning stream has been synchronised, so a
// block is idle when it is reused.  The cache is trimmed (cudaFree) when it
// grows past a limit (RBFD_POOL_LIMIT_MB, default 16384) or when cudaMalloc
// runs out of memory.
namespace {

constexpr int kPoolDevices = 64;

struct DevicePool {
    std::mutex mu;
    std::multimap<size_t, void *> free_blocks[kPoolDevices];
    std::unordered_map<void *, std::pair<int, size_t>> live;
    size_t cached[kPoolDevices] = {};
    size_t limit = 0;
};

DevicePool &pool() {
    static DevicePool *p = [] {
        auto *q = new DevicePool();  // never destroyed: safe to use during process exit
        const char *v = std::getenv("RBFD_POOL_LIMIT_MB");
        q->limit = (v ? std::strtoull(v, nullptr, 10) : 16384ull) << 20;
        return q;
    }();
    return *p;
}

void trim_locked(DevicePool &P, int dev, size_t keep) {
    while (P.cached[dev] > keep && !P.free_blocks[dev].empty()) {
        auto it = std::prev(P.free_blocks[dev].end());  // largest first
        int cur = 0;
        cudaGetDevice(&cur);
        if (cur != dev) cudaSetDevice(dev);
        cudaFree(it->second);
        if (cur != dev) cudaSetDevice(cur);
        P.cached[dev] -= it->first;
        P.free_blocks[dev].erase(it);
    }
}

}  // namespace

// Host-side fault injection for tests: with RBFD_TEST_ENOMEM_AT=N in the
// environment, the N-th device allocation after the variable last changed
// fails as if the device were out of memory (no GPU fault, no real
// exhaustion: the failure path of every caller is exercised on the host).
static bool injected_enomem() {
    static std::mutex mu;
    static std::string seen;
    static long count = 0;
    const char *v = std::getenv("RBFD_TEST_ENOMEM_AT");
    std::lock_guard<std::mutex> lk(mu);
    const std::string cur = v ? v : "";
    if (cur != seen) {
        seen = cur;
        count = 0;
    }
    if (cur.empty()) return false;
    return ++count == std::strtol(cur.c_str(), nullptr, 10);
}

void *dmalloc(size_t bytes, const char *what) {
    if (injected_enomem())
        fail(RBFD_ENOMEM, std::string("allocating ") + what + ": out of device memory (injected by RBFD_TEST_ENOMEM_AT)");
    const size_t sz = ((bytes ? bytes : 1) + 511) / 512 * 512;
    int dev = 0;
    check_cuda(cudaGetDevice(&dev), "cudaGetDevice");
    if (dev < 0 || dev >= kPoolDevices) fail(RBFD_EINVAL, "device index out of range for the memory pool");
    DevicePool &P = pool();
    {
        std::lock_guard<std::mutex> lk(P.mu);
        auto it = P.free_blocks[dev].lower_bound(sz);
        if (it != P.free_blocks[dev].end() && it->first <= 2 * sz) {
            void *p = it->second;
            P.cached[dev] -= it->first;
            P.live[p] = {dev, it->first};
            P.free_blocks[dev].erase(it);
            return p;
        }
    }
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, sz);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        {
            std::lock_guard<std::mutex> lk(P.mu);
            trim_locked(P, dev, 0);
        }
        e = cudaMalloc(&p, sz);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        fail(e == cudaErrorMemoryAllocation ? RBFD_ENOMEM : RBFD_ECUDA,
             std::string("allocating ") + what + " (" + std::to_string(bytes) + " bytes): " + cudaGetErrorString(e));
    }
    std::lock_guard<std::mutex> lk(P.mu);
    P.live[p] = {dev, sz};
    return p;
}

void dfree(void *p) {
    if (!p) return;
    DevicePool &P = pool();
    std::lock_guard<std::mutex> lk(P.mu);
    auto it = P.live.find(p);
    if (it == P.live.end()) {
        cudaFree(p);  // not from the pool
        return;
    }
    const int dev = it->second.first;
    const size_t sz = it->second.second;
    P.live.erase(it);
    P.free_blocks[dev].insert({sz, p});
    P.cached[dev] += sz;
    if (P.cached[dev] > P.limit) trim_locked(P, dev, P.limit / 2);
}

// Pinned host words for the greedy state mirror (cudaMallocHost is slow).
namespace {
std::mutex g_pin_mu;
std::vector<void *> g_pin_free;
}  // namespace

void *pinned_alloc(size_t bytes) {
    if (bytes > 4096) fail(RBFD_EINVAL, "pinned_alloc: block too large");
    {
        std::lock_guard<std::mutex> lk(g_pin_mu);
        if (!g_pin_free.empty()) {
            void *p = g_pin_free.back();
            g_pin_free.pop_back();
            return p;
        }
    }
    void *p = nullptr;
    check_cuda(cudaMallocHost(&p, 4096), "cudaMallocHost");
    return p;
}

void pinned_free(void *p) {
    if (!p) return;
    std::lock_guard<std::mutex> lk(g_pin_mu);
    g_pin_free.push_back(p);
}

cudaEvent_t Profiler::get() {
    if (!free_ev.empty()) {
        cudaEvent_t e = free_ev.back();
        free_ev.pop_back();
        return e;
    }
    cudaEvent_t e;
    RBFD_CUDA(cudaEventCreate(&e));
    return e;
}

cudaEvent_t Profiler::begin(cudaStream_t st) {
    if (!on) return nullptr;
    cudaEvent_t a = get();
    RBFD_CUDA(cudaEventRecord(a, st));
    return a;
}

void Profiler::end(int kind, cudaEvent_t a, cudaStream_t st, int n_launches) {
    launches[kind] += n_launches;
    if (!on || !a) return;
    cudaEvent_t b = get();
    RBFD_CUDA(cudaEventRecord(b, st));
    pend.push_back({kind, a, b});
}

void Profiler::flush() {
    // pairs whose end has not been reached yet (work on another stream) stay pending
    std::vector<Pending> keep;
    for (auto &p : pend) {
        if (cudaEventQuery(p.b) == cudaErrorNotReady) {
            cudaGetLastError();
            keep.push_back(p);
            continue;
        }
        float ms_ = 0.f;
        if (cudaEventElapsedTime(&ms_, p.a, p.b) == cudaSuccess) ms[p.kind] += ms_;
        else cudaGetLastError();
        free_ev.push_back(p.a);
        free_ev.push_back(p.b);
    }
    pend.swap(keep);
}

void Profiler::release() {
    for (auto &p : pend) {
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
    }
    pend.clear();
    for (auto e : free_ev) cudaEventDestroy(e);
    free_ev.clear();
}

void mesh_free(rbfd_mesh *m) {
    if (!m) return;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(m->device);
    if (m->stream) cudaStreamSynchronize(m->stream);
    rbfd::volume_stage_release(m);
    if (m->prep_temps) dfree(m->prep_temps);
    if (m->h_prep) pinned_free(m->h_prep);
    for (auto &L : m->levels) rbfd::level_free(L);
    for (auto &L : m->warm_prev) rbfd::level_free(L);
    // (the mesh's fixed buffers are carved out of d_arena)
    void *ptrs[] = {m->d_arena, m->d_G, m->d_Gt, m->d_vin, m->d_vpos, m->d_vorig, m->d_vflag, m->d_vscan,
                    m->d_vlist, m->d_vkeys, m->d_vacc, m->d_vio, m->d_vreg, m->d_vreg_orig, m->d_pb_fbox,
                    m->d_V, m->d_nrec, m->d_nycol, m->d_nwdf, m->d_ckeys, m->d_vpos4, m->d_wl_list,
                    m->d_wl_cnt};
    for (void *p : ptrs) dfree(p);
    m->sort.release();
    m->prof.release();
    if (m->h_st) pinned_free(m->h_st);
    if (m->h_bar) pinned_free(m->h_bar);
    if (m->h_lvl) pinned_free(m->h_lvl);
    if (m->ev0) cudaEventDestroy(m->ev0);
    if (m->ev1) cudaEventDestroy(m->ev1);
    if (m->ev_g0) cudaEventDestroy(m->ev_g0);
    if (m->ev_g1) cudaEventDestroy(m->ev_g1);
    if (m->own_stream && m->stream) cudaStreamDestroy(m->stream);
    cudaSetDevice(prev);
}

}  // namespace rbfd

using rbfd::Error;

namespace {

template <typename F>
int guarded(F &&f) {
    try {
        f();
        rbfd::g_last_error.clear();
        return RBFD_OK;
    } catch (const Error &e) {
        rbfd::g_last_error = e.msg;
        return e.status;
    } catch (const std::bad_alloc &) {
        rbfd::g_last_error = "host allocation failed";
        return RBFD_ENOMEM;
    } catch (...) {
        rbfd::g_last_error = "unexpected internal error";
        return RBFD_ECUDA;
    }
}

bool is_device_ptr(const void *p) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Host threads for the batch calls, kept for the process (starting a thread
// costs tens of microseconds, waking a waiting one a few).
class WorkerPool {
public:
    static WorkerPool &get() {
        static WorkerPool *p = new WorkerPool;  // (never destroyed: its threads wait for the process to end)
        return *p;
    }
    // run task(i) for 1 <= i < n on the pool, task(0) on the calling thread, and wait
    void run(int n, const std::function<void(int)> &task) {
        if (n <= 0) return;
        int left = n - 1;
        std::mutex done_mu;
        std::condition_variable done_cv;
        {
            std::lock_guard<std::mutex> lk(mu_);
            while (idle_ < n - 1 + (int)queue_.size()) {
                std::thread([this] { loop(); }).detach();
                ++idle_;
            }
            for (int i = 1; i < n; ++i)
                queue_.push_back([&, i] {
                    task(i);
                    std::lock_guard<std::mutex> dl(done_mu);
                    if (--left == 0) done_cv.notify_one();
                });
        }
        cv_.notify_all();
        task(0);
        std::unique_lock<std::mutex> dl(done_mu);
        done_cv.wait(dl, [&] { return left == 0; });
    }

private:
    void loop() {
        for (;;) {
            std::function<void()> job;
            {
                std::unique_lock<std::mutex> lk(mu_);
                cv_.wait(lk, [this] { return !queue_.empty(); });
                job = std::move(queue_.front());
                queue_.pop_front();
                --idle_;
            }
            job();
            std::lock_guard<std::mutex> lk(mu_);
            ++idle_;
        }
    }
    std::mutex mu_;
    std::condition_variable cv_;
    std::deque<std::function<void()>> queue_;
    int idle_ = 0;
};

// Run f(i) for i < n on n host threads (the calling thread takes i = 0);
// returns the statuses, and the message of the first failure in *msg.
template <typename F>
int run_batch(int n, F &&f, const char *name) {
    std::vector<int> rc(n, RBFD_OK);
    std::vector<std::string> msg(n);
    auto body = [&](int i) {
        rc[i] = guarded([&] { f(i); });
        if (rc[i] != RBFD_OK) msg[i] = rbfd::g_last_error;
    };
    WorkerPool::get().run(n, body);
    int worst = RBFD_OK;
    std::string wmsg;
    for (int i = 0; i < n; ++i) {
        if (rc[i] == RBFD_OK) continue;
        if (worst == RBFD_OK || (worst == RBFD_ENOTCONV && rc[i] != RBFD_ENOTCONV)) {
            worst = rc[i];
            wmsg = std::string(name) + ": mesh " + std::to_string(i) + ": " + msg[i];
        }
    }
    rbfd::g_last_error = wmsg;
    return worst;
}

// Meshes whose greedy runs side by side: their persistent grids must be
// resident together, so each takes a share of the blocks.
int share_grid(rbfd_mesh **meshes, int n) {
    int cap = 0;
    if (n > 1) {
        int total = 0;
        int rc = guarded([&] {
            RBFD_CUDA(cudaSetDevice(meshes[0]->device));
            total = rbfd::persist_max_ctas(meshes[0]);
        });
        if (rc != RBFD_OK) return rc;
        cap = std::max(1, total / n);
    }
    for (int i = 0; i < n; ++i) {
        meshes[i]->batch_ctas_cap = cap;
        meshes[i]->batch_share = n;
    }
    return RBFD_OK;
}

void unshare_grid(rbfd_mesh **meshes, int n) {
    for (int i = 0; i < n; ++i) {
        meshes[i]->batch_ctas_cap = 0;
        meshes[i]->batch_share = 0;
    }
}


}  // namespace

extern "C" {

void rbfd_options_default(rbfd_options *opt) {
    if (!opt) return;
    std::memset(opt, 0, sizeof(*opt));
    opt->precision = RBFD_MIXED;
    opt->basis = 2;
    opt->first_point = 0;
    opt->inputs_on_device = 0;
    opt->nc_cap = 0;
    opt->stream = nullptr;
    opt->eps_absolute = 0;
    opt->refine_iters = 3;
    opt->profile = 0;
    opt->engine = 0;
    opt->grid_ctas = 0;
    opt->prune = 1;
}

int rbfd_create(rbfd_mesh **out, int dim, int64_t n_s, const double *xyz_s, const double *dS, int n_levels,
                const double *R, double eps, const rbfd_options *opt) {
    if (out) *out = nullptr;
    rbfd_mesh *m = nullptr;
    int rc = guarded([&] {
        if (!out) rbfd::fail(RBFD_EINVAL, "rbfd_create: out is NULL");
        if (dim != 2 && dim != 3) rbfd::fail(RBFD_EINVAL, "rbfd_create: dim must be 2 or 3");
        if (n_s < 1 || n_s > (int64_t)1 << 30) rbfd::fail(RBFD_EINVAL, "rbfd_create: n_s must be in [1, 2^30]");
        if (!xyz_s || !dS || !R) rbfd::fail(RBFD_EINVAL, "rbfd_create: NULL input pointer");
        if (n_levels < 1 || n_levels > 64) rbfd::fail(RBFD_EINVAL, "rbfd_create: n_levels must be in [1, 64]");
        rbfd_options o;
        rbfd_options_default(&o);
        if (opt) o = *opt;
        if (o.basis != 0 && o.basis != 2 && o.basis != 4 && o.basis != 6)
            rbfd::fail(RBFD_EINVAL, "rbfd_create: basis must be 0, 2, 4 or 6");
        if (o.precision != RBFD_FP64 && o.precision != RBFD_MIXED)
            rbfd::fail(RBFD_EINVAL, "rbfd_create: unknown precision");
        // C4 and C6 run in FP64 whatever the precision asked: their weights
        // reach about 1e9 max|dS| on the 2D ice cases, beyond what the
        // double-float sweeps (about 2^-44 relative) resolve
        if (o.basis >= 4) o.precision = RBFD_FP64;
        if (o.nc_cap < 0) rbfd::fail(RBFD_EINVAL, "rbfd_create: nc_cap must be >= 0");
        if (o.engine < 0 || o.engine > 2) rbfd::fail(RBFD_EINVAL, "rbfd_create: engine must be 0, 1 or 2");
        if (o.grid_ctas < 0 || o.grid_ctas > rbfd::kMaxPersistCTAs)
            rbfd::fail(RBFD_EINVAL, "rbfd_create: grid_ctas must be in [0, 2048]");
        if (o.prune != 0 && o.prune != 1) rbfd::fail(RBFD_EINVAL, "rbfd_create: prune must be 0 or 1");
        if (!(eps > 0.0) || (!o.eps_absolute && !(eps < 1.0)) || !std::isfinite(eps))
            rbfd::fail(RBFD_EINVAL, "rbfd_create: eps must be in (0, 1) (or > 0 when absolute)");
        for (int l = 0; l < n_levels; ++l)
            if (!(R[l] > 0.0) || !std::isfinite(R[l])) rbfd::fail(RBFD_EINVAL, "rbfd_create: every R must be > 0");
        if (o.inputs_on_device && (!is_device_ptr(xyz_s) || !is_device_ptr(dS)))
            rbfd::fail(RBFD_EINVAL, "rbfd_create: inputs_on_device set but inputs are not device memory");
        m = new rbfd_mesh();
        m->dim = dim;
        m->n_s = n_s;
        m->n_levels_req = n_levels;
        m->eps = eps;
        m->opt = o;
        m->R.assign(R, R + n_levels);
        RBFD_CUDA(cudaGetDevice(&m->device));
        if (o.stream) {
            m->stream = static_cast<cudaStream_t>(o.stream);
        } else {
            // the highest priority: the greedy's launches go ahead of the
            // volume work the library queues on its staging streams
            int lo = 0, hi = 0;
            RBFD_CUDA(cudaDeviceGetStreamPriorityRange(&lo, &hi));
            RBFD_CUDA(cudaStreamCreateWithPriority(&m->stream, cudaStreamNonBlocking, hi));
            m->own_stream = true;
        }
        RBFD_CUDA(cudaEventCreate(&m->ev0));
        RBFD_CUDA(cudaEventCreate(&m->ev1));
        RBFD_CUDA(cudaEventCreate(&m->ev_g0));
        RBFD_CUDA(cudaEventCreate(&m->ev_g1));
        m->prof.on = o.profile != 0;
        m->sort.launches = &m->stats.launches;
        rbfd::mesh_prepare(m, xyz_s, dS);
        *out = m;
    });
    if (rc != RBFD_OK && m) {
        rbfd::mesh_free(m);
        delete m;
    }
    return rc;
}

int rbfd_greedy(rbfd_mesh *m) {
    return guarded([&] {
        if (!m) rbfd::fail(RBFD_EINVAL, "rbfd_greedy: NULL mesh");
        RBFD_CUDA(cudaSetDevice(m->device));
        rbfd::greedy_run(m);
    });
}

int rbfd_greedy_warm(rbfd_mesh *m) {
    return guarded([&] {
        if (!m) rbfd::fail(RBFD_EINVAL, "rbfd_greedy_warm: NULL mesh");
        RBFD_CUDA(cudaSetDevice(m->device));
        m->keep_factors = true;
        rbfd::greedy_run(m, true, true);
    });
}

int rbfd_greedy_split(rbfd_mesh *m, int rank, int world, rbfd_maxloc_fn maxloc, void *user) {
    return guarded([&] {
        if (!m) rbfd::fail(RBFD_EINVAL, "rbfd_greedy_split: NULL mesh");
        if (world < 1 || rank < 0 || rank >= world)
            rbfd::fail(RBFD_EINVAL, "rbfd_greedy_split: rank " + std::to_string(rank) + " outside [0, world = " +
                                        std::to_string(world) + ")");
        if (!maxloc) rbfd::fail(RBFD_EINVAL, "rbfd_greedy_split: NULL maxloc callback");
        RBFD_CUDA(cudaSetDevice(m->device));
        // the split runs the step engine (one launch per sweep), whatever the options say
        const int engine = m->opt.engine;
        m->opt.engine = 1;
        m->split_world = world;
        m->split_rank = rank;
        m->split_maxloc = maxloc;
        m->split_user = user;
        struct Restore {
            rbfd_mesh *m;
            int engine;
            ~Restore() {
                m->opt.engine = engine;
                m->split_world = 1;
                m->split_rank = 0;
                m->split_maxloc = nullptr;
                m->split_user = nullptr;
            }
        } restore{m, engine};
        rbfd::greedy_run(m);
    });
}

int rbfd_num_levels(rbfd_mesh *m, int *n_levels) {
    return guarded([&] {
        if (!m || !n_levels) rbfd::fail(RBFD_EINVAL, "rbfd_num_levels: NULL argument");
        if (!m->greedy_done) rbfd::fail(RBFD_ESTATE, "rbfd_num_levels: run rbfd_greedy first");
        *n_levels = (int)m->levels.size();
    });
}

int rbfd_get_level(rbfd_mesh *m, int l, int64_t *n_c, int64_t *idx, double *alpha, double *e_max) {
    return guarded([&] {
        if (!m) rbfd::fail(RBFD_EINVAL, "rbfd_get_level: NULL mesh");
        if (!m->greedy_done) rbfd::fail(RBFD_ESTATE, "rbfd_get_level: run rbfd_greedy first");
        if (l < 0 || l >= (int)m->levels.size()) rbfd::fail(RBFD_EINVAL, "rbfd_get_level: level out of range");
        rbfd::Level &L = m->levels[l];
        if (idx || alpha) rbfd::level_fetch(m, L);
        if (n_c) *n_c = L.nc;
        if (idx) std::memcpy(idx, L.idx.data(), sizeof(int64_t) * L.idx.size());
        if (alpha) std::memcpy(alpha, L.alpha.data(), sizeof(double) * L.alpha.size());
        if (e_max) *e_max = L.emax;
    });
}

int rbfd_level_info(rbfd_mesh *m, int l, double *R, double *smax, double *tau) {
    return guarded([&] {
        if (!m) rbfd::fail(RBFD_EINVAL, "rbfd_level_info: NULL mesh");
        if (!m->greedy_done) rbfd::fail(RBFD_ESTATE, "rbfd_level_info: run rbfd_greedy first");
        if (l < 0 || l >= (int)m->levels.size()) rbfd::fail(RBFD_EINVAL, "rbfd_level_info: level out of range");
        const rbfd::Level &L = m->levels[l];
        if (R) *R = L.R;
        if (smax) *smax = L.smax;
        if (tau) *tau = L.tau;
    });
}

int rbfd_get_stats(rbfd_mesh *m, rbfd_stats *st) {
    return guarded([&] {
        if (!m || !st) rbfd::fail(RBFD_EINVAL, "rbfd_get_stats: NULL argument");
        RBFD_CUDA(cudaSetDevice(m->device));
        unsigned long long pr[16] = {};
        RBFD_CUDA(cudaStreamSynchronize(m->stream));
        RBFD_CUDA(cudaMemcpy(pr, m->d_pairs, sizeof(pr), cudaMemcpyDeviceToHost));
        m->prof.flush();
        *st = m->stats;
        st->deform_points += (int64_t)pr[7];
        st->sweep_pairs_useful = (int64_t)pr[0];
        st->sweep_pairs_visited = (int64_t)pr[1];
        st->vol_pairs_useful = (int64_t)pr[2];
        st->vol_pairs_visited = (int64_t)pr[3];
        st->newton_pairs_useful = (int64_t)pr[8];
        st->newton_pairs_formed = (int64_t)pr[9];
        st->eq12_pairs = (int64_t)(pr[0] + pr[10]);
        st->sweep_pairs_skipped = (int64_t)pr[11];
        st->sweep_warps_skipped = (int64_t)pr[12];
        st->pairs_useful = (int64_t)(pr[0] + pr[2] + pr[8]);
        st->pairs_visited = (int64_t)(pr[1] + pr[3] + pr[9]);
        st->sweep_ms = m->prof.ms[rbfd::kProfSweep];
        st->grow_ms = m->prof.ms[rbfd::kProfGrow];
        st->vol_ms = m->prof.ms[rbfd::kProfVol];
        st->sweep_launches = m->prof.launches[rbfd::kProfSweep];
        st->grow_launches = m->prof.launches[rbfd::kProfGrow];
        st->vol_launches = m->prof.launches[rbfd::kProfVol];
        st->persist_ms = m->prof.ms[rbfd::kProfPersist];
        st->persist_launches = m->prof.launches[rbfd::kProfPersist];
        st->wall_ms = m->prof.ms[rbfd::kProfWall];
        st->wall_launches = m->prof.launches[rbfd::kProfWall];
        st->wall_pairs_search = (int64_t)pr[4];
        st->wall_pairs_exact = (int64_t)pr[5];
        st->newton_ms = m->prof.ms[rbfd::kProfNewton];
        st->newton_launches = m->prof.launches[rbfd::kProfNewton];
        st->newton_terms = (int64_t)pr[6];
        unsigned long long ph[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        if (m->d_phase_ns) RBFD_CUDA(cudaMemcpy(ph, m->d_phase_ns, sizeof(ph), cudaMemcpyDeviceToHost));
        for (int q = 0; q < 8; ++q) st->persist_phase_ms[q] = ph[q] * 1e-6;
    });
}

// The argument checks of a volume update (everything but the greedy state).
static void deform_check(rbfd_mesh *m, int64_t n_v, const void *xyz_v, const void *d_v, double D, double k,
                         const void *out) {
    if (!m) rbfd::fail(RBFD_EINVAL, "rbfd_deform: NULL mesh");
    if (n_v < 0 || n_v > ((int64_t)1 << 31) - 1) rbfd::fail(RBFD_EINVAL, "rbfd_deform: n_v out of range");
    if (n_v > 0 && (!xyz_v || !out)) rbfd::fail(RBFD_EINVAL, "rbfd_deform: NULL array");
    if (!(D >= 0.0) || !(k >= 0.0) || !std::isfinite(D) || !std::isfinite(k))
        rbfd::fail(RBFD_EINVAL, "rbfd_deform: D and k must be finite and >= 0");
    if (D == 0.0 && k == 0.0) rbfd::fail(RBFD_EINVAL, "rbfd_deform: D and k cannot both be 0");
    RBFD_CUDA(cudaSetDevice(m->device));
    if (m->opt.inputs_on_device && n_v > 0 &&
        (!is_device_ptr(xyz_v) || (d_v && !is_device_ptr(d_v)) || !is_device_ptr(out)))
        rbfd::fail(RBFD_EINVAL, "rbfd_deform: inputs_on_device set but arrays are not device memory");
}

static int deform_common(rbfd_mesh *m, int64_t n_v, const void *xyz_v, const void *d_v, double D, double k,
                         void *out, bool f64) {
    return guarded([&] {
        deform_check(m, n_v, xyz_v, d_v, D, k, out);
        if (!m->greedy_done) rbfd::fail(RBFD_ESTATE, "rbfd_deform: run rbfd_greedy first");
        rbfd::deform_run(m, n_v, xyz_v, d_v, f64, D, k, out);
    });
}

// The greedy then the volume update of one mesh of a batch, on the calling
// host thread: the volume's copies, packing and Morton order run on a second
// stream while the greedy runs, and the update is queued behind the greedy's
// last launches without a host wait between the two (its D_l are computed
// on the device from the levels' scalars).
static void greedy_deform_one(rbfd_mesh *m, int64_t n_v, const float *xyz_v, const float *dv, double D, double k,
                       float *out) {
    RBFD_CUDA(cudaSetDevice(m->device));
    deform_check(m, n_v, xyz_v, dv, D, k, out);
    rbfd::volume_stage(m, n_v, xyz_v, dv, false, D, k);
    bool notconv = false;
    try {
        rbfd::greedy_run(m, false);
    } catch (const Error &e) {
        if (e.status != RBFD_ENOTCONV) {
            rbfd::volume_unstage(m);
            throw;
        }
        notconv = true;  // the levels are valid: deform with them, report it after
    }
    const int drc = deform_common(m, n_v, xyz_v, dv, D, k, out, false);
    rbfd::greedy_finish(m);  // (done by the update unless it failed first)
    if (drc != RBFD_OK) rbfd::fail(drc, rbfd::g_last_error);
    if (notconv) rbfd::fail(RBFD_ENOTCONV, "greedy selection did not reach eps before the control cap");
}

int rbfd_set_displacement(rbfd_mesh *m, const double *dS) {
    return guarded([&] {
        if (!m || !dS) rbfd::fail(RBFD_EINVAL, "rbfd_set_displacement: NULL argument");
        RBFD_CUDA(cudaSetDevice(m->device));
        if (m->opt.inputs_on_device && !is_device_ptr(dS))
            rbfd::fail(RBFD_EINVAL, "rbfd_set_displacement: inputs_on_device set but dS is not device memory");
        rbfd::mesh_set_displacement(m, dS);
    });
}

int rbfd_set_volume(rbfd_mesh *m, int64_t n_v, const float *xyz_v, const float *d_v) {
    return guarded([&] {
        if (!m) rbfd::fail(RBFD_EINVAL, "rbfd_set_volume: NULL mesh");
        if (n_v < 0 || n_v > ((int64_t)1 << 31) - 1) rbfd::fail(RBFD_EINVAL, "rbfd_set_volume: n_v out of range");
        if (n_v > 0 && !xyz_v) rbfd::fail(RBFD_EINVAL, "rbfd_set_volume: NULL array");
        RBFD_CUDA(cudaSetDevice(m->device));
        if (m->opt.inputs_on_device && n_v > 0 && (!is_device_ptr(xyz_v) || (d_v && !is_device_ptr(d_v))))
            rbfd::fail(RBFD_EINVAL, "rbfd_set_volume: inputs_on_device set but arrays are not device memory");
        rbfd::volume_register(m, n_v, xyz_v, d_v);
    });
}

int rbfd_deform_volume(rbfd_mesh *m, double D, double k, float *out) {
    return guarded([&] {
        if (!m) rbfd::fail(RBFD_EINVAL, "rbfd_deform_volume: NULL mesh");
        if (!(D >= 0.0) || !(k >= 0.0) || !std::isfinite(D) || !std::isfinite(k) || (D == 0.0 && k == 0.0))
            rbfd::fail(RBFD_EINVAL, "rbfd_deform_volume: D and k must be finite, >= 0 and not both 0");
        if (!m->greedy_done) rbfd::fail(RBFD_ESTATE, "rbfd_deform_volume: run rbfd_greedy first");
        if (m->vreg_n > 0 && !out) rbfd::fail(RBFD_EINVAL, "rbfd_deform_volume: NULL out");
        RBFD_CUDA(cudaSetDevice(m->device));
        if (m->opt.inputs_on_device && m->vreg_n > 0 && !is_device_ptr(out))
            rbfd::fail(RBFD_EINVAL, "rbfd_deform_volume: inputs_on_device set but out is not device memory");
        rbfd::deform_registered(m, D, k, out);
    });
}

static int wall_common(rbfd_mesh *m, int64_t n_v, const void *xyz_v, double *d_out, bool f64) {
    return guarded([&] {
        if (!m) rbfd::fail(RBFD_EINVAL, "rbfd_wall_distance: NULL mesh");
        if (n_v < 0 || n_v > ((int64_t)1 << 31) - 1) rbfd::fail(RBFD_EINVAL, "rbfd_wall_distance: n_v out of range");
        if (n_v > 0 && (!xyz_v || !d_out)) rbfd::fail(RBFD_EINVAL, "rbfd_wall_distance: NULL array");
        RBFD_CUDA(cudaSetDevice(m->device));
        if (m->opt.inputs_on_device && n_v > 0 && (!is_device_ptr(xyz_v) || !is_device_ptr(d_out)))
            rbfd::fail(RBFD_EINVAL, "rbfd_wall_distance: inputs_on_device set but arrays are not device memory");
        rbfd::wall_distance_run(m, n_v, xyz_v, f64, d_out);
    });
}

int rbfd_wall_distance(rbfd_mesh *m, int64_t n_v, const float *xyz_v, double *d_out) {
    return wall_common(m, n_v, xyz_v, d_out, false);
}

int rbfd_wall_distance_f64(rbfd_mesh *m, int64_t n_v, const double *xyz_v, double *d_out) {
    return wall_common(m, n_v, xyz_v, d_out, true);
}

int rbfd_orthogonality(int dim, int64_t n_i, int64_t n_k, int64_t n_layers, int periodic_i, const double *wall,
                       const double *wall_disp, const float *vol, const float *vol_disp, float *theta,
                       rbfd_quality *q, int on_device, void *stream) {
    return guarded([&] {
        if (dim != 2 && dim != 3) rbfd::fail(RBFD_EINVAL, "rbfd_orthogonality: dim must be 2 or 3");
        if (dim == 2) n_k = 1;
        if (n_i < 2 || n_layers < 1 || n_k < 1 || (dim == 3 && n_k < 2))
            rbfd::fail(RBFD_EINVAL, "rbfd_orthogonality: grid too small");
        if (n_k * n_i * (n_layers + 1) > ((int64_t)1 << 40)) rbfd::fail(RBFD_EINVAL, "rbfd_orthogonality: grid too large");
        if (!wall || !vol) rbfd::fail(RBFD_EINVAL, "rbfd_orthogonality: NULL wall or vol");
        if (on_device) {
            const void *ptrs[] = {wall, wall_disp, vol, vol_disp, theta};
            for (const void *p : ptrs)
                if (p && !is_device_ptr(p))
                    rbfd::fail(RBFD_EINVAL, "rbfd_orthogonality: on_device set but an array is not device memory");
        }
        cudaStream_t st = stream ? static_cast<cudaStream_t>(stream) : cudaStreamPerThread;
        rbfd::orthogonality_run(dim, n_i, n_k, n_layers, periodic_i, wall, wall_disp, vol, vol_disp, on_device != 0,
                                st, theta, q);
    });
}

int rbfd_sort_pairs(uint32_t *keys, uint32_t *vals, int64_t n, int key_bits, void *stream) {
    return guarded([&] {
        if (n < 0 || n > ((int64_t)1 << 31) - 1) rbfd::fail(RBFD_EINVAL, "rbfd_sort_pairs: n out of range");
        if (key_bits < 1 || key_bits > 32) rbfd::fail(RBFD_EINVAL, "rbfd_sort_pairs: key_bits must be 1..32");
        if (n == 0) return;
        if (!keys || !vals || !is_device_ptr(keys) || !is_device_ptr(vals))
            rbfd::fail(RBFD_EINVAL, "rbfd_sort_pairs: keys and vals must be device memory");
        cudaPointerAttributes at{};
        RBFD_CUDA(cudaPointerGetAttributes(&at, keys));
        RBFD_CUDA(cudaSetDevice(at.device));
        cudaStream_t st = stream ? static_cast<cudaStream_t>(stream) : cudaStreamPerThread;
        rbfd::SortScratch ss;
        try {
            rbfd::radix_sort_pairs(keys, vals, (size_t)n, key_bits, ss, st);
            RBFD_CUDA(cudaStreamSynchronize(st));
        } catch (...) {
            cudaStreamSynchronize(st);
            ss.release();
            throw;
        }
        ss.release();
    });
}

int rbfd_deform(rbfd_mesh *m, int64_t n_v, const float *xyz_v, const float *d_v, double D, double k, float *out) {
    return deform_common(m, n_v, xyz_v, d_v, D, k, out, false);
}

int rbfd_deform_f64(rbfd_mesh *m, int64_t n_v, const double *xyz_v, const double *d_v, double D, double k,
                    double *out) {
    return deform_common(m, n_v, xyz_v, d_v, D, k, out, true);
}

int rbfd_greedy_batch(rbfd_mesh **meshes, int n) {
    if (n < 0 || (n > 0 && !meshes)) {
        rbfd::g_last_error = "rbfd_greedy_batch: bad arguments";
        return RBFD_EINVAL;
    }
    for (int i = 0; i < n; ++i)
        if (!meshes[i]) {
            rbfd::g_last_error = "rbfd_greedy_batch: NULL mesh";
            return RBFD_EINVAL;
        }
    int rc = share_grid(meshes, n);
    if (rc != RBFD_OK) return rc;
    // the meshes still in their greedy share the persistent blocks: a finished
    // mesh's share goes to the others' next launches (on one device only)
    std::atomic<int> active{n};
    bool one_device = n > 1;
    for (int i = 1; i < n; ++i) one_device = one_device && meshes[i]->device == meshes[0]->device;
    if (one_device) {
        int total = 0;
        rc = guarded([&] { total = rbfd::persist_max_ctas(meshes[0]); });
        if (rc != RBFD_OK) {
            unshare_grid(meshes, n);
            return rc;
        }
        for (int i = 0; i < n; ++i) {
            meshes[i]->batch_active = &active;
            meshes[i]->batch_total = total;
        }
    }
    rc = run_batch(n, [&](int i) {
        struct Leave {  // (also when the greedy fails)
            std::atomic<int> &a;
            ~Leave() { a.fetch_sub(1); }
        } leave{active};
        RBFD_CUDA(cudaSetDevice(meshes[i]->device));
        rbfd::greedy_run(meshes[i]);
    }, "rbfd_greedy_batch");
    for (int i = 0; i < n; ++i) {
        meshes[i]->batch_active = nullptr;
        meshes[i]->batch_total = 0;
    }
    unshare_grid(meshes, n);
    return rc;
}

int rbfd_deform_worklist(rbfd_mesh **meshes, int n, const int64_t *n_v, const float *const *xyz_v,
                         const float *const *d_v, const double *D, const double *k, float *const *out,
                         rbfd_worklist_tune *tune) {
    return guarded([&] {
        if (n < 1 || !meshes || !n_v || !xyz_v || !D || !k || !out)
            rbfd::fail(RBFD_EINVAL, "rbfd_deform_worklist: bad arguments");
        for (int i = 0; i < n; ++i)
            if (!meshes[i]) rbfd::fail(RBFD_EINVAL, "rbfd_deform_worklist: NULL mesh");
        rbfd::deform_worklist(meshes, n, n_v, xyz_v, d_v, D, k, out, tune);
    });
}

int rbfd_greedy_deform_batch(rbfd_mesh **meshes, int n, const int64_t *n_v, const float *const *xyz_v,
                             const float *const *d_v, const double *D, const double *k, float *const *out) {
    if (n < 0 || (n > 0 && (!meshes || !n_v || !xyz_v || !D || !k || !out))) {
        rbfd::g_last_error = "rbfd_greedy_deform_batch: bad arguments";
        return RBFD_EINVAL;
    }
    for (int i = 0; i < n; ++i)
        if (!meshes[i]) {
            rbfd::g_last_error = "rbfd_greedy_deform_batch: NULL mesh";
            return RBFD_EINVAL;
        }
    int rc = share_grid(meshes, n);
    if (rc != RBFD_OK) return rc;
    rc = run_batch(n, [&](int i) {
        greedy_deform_one(meshes[i], n_v[i], xyz_v[i], d_v ? d_v[i] : nullptr, D[i], k[i], out[i]);
    }, "rbfd_greedy_deform_batch");
    unshare_grid(meshes, n);
    return rc;
}

int rbfd_run_jobs(const rbfd_job *jobs, int n, rbfd_mesh **meshes) {
    if (n < 0 || (n > 0 && (!jobs || !meshes))) {
        rbfd::g_last_error = "rbfd_run_jobs: bad arguments";
        return RBFD_EINVAL;
    }
    for (int i = 0; i < n; ++i) meshes[i] = nullptr;
    const int rc = run_batch(n, [&](int i) {
        const rbfd_job &J = jobs[i];
        rbfd_mesh *m = nullptr;
        const int crc = rbfd_create(&m, J.dim, J.n_s, J.xyz_s, J.dS, J.n_levels, J.R, J.eps, J.opt);
        if (crc != RBFD_OK) rbfd::fail(crc, rbfd::g_last_error);
        meshes[i] = m;
        if (n > 1) {  // the jobs run side by side: each mesh takes a share of the blocks
            m->batch_ctas_cap = std::max(1, rbfd::persist_max_ctas(m) / n);
            m->batch_share = n;
        }
        greedy_deform_one(m, J.n_v, J.xyz_v, J.d_v, J.D, J.k, J.out);
    }, "rbfd_run_jobs");
    for (int i = 0; i < n; ++i)
        if (meshes[i]) unshare_grid(&meshes[i], 1);
    return rc;
}

int rbfd_deform_batch(rbfd_mesh **meshes, int n, const int64_t *n_v, const float *const *xyz_v,
                      const float *const *d_v, const double *D, const double *k, float *const *out) {
    if (n < 0 || (n > 0 && (!meshes || !n_v || !xyz_v || !d_v || !D || !k || !out))) {
        rbfd::g_last_error = "rbfd_deform_batch: bad arguments";
        return RBFD_EINVAL;
    }
    return run_batch(n, [&](int i) {
        int rc = deform_common(meshes[i], n_v[i], xyz_v[i], d_v[i], D[i], k[i], out[i], false);
        if (rc != RBFD_OK) rbfd::fail(rc, rbfd::g_last_error);
    }, "rbfd_deform_batch");
}

int rbfd_destroy(rbfd_mesh *m) {
    if (!m) return RBFD_OK;
    rbfd::mesh_free(m);
    delete m;
    return RBFD_OK;
}

const char *rbfd_last_error(void) { return rbfd::g_last_error.c_str(); }

const char *rbfd_version(void) { return "rbfd 0.1 (sm_103a)"; }

}  // extern "C"
