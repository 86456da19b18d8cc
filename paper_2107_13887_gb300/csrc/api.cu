// api.cu -- the extern "C" boundary declared in include/rbfd.h.  Every entry
// point validates its arguments, converts internal errors into an
// rbfd_status, and records a thread-local message for rbfd_last_error().
#include <cmath>
#include <cstring>
#include <new>
#include <string>

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

void *dmalloc(size_t bytes, const char *what) {
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes ? bytes : 1);
    if (e != cudaSuccess) {
        cudaGetLastError();
        fail(e == cudaErrorMemoryAllocation ? RBFD_ENOMEM : RBFD_ECUDA,
             std::string("allocating ") + what + " (" + std::to_string(bytes) + " bytes): " + cudaGetErrorString(e));
    }
    return p;
}

void dfree(void *p) {
    if (p) cudaFree(p);
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
    for (auto &p : pend) {
        float ms_ = 0.f;
        if (cudaEventElapsedTime(&ms_, p.a, p.b) == cudaSuccess) ms[p.kind] += ms_;
        else cudaGetLastError();
        free_ev.push_back(p.a);
        free_ev.push_back(p.b);
    }
    pend.clear();
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
    for (auto &L : m->levels) {
        dfree(L.d_cx);
        dfree(L.d_alpha);
        dfree(L.d_cell_start);
        dfree(L.d_cell_ctrl);
    }
    void *ptrs[] = {m->d_perm, m->d_inv, m->d_xs, m->d_dS, m->d_cur, m->d_E, m->d_pb_lo, m->d_pb_hi,
                    m->d_pb_org, m->d_xs_hi, m->d_xs_lo, m->d_sel, m->d_G, m->d_w, m->d_alpha, m->d_cx,
                    m->d_cid, m->d_phi, m->d_y, m->d_red, m->d_gpart, m->d_vec, m->d_vec2, m->d_v4part,
                    m->d_nb_cnt, m->d_nb_list, m->d_part, m->d_pb_done, m->d_pb_key, m->d_pb_idx, m->d_pairs,
                    m->d_st, m->d_vin, m->d_vpos, m->d_vorig, m->d_vflag, m->d_vscan, m->d_vlist, m->d_vkeys,
                    m->d_vacc, m->d_vio, m->d_misc, m->d_bbox};
    for (void *p : ptrs) dfree(p);
    m->sort.release();
    m->prof.release();
    if (m->h_st) cudaFreeHost(m->h_st);
    if (m->ev0) cudaEventDestroy(m->ev0);
    if (m->ev1) cudaEventDestroy(m->ev1);
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
        if (o.nc_cap < 0) rbfd::fail(RBFD_EINVAL, "rbfd_create: nc_cap must be >= 0");
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
            RBFD_CUDA(cudaStreamCreateWithFlags(&m->stream, cudaStreamNonBlocking));
            m->own_stream = true;
        }
        RBFD_CUDA(cudaEventCreate(&m->ev0));
        RBFD_CUDA(cudaEventCreate(&m->ev1));
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
        const rbfd::Level &L = m->levels[l];
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
        unsigned long long pr[4] = {0, 0, 0, 0};
        RBFD_CUDA(cudaStreamSynchronize(m->stream));
        RBFD_CUDA(cudaMemcpy(pr, m->d_pairs, sizeof(pr), cudaMemcpyDeviceToHost));
        m->prof.flush();
        *st = m->stats;
        st->sweep_pairs_useful = (int64_t)pr[0];
        st->sweep_pairs_visited = (int64_t)pr[1];
        st->vol_pairs_useful = (int64_t)pr[2];
        st->vol_pairs_visited = (int64_t)pr[3];
        st->pairs_useful = (int64_t)(pr[0] + pr[2]);
        st->pairs_visited = (int64_t)(pr[1] + pr[3]);
        st->sweep_ms = m->prof.ms[rbfd::kProfSweep];
        st->grow_ms = m->prof.ms[rbfd::kProfGrow];
        st->vol_ms = m->prof.ms[rbfd::kProfVol];
        st->sweep_launches = m->prof.launches[rbfd::kProfSweep];
        st->grow_launches = m->prof.launches[rbfd::kProfGrow];
        st->vol_launches = m->prof.launches[rbfd::kProfVol];
    });
}

static int deform_common(rbfd_mesh *m, int64_t n_v, const void *xyz_v, const void *d_v, double D, double k,
                         void *out, bool f64) {
    return guarded([&] {
        if (!m) rbfd::fail(RBFD_EINVAL, "rbfd_deform: NULL mesh");
        if (n_v < 0 || n_v > ((int64_t)1 << 31) - 1) rbfd::fail(RBFD_EINVAL, "rbfd_deform: n_v out of range");
        if (n_v > 0 && (!xyz_v || !d_v || !out)) rbfd::fail(RBFD_EINVAL, "rbfd_deform: NULL array");
        if (!(D >= 0.0) || !(k >= 0.0) || !std::isfinite(D) || !std::isfinite(k))
            rbfd::fail(RBFD_EINVAL, "rbfd_deform: D and k must be finite and >= 0");
        if (D == 0.0 && k == 0.0) rbfd::fail(RBFD_EINVAL, "rbfd_deform: D and k cannot both be 0");
        if (!m->greedy_done) rbfd::fail(RBFD_ESTATE, "rbfd_deform: run rbfd_greedy first");
        RBFD_CUDA(cudaSetDevice(m->device));
        if (m->opt.inputs_on_device && n_v > 0 &&
            (!is_device_ptr(xyz_v) || !is_device_ptr(d_v) || !is_device_ptr(out)))
            rbfd::fail(RBFD_EINVAL, "rbfd_deform: inputs_on_device set but arrays are not device memory");
        rbfd::deform_run(m, n_v, xyz_v, d_v, f64, D, k, out);
    });
}

int rbfd_deform(rbfd_mesh *m, int64_t n_v, const float *xyz_v, const float *d_v, double D, double k, float *out) {
    return deform_common(m, n_v, xyz_v, d_v, D, k, out, false);
}

int rbfd_deform_f64(rbfd_mesh *m, int64_t n_v, const double *xyz_v, const double *d_v, double D, double k,
                    double *out) {
    return deform_common(m, n_v, xyz_v, d_v, D, k, out, true);
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
