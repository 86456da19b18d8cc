// server.cu -- continuous-batching request loop for deformation requests
// (rbfd_server_* / rbfd_submit / rbfd_poll in include/rbfd.h).
//
// A request is one time step of an icing computation: a new surface
// displacement dS on a registered mesh.  The server runs up to `slots`
// requests at a time, each on a worker thread with its own CUDA stream, so
// the greedy launches of different requests overlap on the GPU (their
// persistent grids are sized to be resident together).  Requests that arrive
// while others run wait in a FIFO queue and are admitted as soon as a slot is
// free and their device-memory footprint fits the budget; a request whose
// mesh is busy waits for that mesh's instance, while requests on other
// meshes go ahead.  Each registered mesh keeps its resident instance
// (Morton-ordered surface, point blocks, workspace, sorted volume) on the
// device between time steps: a new step only uploads dS, runs the greedy
// selection (Section 3) warm -- every level starts from the previous step's
// controls and inverse factor and continues the greedy only if they miss
// tau_l -- and the volume update (Section 4).
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <functional>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "internal.h"

namespace {

using clk = std::chrono::steady_clock;

struct MeshSpec {
    int dim = 2;
    int64_t n_s = 0, n_v = 0;
    std::vector<double> xyz_s, R;
    std::vector<float> xyz_v, d_v;
    double eps = 0, D = 0, k = 0;
    size_t footprint = 0;
    std::vector<rbfd_mesh *> idle;  // resident instances not running a request
    int instances = 0;
};

// A request's volume update waiting for the fused launch.
struct VolumeJob {
    rbfd_mesh *inst = nullptr;
    double D = 0, k = 0;
    float *out = nullptr;
    int status = RBFD_OK;
    std::string msg;
    bool done = false;
};

struct Request {
    int mesh = -1;
    std::vector<double> dS;
    float *out = nullptr;
    int state = RBFD_REQ_QUEUED;
    int status = RBFD_OK;
    std::string msg;
    clk::time_point t_submit, t_start, t_done;
};

}  // namespace

struct rbfd_server {
    rbfd_server_options opt{};
    int device = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::vector<std::unique_ptr<MeshSpec>> meshes;
    std::map<uint64_t, Request> reqs;
    std::deque<uint64_t> queue;
    uint64_t next_ticket = 1;
    size_t used_bytes = 0;
    int running = 0;
    bool shutdown = false;
    std::vector<std::thread> workers;
    // the volume stage: requests whose greedy is done queue their volume
    // updates here; a worker runs its own with every other queued update of
    // its dimension and basis in one work-list launch
    std::mutex vmu;
    std::condition_variable vcv;
    std::deque<VolumeJob *> vq;
};

namespace rbfd {

// Device bytes one resident instance of a mesh holds (greedy workspace, the
// inverse factor, block lists, sorted surface and volume, deform buffers).
size_t mesh_footprint(int dim, int64_t n_s, int64_t n_v, int64_t cap) {
    (void)dim;
    const int64_t n_pb = (n_s + kPB - 1) / kPB;
    const int64_t nch = std::max<int64_t>(128, (608 + n_pb - 1) / n_pb);
    size_t b = 0;
    b += 16ull * cap * cap;                         // G and its transpose
    b += 8ull * n_pb * cap;                         // block lists and their reverse (pruned sweep)
    b += (size_t)n_s * (4 * 32 + 2 * 16 + 16);      // sorted surface, targets, error, df coords, perms
    b += (size_t)(nch + (nch + 15) / 16) * n_s * 32;  // sweep partials and their group sums
    b += (size_t)cap * (6 * 32 + 8 * 8) + 32ull * (cap / 256 + 2) * cap;
    b += (size_t)n_v * (32 * 3 + 4 * 6);            // registered + working volume buffers
    // Newton-basis values V: n_s doubles per column, at most kNewtonCols columns and 1 GB
    b += std::min<size_t>((size_t)n_s * 8 * std::min<int64_t>(cap, kNewtonCols), (size_t)1 << 30);
    return b + (64ull << 20);                       // small buffers and pool rounding
}

// The volume update of a request whose greedy is done: queued for a fused
// launch.  A worker whose update is still queued takes it together with every
// other queued update of its dimension and basis (up to 16 meshes), runs them
// in one work-list launch on the registered volumes (cells of size R_l: the
// same sums as the request's own rbfd_deform_volume, bit for bit) and wakes
// their workers; a worker whose update another one took waits for it.
// Several fused launches may run at once (one per leading worker, each on its
// meshes' streams), so a small request never waits behind a large launch.
// Requests in FP64 (or C4 / C6) run theirs alone, and so does every request
// unless the server's fuse_volume option is set: on a stream of mixed-size
// meshes the fused launch (a persistent grid over every SM, host waits for
// its completion) measured higher latency than the requests' own launches
// side by side (p50 6.5 against 2.7 ms, p99 50 against 31 ms at 50 requests/s).
static void volume_stage(rbfd_server *S, rbfd_mesh *inst, double D, double k, float *out) {
    if (!S->opt.fuse_volume || inst->opt.precision == RBFD_FP64) {
        deform_registered(inst, D, k, out);
        return;
    }
    VolumeJob job;
    job.inst = inst;
    job.D = D;
    job.k = k;
    job.out = out;
    std::unique_lock<std::mutex> lk(S->vmu);
    S->vq.push_back(&job);
    for (;;) {
        if (job.done) break;
        if (std::find(S->vq.begin(), S->vq.end(), &job) == S->vq.end()) {  // another worker runs it
            S->vcv.wait(lk);
            continue;
        }
        std::vector<VolumeJob *> batch;
        const int dim = inst->dim, basis = inst->opt.basis;
        S->vq.erase(std::find(S->vq.begin(), S->vq.end(), &job));
        batch.push_back(&job);
        for (auto it = S->vq.begin(); it != S->vq.end() && batch.size() < 16;) {
            if ((*it)->inst->dim == dim && (*it)->inst->opt.basis == basis) {
                batch.push_back(*it);
                it = S->vq.erase(it);
            } else {
                ++it;
            }
        }
        lk.unlock();
        int status = RBFD_OK;
        std::string msg;
        try {
            NvtxRange nvtx("rbfd fused volume stage");
            const int n = (int)batch.size();
            std::vector<rbfd_mesh *> ms(n);
            std::vector<double> Dv(n), kv(n);
            std::vector<float *> outs(n);
            for (int i = 0; i < n; ++i) {
                ms[i] = batch[i]->inst;
                Dv[i] = batch[i]->D;
                kv[i] = batch[i]->k;
                outs[i] = batch[i]->out;
            }
            rbfd_worklist_tune t{};
            t.autotune = 0;
            t.ctas_per_sm = 8;
            t.item_blocks = 1;
            for (int i = 0; i < 16; ++i) t.cell_div[i] = 1;
            deform_worklist(ms.data(), n, nullptr, nullptr, nullptr, Dv.data(), kv.data(), outs.data(), &t, true);
        } catch (const Error &e) {
            status = e.status;
            msg = e.msg;
        } catch (...) {
            status = RBFD_ECUDA;
            msg = "server: unexpected internal error in the volume stage";
        }
        lk.lock();
        for (VolumeJob *j : batch) {
            j->status = status;
            j->msg = msg;
            j->done = true;
        }
        S->vcv.notify_all();
    }
    if (job.status != RBFD_OK) fail(job.status, job.msg);
}

// Run one admitted request.  inst is an idle resident instance of its mesh,
// or nullptr when a new instance (already counted in used_bytes) is to be made.
static void run_request(rbfd_server *S, uint64_t ticket, rbfd_mesh *inst) {
    NvtxRange nvtx("rbfd serving request");
    int mesh_id;
    std::vector<double> dS;
    float *out;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        Request &r = S->reqs[ticket];
        mesh_id = r.mesh;
        dS.swap(r.dS);
        out = r.out;
    }
    MeshSpec &M = *S->meshes[mesh_id];
    const bool fresh = inst == nullptr;
    int status = RBFD_OK;
    std::string msg;
    try {
        RBFD_CUDA(cudaSetDevice(S->device));
        if (fresh) {
            rbfd_options o;
            rbfd_options_default(&o);
            o.precision = S->opt.precision;
            int rc = rbfd_create(&inst, M.dim, M.n_s, M.xyz_s.data(), dS.data(), (int)M.R.size(), M.R.data(), M.eps,
                                 &o);
            if (rc != RBFD_OK) fail(rc, std::string("server: creating a mesh instance: ") + rbfd_last_error());
            volume_register(inst, M.n_v, M.xyz_v.data(), M.d_v.empty() ? nullptr : M.d_v.data());
            inst->keep_factors = true;  // the next time step starts warm
        } else {
            mesh_set_displacement(inst, dS.data());
        }
        // the persistent grids of all slots must be resident together
        inst->batch_ctas_cap = std::max(1, persist_max_ctas(inst) / std::max(1, S->opt.slots));
        inst->batch_share = S->opt.slots;
        try {
            // a resident instance starts every level from its previous time
            // step's controls and factor (rbfd_greedy_warm)
            greedy_run(inst, true, !fresh);
        } catch (const Error &e) {
            if (e.status != RBFD_ENOTCONV) throw;
            status = RBFD_ENOTCONV;  // results valid
            msg = e.msg;
        }
        volume_stage(S, inst, M.D, M.k, out);
    } catch (const Error &e) {
        status = e.status;
        msg = e.msg;
    } catch (...) {
        status = RBFD_ECUDA;
        msg = "server: unexpected internal error";
    }
    const bool ok = status == RBFD_OK || status == RBFD_ENOTCONV;
    if (!ok && inst) {  // a failed instance is not reused
        rbfd_destroy(inst);
        inst = nullptr;
    }
    std::lock_guard<std::mutex> lk(S->mu);
    Request &r = S->reqs[ticket];
    r.status = status;
    r.msg = msg;
    r.state = ok ? RBFD_REQ_DONE : RBFD_REQ_FAILED;
    r.t_done = clk::now();
    if (inst) {
        M.idle.push_back(inst);
    } else {  // the instance is gone (or was never made): release its share
        M.instances--;
        S->used_bytes -= M.footprint;
    }
    S->running--;
    S->cv_done.notify_all();
    S->cv_work.notify_all();
}

// First queued request that can start now: its mesh has an idle instance,
// or it has no instance yet and a new one fits the memory budget.  A mesh
// whose only instance is busy makes its request wait for that instance (the
// same mesh's time steps run in order): creating a second instance on the
// request path (allocations, the volume's Morton order) cost tens of
// milliseconds and was the whole tail of the latency.  Called with the lock
// held.
static bool pick_request(rbfd_server *S, uint64_t &ticket, rbfd_mesh *&inst) {
    for (auto it = S->queue.begin(); it != S->queue.end(); ++it) {
        Request &r = S->reqs[*it];
        MeshSpec &M = *S->meshes[r.mesh];
        bool ok = false;
        if (!M.idle.empty()) {
            inst = M.idle.back();
            M.idle.pop_back();
            ok = true;
        } else if (M.instances == 0 && S->used_bytes + M.footprint <= (size_t)S->opt.mem_budget_bytes) {
            inst = nullptr;  // reserve for a new instance
            S->used_bytes += M.footprint;
            M.instances++;
            ok = true;
        }
        if (ok) {
            ticket = *it;
            S->queue.erase(it);
            r.state = RBFD_REQ_RUNNING;
            r.t_start = clk::now();
            S->running++;
            return true;
        }
    }
    return false;
}

static void worker(rbfd_server *S) {
    cudaSetDevice(S->device);
    for (;;) {
        uint64_t ticket = 0;
        rbfd_mesh *inst = nullptr;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv_work.wait(lk, [&] { return S->shutdown || (!S->queue.empty() && pick_request(S, ticket, inst)); });
            if (ticket == 0) {
                if (S->shutdown) return;
                continue;
            }
        }
        run_request(S, ticket, inst);
    }
}

}  // namespace rbfd

namespace {

int guarded_srv(const std::function<void()> &f) {
    try {
        f();
        rbfd::set_last_error("");
        return RBFD_OK;
    } catch (const rbfd::Error &e) {
        rbfd::set_last_error(e.msg);
        return e.status;
    } catch (...) {
        rbfd::set_last_error("server: unexpected internal error");
        return RBFD_ECUDA;
    }
}

}  // namespace

extern "C" {

void rbfd_server_options_default(rbfd_server_options *o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->slots = 4;
    o->mem_budget_bytes = 0;
    o->precision = RBFD_MIXED;
    o->max_queue = 4096;
}

int rbfd_server_create(rbfd_server **out, const rbfd_server_options *opt) {
    if (out) *out = nullptr;
    return guarded_srv([&] {
        if (!out) rbfd::fail(RBFD_EINVAL, "rbfd_server_create: out is NULL");
        rbfd_server_options o;
        rbfd_server_options_default(&o);
        if (opt) o = *opt;
        if (o.slots < 1 || o.slots > 64) rbfd::fail(RBFD_EINVAL, "rbfd_server_create: slots must be in [1, 64]");
        if (o.max_queue < 1) rbfd::fail(RBFD_EINVAL, "rbfd_server_create: max_queue must be >= 1");
        auto *S = new rbfd_server();
        S->opt = o;
        RBFD_CUDA(cudaGetDevice(&S->device));
        if (S->opt.mem_budget_bytes <= 0) {
            size_t fr = 0, tot = 0;
            RBFD_CUDA(cudaMemGetInfo(&fr, &tot));
            S->opt.mem_budget_bytes = (int64_t)(0.8 * (double)fr);
        }
        for (int i = 0; i < o.slots; ++i) S->workers.emplace_back(rbfd::worker, S);
        *out = S;
    });
}

int rbfd_server_add_mesh(rbfd_server *S, int dim, int64_t n_s, const double *xyz_s, int64_t n_v, const float *xyz_v,
                         const float *d_v, int n_levels, const double *R, double eps, double D, double k,
                         int *mesh_id) {
    return guarded_srv([&] {
        if (!S || !mesh_id) rbfd::fail(RBFD_EINVAL, "rbfd_server_add_mesh: NULL argument");
        if (dim != 2 && dim != 3) rbfd::fail(RBFD_EINVAL, "rbfd_server_add_mesh: dim must be 2 or 3");
        if (n_s < 1 || !xyz_s || n_levels < 1 || n_levels > 64 || !R || !(eps > 0.0 && eps < 1.0))
            rbfd::fail(RBFD_EINVAL, "rbfd_server_add_mesh: bad surface or level arguments");
        if (n_v < 0 || (n_v > 0 && !xyz_v)) rbfd::fail(RBFD_EINVAL, "rbfd_server_add_mesh: bad volume");
        if (!(D >= 0.0) || !(k >= 0.0) || (D == 0.0 && k == 0.0))
            rbfd::fail(RBFD_EINVAL, "rbfd_server_add_mesh: D and k must be >= 0 and not both 0");
        for (int l = 0; l < n_levels; ++l)
            if (!(R[l] > 0.0)) rbfd::fail(RBFD_EINVAL, "rbfd_server_add_mesh: every R must be > 0");
        auto M = std::make_unique<MeshSpec>();
        M->dim = dim;
        M->n_s = n_s;
        M->n_v = n_v;
        M->xyz_s.assign(xyz_s, xyz_s + n_s * dim);
        M->R.assign(R, R + n_levels);
        M->xyz_v.assign(xyz_v, xyz_v + n_v * dim);
        if (d_v) M->d_v.assign(d_v, d_v + n_v);  // empty: wall distance computed on the device
        M->eps = eps;
        M->D = D;
        M->k = k;
        M->footprint = rbfd::mesh_footprint(dim, n_s, n_v, std::min<int64_t>(n_s, 32768));
        if (M->footprint > (size_t)S->opt.mem_budget_bytes)
            rbfd::fail(RBFD_ENOMEM, "rbfd_server_add_mesh: one instance of this mesh exceeds the memory budget");
        std::lock_guard<std::mutex> lk(S->mu);
        S->meshes.push_back(std::move(M));
        *mesh_id = (int)S->meshes.size() - 1;
    });
}

int rbfd_submit(rbfd_server *S, int mesh_id, const rbfd_request *req, uint64_t *ticket) {
    return guarded_srv([&] {
        if (!S || !req || !ticket || !req->dS || !req->out) rbfd::fail(RBFD_EINVAL, "rbfd_submit: NULL argument");
        std::lock_guard<std::mutex> lk(S->mu);
        if (mesh_id < 0 || mesh_id >= (int)S->meshes.size()) rbfd::fail(RBFD_EINVAL, "rbfd_submit: unknown mesh");
        if ((int64_t)S->queue.size() >= S->opt.max_queue) rbfd::fail(RBFD_EBUSY, "rbfd_submit: queue full");
        const MeshSpec &M = *S->meshes[mesh_id];
        Request r;
        r.mesh = mesh_id;
        r.dS.assign(req->dS, req->dS + M.n_s * M.dim);
        r.out = req->out;
        r.t_submit = clk::now();
        const uint64_t t = S->next_ticket++;
        S->reqs.emplace(t, std::move(r));
        S->queue.push_back(t);
        *ticket = t;
        S->cv_work.notify_one();
    });
}

int rbfd_poll(rbfd_server *S, uint64_t ticket, int *state) {
    if (!S || !state) return RBFD_EINVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) {
        rbfd::set_last_error("rbfd_poll: unknown ticket");
        return RBFD_EINVAL;
    }
    *state = it->second.state;
    if (it->second.state >= RBFD_REQ_FAILED) rbfd::set_last_error(it->second.msg);
    return it->second.state >= RBFD_REQ_DONE ? it->second.status : RBFD_OK;
}

int rbfd_wait(rbfd_server *S, uint64_t ticket, double timeout_s, int *state) {
    if (!S || !state) return RBFD_EINVAL;
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) {
        rbfd::set_last_error("rbfd_wait: unknown ticket");
        return RBFD_EINVAL;
    }
    const bool done = S->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s > 0 ? timeout_s : 1e9),
                                          [&] { return it->second.state >= RBFD_REQ_DONE; });
    *state = it->second.state;
    if (!done) {
        rbfd::set_last_error("rbfd_wait: timed out");
        return RBFD_ETIMEOUT;
    }
    if (it->second.state >= RBFD_REQ_FAILED) rbfd::set_last_error(it->second.msg);
    return it->second.status;
}

int rbfd_cancel(rbfd_server *S, uint64_t ticket) {
    return guarded_srv([&] {
        if (!S) rbfd::fail(RBFD_EINVAL, "rbfd_cancel: NULL server");
        std::lock_guard<std::mutex> lk(S->mu);
        auto it = S->reqs.find(ticket);
        if (it == S->reqs.end()) rbfd::fail(RBFD_EINVAL, "rbfd_cancel: unknown ticket");
        Request &r = it->second;
        if (r.state == RBFD_REQ_RUNNING) rbfd::fail(RBFD_EBUSY, "rbfd_cancel: the request is running");
        if (r.state != RBFD_REQ_QUEUED) rbfd::fail(RBFD_ESTATE, "rbfd_cancel: the request has finished");
        for (auto q = S->queue.begin(); q != S->queue.end(); ++q)
            if (*q == ticket) {
                S->queue.erase(q);
                break;
            }
        r.state = RBFD_REQ_CANCELLED;
        r.status = RBFD_ECANCELED;
        r.msg = "rbfd_cancel: cancelled before it started";
        r.t_start = r.t_done = clk::now();
        r.dS.clear();
        S->cv_done.notify_all();
    });
}

int rbfd_request_times(rbfd_server *S, uint64_t ticket, double *queue_ms, double *run_ms, double *total_ms) {
    if (!S) return RBFD_EINVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end() || it->second.state < RBFD_REQ_DONE) {
        rbfd::set_last_error("rbfd_request_times: unknown or unfinished ticket");
        return RBFD_EINVAL;
    }
    const Request &r = it->second;
    auto ms = [](clk::duration d) { return std::chrono::duration<double, std::milli>(d).count(); };
    if (queue_ms) *queue_ms = ms(r.t_start - r.t_submit);
    if (run_ms) *run_ms = ms(r.t_done - r.t_start);
    if (total_ms) *total_ms = ms(r.t_done - r.t_submit);
    return RBFD_OK;
}

int rbfd_server_destroy(rbfd_server *S) {
    if (!S) return RBFD_OK;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->shutdown = true;
        S->queue.clear();
        S->cv_work.notify_all();
    }
    for (auto &t : S->workers) t.join();
    for (auto &M : S->meshes)
        for (rbfd_mesh *m : M->idle) rbfd_destroy(m);
    delete S;
    return RBFD_OK;
}

}  // extern "C"
