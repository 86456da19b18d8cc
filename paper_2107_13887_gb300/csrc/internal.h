// internal.h -- host-side state of an rbfd mesh and the launch wrappers that
// the C ABI (api.cu) drives.  Not part of the public interface.
#pragma once

#include <atomic>
#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "../../include/rbfd.h"
#include "common.cuh"

namespace rbfd {

// Error carrying an rbfd_status; thrown inside the library, converted to a
// status + thread-local message at the C boundary.
struct Error {
    int status;
    std::string msg;
};

void set_last_error(const std::string &msg);
[[noreturn]] void fail(int status, const std::string &msg);
void check_cuda(cudaError_t e, const char *what);
#define RBFD_CUDA(call) ::rbfd::check_cuda((call), #call)

// An NVTX range for the scope (greedy levels and steps, volume updates,
// serving requests): named spans on a profiler's timeline, nothing without one.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
    ~NvtxRange() { nvtxRangePop(); }
};

// Device allocation from the library's per-device caching pool; reports
// RBFD_ENOMEM through Error.  dfree returns the block to the pool: call it
// only once the stream that used the block has been synchronised.
void *dmalloc(size_t bytes, const char *what);
void dfree(void *p);
// Small pinned host blocks (<= 4 KB), pooled.
void *pinned_alloc(size_t bytes);
void pinned_free(void *p);

template <typename T>
T *dalloc(size_t n, const char *what) {
    return static_cast<T *>(dmalloc(sizeof(T) * (n ? n : 1), what));
}

// ------------------------------------------------------------ spatial prep

// Tile sizes of the radix sort and of the scan (keys per block), and the
// scratch capacities they need for n keys: SortScratch::reserve grows to
// these, and fixed scratch arrays are sized by them.
constexpr int kSortTile = 2048;
constexpr int kScanTile = 2048;
constexpr size_t sort_hist_need(size_t n) { return 256 * ((n + kSortTile - 1) / kSortTile + 1); }
constexpr size_t sort_sums_need(size_t n) {
    return ((sort_hist_need(n) + kScanTile - 1) / kScanTile > (n + kScanTile - 1) / kScanTile
                ? (sort_hist_need(n) + kScanTile - 1) / kScanTile
                : (n + kScanTile - 1) / kScanTile) + 2;
}

// Scratch for the radix sort / scan / compaction primitives (grown on demand).
struct SortScratch {
    int64_t *launches = nullptr;  // kernel launch counter of the owning mesh
    uint32_t *keys_alt = nullptr;
    uint32_t *vals_alt = nullptr;
    uint32_t *hist = nullptr;   // 256 * n_blocks
    uint32_t *block_sums = nullptr;
    size_t cap_items = 0, cap_hist = 0, cap_sums = 0;
    void reserve(size_t n_items);
    void release();
};

// Stable LSD radix sort of (key, value) pairs by the low key_bits bits of key.
// The sorted result ends up in keys/vals.
void radix_sort_pairs(uint32_t *keys, uint32_t *vals, size_t n, int key_bits, SortScratch &s,
                      cudaStream_t st);

// Exclusive scan of n uint32 values (out may alias in); returns nothing,
// total written to *total_dev if non-null.
void exclusive_scan_u32(const uint32_t *in, uint32_t *out, size_t n, uint32_t *total_dev, SortScratch &s,
                        cudaStream_t st);

// Morton keys of points relative to the box bbox[6] in device memory: 2D 16
// bits per axis, 3D 10 bits, shifted right by `shift` bits (coarser keys,
// fewer radix passes); iso: cubic cells of the box's longest extent.
void morton_keys_f64_dev(const double4 *xyz, size_t n, int dim, const double *bbox, uint32_t *keys, uint32_t *vals,
                         cudaStream_t st, int shift = 0, bool iso = false);
// Volume points: 24-bit Morton keys (12 bits per axis in 2D, 8 in 3D), three radix passes.
constexpr int kVolKeyBits = 24;
inline int vol_key_shift(int dim) { return dim == 2 ? 32 - kVolKeyBits : 30 - kVolKeyBits; }
void morton_keys_f32(const float4 *xyzd, const uint32_t *idx, size_t n, int dim, double3 lo, double3 hi,
                     uint32_t *keys, uint32_t *vals, cudaStream_t st);

// ------------------------------------------------------------ mesh state

struct Level {
    double R = 0, tau = 0, smax = 0, emax = 0;
    int64_t nc = 0;
    int status = RBFD_OK;
    // host copies of the original surface indices (selection order) and the
    // weights [nc][dim], fetched from the device on first request
    std::vector<int64_t> idx;
    std::vector<double> alpha;
    bool fetched = false;
    uint32_t *d_orig = nullptr;   // original surface indices (device)
    double *h_scal = nullptr;     // pinned: the level's scalars (max |dS_l|^2, ..., corrections)
    double4 *d_cx = nullptr;      // control coordinates (FP64)
    double4 *d_alpha = nullptr;   // weights (FP64)
    float4 *d_cdf = nullptr;      // [2 nc] the coordinates as double-float (hi xyz, lo xyz)
    float4 *d_adf = nullptr;      // [2 nc] the weights as double-float ((ax, ay) hi/lo pairs, az pair)
    // uniform cell grid over the surface's box (cell size h) for the volume sweep
    double3 g0{0, 0, 0};
    double h = 0;
    int3 gdim{0, 0, 0};
    int ncell = 0;
    uint32_t *d_cell_start = nullptr;  // [ncell + 1]
    uint32_t *d_cell_ctrl = nullptr;   // [nc] control ids ordered by cell
    // the controls' double-float records in that cell order, 64 bytes each
    // (coordinates hi, lo; weights (ax, ay) hi/lo pairs, az pair): the volume
    // sweep stages a cell's controls with one bulk copy
    float4 *d_rec = nullptr;
    // kept for a warm start of the next time step (rbfd_greedy_warm): the
    // level's inverse factor G = L^{-1} and its transpose, packed n x n rows,
    // and the controls' sorted positions
    double *d_Gs = nullptr, *d_Gts = nullptr;
    uint32_t *d_cids = nullptr;
    // the same with cell size h / 2 (made on request: level_fine_grid)
    double3 f_g0{0, 0, 0};
    double f_h = 0;
    int3 f_gdim{0, 0, 0};
    uint32_t *f_cell_start = nullptr, *f_cell_ctrl = nullptr;
    float4 *f_rec = nullptr;
};

// Optional per-kernel-class timing with CUDA events on the mesh's stream.
enum ProfKind { kProfSweep = 0, kProfGrow = 1, kProfVol = 2, kProfPersist = 3, kProfWall = 4, kProfNewton = 5,
                kProfKinds = 6 };

struct Profiler {
    bool on = false;
    std::vector<cudaEvent_t> free_ev;
    struct Pending {
        int kind;
        cudaEvent_t a, b;
    };
    std::vector<Pending> pend;
    double ms[kProfKinds] = {};
    int64_t launches[kProfKinds] = {};
    cudaEvent_t get();
    cudaEvent_t begin(cudaStream_t st);            // records and returns the start event (or nullptr)
    void end(int kind, cudaEvent_t a, cudaStream_t st, int n_launches);
    void flush();                                  // after a stream sync: accumulate finished pairs
    void release();
};

}  // namespace rbfd

struct rbfd_mesh {
    int dim = 3;
    int64_t n_s = 0;
    int n_levels_req = 0;
    double eps = 0, S0 = 0;
    double h_sbox[6] = {0, 0, 0, 0, 0, 0};  // box of the surface points (lo xyz, hi xyz)
    rbfd_options opt{};
    std::vector<double> R;
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;

    // Morton-sorted surface
    int n_pb = 0;
    uint32_t *d_perm = nullptr;  // sorted position -> original index
    uint32_t *d_inv = nullptr;   // original index -> sorted position
    double4 *d_xs = nullptr;     // sorted coordinates (FP64, z = 0 in 2D)
    double4 *d_dS = nullptr;     // sorted displacements
    double4 *d_cur = nullptr;    // current level target dS_l
    double4 *d_E = nullptr;      // error of the last confirm sweep
    double4 *d_pb_lo = nullptr, *d_pb_hi = nullptr, *d_pb_org = nullptr;
    float4 *d_xs_hi = nullptr, *d_xs_lo = nullptr;  // coordinates relative to the block origin (df)
    float4 *d_pb_fbox = nullptr;  // [4][n_pb] FP32 block boxes for the wall distance (made on first use)

    // greedy workspace
    int cap = 0;
    unsigned char *d_sel = nullptr;
    double *d_G = nullptr;        // inverse Cholesky factor, cap x cap, row-major lower
    double *d_Gt = nullptr;       // its transpose, row-major (row k = column k of G)
    uint32_t *d_nz_k = nullptr;   // nonzeros of the newest phi column: control ids
    double *d_nz_v = nullptr;     //   and values
    double4 *d_w = nullptr;       // L^{-1} dS_c
    double4 *d_alpha = nullptr;   // weights of the current level
    double4 *d_cx = nullptr;      // control coordinates
    float4 *d_cdf = nullptr;      // the same split into double-float hi [0..cap] and lo [cap+1..]
    uint32_t *d_cid = nullptr;    // control sorted positions
    double *d_phi = nullptr;      // phi(c_new, c_k)
    double *d_y = nullptr;        // G phi
    double *d_red = nullptr;      // per-block partial dot products
    double *d_gpart = nullptr;    // per-row-tile partial column sums
    double4 *d_vec = nullptr;     // refinement vectors
    double4 *d_vec2 = nullptr;
    uint32_t *d_nb_cnt = nullptr; // controls listed per point block
    uint32_t *d_nb_list = nullptr;// [n_pb][cap]
    double4 *d_part = nullptr;    // sweep partial sums [n_chunk_max][n_s]
    double4 *d_gpart4 = nullptr;  // their group sums [ceil(n_chunk_max / 16)][n_s] (persistent sweep)
    unsigned int *d_grp_done = nullptr;  // [n_pb][ceil(n_chunk_max / 16)] chunk counters of the groups
    int n_chunk_max = 1;
    unsigned int *d_pb_done = nullptr;
    double *d_pb_key = nullptr;
    int *d_pb_idx = nullptr;
    // pruned list sweep (meshes of at most kPfxMax point blocks): per step
    // parity and warp of points (32 points, 4 per point block) the warp's max
    // |E| at its last sweep (rounded up, down), the bound accumulated since,
    // the largest sum_c phi |alpha_c| at its points then, in FP32
    // ([2][4 n_pb]); each warp's box
    // in FP32 rounded outward ([4 n_pb][lo, hi]); the point blocks listing
    // each control ([cap + 1][n_pb], counts [cap + 1])
    float4 *d_bnd = nullptr;
    double *d_bacc = nullptr;  // the bound accumulated since, summed in FP64 ([2][4 n_pb])
    float4 *d_wbox = nullptr;
    uint32_t *d_rev = nullptr;
    uint32_t *d_rev_cnt = nullptr;
    unsigned long long *d_pairs = nullptr;  // [16]: surface sweep useful, visited; volume useful, visited;
                                            //     wall distance search, exact pass; Newton basis terms;
                                            //     deform points; Newton phi values within R, all formed;
                                            //     Eq. 12 nonzeros of the Newton steps; pairs and block
                                            //     steps the pruned sweep skipped
    rbfd::GreedyState *d_st = nullptr;
    rbfd::GreedyState *h_st = nullptr;  // pinned
    rbfd::GridBarrier *h_bar = nullptr; // pinned
    double *d_lvl = nullptr;            // [8] level scalars: max|dS_l|^2, its argmax, refinement flag and count
    double *h_lvl = nullptr;            // pinned copy
    uint32_t *d_ckeys = nullptr;        // [cap + 1] control cell keys
    // persistent engine
    int batch_ctas_cap = 0;          // set by the batch calls: blocks this mesh may use
    // rbfd_greedy_batch: the batch's meshes still in their greedy and the
    // blocks they share (a finished mesh's share goes to the others)
    std::atomic<int> *batch_active = nullptr;
    int batch_total = 0;
    int batch_share = 0;             // meshes whose greedy runs beside this one (batch calls, server)
    rbfd::GridBarrier *d_bar = nullptr;
    double *d_pred = nullptr;       // [kMaxPersistCTAs][4] per-block y.y, y.w; then the pivot and w_n (8)
    // Newton-basis launch (made on first use): V[k][i] = v_k(x_i) for k < newton_cols
    int newton_cols = 0;
    double *d_V = nullptr;
    float4 *d_nwdf = nullptr;       // [cap + 1][2] w in double-float (mixed-mode Newton launch)
    int newton_rec_rows = 0;        // blocks the records below are sized for
    int newton_shape_key = -1;      // launch shape of the Newton kernel, cached per (blocks asked, sharing)
    int newton_ctas = 0, newton_ppb = 0, newton_cs = 0;
    size_t newton_smem = 0;
    double4 *d_nrec = nullptr;      // [blocks][3] per-block candidate records
    double *d_nycol = nullptr;      // [blocks][newton_cols + 1] their columns of V
    unsigned long long *d_phase_ns = nullptr;  // [8] persistent phase timing (profile mode)

    // surface split of the greedy over ranks (rbfd_greedy_split): this rank's
    // share of the Morton point blocks and the caller's all-reduce-maxloc of
    // each step's candidate; split_world = 1 outside that call
    int split_world = 1, split_rank = 0;
    // keep every level's inverse factor after the greedy (rbfd_greedy_warm)
    bool keep_factors = false;
    rbfd_maxloc_fn split_maxloc = nullptr;
    void *split_user = nullptr;

    std::vector<rbfd::Level> levels;
    // levels of the run before a new displacement, kept (with their factors)
    // for the warm start of the next greedy
    std::vector<rbfd::Level> warm_prev;
    bool greedy_done = false;
    rbfd_stats stats{};
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    cudaEvent_t ev_g0 = nullptr, ev_g1 = nullptr;  // the greedy's start and end
    bool greedy_pending = false;   // the greedy's last wait and epilogue not yet done (greedy_finish)
    double *d_lvl_hist = nullptr;  // [levels] max |dS_l|^2 of each level
    double *d_Dl = nullptr;        // [levels] D_l on the device (volume update after a pending greedy)
    float *d_invDlf = nullptr;     // [levels] 1 / D_l in FP32
    rbfd::SortScratch sort;
    rbfd::Profiler prof;

    // deform workspace (grown on demand)
    size_t vol_cap = 0;
    float4 *d_vin = nullptr;       // input points (x, y, z, d), caller order
    float4 *d_vpos = nullptr;      // compacted + Morton-sorted points
    float4 *d_vpos4 = nullptr;     // the same as float4 (FP32-input volume sweep)
    uint32_t *d_vorig = nullptr;   // their caller indices
    uint32_t *d_wl_list = nullptr; // work-list volume update: the lists d < D_l of every level [levels][wl_cap]
    size_t wl_cap = 0;
    int wl_levels = 0;
    uint32_t *d_wl_cnt = nullptr;  // [64] their lengths
    uint32_t *d_vflag = nullptr, *d_vscan = nullptr, *d_vlist = nullptr, *d_vkeys = nullptr;
    double4 *d_vacc = nullptr;     // accumulated displacement per sorted point
    void *d_vio = nullptr;         // staging for host inputs/outputs
    size_t vio_bytes = 0;
    // registered volume (rbfd_set_volume): Morton-sorted once, deformed per displacement
    int64_t vreg_n = 0;
    double4 *d_vreg = nullptr;     // sorted points (x, y, z, d)
    uint32_t *d_vreg_orig = nullptr;
    void *d_arena = nullptr;       // one block holding the fixed buffers of the set-up
    bool prep_pending = false;     // the set-up's S0 and surface box not yet read (mesh_ready)
    double *h_prep = nullptr;      // pinned: their copy
    void *prep_temps = nullptr;    // the set-up's temporaries, freed by mesh_ready
    uint32_t *d_misc = nullptr;    // small counters
    double *d_bbox = nullptr;      // 8 doubles
    // volume staged ahead of the greedy (copies, packing, Morton order of every
    // point on a second stream while the greedy runs): valid for one deform
    // call with the same arguments
    cudaStream_t vstream = nullptr;
    cudaEvent_t ev_vfork = nullptr, ev_vdone = nullptr;
    rbfd::SortScratch vsort;
    double *d_vred = nullptr;      // box partials of the staging (6 x 256)
    double *d_vbox = nullptr;      // box of the staged points (8 doubles)
    bool vst_ok = false;
    int64_t vst_n = 0;
    const void *vst_x = nullptr, *vst_d = nullptr;
    bool vst_f64 = false;
    void *vst_dout = nullptr;      // device output (the staging buffer for host outputs)
    const void *vst_io_x = nullptr, *vst_io_d = nullptr;  // device copies of the inputs
    bool vst_queued = false;       // the staging work is on the staging stream
    double vst_D0 = 0.0;           // D_0 of the staged call
    bool vst_l0 = false;           // level 0 already swept on the staging stream
};

namespace rbfd {
constexpr int kMaxPersistCTAs = 2048;
constexpr int kPfxMax = 2048;  // point blocks up to which the persistent sweep balances its items (and prunes)
constexpr int kNewtonCols = 4096;  // most controls a Newton-basis launch carries (y staged in shared memory)
int newton_columns(rbfd_mesh *m);
void newton_reserve(rbfd_mesh *m);
// false if a Newton launch of this mesh does not fit its share of the GPU
bool newton_fits(rbfd_mesh *m, int ctas);
void newton_run_level(rbfd_mesh *m, double R, double tau, int ctas);
int persist_max_ctas(rbfd_mesh *m);
// max_steps > 0: the launch ends after that many steps with st->handoff set
// (the level goes on in the next launch)
void persist_run_level(rbfd_mesh *m, double R, double tau, int ctas, int max_steps = 0);
constexpr int kYieldSteps = 1024;  // steps of a batch mesh's launch while other meshes still run
// wait = false: the greedy returns once its work is queued; its last wait and
// epilogue (level scalars, timing) happen in greedy_finish
// warm = true: start every level from the previous run's controls and
// factor (kept with keep_factors), re-solve the weights for the current
// displacement, and continue the greedy only where the level's confirm
// sweep is not below tau_l (rbfd_greedy_warm)
void greedy_run(rbfd_mesh *m, bool wait = true, bool warm = false);
void greedy_finish(rbfd_mesh *m);
// a level's device and pinned buffers back to the pools (its stream synchronised)
void level_free(Level &L);
// the level's control grid of half the cell size (f_* fields), queued on
// the mesh's stream if not made yet
void level_fine_grid(rbfd_mesh *m, Level &L);
// the host copies of a level's indices and weights (one synchronised copy, first call only)
void level_fetch(rbfd_mesh *m, Level &L);
void deform_run(rbfd_mesh *m, int64_t n_v, const void *xyz_v, const void *d_v, bool f64, double D, double k,
                void *out);
// rbfd_deform_worklist: the volume updates of n meshes in one work-list launch
// registered = true: every mesh's registered volume (rbfd_set_volume; n_v,
// xyz_v and d_v are then ignored), the serving loop's fused volume stage
void deform_worklist(rbfd_mesh **ms, int n, const int64_t *n_v, const float *const *xyz_v,
                     const float *const *d_v, const double *D, const double *k, float *const *out,
                     rbfd_worklist_tune *tune, bool registered = false);
// Stage a volume for the next deform_run with the same arguments: copies,
// packing and the Morton order of every point, on a second stream that
// starts after the work queued so far on the mesh's stream (the greedy can
// run meanwhile).  Only with wall distances given.
void volume_stage(rbfd_mesh *m, int64_t n_v, const void *xyz_v, const void *d_v, bool f64, double D, double k);
// After level l is saved: with a staged volume, queue that level's volume
// sweep on the staging stream (level 0 only: its D_0 follows from S0), so it
// runs while the greedy continues.
void volume_level_early(rbfd_mesh *m, int l);
// Queue the staging work of a staged volume (copies, packing, Morton order)
// on its stream, if not yet done: the greedy calls it after its first launch.
void volume_stage_enqueue(rbfd_mesh *m);
// Drop a staged volume that will not be used (the mesh's stream waits for it).
void volume_unstage(rbfd_mesh *m);
// Return the staging stream and events (mesh destruction).
void volume_stage_release(rbfd_mesh *m);
void mesh_prepare(rbfd_mesh *m, const double *xyz_s, const double *dS);
// Wait for the set-up queued by mesh_prepare and read S0 and the surface box
// (first call only).
void mesh_ready(rbfd_mesh *m);
void mesh_set_displacement(rbfd_mesh *m, const double *dS);
void volume_register(rbfd_mesh *m, int64_t n_v, const float *xyz_v, const float *d_v);
void deform_registered(rbfd_mesh *m, double D, double k, float *out);
void mesh_free(rbfd_mesh *m);
// wall distance of n Morton-sorted points: min(d, cap) into d_out (sorted
// order) or, with d_out null, into vpos[i].w
void wall_distance_sorted(rbfd_mesh *m, int64_t n, double4 *vpos, double cap, double *d_out);
void wall_distance_run(rbfd_mesh *m, int64_t n_v, const void *xyz_v, bool f64, double *out);
void orthogonality_run(int dim, int64_t n_i, int64_t n_k, int64_t n_layers, int periodic_i, const double *wall,
                       const double *wall_disp, const float *vol, const float *vol_disp, bool on_device,
                       cudaStream_t st, float *theta, rbfd_quality *q);
}  // namespace rbfd
