/*
 * rbfd.h -- C ABI of the GB300 library for multi-level greedy compact-support
 * RBF mesh deformation with volume point reduction (Morelli, Bellosta,
 * Guardone, "Efficient Radial Basis Function Mesh Deformation Methods for
 * Aircraft Icing").
 *
 * The library runs every step of the method in its own CUDA kernels on one
 * GPU.  Plain pointers and sizes only; no C++ or framework types.
 *
 * Conventions for every function:
 *   - the return value is an rbfd_status; on failure rbfd_last_error() gives a
 *     human-readable, thread-local message describing the most recent error;
 *   - point arrays are row-major [n][dim] (x, y[, z] per point), dim 2 or 3;
 *   - the caller owns every buffer it passes; the library copies what it keeps;
 *   - buffers are host pointers unless rbfd_options.inputs_on_device is set
 *     at rbfd_create, in which case every array argument of that mesh's calls
 *     (create, deform) must be device memory of the current CUDA device;
 *   - a mesh handle is not thread-safe: one host thread at a time per handle.
 */
#ifndef RBFD_H
#define RBFD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum rbfd_status {
    RBFD_OK = 0,
    RBFD_EINVAL = 1,     /* bad argument: dim not 2/3, R <= 0, eps not in (0,1), NULL pointer, ... */
    RBFD_ENOMEM = 2,     /* a device or host allocation failed */
    RBFD_ESINGULAR = 3,  /* Phi_cc lost positive definiteness: coincident or near-coincident controls */
    RBFD_ENOTCONV = 4,   /* the control cap was reached before eps; results are valid, e_max reports the error */
    RBFD_ETIMEOUT = 5,   /* a bounded device-side or host-side wait hit its limit */
    RBFD_EBUSY = 6,      /* serving admission refused for now (device memory); retry later */
    RBFD_ECUDA = 7,      /* a CUDA runtime call failed (message in rbfd_last_error) */
    RBFD_ESTATE = 8,     /* call out of order (e.g. deform before greedy) */
    RBFD_ECOMM = 9,      /* the caller's reduction callback failed (rbfd_greedy_split) */
    RBFD_ECANCELED = 10  /* the serving request was cancelled before it started (rbfd_cancel) */
} rbfd_status;

typedef enum rbfd_precision {
    RBFD_FP64 = 0,  /* every step in IEEE double: the reference mode */
    RBFD_MIXED = 1  /* evaluation sweeps on the FP32 pipe in double-float (FP32 pair)
                       arithmetic; FP64 kept for the control-system growth, the
                       iterative-refinement residual and the stop test */
} rbfd_precision;

typedef struct rbfd_options {
    int precision;         /* rbfd_precision; default RBFD_MIXED */
    int basis;             /* Wendland basis of Table 1: 0 = C0, 2 = C2 (Eq. 2, default), 4 = C4, 6 = C6.
                              C4 and C6 always run in FP64 (RBFD_MIXED applies to C0 and C2): their
                              control systems carry weights up to about 1e9 max|dS| on ice shapes,
                              beyond what the double-float sweeps resolve */
    int first_point;       /* 0: surface point 0 starts every level (Section 3, default);
                              1: the point of largest |dS_l| starts level l */
    int inputs_on_device;  /* 0: host pointers (default); 1: device pointers */
    int64_t nc_cap;        /* controls per level at most; 0 = min(n_s, 32768).  Device memory grows
                              as 16 * nc_cap^2 bytes (the inverse factor and its transpose) */
    void *stream;          /* cudaStream_t to run on; NULL = a stream the mesh creates */
    int eps_absolute;      /* 0: eps is relative to max_i |dS_i| (default); 1: absolute length */
    int refine_iters;      /* iterative-refinement sweeps at level close (default 3) */
    int profile;           /* 1: time each kernel class with CUDA events on the mesh's stream
                              (rbfd_stats.*_ms / *_launches); adds two event records per launch */
    int engine;            /* greedy engine: 0 (default) = persistent cooperative launches: a
                              level starts in the Newton basis (one FP64 update per point
                              and step) and goes on with the control-list sweep once that
                              is cheaper; 2 = the persistent list sweep only; 1 = separate
                              launches for every step */
    int grid_ctas;         /* blocks of the persistent launch (0 = chosen from the mesh size) */
    int prune;             /* 1 (default): the persistent list sweep skips a warp of 32
                              points while a bound shows that none of them can hold the
                              step's argmax (the bound: the warp's max |E| at its last sweep
                              plus, for every step since, |w_n| times the sum over the
                              controls of |G row n| phi(distance to the warp's box / R), plus
                              the sweep's rounding).  The picks and the stop test are those
                              of a full sweep; fewer pairs are evaluated.  Meshes of up to
                              2,048 point blocks (262,144 surface points).  0: every point
                              every step */
} rbfd_options;

typedef struct rbfd_mesh rbfd_mesh;

/* Fill *opt with the defaults listed above. */
void rbfd_options_default(rbfd_options *opt);

/*
 * rbfd_create -- set up one surface for deformation (Section 2: surface
 * points r_s and displacements dS = (dX_s, dY_s, dZ_s); Section 3: support
 * radius R_l for each of the n_levels levels of the multi-level greedy
 * selection, final tolerance eps on max_i |E_i| / max_i |dS_i|).
 *
 *   out      receives the new handle (set to NULL on failure)
 *   dim      2 or 3
 *   n_s      number of surface points, >= 1
 *   xyz_s    [n_s][dim] surface coordinates (double)
 *   dS       [n_s][dim] surface displacements (double)
 *   n_levels number of greedy levels, >= 1
 *   R        [n_levels] support radius per level, each > 0
 *   eps      final tolerance, 0 < eps < 1 (relative unless opt->eps_absolute)
 *   opt      options, or NULL for the defaults
 *
 * Copies the inputs to the device, Morton-orders the surface points and
 * builds the point blocks the sweeps use.  Errors: RBFD_EINVAL, RBFD_ENOMEM,
 * RBFD_ECUDA.
 */
int rbfd_create(rbfd_mesh **out, int dim, int64_t n_s, const double *xyz_s, const double *dS,
                int n_levels, const double *R, double eps, const rbfd_options *opt);

/*
 * rbfd_greedy -- run the multi-level greedy surface point selection of
 * Section 3 on the device: for each level l, start from one control, then
 * repeatedly solve Phi_cc alpha = dS_l on the controls (Eq. 9), sweep the
 * error E = dS_l - Phi_sc alpha over all surface points (Eq. 12), add the
 * point of largest |E_i| until max |E_i| / max |dS_i| < eps^((l+1)/n_levels);
 * then dS_{l+1} = E.  Blocks until done.  May be called again to re-run.
 * Errors: RBFD_ESINGULAR, RBFD_ENOTCONV (results valid), RBFD_ETIMEOUT (a grid
 * barrier of the persistent launch waited past its bound; the launch ended
 * without hanging), RBFD_ECUDA.
 */
int rbfd_greedy(rbfd_mesh *m);

/*
 * rbfd_get_level -- results of level l (0-based) after rbfd_greedy.
 *   n_c    receives the number of controls (may be NULL)
 *   idx    [n_c] receives their surface indices in selection order (may be NULL)
 *   alpha  [n_c][dim] receives their weights (may be NULL)
 *   e_max  receives max_i |E_i| / max_i |dS_i| after the level (may be NULL)
 * Call first with idx = alpha = NULL to learn n_c.  Host pointers always.
 * Errors: RBFD_EINVAL (l out of range), RBFD_ESTATE (no greedy yet).
 */
int rbfd_get_level(rbfd_mesh *m, int l, int64_t *n_c, int64_t *idx, double *alpha, double *e_max);

/* Number of levels the greedy produced (0 when every dS is zero). */
int rbfd_num_levels(rbfd_mesh *m, int *n_levels);

/*
 * rbfd_level_info -- per-level scalars: R_l, max_i |dS_l,i| (the quantity the
 * support distance D_l = k max |dS_l| of Section 4 uses) and the level's
 * tolerance tau_l.  Any output may be NULL.
 */
int rbfd_level_info(rbfd_mesh *m, int l, double *R, double *smax, double *tau);

typedef struct rbfd_stats {
    double greedy_ms;        /* device time of the last rbfd_greedy (CUDA events) */
    double deform_ms;        /* device time of the last rbfd_deform */
    int64_t greedy_steps;    /* control additions over all levels */
    int64_t pairs_useful;    /* greedy + deform point/control pairs evaluated with |r - r_c| < R */
    int64_t pairs_visited;   /* pairs the kernels evaluated (a superset of the useful ones) */
    int64_t deform_points;   /* volume points updated at least at one level (sum over levels) */
    int64_t refine_sweeps;   /* iterative-refinement sweeps run at level close */
    int64_t confirm_resumes; /* times a level-close confirm sweep reopened the greedy */
    int64_t launches;        /* kernels this mesh launched (all calls since creation) */
    /* per kernel class, since creation (event timing only with opt.profile = 1):
       surface error sweep (Eq. 12 + argmax), control-system growth, volume sweep (Eq. 23) */
    double sweep_ms, grow_ms, vol_ms;
    int64_t sweep_launches, grow_launches, vol_launches;
    int64_t sweep_pairs_useful, sweep_pairs_visited, vol_pairs_useful, vol_pairs_visited;
    double persist_ms;         /* persistent list-sweep launches (engines 0, 2): sweep + growth of every step */
    int64_t persist_launches;
    int64_t persist_ctas;      /* blocks of the last persistent launch */
    /* profile mode: block 0 of the persistent launch, summed over steps, in ms:
       [2p] = work of phase p (sweep, argmax+phi, G phi, G row), [2p+1] = wait at its barrier */
    double persist_phase_ms[8];
    /* wall distance queries (rbfd_wall_distance, or deform/set_volume without d_v) */
    double wall_ms;              /* event time of the query kernels (opt.profile = 1) */
    int64_t wall_launches;
    int64_t wall_pairs_search;   /* point pairs scanned by the FP32 search pass */
    int64_t wall_pairs_exact;    /* point pairs scanned by the exact pass */
    int64_t newton_steps;        /* greedy steps taken in the Newton basis (engine 0) */
    double newton_ms;            /* event time of the Newton-basis launches (opt.profile = 1) */
    int64_t newton_launches;
    int64_t newton_terms;        /* basis values the Newton update read: n_s x controls, summed over steps */
    /* host wall time of the last rbfd_greedy by part, in ms, summed over levels:
       [0] level start, [1] greedy steps (launches and their waits),
       [2] level close (refinement, confirm sweep), [3] level save (results to
       the host, control grid) */
    double greedy_host_ms[4];
    /* pair evaluations the kernels performed with |r - r_c| < R, by kind: the
       Newton-basis update evaluates phi of each step's control at every
       surface point (newton_pairs_useful within R, newton_pairs_formed in all),
       where a list sweep of the same step evaluates the nonzeros of Eq. 12:
       eq12_pairs counts those for every greedy step and the confirm sweeps,
       whichever engine ran (the method's own pair count, as Section 3 states
       it), less the point blocks a pruned sweep skipped (opt.prune; those
       are counted in sweep_pairs_skipped); pairs_useful = sweep_pairs_useful + vol_pairs_useful +
       newton_pairs_useful is what was evaluated */
    int64_t newton_pairs_useful;
    int64_t newton_pairs_formed;
    int64_t eq12_pairs;
    /* FP64 multiply-adds the persistent list sweep spent on the rows of the
       inverse factor G in the last rbfd_greedy (k (k + 1) / 2 for the step that
       adds control k) */
    int64_t persist_grow_fma;
    /* pairs (points x their block's list length, as sweep_pairs_visited
       counts them) and steps of a warp of 32 points that the pruned list
       sweep skipped, since creation */
    int64_t sweep_pairs_skipped;
    int64_t sweep_warps_skipped;
} rbfd_stats;

int rbfd_get_stats(rbfd_mesh *m, rbfd_stats *st);

/*
 * rbfd_deform -- volume update of Eq. 19 with the wall-distance blending of
 * Eq. 23 (Section 4):
 *     out_v = sum_l psi(d_v / D_l) sum_j alpha_j^(l) phi(|r_v - r_cj^(l)| / R_l)
 * with psi(xi) = 1 - xi on [0, 1), 0 beyond, and D_l = k * max_i |dS_l,i|
 * (capped at D when D > 0) if k > 0, else D_l = D.  Only volume points with
 * d_v < D_l take part in level l (volume point reduction).
 *
 *   n_v    number of volume points (0 allowed)
 *   xyz_v  [n_v][dim] volume coordinates (float)
 *   d_v    [n_v] wall distance of each volume point (float, negative read as 0),
 *          or NULL: the library computes it (as rbfd_wall_distance, needed
 *          and computed only below max_l D_l)
 *   D, k   support distance and volume reduction factor (>= 0; not both 0)
 *   out    [n_v][dim] receives the displacement of each volume point (float)
 *
 * Errors: RBFD_EINVAL, RBFD_ESTATE (no greedy yet), RBFD_ENOMEM, RBFD_ECUDA.
 */
int rbfd_deform(rbfd_mesh *m, int64_t n_v, const float *xyz_v, const float *d_v, double D, double k,
                float *out);

/*
 * Time stepping on one surface (an ice shape growing step by step): the
 * surface points and the volume mesh stay the same, the displacement changes.
 *
 * rbfd_set_displacement -- replace dS ([n_s][dim], caller order) of a mesh;
 *   keeps the Morton order, point blocks and workspace; the previous greedy
 *   results are dropped (run rbfd_greedy again).
 * rbfd_set_volume -- register a volume mesh ([n_v][dim] float coordinates,
 *   [n_v] wall distances, or NULL to compute them once with
 *   rbfd_wall_distance) once; it is packed and Morton-sorted on the device
 *   and kept until the next call or rbfd_destroy.
 * rbfd_deform_volume -- rbfd_deform on the registered volume: out [n_v][dim].
 * Pointer kinds follow inputs_on_device.  Errors as for rbfd_deform.
 */
int rbfd_set_displacement(rbfd_mesh *m, const double *dS);
int rbfd_set_volume(rbfd_mesh *m, int64_t n_v, const float *xyz_v, const float *d_v);
int rbfd_deform_volume(rbfd_mesh *m, double D, double k, float *out);

/* Same as rbfd_deform with double coordinates, distances (or NULL) and output. */
int rbfd_deform_f64(rbfd_mesh *m, int64_t n_v, const double *xyz_v, const double *d_v, double D, double k,
                    double *out);

/*
 * rbfd_wall_distance -- the wall distance d of Section 4 (the distance of a
 * volume point from the surface, the argument of psi in Eq. 23, which the
 * paper takes as given): for each volume point r_v,
 *     d_out[v] = min_i |r_v - r_s,i|
 * over the mesh's n_s surface points (as passed to rbfd_create), with the
 * distance evaluated in FP64 as sqrt(dx*dx + dy*dy (+ dz*dz)), each operation
 * rounded once, in axis order.  The result is exact in that sense: the same
 * value as a plain brute-force minimum in FP64, bit for bit.  Needs no greedy.
 *
 *   n_v    number of volume points (0 allowed)
 *   xyz_v  [n_v][dim] coordinates: float (rbfd_wall_distance) or double
 *          (rbfd_wall_distance_f64); host or device per inputs_on_device
 *   d_out  [n_v] result (double), caller order
 *
 * Errors: RBFD_EINVAL (NULL arrays, n_v < 0 or >= 2^31), RBFD_ENOMEM, RBFD_ECUDA.
 */
int rbfd_wall_distance(rbfd_mesh *m, int64_t n_v, const float *xyz_v, double *d_out);
int rbfd_wall_distance_f64(rbfd_mesh *m, int64_t n_v, const double *xyz_v, double *d_out);

/*
 * rbfd_orthogonality -- mesh quality of a deformed structured grid, the
 * orthogonality angle by which Section 5 judges the deformations.  The grid
 * grows off the surface: node layer j = 0 is the wall, layers j = 1..n_layers
 * are volume points; i runs round the section (periodic_i = 1 when it closes
 * on itself, as an O-mesh does), k along the span (3D only).
 *
 *   wall       [n_k][n_i][dim] wall node coordinates (double)
 *   wall_disp  same shape, added to wall (double), or NULL
 *   vol        [n_k][n_i][n_layers][dim] volume node coordinates (float);
 *              the layout rbfd_deform's xyz_v has for these meshes
 *   vol_disp   same shape, added to vol (float; rbfd_deform's out), or NULL
 *   theta      per cell, the angle in degrees (float), or NULL; 2D cells
 *              (i, j) at i * n_layers + j, 3D cells (k, i, j) at
 *              (k * n_ci + i) * n_layers + j, n_ci = n_i if periodic_i else
 *              n_i - 1, k < n_k - 1, j < n_layers
 *   q          summary (below), or NULL
 *   on_device  1: every array is device memory of the current device; 0: host
 *   stream     cudaStream_t to run on, or NULL for the per-thread default stream
 *
 * Each node is the FP64 sum of its coordinate and its displacement.  The
 * orthogonality angle of a cell is the smallest angle between two grid lines
 * (cell edges) meeting at a corner, folded into [0, 90] degrees: 90 for a
 * rectangular cell, 0 for a collapsed one.  A cell whose corners disagree in
 * orientation (2D: the cross product of the edges round the cell; 3D: the
 * triple product of the three edges at a corner) is tangled.  Angles are
 * within 1e-4 degrees of an FP64 evaluation; tangled decisions equal it.
 * Errors: RBFD_EINVAL (dim not 2 or 3, n_i < 2, n_layers < 1, n_k < 2 in 3D,
 * NULL wall or vol), RBFD_ENOMEM, RBFD_ECUDA.
 */
typedef struct rbfd_quality {
    double min_deg;   /* smallest cell angle */
    double mean_deg;  /* mean cell angle */
    int64_t argmin;   /* cell of the smallest angle (lowest index on ties) */
    int64_t cells;
    int64_t tangled;  /* tangled cells */
    int64_t hist[9];  /* cells per 10-degree bin: [0,10), [10,20), ..., [80,90] */
} rbfd_quality;

int rbfd_orthogonality(int dim, int64_t n_i, int64_t n_k, int64_t n_layers, int periodic_i, const double *wall,
                       const double *wall_disp, const float *vol, const float *vol_disp, float *theta,
                       rbfd_quality *q, int on_device, void *stream);

/*
 * rbfd_sort_pairs -- the stable sort of (key, value) pairs that orders the
 * surface, volume and control points by Morton key (spatial preparation: the
 * neighbour lists of the compact-support sums of Section 3 and Eq. 23 are
 * read in this order).  Exposed so that callers can order their own points
 * the same way.
 *
 * keys, vals: n uint32 each, DEVICE memory, sorted in place by the low
 * key_bits bits of the key (1..32), equal keys kept in input order; values
 * follow their keys.  Up to 8,192 pairs one block sorts them in registers and
 * shared memory; beyond, an LSD radix sort of 8-bit digits.  stream: a
 * cudaStream_t (NULL: the per-thread default stream); the call returns after
 * the sort has finished.  Scratch memory is allocated and freed by the call.
 * Errors: RBFD_EINVAL (n < 0 or above 2^31 - 1, key_bits outside 1..32, NULL
 * or non-device arrays with n > 0), RBFD_ENOMEM, RBFD_ECUDA.
 */
int rbfd_sort_pairs(uint32_t *keys, uint32_t *vals, int64_t n, int key_bits, void *stream);

/*
 * rbfd_deform_noalloc -- the volume update of rbfd_deform for callers that
 * cannot allocate device memory while they run: a solver loop whose device
 * memory was reserved up front (a pool or a fixed budget), or a host that keeps
 * cudaMalloc/cudaFree off its hot path because those calls synchronise the
 * device and can fail in the middle of a run.  The paper has no counterpart;
 * this is a deployment variant of the same computation.
 *
 * Same arguments as rbfd_deform, with these differences:
 *   - xyz_v, d_v and out must be device memory of the mesh's GPU (float32,
 *     n_v x dim, n_v and n_v x dim values); anything else returns RBFD_EINVAL;
 *   - d_v is required (rbfd_deform computes missing wall distances; this call
 *     cannot, since that needs scratch of its own): NULL returns RBFD_EINVAL;
 *   - n_v must not exceed 131072: every per-call buffer lives in one fixed
 *     device array of about 16 MB that each GPU loading the library holds
 *     until the process exits; larger n_v returns RBFD_EINVAL;
 *   - the call allocates nothing (no cudaMalloc/cudaFree, no allocating
 *     library routine).  On each device the first call looks up the array's
 *     device address once (cudaGetSymbolAddress); make that first call before
 *     any stream capture;
 *   - it returns once its work on the mesh's stream has finished (it reads
 *     one count back to size its sort, and waits for its end event);
 *   - results: in FP64 mode the same per-point FP64 sums as rbfd_deform (only
 *     the grouping of points into blocks differs: agreement to rounding, far
 *     inside 1e-10 max|dS|); in mixed mode it runs the double-float sweep on
 *     FP64-packed points rather than rbfd_deform's FP32-input sweep, so the two
 *     agree within the mixed-mode bound of 1e-5 max|dS|, not bit for bit.
 * All calls share the array and it keeps the previous call's contents (the
 * call clears what must start at zero).  Calls whose work overlaps on the
 * GPU (two host threads, or two meshes on different streams) race on it: run
 * them one after another.  The mesh itself (rbfd_create, rbfd_greedy) is set up
 * beforehand with the ordinary, allocating calls.
 */
int rbfd_deform_noalloc(rbfd_mesh *m, int64_t n_v, const float *xyz_v, const float *d_v, double D, double k,
                        float *out);

/*
 * rbfd_greedy_warm -- rbfd_greedy for the mesh's current displacement
 * (rbfd_set_displacement), started from the previous run on this mesh: every
 * level begins with the previous run's controls of that level and their
 * inverse Cholesky factor, solves Eq. 9 for the new targets on it, and runs
 * the level close (FP64 refinement and the confirm sweep of Eq. 12).  If the
 * level's error is below tau_l the level keeps those controls; otherwise the
 * greedy of Section 3 continues from them.  A time step of an ice-growth
 * sequence, whose displacement changes little, then costs a few triangular
 * products and one sweep per level instead of the whole selection.  The
 * controls of a warm run are valid (every level below tau_l, Eq. 9 solved)
 * but they are the previous run's, not the greedy's own choice for the new
 * displacement.
 *
 * The first call on a mesh, or one after the levels changed, runs the plain
 * greedy.  From the first call on, every greedy on the mesh keeps each
 * level's factor on the device for the next call: 16 n_l^2 bytes per level
 * (about 80 MB for 2,300 controls).  Errors: as rbfd_greedy.
 */
int rbfd_greedy_warm(rbfd_mesh *m);

/*
 * rbfd_greedy_split -- rbfd_greedy with the surface points split over `world`
 * ranks (one GPU each), for the argmax of Section 3: at every greedy step
 * E = dS_l - Phi_sc alpha (Eq. 12) is swept over this rank's share of the
 * surface only -- a contiguous range of the Morton-ordered point blocks,
 * [rank n_pb / world, (rank + 1) n_pb / world) -- and the ranks combine their
 * best candidates with one all-reduce-maxloc of 16 bytes per step, which the
 * caller performs in `maxloc` (over NCCL, gloo, MPI, ...).
 *
 * Every rank creates the same mesh (rbfd_create with the full surface: the
 * coordinates and displacements are replicated, a few MB) and calls this
 * function with its own rank; the control system (the inverse factor G, the
 * weights alpha, the per-block control lists) is then updated identically and
 * deterministically on every rank, and the once-per-level confirm sweep runs
 * over the whole surface on every rank, so every rank ends with the same
 * levels: the controls and weights of rbfd_greedy with options.engine = 1,
 * bit for bit.  rbfd_deform can then be split by volume points (Morton ranges)
 * with no collective at all.
 *
 * maxloc(user, key, idx): on entry *key is the rank's largest |E_i|^2 over its
 * unselected points (-1 if it has none) and *idx that point's original
 * surface index (-1 if none); it must store the largest key over all ranks
 * and its index, the lowest index among equal keys, identically on every
 * rank, and return 0 (nonzero: the call fails with RBFD_ECOMM).  It is called
 * once per greedy step, from the calling thread.
 *
 * The steps run as separate launches with one host round trip each (the
 * exchange), so this form pays off when a rank's surface sweep is long
 * against that round trip; world = 1 is rbfd_greedy with engine 1.
 * Errors: as rbfd_greedy, plus RBFD_EINVAL (rank outside [0, world), world < 1,
 * NULL callback) and RBFD_ECOMM.
 */
typedef int (*rbfd_maxloc_fn)(void *user, double *key, int64_t *idx);
int rbfd_greedy_split(rbfd_mesh *m, int rank, int world, rbfd_maxloc_fn maxloc, void *user);

/*
 * rbfd_greedy_batch -- rbfd_greedy on n meshes at once.  Each greedy is a
 * chain of small, latency-bound steps (Section 3); independent meshes (several
 * ice shapes, several grids) run side by side: one host thread per mesh, each
 * on the mesh's own stream, the persistent launches sized so that they are
 * resident together.  On one device the meshes still in their greedy share
 * the blocks: while several run, a mesh's persistent launch ends every 1,024
 * steps and the next one takes the share that finished meshes left (the
 * controls are those of the mesh alone; the weights agree to rounding).
 * Give every mesh its own stream (the default) for overlap.  Returns the first failing mesh's status (RBFD_ENOTCONV only if no
 * mesh failed otherwise); every mesh that succeeded holds its results.
 */
int rbfd_greedy_batch(rbfd_mesh **meshes, int n);

/*
 * rbfd_deform_batch -- rbfd_deform on n meshes at once (one host thread and
 * stream per mesh).  Array i of each argument belongs to mesh i; the pointer
 * kinds follow each mesh's inputs_on_device option.
 */
int rbfd_deform_batch(rbfd_mesh **meshes, int n, const int64_t *n_v, const float *const *xyz_v,
                      const float *const *d_v, const double *D, const double *k, float *const *out);

/*
 * rbfd_deform_worklist -- the volume update of Eq. 19 with the blending of
 * Eq. 23 (Section 4) for n meshes (several wings of uneven size, say) in ONE
 * persistent launch.  Per mesh, its points are packed and Morton-sorted and
 * the lists V_l = {d < D_l} are formed on the mesh's own stream; then one
 * work-list kernel sweeps every (mesh, level) pair: blocks of 128 list
 * entries are handed out from a global counter, level by level, so small and
 * large meshes share the SMs with no tail of one mesh's launch; a level of a
 * mesh waits (bounded) for that mesh's previous level before it adds into the
 * same accumulator.  The results are those of rbfd_deform for each mesh,
 * within the mixed-mode bound (1e-5 max|dS|): the pair arithmetic is the
 * same, only the cell grid may differ (cell_div).
 *
 * Requirements: every mesh in mixed precision (RBFD_MIXED), all of one
 * dimension and basis, greedy done, on one device; float32 volume arrays
 * (host or device per each mesh's inputs_on_device); d_v (or any d_v[i]) may
 * be NULL: wall distances are then computed on the device.  n <= 16 meshes
 * and at most 64 (mesh, level) pairs.
 *
 * tune (in/out, may be NULL: autotune): with tune->autotune = 1 the call
 * times candidate settings on this call's own work (per mesh the cell size
 * R_l or R_l / 2 of its control grid; then blocks per SM; then list blocks per
 * work item) by coordinate descent, keeps the fastest, and caches it for later
 * calls on meshes of the same sizes; with autotune = 0 the given settings are
 * used.  On return the fields hold the settings used and the launch's
 * device time.
 * Errors: RBFD_EINVAL, RBFD_ESTATE (no greedy), RBFD_ETIMEOUT (a level's wait
 * ran out: not expected), RBFD_ENOMEM, RBFD_ECUDA.
 */
typedef struct rbfd_worklist_tune {
    int autotune;        /* 1: choose the fields below by timing candidates (cached per batch shape) */
    int ctas_per_sm;     /* resident blocks per SM of the work-list launch (1..8) */
    int item_blocks;     /* 128-entry list blocks per work item (1, 2 or 4) */
    int cell_div[16];    /* per mesh: control cell size R_l / cell_div, 1 or 2 */
    int cached;          /* out: 1 if the settings came from the cache */
    int trials;          /* out: candidate launches timed by this call */
    double launch_ms;    /* out: device time of the work-list launch */
    int64_t items;       /* out: list blocks the launch swept */
} rbfd_worklist_tune;

int rbfd_deform_worklist(rbfd_mesh **meshes, int n, const int64_t *n_v, const float *const *xyz_v,
                         const float *const *d_v, const double *D, const double *k, float *const *out,
                         rbfd_worklist_tune *tune);

/*
 * rbfd_greedy_deform_batch -- rbfd_greedy then rbfd_deform for each of n
 * meshes, mesh i's two calls one after the other on its own host thread and
 * stream, so that one mesh's volume update overlaps another's greedy.  With
 * wall distances given, a mesh's volume (host copies, packing, Morton order)
 * is prepared on a second stream while its own greedy runs; the results are
 * those of rbfd_greedy + rbfd_deform bit for bit.  The volume arrays are read
 * from the start of the call.  Arguments as rbfd_deform_batch (d_v may be
 * NULL, or any d_v[i], to compute wall distances).  Returns RBFD_ENOTCONV,
 * after deforming with the valid levels, if a greedy hit its control cap;
 * otherwise the worst status.
 */
int rbfd_greedy_deform_batch(rbfd_mesh **meshes, int n, const int64_t *n_v, const float *const *xyz_v,
                             const float *const *d_v, const double *D, const double *k, float *const *out);

/*
 * rbfd_job -- one whole deformation: the arguments of rbfd_create (surface,
 * displacement, levels, eps, options) and of rbfd_deform (FP32 volume points,
 * wall distances or NULL, D, k, output).  Pointer kinds follow
 * opt->inputs_on_device; the caller owns every array.
 */
typedef struct rbfd_job {
    int dim;                 /* 2 or 3 */
    int n_levels;            /* entries of R */
    int64_t n_s;             /* surface points */
    const double *xyz_s;     /* [n_s][dim] surface coordinates */
    const double *dS;        /* [n_s][dim] surface displacements */
    const double *R;         /* [n_levels] support radius per level */
    double eps;              /* final tolerance of the greedy */
    const rbfd_options *opt; /* NULL: rbfd_options_default */
    int64_t n_v;             /* volume points */
    const float *xyz_v;      /* [n_v][dim] volume coordinates */
    const float *d_v;        /* [n_v] wall distances, or NULL to compute them */
    double D, k;             /* as rbfd_deform */
    float *out;              /* [n_v][dim] volume displacements (written) */
} rbfd_job;

/*
 * rbfd_run_jobs -- rbfd_create, rbfd_greedy and rbfd_deform for each of n
 * jobs, the jobs side by side (one host thread and stream each, as
 * rbfd_greedy_deform_batch), with no return to the caller in between.
 * meshes[i] receives job i's mesh (NULL if its creation failed): the caller
 * reads it (levels, statistics) and destroys it.  Returns RBFD_ENOTCONV, after
 * deforming with the valid levels, if a greedy hit its control cap; otherwise
 * the worst status (the message names the job).
 */
int rbfd_run_jobs(const rbfd_job *jobs, int n, rbfd_mesh **meshes);

/* ------------------------------------------------------------- serving ---
 *
 * A request loop for deformation requests as icing time steps produce them:
 * each request is a new surface displacement on a registered mesh (2D or 3D,
 * any size).  Up to `slots` requests run at once, each on its own worker
 * thread and CUDA stream, so their GPU work overlaps; requests arriving
 * meanwhile wait in a FIFO queue and start as soon as a slot is free and the
 * device memory their mesh needs fits the budget (admission by footprint).
 * Each mesh keeps resident instances (sorted surface and volume, workspace)
 * on the device between time steps.  A request's result does not depend on
 * which other requests run beside it (up to the rounding of the growth
 * reductions, far below the stated tolerances).
 */
typedef struct rbfd_server rbfd_server;

typedef struct rbfd_server_options {
    int slots;                 /* requests in flight at most (default 4) */
    int precision;             /* rbfd_precision of every request (default RBFD_MIXED) */
    int64_t mem_budget_bytes;  /* device memory the resident instances may hold (0 = 80% of free memory) */
    int64_t max_queue;         /* queued requests at most; rbfd_submit returns RBFD_EBUSY beyond (default 4096) */
    int fuse_volume;           /* 1: the volume updates of requests whose greedy is done at the same time run
                                  fused in one work-list launch (rbfd_deform_worklist on the registered
                                  volumes; the same results bit for bit); 0 (default): each request's own
                                  launches, side by side -- measured lower latency on mixed-size streams */
} rbfd_server_options;

typedef struct rbfd_request {
    const double *dS;  /* [n_s][dim] host displacement of the registered surface; copied by rbfd_submit */
    float *out;        /* [n_v][dim] host buffer; written when the request completes, untouched before */
} rbfd_request;

typedef enum rbfd_request_state {
    RBFD_REQ_QUEUED = 0,
    RBFD_REQ_RUNNING = 1,
    RBFD_REQ_DONE = 2,   /* out holds the result (status RBFD_OK or RBFD_ENOTCONV) */
    RBFD_REQ_FAILED = 3,    /* rbfd_poll returns the error status */
    RBFD_REQ_CANCELLED = 4  /* removed from the queue by rbfd_cancel; out untouched (RBFD_ECANCELED) */
} rbfd_request_state;

void rbfd_server_options_default(rbfd_server_options *opt);

/* Start the worker threads on the current CUDA device. */
int rbfd_server_create(rbfd_server **out, const rbfd_server_options *opt);

/*
 * Register a mesh: surface points xyz_s [n_s][dim] (double), volume points
 * xyz_v [n_v][dim] with wall distances d_v [n_v] (float; NULL: computed on the
 * device when an instance is made), the greedy levels
 * (R [n_levels], eps) and the support distance rule (D, k) of rbfd_deform.
 * Host pointers; the server copies them.  *mesh_id names the mesh in rbfd_submit.
 */
int rbfd_server_add_mesh(rbfd_server *s, int dim, int64_t n_s, const double *xyz_s, int64_t n_v, const float *xyz_v,
                         const float *d_v, int n_levels, const double *R, double eps, double D, double k,
                         int *mesh_id);

/* Queue one request; *ticket identifies it.  RBFD_EBUSY if the queue is full. */
int rbfd_submit(rbfd_server *s, int mesh_id, const rbfd_request *req, uint64_t *ticket);

/* Non-blocking: *state = rbfd_request_state; returns the request's status once done. */
int rbfd_poll(rbfd_server *s, uint64_t ticket, int *state);

/* Block until the request is done or timeout_s passes (<= 0: no limit; RBFD_ETIMEOUT). */
int rbfd_wait(rbfd_server *s, uint64_t ticket, double timeout_s, int *state);

/*
 * Cancel a queued request: it leaves the queue, its out buffer is never
 * written, and rbfd_poll / rbfd_wait report RBFD_REQ_CANCELLED with status
 * RBFD_ECANCELED.  A request that already runs is not interrupted (its
 * kernels finish): RBFD_EBUSY; one that finished: RBFD_ESTATE; an unknown
 * ticket: RBFD_EINVAL.
 */
int rbfd_cancel(rbfd_server *s, uint64_t ticket);

/* Host-clock times of a finished request: queued, running, and submit-to-done. */
int rbfd_request_times(rbfd_server *s, uint64_t ticket, double *queue_ms, double *run_ms, double *total_ms);

/* Finish the running requests, drop the queued ones, free everything. */
int rbfd_server_destroy(rbfd_server *s);

/* Release every device and host resource of the mesh.  NULL is allowed. */
int rbfd_destroy(rbfd_mesh *m);

/* Message of the most recent failing call on this thread ("" if none). */
const char *rbfd_last_error(void);

/* Library version string. */
const char *rbfd_version(void);

#ifdef __cplusplus
}
#endif

#endif /* RBFD_H */
