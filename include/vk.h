/*
 * vk.h -- C ABI of libvk_nm: non-metric (k-nearest and Voronoi) neighbor
 * lists fused with the Vicsek alignment + position update, on one GB300.
 *
 * The method is the topological Vicsek model of arxiv 2103.10239 ("Non-metric
 * interaction rules in models of active matter", Sec. "Metric and
 * topological flocking models" and Sec. "Computational tools: Voronoi
 * neighbor lists"):
 *   Eq. (1)  Delta r_i = (v0 dt) n_i(t)
 *   Eq. (2)  n_i(t+dt) = N( eta xi_i^t + (1/m_i^t) sum_<ij> n_j(t) )
 * where the neighbors <ij> of particle i are either its k nearest particles
 * at any distance (not reciprocal) or its Voronoi neighbors (reciprocal).
 *
 * Conventions shared by every call
 *   - Positions are fixed-point grid coordinates: int32 pos_q in [0, L_q) per
 *     axis, real coordinate = pos_q * 2^-F.  The box is periodic with edge
 *     L_q <= 2^31 grid units (<= 2^30 for the 2D Voronoi rule, <= 2^23 for the
 *     3D one, whose exact int128 predicates need it).  Distances use the
 *     minimum image, differences mapped into (-L_q/2, L_q/2], and are compared
 *     as exact integer squared distances D.
 *   - kNN lists are ordered by (D, id) ascending (ties broken by the smaller
 *     particle id); self is excluded.  Voronoi lists hold the ids whose
 *     Voronoi cell shares an edge of positive length (2D) or a face of positive
 *     area (3D) with the particle's cell (Delaunay edges between cocircular or
 *     cospherical points are dropped), sorted by id.
 *   - Headings are FP32 unit vectors (the authoritative state).  In 2D the
 *     angle theta = atan2(n_y, n_x) in [0, 2pi) is also exported.
 *   - Noise: Philox4x32-10 keyed by the 64-bit seed, counter (particle id,
 *     step, replica, 0); u = (word0 >> 8) * 2^-24.  Angular noise (2D
 *     default): theta' = atan2(S) + eta (u - 1/2), S = sum of neighbor
 *     headings.  Vectorial noise (Eq. 2 literally): n' = N(eta xi + S/m).
 *   - Advection uses the heading before the update (Eq. 1): the grid step
 *     Delta_q = round-half-even(s * n_a) with s = fl32(v0*dt) * 2^F, exact;
 *     requires s <= 2^22.  Positions wrap modulo L_q.
 *
 * Memory and ownership
 *   - Every array argument may be a host or a device pointer (detected with
 *     cudaPointerGetAttributes).  The caller owns it; the library copies what
 *     it needs before the call returns (device copies are stream-ordered).
 *   - The library owns all device state of a vk_sim; vk_destroy frees it.
 *   - All device work runs on the stream given at init (NULL: the library
 *     creates its own non-blocking stream).  vk_step is asynchronous.
 *
 * Errors
 *   - Every call returns a vk_status and never aborts.  Device-side failures
 *     (capacity overflow, values out of range) latch a sticky status word on
 *     the device; it is returned by the next vk_sync or vk_get_* call.
 *     vk_last_error gives a message for the last failure.
 *   - Coincident particles are valid input under both rules in 2D.  The paper
 *     leaves the Voronoi cell of coincident points undefined; this library
 *     reads them as one Voronoi site: they are each other's neighbors and
 *     share the site's other neighbors.  (An earlier reading returned
 *     VK_ERR_DEGENERATE; coincident points do occur on the fixed-point grid
 *     in long runs, so an error would end the simulation.)  The 3D Voronoi
 *     rule reports coincident particles as VK_ERR_DEGENERATE (latched by the
 *     step, returned by the next synchronising call); there a collision on the
 *     2^-F grid needs ~2^(3F) / N^2 steps.
 */
#ifndef VK_NM_H
#define VK_NM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct vk_sim vk_sim; /* opaque; owned by the library */

typedef enum {
  VK_OK = 0,
  VK_ERR_ARG = 1,        /* invalid argument (null pointer, k >= N, bad rule ...) */
  VK_ERR_CUDA = 2,       /* a CUDA runtime call failed */
  VK_ERR_OOM = 3,        /* device allocation failed */
  VK_ERR_CAPACITY = 4,   /* an output buffer or an internal bound was too small */
  VK_ERR_RANGE = 5,      /* box / fixed-point range outside the supported limits */
  VK_ERR_DEGENERATE = 6, /* the tissue model met coincident particles or a zero-length Voronoi edge
                            (the 2D Voronoi rule itself treats coincident points as one site),
                            or the 3D Voronoi rule met coincident particles */
  VK_ERR_TIMEOUT = 7,    /* a bounded device wait gave up */
  VK_ERR_STATE = 8       /* call not valid in the current state */
} vk_status;

/* Neighbor rules (Sec. "Metric and topological flocking models"): the k
 * nearest particles at any distance (optionally only those inside a field of
 * view, 2D), the Voronoi neighbors (2D and 3D), or every particle within the
 * metric radius r0 (the original Vicsek rule, 2D and 3D). */
typedef enum { VK_RULE_KNN = 0, VK_RULE_VORONOI = 1, VK_RULE_METRIC = 2 } vk_rule;
typedef enum { VK_NOISE_ANGULAR = 0, VK_NOISE_VECTORIAL = 1 } vk_noise;
typedef enum { VK_SUM_PLAIN = 0, VK_SUM_COMPENSATED = 1, VK_SUM_FP64 = 2 } vk_sum_mode;
typedef enum { VK_HEADING_DIR = 0, VK_HEADING_THETA = 1 } vk_heading_kind;

/* Periodic box: dim (2 or 3), fractional bits F (0..30) and L_q per axis. */
typedef struct {
  int32_t dim;
  int32_t frac_bits;
  uint32_t box_q[3];
} vk_box;

/* Run parameters (Eq. 1 and Eq. 2).  eta is the noise strength: radians of
 * the uniform angular kick in angular mode, the weight of the random unit
 * vector in vectorial mode. */
typedef struct {
  int32_t rule;         /* vk_rule */
  int32_t k;            /* neighbors for VK_RULE_KNN, 1..32, k <= N-1 (unused by the others) */
  float v0;             /* self-propulsion speed (length units per time) */
  float dt;             /* time step */
  float eta;            /* noise strength (per-replica values override in batches) */
  uint64_t seed;        /* Philox key */
  int32_t noise;        /* vk_noise; 3D requires VK_NOISE_VECTORIAL */
  int32_t include_self; /* 1: add n_i(t) to the sum (default 0, Eq. 2 literally) */
  int32_t advect_new;   /* 1: advect with n_i(t+dt) instead of n_i(t) (default 0) */
  int32_t sum_mode;     /* vk_sum_mode for the heading sums (default compensated) */
  float cell_occupancy; /* target particles per coarse cell of the search grid at the mean
                           density; 0 = default (256 in 2D, 2 for Voronoi, 1.5 in 3D).
                           Dense coarse cells get sub-grids of about 2 particles per sub-cell.
                           Results never depend on it; only the speed does. */
  int32_t phi_capacity; /* order-parameter history kept per replica; 0 = 4096 steps */
  int32_t knn_search;   /* kNN search: 0 = radius first (default; a square in 2D, a cube in 3D),
                           1 = the ring walk only.  Results never depend on it; only the speed does. */
  float search_halo;    /* radius first: half-width of a particle's search square (cube), as a multiple
                           of its k-th neighbor distance at the previous step; 0 = default (1.15 in 2D, 1.3 in 3D).
                           Results never depend on it; only the speed does. */
  float search_halo_step; /* radius first: plus this multiple of the distance a particle moves
                           in one step (v0 dt); < 0 = default (0).  Speed only. */
  int32_t replica_offset; /* noise counter index of the first replica (default 0): replica r
                           draws with index replica_offset + r, so a single-replica sim with
                           replica_offset = r reproduces replica r of a batch exactly */
  float r0;             /* VK_RULE_METRIC: interaction radius in length units; the exact test is
                           D <= r0q^2 with r0q = rint(r0 * 2^F) grid units (round half to even,
                           per replica's F), r0q <= 2^31.  Self is not a neighbor (include_self
                           adds it).  The heading sum of the metric rule is exact: every
                           component is rounded to 2^-32 and summed in int64 (order-free, so
                           bit-identical run to run), then converted to FP64; sum_mode is not
                           used by this rule. */
  int32_t fov;          /* VK_RULE_KNN, 2D: 1 = only particles inside the field of view count
                           (default 0).  j is in view of i iff d.nq >= cq |d| for the minimum-
                           image offset d = r_j - r_i, with nq = rint(n_i(t) * 2^24) and
                           cq = rint(fov_cos * 2^24) (round half to even), decided exactly in
                           integers; d = 0 is in view.  A particle with fewer than k particles
                           in view aligns with those it has (its list is shorter). */
  float fov_cos;        /* cosine of the half-angle of the field of view, in [-1, 1]; -1 is the
                           full circle (the plain rule), 0 the half-plane ahead */
  int32_t voronoi_rebuild; /* VK_RULE_VORONOI, 2D: 0 (default) = start every cell from last step's
                           neighbors and re-check it (Sec. "Computational tools: Voronoi neighbor
                           lists": the old triangulation is kept where every circumcircle is still
                           empty and repaired where it is not); 1 = build every cell from scratch.
                           Results never depend on it; only the speed does. */
  int32_t voronoi3_kernel; /* VK_RULE_VORONOI, 3D: 0 (default) = one thread builds each cell (in
                           thread-local memory); 1 = one warp builds each cell (in shared memory:
                           the lanes test the vertices and solve new vertices in parallel).  Both
                           use the same exact predicates and give the same results; only the speed
                           differs. */
} vk_params;

/* Fills p with the defaults: kNN, k = 7, v0 = 0.5, dt = 1, eta = 0.3, seed = 1,
 * angular noise, compensated sums, default cell occupancy and history. */
void vk_default_params(vk_params* p);

/* Create a simulation of one periodic system (Sec. "Metric and topological
 * flocking models").  pos_q: n*dim int32, row-major (particle-major);
 * heading: n*dim FP32 unit vectors (VK_HEADING_DIR) or n angles in radians
 * (VK_HEADING_THETA, 2D only; converted on the device with sincosf).
 * The particle id is the row index.  The step counter starts at 0. */
vk_status vk_init(const int32_t* pos_q, const float* heading, int32_t heading_kind, int64_t n,
                  const vk_box* box, const vk_params* params, void* cuda_stream, vk_sim** out);

/* Create n_rep independent systems (replicas) that step together in one
 * launch per kernel.  Replica r has n_r[r] particles stored contiguously in
 * pos_q / heading after those of replicas 0..r-1, its own box boxes[r] and its
 * own noise strength eta_r[r] (NULL: params->eta for all).  Particle ids are
 * local to each replica (0..n_r-1); the replica index enters the noise
 * counter.  All replicas share the other parameters and the dimension. */
vk_status vk_batch_init(int32_t n_rep, const int64_t* n_r, const int32_t* pos_q,
                        const float* heading, int32_t heading_kind, const vk_box* boxes,
                        const float* eta_r, const vk_params* params, void* cuda_stream,
                        vk_sim** out);

/* Advance nsteps time steps of Alg. 1 (build the neighbor lists, align with
 * noise, advect).  Asynchronous on the sim's stream. */
vk_status vk_step(vk_sim* sim, int64_t nsteps);

/* Neighbor lists of the CURRENT positions of one replica, in id order:
 * offsets (n+1 int64, CSR) and ids (int32).  kNN rule: the k nearest other
 * particles at any distance, not reciprocal (Sec. "Metric and topological
 * flocking models"), row i ordered by (D, id); with a field of view, the k
 * nearest in view, so a row may be shorter than k.  Metric rule: every other
 * particle at exact squared distance <= r0q^2 (reciprocal), row i sorted by
 * id.  Voronoi rule: the particles
 * whose Voronoi cell shares an edge of positive length (2D) or a face of
 * positive area (3D) with i's, i.e. the Delaunay neighbors by the
 * empty-circumcircle (circumsphere) property (Sec. "Computational tools:
 * Voronoi neighbor lists"), row i sorted by id.  These are the lists
 * the next vk_step uses.  If ids_capacity is too small (or ids is NULL),
 * *nnz_needed receives the count and VK_ERR_CAPACITY is returned (VK_OK when
 * ids is NULL).  Synchronous. */
vk_status vk_get_neighbors(vk_sim* sim, int32_t replica, int64_t* offsets, int32_t* ids,
                           int64_t ids_capacity, int64_t* nnz_needed);

/* Polar order parameter phi(t) = |sum_i n_i(t)| / N of one replica after
 * each of the last *count steps (oldest first; at most phi_capacity and at
 * most max_values are written).  The paper does not define it: it is the
 * standard observable of the Vicsek model whose dynamics Eq. (1)-(2) state.
 * Sums are FP32 compensated per block and FP64 across blocks.  Synchronous. */
vk_status vk_get_order_parameter(vk_sim* sim, int32_t replica, double* phi, int64_t max_values,
                                 int64_t* count);

/* Current state of one replica in id order: the positions r_i of Eq. (1)
 * as pos_q (n*dim int32), the headings n_i of Eq. (2) as dir (n*dim FP32),
 * theta = atan2(n_y, n_x) in [0, 2pi) (n FP32, 2D; may be NULL), and the
 * step counter t.  Any output may be NULL.  Synchronous. */
vk_status vk_get_state(vk_sim* sim, int32_t replica, int32_t* pos_q, float* dir, float* theta,
                       int64_t* step);

/* Overwrite the state (r_i, n_i) of Eq. (1)-(2) of one replica (id order,
 * same layout as vk_get_state) and, if step >= 0, the step counter of the
 * whole simulation (teacher forcing, checkpoint resume).  Positions outside
 * [0, L_q) give VK_ERR_RANGE and non-finite headings VK_ERR_ARG.  The
 * per-particle search state (2D kNN: last step's k-th distance; Voronoi: last
 * step's neighbors) stays attached to each id, so a state read and written
 * back steps at full speed; it only guides the search, so results are the
 * same for any state.  Synchronous. */
vk_status vk_set_state(vk_sim* sim, int32_t replica, const int32_t* pos_q, const float* dir,
                       int64_t step);

/* Voronoi tissue model (Sec. "Geometric models of dense tissue"; Sec.
 * "Voronoi model forces") for the CURRENT positions of one replica (2D, any
 * rule): every particle generates its Voronoi cell, of area A_i and
 * perimeter P_i; E = sum_i KA (A_i - A0)^2 + KP (P_i - P0)^2 (Eq. vmEnergy)
 * and F_i = -dE/dr_i, by the chain rule through the Voronoi vertices.  All in
 * length units (one grid unit = 2^-F) and FP64, by id: area and perimeter n
 * doubles, force 2n doubles ((x, y) per particle), energy one double; each
 * may be NULL (not computed or not written), host or device memory.  The
 * cells are built with the exact predicates of the Voronoi rule; the FP64
 * geometry follows from the exact integer offsets.  Needs n >= 3, box edges
 * <= 2^30, distinct particles and no Voronoi edge of zero length (four
 * cocircular particles), else VK_ERR_DEGENERATE; cells of more than 32
 * edges give VK_ERR_CAPACITY.  Synchronous. */
vk_status vk_get_tissue(vk_sim* sim, int32_t replica, double KA, double KP, double A0, double P0,
                        double* area, double* perimeter, double* force, double* energy);

/* Wait for the sim's stream and return the sticky device status. */
vk_status vk_sync(vk_sim* sim);

/* Message for the last failure of this sim (or of the last init when sim is
 * NULL); never NULL. */
const char* vk_last_error(const vk_sim* sim);
const char* vk_status_string(int32_t status);

void vk_destroy(vk_sim* sim);

/* Capture vk_step's launches in CUDA graphs of `steps_per_graph` steps (0
 * turns graphs off; default 0).  Each replay advances a device-side step
 * counter, so a graph is reused for any number of steps. */
vk_status vk_set_graph_steps(vk_sim* sim, int32_t steps_per_graph);

/* Tracing: when enabled (1), vk_step launches kernels directly (no graph) and
 * brackets every kernel phase with CUDA events on the sim's stream; level 2
 * also collects the search counters of vk_get_search_stats.
 * vk_get_profile returns, per phase, the summed event time in ms and the
 * launch count since profiling was enabled, plus the phase names.  Phases:
 * 0 search_update (the search + update kernel of every particle), 1 build
 * (grid scans), 2 scatter, 3 load_sort (init / set_state), 4 export
 * (vk_get_neighbors), 5 search_deferred (2D kNN radius first: the particles
 * the first kernel listed for larger squares or the walk). */
vk_status vk_set_profiling(vk_sim* sim, int32_t enable);
vk_status vk_get_profile(vk_sim* sim, double* ms, int64_t* launches, int32_t max_phases,
                         int32_t* n_phases);
const char* vk_phase_name(int32_t phase);

/* Search counters of the neighbor search while tracing was on (level 2):
 * mean candidates examined per particle update, mean contiguous slot runs
 * read per particle update (2D kNN radius first: mean squares scanned), the
 * largest candidate count of one particle, and the fraction of particle
 * updates whose own coarse cell was split into sub-cells (2D kNN radius
 * first: that fell back to the per-particle walk).  Any output may be NULL. */
vk_status vk_get_search_stats(vk_sim* sim, double* mean_candidates, double* mean_runs,
                              int64_t* max_candidates, double* split_fraction);

/* Raw totals of the search counters collected while tracing at level 2, in
 * this order: 0 candidates examined (summed over particle updates), 1 slot
 * runs (walk) or squares scanned (radius first), 2 largest candidate count
 * of one particle update, 3 particle updates, 4 updates whose own coarse
 * cell was split (walk) or that fell back to the walk (radius first); radius
 * first only, over the particles it served or handed on: 5 squares scanned,
 * 6 slot runs, 7 candidates, 8 coarse cells visited, 9 hits merged, and the
 * particles the step kernel deferred because 10 the square was too wide for
 * the box or listed too many slot runs (these go straight to the walk),
 * 11 the square held fewer than k hits (a larger square follows), 12 two
 * candidates were at the same distance (walk), 13 (unused, 0).  Writes
 * min(max_values, 14) values; *n (may be NULL) receives 14. */
vk_status vk_get_search_counters(vk_sim* sim, int64_t* values, int32_t max_values, int32_t* n);

/* Sizes chosen at init: total particles, replicas, cells of the search grid. */
typedef struct {
  int64_t n_total;
  int32_t n_rep;
  int32_t dim;
  int64_t n_cells;
  int64_t step;
  int32_t kernels_per_step;
  int32_t rule;
  int32_t k;
} vk_info;
vk_status vk_get_info(vk_sim* sim, vk_info* out);

/* Re-pick the search grid (particles per cell) by timing `trial_steps` steps
 * for each candidate occupancy on a scratch copy of the state; the state and
 * the step counter are restored afterwards.  Results never depend on the
 * grid; only the speed does.  On return *best holds the chosen occupancy.
 * The choice is remembered for the process, keyed by (dimension, rule, k,
 * floor(log2(mean particles per replica))): later sims of the same kind
 * whose params leave cell_occupancy at 0 start from it. */
vk_status vk_autotune(vk_sim* sim, const float* candidates, int32_t n_candidates,
                      int32_t trial_steps, float* best);

/* Forget every occupancy vk_autotune has chosen in this process (see
 * vk_autotune: later sims then start from the built-in defaults again). */
void vk_autotune_forget(void);

/* ------------------------------------------------------------------------
 * Allocation-free kNN lists.  (The paper has no counterpart: this is a
 * deployment entry point.)
 *
 * Some callers cannot allocate GPU memory at the moment they need neighbor
 * lists: code that is recording a CUDA graph (cudaMalloc/cudaFree are not
 * allowed during stream capture), real-time loops that cannot afford the
 * blocking and device synchronisation of cudaMalloc/cudaFree, and hosts that
 * manage the whole device memory budget themselves.  This call allocates
 * nothing: the caller passes the input and output arrays, and every
 * intermediate array lives in one fixed static scratch array of about 6 MiB
 * compiled into the library, which each GPU that loads the library holds
 * until the process exits.
 *
 * Computes, for n <= VK_NOALLOC_MAX_N points of a periodic 2D box, the same
 * lists as vk_init + vk_get_neighbors with VK_RULE_KNN: out_ids[i*k + j] is
 * the j-th nearest other point of point i, ordered by (exact squared
 * minimum-image distance, id).
 *   pos_q    device pointer, n*2 int32 in [0, L_q) (points outside are
 *            wrapped into the box and reported through dev_status)
 *   out_ids  device pointer, n*k int32
 *   dev_status  optional pointer (device or host-pinned) receiving 0, or
 *            VK_ERR_RANGE when a point lay outside the box
 * Asynchronous on cuda_stream (NULL: the legacy default stream).  Returns
 * VK_ERR_ARG for n > VK_NOALLOC_MAX_N, n < 2, k outside [1, min(32, n-1)] or
 * a non-2D box; these checks, and the check that the intermediates fit the
 * scratch (VK_ERR_CAPACITY, which no valid n reaches), run on the host before
 * any device work.  An error left pending by earlier CUDA work of the caller
 * gives VK_ERR_CUDA and stays pending.  The first call on each device looks
 * up the device address of the scratch array and keeps it for the life of
 * the process, so make that first call outside stream capture, and do not
 * call this entry point again after cudaDeviceReset (the kept address is
 * then stale).  All calls share the one scratch array and leave their
 * intermediates in it: calls that can overlap on the GPU (different streams,
 * different host threads) race and must be serialised by the caller. */
#define VK_NOALLOC_MAX_N 65536
vk_status vk_knn_lists_noalloc(const int32_t* pos_q, int64_t n, const vk_box* box, int32_t k,
                               int32_t* out_ids, int32_t* dev_status, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* VK_NM_H */
