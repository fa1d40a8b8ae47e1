// vk_capi.cu -- host runtime behind the C ABI declared in include/vk.h.
//
// One vk_sim owns the device state of one or more replicas, a stream, the
// optional CUDA graph of a multi-step sequence and the tracing events.  A
// time step (Alg. 1 of the paper: build the neighbor relation, then update) is
//   search+update kernel (kNN or Voronoi; writes the next state and the
//   histogram of the new coarse cells) -> build of the two-level grid (coarse
//   scan with sub-grid sides, sub-cell histogram, sub-cell scan) -> scatter
//   into (coarse, sub-cell) order (also advances the device step counter).
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/vk.h"
#include "vk_internal.cuh"
#include "vk_voronoi3_api.cuh"

using namespace vk;

namespace {

constexpr int kPhases = 6;
constexpr int kCounters = 14;  // search counters (tracing level 2)
const char* kPhaseNames[kPhases] = {"search_update", "build", "scatter", "load_sort", "export", "search_deferred"};

thread_local std::string g_init_error;

}  // namespace

struct vk_sim {
  vk_params prm;
  int dim = 2;
  int n_rep = 0;
  int64_t n_total = 0;
  int64_t n_cells = 0;
  // staging of vk_get_state / vk_set_state, allocated at the first call
  int32_t* st_pos = nullptr;
  float* st_dir = nullptr;
  float* st_theta = nullptr;
  // tissue model scratch, allocated at the first vk_get_tissue call: per-slot
  // cells and the outputs by id (area n, perimeter n, force 2n, energy 1)
  TissueScratch tis{};
  double* tis_out = nullptr;
  int64_t cells_cap = 0;
  std::vector<Rep> reps_h;
  std::vector<BlockTask> tasks_h;
  std::vector<uint32_t> bounds_h;  // cell boundary tables of all replicas
  std::vector<int64_t> n_r;
  std::vector<vk_box> boxes;
  std::vector<float> eta_r;
  Rep* reps_d = nullptr;
  BlockTask* tasks_d = nullptr;
  Buffers b{};
  Geometry g{};
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int64_t step = 0;
  int64_t phi_first = 0;
  int phi_cap = 4096;
  float occupancy = 0.f;
  // graphs
  int graph_steps = 0;
  cudaGraphExec_t gexec = nullptr;
  int gexec_steps = 0;
  // tracing
  bool prof = false;
  bool prof_counters = false;  // search counters (tracing level 2)
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev[kPhases];
  double prof_ms[kPhases] = {0, 0, 0, 0, 0, 0};
  int64_t prof_launches[kPhases] = {0, 0, 0, 0, 0, 0};
  unsigned long long* d_stats = nullptr;  // search counters, collected while tracing
  std::string err;
};

namespace {

vk_status fail(vk_sim* s, vk_status st, const std::string& msg) {
  if (s) s->err = msg;
  else g_init_error = msg;
  return st;
}

vk_status cuda_fail(vk_sim* s, cudaError_t e, const char* where) {
  cudaGetLastError();
  return fail(s, e == cudaErrorMemoryAllocation ? VK_ERR_OOM : VK_ERR_CUDA,
              std::string(where) + ": " + cudaGetErrorString(e));
}

#define VK_CUDA(sim, call)                                  \
  do {                                                      \
    cudaError_t e_ = (call);                                \
    if (e_ != cudaSuccess) return cuda_fail(sim, e_, #call); \
  } while (0)

template <class T>
cudaError_t dalloc(T** p, size_t count) {
  return cudaMalloc((void**)p, sizeof(T) * (count ? count : 1));
}

// the field of view's half-angle cosine in 2^-24 units (round half to even),
// or the full circle
int32_t fov_cq(const vk_params& p) {
  if (p.rule != VK_RULE_KNN || !p.fov) return kViewAll;
  return (int32_t)std::nearbyint((double)p.fov_cos * 16777216.0);
}

StepParams step_params(const vk_sim* s) {
  StepParams P;
  P.k = s->prm.k;
  P.noise = s->prm.noise;
  P.include_self = s->prm.include_self;
  P.advect_new = s->prm.advect_new;
  P.sum_mode = s->prm.sum_mode;
  P.seed_lo = (uint32_t)s->prm.seed;
  P.seed_hi = (uint32_t)(s->prm.seed >> 32);
  P.n_rep = s->n_rep;
  P.phi_cap = s->phi_cap;
  P.knn_search = s->prm.knn_search;
  // measured defaults: squares 1.15 x the last k-th distance (2D), cubes 1.3 x (3D)
  P.halo_alpha = s->prm.search_halo > 0.f ? s->prm.search_halo : (s->dim == 3 ? 1.3f : 1.15f);
  P.halo_beta = s->prm.search_halo_step >= 0.f ? s->prm.search_halo_step : 0.f;
  P.fov_cq = fov_cq(s->prm);
  P.stats = (s->prof && s->prof_counters) ? s->d_stats : nullptr;
  return P;
}

// Occupancies chosen by vk_autotune, keyed by (dimension, rule, k, size
// bucket = floor(log2(mean particles per replica))): a later sim of the same
// kind whose caller leaves cell_occupancy at 0 starts from the tuned value.
// Process-wide; speed only.
using TuneKey = std::tuple<int, int, int, int>;
std::map<TuneKey, float> g_tuned;
std::mutex g_tuned_mu;

TuneKey tune_key(const vk_params& p, int dim, int64_t n_total, int n_rep) {
  const int64_t mean = std::max<int64_t>(1, n_total / std::max(1, n_rep));
  int bucket = 0;
  while ((int64_t)1 << (bucket + 1) <= mean) ++bucket;
  return TuneKey(dim, p.rule, p.rule == VK_RULE_KNN ? p.k : 0, bucket);
}

float default_occupancy(const vk_params& p, int dim, int64_t n_total, int n_rep) {
  if (p.cell_occupancy > 0.f) return p.cell_occupancy;
  {
    std::lock_guard<std::mutex> lock(g_tuned_mu);
    auto it = g_tuned.find(tune_key(p, dim, n_total, n_rep));
    if (it != g_tuned.end()) return it->second;
  }
  // Voronoi: 2 particles per cell in 2D; 1 in 3D (a sweep of 1, 1.5, 2 and 3
  // at N = 2^18 uniform: 83, 89, 96, 109 ms per step)
  if (p.rule == VK_RULE_VORONOI) return dim == 2 ? 2.0f : 1.0f;
  // 2D kNN and metric: coarse cells of a few hundred particles split into
  // sub-grids (the radius-first search measured fastest at 256 on uniform
  // and clustered flocks); 3D: cells of about 1.5 particles (the cube search)
  return dim == 2 ? 256.0f : 1.5f;
}

// per-replica search grid for a target occupancy; fills nc, c0 and the cell
// boundary tables (bnd[b] = ceil(b * L / nc), the first coordinate of cell b)
void plan_cells(vk_sim* s, float occ) {
  int64_t c0 = 0;
  s->bounds_h.clear();
  for (int r = 0; r < s->n_rep; ++r) {
    Rep& R = s->reps_h[r];
    double vol = 1.0;
    for (int a = 0; a < s->dim; ++a) vol *= (double)R.L[a];
    const double side = std::pow((double)occ * vol / (double)std::max<int64_t>(1, R.n), 1.0 / s->dim);
    int64_t cells = 1;
    for (int a = 0; a < 3; ++a) {
      if (a >= s->dim) {
        R.nc[a] = 1;
        continue;
      }
      double ncd = std::floor((double)R.L[a] / side);
      ncd = std::max(1.0, std::min(ncd, std::min((double)R.L[a], 65536.0)));
      R.nc[a] = (int32_t)ncd;
      cells *= R.nc[a];
    }
    for (int a = 0; a < 3; ++a) {
      R.bnd[a] = (int32_t)s->bounds_h.size();
      R.inv_w[a] = (float)R.nc[a] / (float)R.L[a];
      for (int64_t b = 0; b <= R.nc[a]; ++b)
        s->bounds_h.push_back((uint32_t)((b * (int64_t)R.L[a] + R.nc[a] - 1) / R.nc[a]));
    }
    R.c0 = c0;
    c0 += cells;
  }
  s->n_cells = c0;
}

vk_status record_begin(vk_sim* s, int phase, cudaEvent_t* e0) {
  if (!s->prof) return VK_OK;
  VK_CUDA(s, cudaEventCreate(e0));
  VK_CUDA(s, cudaEventRecord(*e0, s->stream));
  (void)phase;
  return VK_OK;
}

vk_status record_end(vk_sim* s, int phase, cudaEvent_t e0, int launches) {
  if (!s->prof) return VK_OK;
  cudaEvent_t e1;
  VK_CUDA(s, cudaEventCreate(&e1));
  VK_CUDA(s, cudaEventRecord(e1, s->stream));
  s->ev[phase].push_back({e0, e1});
  s->prof_launches[phase] += launches;
  return VK_OK;
}

int64_t sub_cells_bound(const vk_sim* s) { return s->n_cells + s->n_total / kSubTarget + 1; }

vk_status ensure_cells_capacity(vk_sim* s) {
  if (s->n_cells <= s->cells_cap) return VK_OK;
  void* old[] = {s->b.counts, s->b.offsets, s->b.bsum, s->b.sub_s, s->b.sub_base,
                 s->b.sub_count, s->b.sub_off, s->b.bsum2};
  for (void* p : old)
    if (p) cudaFree(p);
  s->b.counts = s->b.offsets = s->b.bsum = s->b.sub_base = s->b.sub_count = s->b.sub_off = s->b.bsum2 = nullptr;
  s->b.sub_s = nullptr;
  const int64_t cap = s->n_cells;
  const int64_t scap = sub_cells_bound(s);
  VK_CUDA(s, dalloc(&s->b.counts, cap));
  VK_CUDA(s, dalloc(&s->b.offsets, cap + 1));
  VK_CUDA(s, dalloc(&s->b.bsum, 2 * ((cap + 2047) / 2048 + 1)));
  VK_CUDA(s, dalloc(&s->b.sub_s, cap));
  VK_CUDA(s, dalloc(&s->b.sub_base, cap + 1));
  VK_CUDA(s, dalloc(&s->b.sub_count, scap));
  VK_CUDA(s, dalloc(&s->b.sub_off, scap + 1));
  VK_CUDA(s, dalloc(&s->b.bsum2, (scap + 2047) / 2048 + 1));
  VK_CUDA(s, cudaMemsetAsync(s->b.counts, 0, sizeof(uint32_t) * cap, s->stream));
  VK_CUDA(s, cudaMemsetAsync(s->b.sub_count, 0, sizeof(uint32_t) * scap, s->stream));
  s->cells_cap = cap;
  return VK_OK;
}

void refresh_geometry(vk_sim* s) {
  s->g.dim = s->dim;
  s->g.rule = s->prm.rule;
  s->g.n_rep = s->n_rep;
  s->g.n_total = s->n_total;
  s->g.n_cells = s->n_cells;
  s->g.n_sub_max = sub_cells_bound(s);
  s->g.n_tasks = (int)s->tasks_h.size();
  s->g.reps = s->reps_d;
  s->g.tasks = s->tasks_d;
}

vk_status upload_reps(vk_sim* s) {
  VK_CUDA(s, cudaMemcpyAsync(s->reps_d, s->reps_h.data(), sizeof(Rep) * s->n_rep, cudaMemcpyHostToDevice,
                             s->stream));
  if (s->b.bounds) cudaFree(s->b.bounds);
  s->b.bounds = nullptr;
  VK_CUDA(s, dalloc(&s->b.bounds, s->bounds_h.size()));
  VK_CUDA(s, cudaMemcpyAsync(s->b.bounds, s->bounds_h.data(), sizeof(uint32_t) * s->bounds_h.size(),
                             cudaMemcpyHostToDevice, s->stream));
  VK_CUDA(s, cudaStreamSynchronize(s->stream));
  refresh_geometry(s);
  return VK_OK;
}

// U (+ ranks from a fresh histogram) -> S, sorted by the current grid
// keep_search_state: the search hints (already moved into U's order) and the
// Voronoi seeds (kept by id) follow their particles through the re-sort;
// otherwise they are cleared.  Results never depend on them, only the speed.
vk_status sort_from_U(vk_sim* s, bool keep_search_state = false) {
  cudaEvent_t e0 = nullptr;
  vk_status st = record_begin(s, 3, &e0);
  if (st) return st;
  if (!keep_search_state) {
    if (s->b.U_hint) VK_CUDA(s, cudaMemsetAsync(s->b.U_hint, 0, sizeof(float) * (size_t)s->n_total, s->stream));
    if (s->b.vor_seed_n)
      VK_CUDA(s, cudaMemsetAsync(s->b.vor_seed_n, 0, sizeof(int32_t) * (size_t)s->n_total, s->stream));
  }
  VK_CUDA(s, launch_count(s->g, s->b, s->stream));
  VK_CUDA(s, launch_build(s->g, s->b, s->stream));
  VK_CUDA(s, launch_scatter(s->g, s->b, step_params(s), 0, s->stream));
  return record_end(s, 3, e0, 9);
}

vk_status read_status(vk_sim* s) {
  int32_t h = 0;
  VK_CUDA(s, cudaMemcpyAsync(&h, s->b.d_status, sizeof(int32_t), cudaMemcpyDeviceToHost, s->stream));
  VK_CUDA(s, cudaStreamSynchronize(s->stream));
  if (h == 0) return VK_OK;
  const char* what = h == VK_ERR_CAPACITY     ? "device: capacity exceeded (Voronoi polygon or buffer)"
                     : h == VK_ERR_DEGENERATE ? "device: coincident particles or a zero-length Voronoi edge"
                     : h == VK_ERR_RANGE      ? "device: value outside the supported range"
                                              : "device: invalid input value";
  return fail(s, (vk_status)h, what);
}

vk_status clear_phi(vk_sim* s) {
  VK_CUDA(s, cudaMemsetAsync(s->b.phi_acc, 0, sizeof(PhiAcc) * 3 * (size_t)s->phi_cap * s->n_rep, s->stream));
  s->phi_first = s->step;
  return VK_OK;
}

// kernels of the search+update phase: for 2D kNN the radius-first kernel,
// the deferred-particle kernel and the walk-list kernel (one kernel with the
// walk only); one for 3D kNN and for the metric rule; the Voronoi kernel and
// its overflow kernel
int search_launches(const vk_sim* s) {
  if (s->prm.rule == VK_RULE_KNN) return (s->dim == 2 && s->prm.knn_search == 0) ? 3 : 1;
  if (s->prm.rule == VK_RULE_METRIC) return 1;
  return 2;
}

vk_status enqueue_step(vk_sim* s) {
  const StepParams P = step_params(s);
  cudaEvent_t e0 = nullptr;
  vk_status st = record_begin(s, 0, &e0);
  if (st) return st;
  if (s->prm.rule == VK_RULE_KNN && s->dim == 2) VK_CUDA(s, launch_knn2_step(s->g, s->b, P, s->stream));
  else if (s->prm.rule == VK_RULE_KNN) VK_CUDA(s, launch_knn_step(s->g, s->b, P, s->stream));
  else if (s->prm.rule == VK_RULE_METRIC) VK_CUDA(s, launch_metric_step(s->g, s->b, P, s->stream));
  else if (s->dim == 2) VK_CUDA(s, launch_voronoi_step(s->g, s->b, P, s->stream));
  else VK_CUDA(s, launch_voronoi3_step(s->g, s->b, P, s->prm.voronoi3_kernel, s->stream));
  const int deferred_launches = (s->prm.rule == VK_RULE_KNN && s->dim == 2 && s->prm.knn_search == 0) ? 2 : 0;
  if ((st = record_end(s, 0, e0, search_launches(s) - deferred_launches))) return st;
  if (deferred_launches) {
    if ((st = record_begin(s, 5, &e0))) return st;
    VK_CUDA(s, launch_knn2_finish(s->g, s->b, P, s->stream));
    if ((st = record_end(s, 5, e0, deferred_launches))) return st;
  }
  if ((st = record_begin(s, 1, &e0))) return st;
  VK_CUDA(s, launch_build(s->g, s->b, s->stream));
  if ((st = record_end(s, 1, e0, 7))) return st;
  if ((st = record_begin(s, 2, &e0))) return st;
  VK_CUDA(s, launch_scatter(s->g, s->b, P, 1, s->stream));
  return record_end(s, 2, e0, 1);
}

void drop_graph(vk_sim* s) {
  if (s->gexec) cudaGraphExecDestroy(s->gexec);
  s->gexec = nullptr;
  s->gexec_steps = 0;
}

vk_status capture_graph(vk_sim* s, int steps) {
  drop_graph(s);
  cudaGraph_t graph = nullptr;
  VK_CUDA(s, cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal));
  vk_status st = VK_OK;
  for (int i = 0; i < steps && st == VK_OK; ++i) st = enqueue_step(s);
  cudaError_t e = cudaStreamEndCapture(s->stream, &graph);
  if (st != VK_OK) {
    if (graph) cudaGraphDestroy(graph);
    return st;
  }
  if (e != cudaSuccess) return cuda_fail(s, e, "cudaStreamEndCapture");
  e = cudaGraphInstantiate(&s->gexec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return cuda_fail(s, e, "cudaGraphInstantiate");
  s->gexec_steps = steps;
  return VK_OK;
}

bool valid_params(const vk_params* p, int dim, std::string* why) {
  if (p->rule != VK_RULE_KNN && p->rule != VK_RULE_VORONOI && p->rule != VK_RULE_METRIC)
    return *why = "unknown rule", false;
  if (p->rule == VK_RULE_KNN && (p->k < 1 || p->k > kMaxK)) return *why = "k must be in [1, 32]", false;
  if (p->noise != VK_NOISE_ANGULAR && p->noise != VK_NOISE_VECTORIAL) return *why = "unknown noise", false;
  if (dim == 3 && p->noise != VK_NOISE_VECTORIAL) return *why = "3D needs vectorial noise", false;
  if (p->sum_mode < 0 || p->sum_mode > 2) return *why = "unknown sum mode", false;
  if (!std::isfinite(p->v0) || !std::isfinite(p->dt) || !std::isfinite(p->eta))
    return *why = "v0, dt and eta must be finite", false;
  if (p->phi_capacity < 0 || p->phi_capacity == 1) return *why = "phi_capacity must be 0 or >= 2", false;
  if (p->knn_search != 0 && p->knn_search != 1) return *why = "knn_search must be 0 or 1", false;
  if (!(p->search_halo >= 0.f) || !std::isfinite(p->search_halo)) return *why = "search_halo must be >= 0", false;
  if (!std::isfinite(p->search_halo_step)) return *why = "search_halo_step must be finite", false;
  if (p->replica_offset < 0) return *why = "replica_offset must be >= 0", false;
  if (p->rule == VK_RULE_METRIC && !(p->r0 >= 0.f && std::isfinite(p->r0)))
    return *why = "r0 must be finite and >= 0", false;
  if (p->fov != 0 && p->fov != 1) return *why = "fov must be 0 or 1", false;
  if (p->voronoi_rebuild != 0 && p->voronoi_rebuild != 1) return *why = "voronoi_rebuild must be 0 or 1", false;
  if (p->voronoi3_kernel != 0 && p->voronoi3_kernel != 1) return *why = "voronoi3_kernel must be 0 or 1", false;
  if (p->fov && (p->rule != VK_RULE_KNN || dim != 2)) return *why = "a field of view needs the 2D kNN rule", false;
  if (p->fov && !(p->fov_cos >= -1.f && p->fov_cos <= 1.f)) return *why = "fov_cos must be in [-1, 1]", false;
  return true;
}

vk_status build_sim(int32_t n_rep, const int64_t* n_r, const int32_t* pos_q, const float* heading,
                    int32_t heading_kind, const vk_box* boxes, const float* eta_r, const vk_params* params,
                    void* cuda_stream, vk_sim** out) {
  if (!out) return fail(nullptr, VK_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (n_rep < 1 || !n_r || !pos_q || !heading || !boxes || !params)
    return fail(nullptr, VK_ERR_ARG, "null argument or n_rep < 1");
  const int dim = boxes[0].dim;
  if (dim != 2 && dim != 3) return fail(nullptr, VK_ERR_ARG, "dim must be 2 or 3");
  if (heading_kind != VK_HEADING_DIR && heading_kind != VK_HEADING_THETA)
    return fail(nullptr, VK_ERR_ARG, "unknown heading kind");
  if (heading_kind == VK_HEADING_THETA && dim != 2) return fail(nullptr, VK_ERR_ARG, "theta input is 2D only");
  std::string why;
  if (!valid_params(params, dim, &why)) return fail(nullptr, VK_ERR_ARG, why);
  int64_t total = 0;
  for (int r = 0; r < n_rep; ++r) {
    const vk_box& B = boxes[r];
    if (B.dim != dim) return fail(nullptr, VK_ERR_ARG, "all replicas must share the dimension");
    if (B.frac_bits < 0 || B.frac_bits > 30) return fail(nullptr, VK_ERR_RANGE, "frac_bits must be in [0, 30]");
    for (int a = 0; a < dim; ++a) {
      const uint64_t lim = params->rule != VK_RULE_VORONOI ? (1ull << 31) : (dim == 2 ? (1ull << 30) : (1ull << 23));
      if (B.box_q[a] < 1 || B.box_q[a] > lim)
        return fail(nullptr, VK_ERR_RANGE,
                    "box edge outside [1, 2^31] (2^30 for the 2D Voronoi rule, 2^23 for the 3D one)");
    }
    const float vdt = params->v0 * params->dt;
    const double sgrid = std::ldexp((double)vdt, B.frac_bits);
    if (!(std::fabs(sgrid) <= 4194304.0))
      return fail(nullptr, VK_ERR_RANGE, "v0*dt*2^F must not exceed 2^22 grid units");
    if (n_r[r] < 1) return fail(nullptr, VK_ERR_ARG, "every replica needs at least one particle");
    if (params->rule == VK_RULE_KNN && params->k > n_r[r] - 1)
      return fail(nullptr, VK_ERR_ARG, "k must be smaller than the number of particles");
    if (params->rule == VK_RULE_METRIC && !(std::nearbyint(std::ldexp((double)params->r0, B.frac_bits)) <= 2147483648.0))
      return fail(nullptr, VK_ERR_RANGE, "r0 * 2^F must not exceed 2^31 grid units");
    total += n_r[r];
  }
  if (total >= (1ll << 31) - 1) return fail(nullptr, VK_ERR_RANGE, "too many particles (>= 2^31)");

  vk_sim* s = new vk_sim();
  s->prm = *params;
  s->dim = dim;
  s->n_rep = n_rep;
  s->n_total = total;
  s->phi_cap = params->phi_capacity > 0 ? params->phi_capacity : 4096;
  s->n_r.assign(n_r, n_r + n_rep);
  s->boxes.assign(boxes, boxes + n_rep);
  s->eta_r.resize(n_rep);
  int64_t p0 = 0;
  s->reps_h.resize(n_rep);
  for (int r = 0; r < n_rep; ++r) {
    Rep& R = s->reps_h[r];
    std::memset(&R, 0, sizeof(R));
    R.p0 = p0;
    R.n = (int32_t)n_r[r];
    for (int a = 0; a < 3; ++a) R.L[a] = a < dim ? boxes[r].box_q[a] : 1u;
    R.eta = eta_r ? eta_r[r] : params->eta;
    s->eta_r[r] = R.eta;
    const float vdt = params->v0 * params->dt;
    R.s = (float)std::ldexp((double)vdt, boxes[r].frac_bits);
    R.replica = (uint32_t)(r + params->replica_offset);
    R.r0q = params->rule == VK_RULE_METRIC
                ? (uint32_t)std::nearbyint(std::ldexp((double)params->r0, boxes[r].frac_bits))
                : 0u;
    for (int first = 0; first < R.n; first += kBlock) s->tasks_h.push_back({r, first});
    p0 += n_r[r];
  }
  s->occupancy = default_occupancy(*params, dim, total, n_rep);
  plan_cells(s, s->occupancy);

  if (cuda_stream) {
    s->stream = (cudaStream_t)cuda_stream;
  } else {
    cudaError_t e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      vk_status st = cuda_fail(nullptr, e, "cudaStreamCreate");
      delete s;
      return st;
    }
    s->own_stream = true;
  }
  // let work queued on the legacy default stream (e.g. by PyTorch) finish first
  cudaStreamSynchronize(cudaStreamLegacy);

  auto bail = [&](vk_status st) {
    g_init_error = s->err;
    vk_destroy(s);
    return st;
  };
  const size_t pv = dim == 2 ? sizeof(int2) : sizeof(int4);
  const size_t fv = dim == 2 ? sizeof(float2) : sizeof(float4);
  cudaError_t e = cudaSuccess;
  const size_t N = (size_t)total;
  if ((e = cudaMalloc(&s->b.S_pos, pv * N)) || (e = cudaMalloc(&s->b.S_dir, fv * N)) ||
      (e = dalloc(&s->b.S_id, N)) || (e = cudaMalloc(&s->b.U_pos, pv * N)) || (e = cudaMalloc(&s->b.U_dir, fv * N)) ||
      (e = dalloc(&s->b.U_id, N)) || (e = dalloc(&s->b.U_rank, N)) ||
      (e = dalloc(&s->b.phi_acc, 3 * (size_t)s->phi_cap * n_rep)) || (e = dalloc(&s->b.d_step, 1)) ||
      (e = dalloc(&s->b.d_status, 1)) || (e = dalloc(&s->reps_d, n_rep)) ||
      (e = dalloc(&s->b.ovf_list, 2 * N)) || (e = dalloc(&s->b.ovf_count, 2)) ||
      (e = dalloc(&s->d_stats, kCounters)) ||
      (e = dalloc(&s->tasks_d, s->tasks_h.size())))
    return bail(cuda_fail(s, e, "cudaMalloc"));
  if (params->rule == VK_RULE_KNN) {
    if ((e = dalloc(&s->b.S_hint, N)) || (e = dalloc(&s->b.U_hint, N)) || (dim == 2 && (e = prepare_knn2())))
      return bail(cuda_fail(s, e, "kNN search buffers"));
  }
  if (params->rule == VK_RULE_VORONOI && dim == 2 && !params->voronoi_rebuild) {
    if ((e = dalloc(&s->b.vor_seed, N * kVorSeed)) || (e = dalloc(&s->b.vor_seed_n, N)) ||
        (e = dalloc(&s->b.slot_of, N)))
      return bail(cuda_fail(s, e, "Voronoi seed buffers"));
  }
  if (ensure_cells_capacity(s)) return bail(VK_ERR_OOM);
  if ((e = cudaMemsetAsync(s->b.d_step, 0, sizeof(int64_t), s->stream)) ||
      (e = cudaMemsetAsync(s->b.ovf_count, 0, 2 * sizeof(int32_t), s->stream)) ||
      (e = cudaMemsetAsync(s->b.d_status, 0, sizeof(int32_t), s->stream)) ||
      (e = cudaMemcpyAsync(s->tasks_d, s->tasks_h.data(), sizeof(BlockTask) * s->tasks_h.size(),
                           cudaMemcpyHostToDevice, s->stream)))
    return bail(cuda_fail(s, e, "init copies"));
  if (upload_reps(s)) return bail(VK_ERR_CUDA);
  if (clear_phi(s)) return bail(VK_ERR_CUDA);

  // stage the caller's arrays (host or device) and load them into U
  int32_t* pos_d = nullptr;
  float* head_d = nullptr;
  const size_t nh = heading_kind == VK_HEADING_THETA ? N : N * dim;
  if ((e = dalloc(&pos_d, N * dim)) || (e = dalloc(&head_d, nh))) {
    cudaFree(pos_d);
    return bail(cuda_fail(s, e, "cudaMalloc staging"));
  }
  vk_status st = VK_OK;
  if ((e = cudaMemcpyAsync(pos_d, pos_q, sizeof(int32_t) * N * dim, cudaMemcpyDefault, s->stream)) ||
      (e = cudaMemcpyAsync(head_d, heading, sizeof(float) * nh, cudaMemcpyDefault, s->stream)) ||
      (e = launch_load(s->g, s->b, pos_d, head_d, heading_kind, s->stream)))
    st = cuda_fail(s, e, "load");
  if (st == VK_OK) st = read_status(s);
  cudaStreamSynchronize(s->stream);
  cudaFree(pos_d);
  cudaFree(head_d);
  if (st != VK_OK) return bail(st);
  if ((st = sort_from_U(s)) || (st = read_status(s))) return bail(st);
  *out = s;
  return VK_OK;
}

}  // namespace

extern "C" {

void vk_default_params(vk_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->rule = VK_RULE_KNN;
  p->k = 7;
  p->v0 = 0.5f;
  p->dt = 1.0f;
  p->eta = 0.3f;
  p->seed = 1;
  p->noise = VK_NOISE_ANGULAR;
  p->include_self = 0;
  p->advect_new = 0;
  p->sum_mode = VK_SUM_COMPENSATED;
  p->cell_occupancy = 0.f;
  p->phi_capacity = 0;
  p->knn_search = 0;
  p->search_halo = 0.f;
  p->search_halo_step = -1.f;
  p->replica_offset = 0;
  p->r0 = 1.0f;
  p->fov = 0;
  p->fov_cos = -1.0f;
  p->voronoi3_kernel = 0;
}

vk_status vk_init(const int32_t* pos_q, const float* heading, int32_t heading_kind, int64_t n,
                  const vk_box* box, const vk_params* params, void* cuda_stream, vk_sim** out) {
  return build_sim(1, &n, pos_q, heading, heading_kind, box, nullptr, params, cuda_stream, out);
}

vk_status vk_batch_init(int32_t n_rep, const int64_t* n_r, const int32_t* pos_q, const float* heading,
                        int32_t heading_kind, const vk_box* boxes, const float* eta_r, const vk_params* params,
                        void* cuda_stream, vk_sim** out) {
  return build_sim(n_rep, n_r, pos_q, heading, heading_kind, boxes, eta_r, params, cuda_stream, out);
}

vk_status vk_step(vk_sim* s, int64_t nsteps) {
  if (!s || nsteps < 0) return fail(s, VK_ERR_ARG, "bad arguments to vk_step");
  int64_t left = nsteps;
  if (s->graph_steps > 0 && !s->prof && left >= s->graph_steps) {
    if (!s->gexec || s->gexec_steps != s->graph_steps) {
      vk_status st = capture_graph(s, s->graph_steps);
      if (st) return st;
    }
    while (left >= s->gexec_steps) {
      VK_CUDA(s, cudaGraphLaunch(s->gexec, s->stream));
      left -= s->gexec_steps;
    }
  }
  for (; left > 0; --left) {
    vk_status st = enqueue_step(s);
    if (st) return st;
  }
  s->step += nsteps;
  return VK_OK;
}

vk_status vk_sync(vk_sim* s) {
  if (!s) return fail(s, VK_ERR_ARG, "sim is NULL");
  VK_CUDA(s, cudaStreamSynchronize(s->stream));
  return read_status(s);
}

vk_status vk_get_neighbors(vk_sim* s, int32_t replica, int64_t* offsets, int32_t* ids, int64_t ids_capacity,
                           int64_t* nnz_needed) {
  if (!s || replica < 0 || replica >= s->n_rep || !offsets) return fail(s, VK_ERR_ARG, "bad arguments");
  cudaStreamSynchronize(cudaStreamLegacy);
  const Rep& R = s->reps_h[replica];
  const int64_t n = R.n;
  cudaEvent_t e0 = nullptr;
  vk_status st = record_begin(s, 4, &e0);
  if (st) return st;
  std::vector<int64_t> off_h(n + 1);
  std::vector<int32_t> ids_h;
  if (s->prm.rule == VK_RULE_KNN) {
    const int k = s->prm.k;
    int32_t* out_d = nullptr;
    VK_CUDA(s, dalloc(&out_d, (size_t)n * k));
    cudaError_t e = s->dim == 2 ? launch_knn2_export(s->g, s->b, k, replica, (int)n, out_d, s->stream,
                                                     step_params(s))
                                : launch_knn_export(s->g, s->b, k, replica, (int)n, out_d, s->stream);
    if (e == cudaSuccess) {
      ids_h.resize((size_t)n * k);
      e = cudaMemcpyAsync(ids_h.data(), out_d, sizeof(int32_t) * n * k, cudaMemcpyDeviceToHost, s->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    cudaFree(out_d);
    if (e != cudaSuccess) return cuda_fail(s, e, "knn export");
    for (int64_t i = 0; i <= n; ++i) off_h[i] = i * k;
    if (s->prm.fov) {
      // rows with fewer than k particles in view end in -1: drop those entries
      int64_t w = 0;
      for (int64_t i = 0; i < n; ++i) {
        off_h[i] = w;
        for (int j = 0; j < k; ++j)
          if (ids_h[(size_t)(i * k + j)] >= 0) ids_h[(size_t)w++] = ids_h[(size_t)(i * k + j)];
      }
      off_h[n] = w;
      ids_h.resize((size_t)w);
    }
  } else {
    // pass 0: degrees by id; pass 1: ids at the CSR offsets
    const bool metric = s->prm.rule == VK_RULE_METRIC;
    auto exporter = [&](int pass, int32_t* deg, const int64_t* off, int32_t* ids_out) {
      return metric ? launch_metric_export(s->g, s->b, replica, (int)n, pass, deg, off, ids_out, s->stream)
          : s->dim == 2 ? launch_voronoi_export(s->g, s->b, replica, (int)n, pass, deg, off, ids_out, s->stream)
                        : launch_voronoi3_export(s->g, s->b, replica, (int)n, pass, deg, off, ids_out, s->stream);
    };
    int32_t* deg_d = nullptr;
    int64_t* off_d = nullptr;
    int32_t* ids_d = nullptr;
    VK_CUDA(s, dalloc(&deg_d, n));
    std::vector<int32_t> deg(n);
    cudaError_t e = exporter(0, deg_d, nullptr, nullptr);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(deg.data(), deg_d, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e == cudaSuccess) {
      off_h[0] = 0;
      for (int64_t i = 0; i < n; ++i) off_h[i + 1] = off_h[i] + deg[i];
      ids_h.resize(off_h[n]);
      e = dalloc(&off_d, n + 1);
    }
    if (e == cudaSuccess) e = dalloc(&ids_d, std::max<int64_t>(1, off_h[n]));
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(off_d, off_h.data(), sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess) e = exporter(1, deg_d, off_d, ids_d);
    if (e == cudaSuccess && off_h[n] > 0)
      e = cudaMemcpyAsync(ids_h.data(), ids_d, sizeof(int32_t) * off_h[n], cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    cudaFree(deg_d);
    cudaFree(off_d);
    cudaFree(ids_d);
    if (e != cudaSuccess) return cuda_fail(s, e, metric ? "metric export" : "voronoi export");
  }
  if ((st = record_end(s, 4, e0, 1))) return st;
  if ((st = read_status(s))) return st;
  const int64_t nnz = (int64_t)ids_h.size();
  if (nnz_needed) *nnz_needed = nnz;
  VK_CUDA(s, cudaMemcpy(offsets, off_h.data(), sizeof(int64_t) * (n + 1), cudaMemcpyDefault));
  if (!ids) return VK_OK;
  if (ids_capacity < nnz) return fail(s, VK_ERR_CAPACITY, "ids_capacity is smaller than the neighbor count");
  if (nnz) VK_CUDA(s, cudaMemcpy(ids, ids_h.data(), sizeof(int32_t) * nnz, cudaMemcpyDefault));
  return VK_OK;
}

vk_status vk_get_tissue(vk_sim* s, int32_t replica, double KA, double KP, double A0, double P0, double* area,
                        double* perimeter, double* force, double* energy) {
  if (!s || replica < 0 || replica >= s->n_rep) return fail(s, VK_ERR_ARG, "bad arguments");
  if (s->dim != 2) return fail(s, VK_ERR_ARG, "the tissue model is 2D");
  if (!std::isfinite(KA) || !std::isfinite(KP) || !std::isfinite(A0) || !std::isfinite(P0))
    return fail(s, VK_ERR_ARG, "KA, KP, A0 and P0 must be finite");
  const Rep& R = s->reps_h[replica];
  const int64_t n = R.n;
  if (n < 3) return fail(s, VK_ERR_ARG, "the tissue model needs at least 3 particles");
  for (int a = 0; a < 2; ++a)
    if (s->boxes[replica].box_q[a] > (1u << 30)) return fail(s, VK_ERR_RANGE, "box edge above 2^30");
  cudaStreamSynchronize(cudaStreamLegacy);
  cudaEvent_t e0 = nullptr;
  vk_status st = record_begin(s, 4, &e0);
  if (st) return st;
  // per-slot scratch over the whole state (slots of this replica are p0..p0+n-1),
  // kept for later calls
  const size_t N = (size_t)s->n_total;
  TissueScratch& w = s->tis;
  cudaError_t e = cudaSuccess;
  if (!s->tis_out) {
    const bool ok = !((e = dalloc(&w.nb_n, N)) || (e = dalloc(&w.nb_slot, N * kTissueCap)) ||
                      (e = dalloc(&w.nb_off, N * kTissueCap)) || (e = dalloc(&w.area, N)) ||
                      (e = dalloc(&w.perim, N)) || (e = dalloc(&s->tis_out, 4 * N + 1)));
    if (!ok) {
      void* part[] = {w.nb_n, w.nb_slot, w.nb_off, w.area, w.perim, s->tis_out};
      for (void* p : part)
        if (p) cudaFree(p);
      w = TissueScratch{};
      s->tis_out = nullptr;
      return cuda_fail(s, e, "tissue scratch");
    }
  }
  double* area_d = area ? s->tis_out : nullptr;
  double* perim_d = perimeter ? s->tis_out + N : nullptr;
  double* force_d = force ? s->tis_out + 2 * N : nullptr;
  double* energy_d = energy ? s->tis_out + 4 * N : nullptr;
  const double unit = std::ldexp(1.0, -s->boxes[replica].frac_bits);
  e = launch_tissue(s->g, s->b, replica, (int)n, KA, KP, A0, P0, unit, w, area_d, perim_d, force_d, energy_d,
                    s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e == cudaSuccess) st = record_end(s, 4, e0, energy ? 3 : 2);
  if (e == cudaSuccess && st == VK_OK) st = read_status(s);
  if (e == cudaSuccess && st == VK_OK) {
    if (area) e = cudaMemcpy(area, area_d, sizeof(double) * n, cudaMemcpyDefault);
    if (e == cudaSuccess && perimeter) e = cudaMemcpy(perimeter, perim_d, sizeof(double) * n, cudaMemcpyDefault);
    if (e == cudaSuccess && force) e = cudaMemcpy(force, force_d, sizeof(double) * 2 * n, cudaMemcpyDefault);
    if (e == cudaSuccess && energy) e = cudaMemcpy(energy, energy_d, sizeof(double), cudaMemcpyDefault);
  }
  if (e != cudaSuccess) return cuda_fail(s, e, "tissue model");
  return st;
}

vk_status vk_get_order_parameter(vk_sim* s, int32_t replica, double* phi, int64_t max_values, int64_t* count) {
  if (!s || replica < 0 || replica >= s->n_rep || (!phi && max_values > 0)) return fail(s, VK_ERR_ARG, "bad arguments");
  VK_CUDA(s, cudaStreamSynchronize(s->stream));
  // the slot of the upcoming step is already cleared: cap-1 values are kept
  const int64_t have = std::min<int64_t>(s->step - s->phi_first, s->phi_cap - 1);
  const int64_t nout = std::min<int64_t>(have, std::max<int64_t>(0, max_values));
  if (count) *count = nout;
  if (nout == 0) return VK_OK;
  std::vector<long long> ring(3 * (size_t)s->phi_cap * s->n_rep);
  VK_CUDA(s, cudaMemcpy(ring.data(), s->b.phi_acc, sizeof(long long) * ring.size(), cudaMemcpyDeviceToHost));
  std::vector<double> vals(nout);
  const double n = (double)s->reps_h[replica].n;
  for (int64_t i = 0; i < nout; ++i) {
    const int64_t t = s->step - nout + i;  // phi after the update from step t to t+1
    const long long* a = ring.data() + ((size_t)(t % s->phi_cap) * s->n_rep + replica) * 3;
    // fixed-point sums (2^-32 units) -> FP64
    const double x = std::ldexp((double)a[0], -32), y = std::ldexp((double)a[1], -32),
                 z = std::ldexp((double)a[2], -32);
    vals[i] = std::sqrt(x * x + y * y + z * z) / n;
  }
  VK_CUDA(s, cudaMemcpy(phi, vals.data(), sizeof(double) * nout, cudaMemcpyDefault));
  return VK_OK;
}

// device staging for the largest replica (id-ordered arrays), kept for the
// sim's lifetime so that state transfers allocate nothing per call
vk_status ensure_staging(vk_sim* s) {
  if (s->st_pos) return VK_OK;
  int64_t nmax = 0;
  for (const Rep& R : s->reps_h) nmax = std::max<int64_t>(nmax, R.n);
  const size_t n = (size_t)std::max<int64_t>(nmax, 1), d = (size_t)s->dim;
  cudaError_t e = dalloc(&s->st_pos, n * d);
  if (e == cudaSuccess) e = dalloc(&s->st_dir, n * d);
  if (e == cudaSuccess) e = dalloc(&s->st_theta, n);
  if (e != cudaSuccess) return cuda_fail(s, e, "state staging");
  return VK_OK;
}

vk_status vk_get_state(vk_sim* s, int32_t replica, int32_t* pos_q, float* dir, float* theta, int64_t* step) {
  if (!s || replica < 0 || replica >= s->n_rep) return fail(s, VK_ERR_ARG, "bad arguments");
  cudaStreamSynchronize(cudaStreamLegacy);
  if (vk_status st = ensure_staging(s)) return st;
  const Rep& R = s->reps_h[replica];
  const size_t n = (size_t)R.n, d = (size_t)s->dim;
  int32_t* pd = s->st_pos;
  float* dd = s->st_dir;
  float* td = s->st_theta;
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess)
    e = launch_export_state(s->g, s->b, replica, R.p0, R.n, pd, dd, s->dim == 2 ? td : nullptr, s->stream);
  if (e == cudaSuccess && pos_q) e = cudaMemcpyAsync(pos_q, pd, sizeof(int32_t) * n * d, cudaMemcpyDefault, s->stream);
  if (e == cudaSuccess && dir) e = cudaMemcpyAsync(dir, dd, sizeof(float) * n * d, cudaMemcpyDefault, s->stream);
  if (e == cudaSuccess && theta && s->dim == 2)
    e = cudaMemcpyAsync(theta, td, sizeof(float) * n, cudaMemcpyDefault, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_fail(s, e, "get_state");
  if (step) *step = s->step;
  return read_status(s);
}

vk_status vk_set_state(vk_sim* s, int32_t replica, const int32_t* pos_q, const float* dir, int64_t step) {
  if (!s || replica < 0 || replica >= s->n_rep || !pos_q || !dir) return fail(s, VK_ERR_ARG, "bad arguments");
  cudaStreamSynchronize(cudaStreamLegacy);
  const Rep& R = s->reps_h[replica];
  const size_t n = (size_t)R.n, d = (size_t)s->dim, N = (size_t)s->n_total;
  const size_t pv = s->dim == 2 ? sizeof(int2) : sizeof(int4);
  const size_t fv = s->dim == 2 ? sizeof(float2) : sizeof(float4);
  if (vk_status st = ensure_staging(s)) return st;
  int32_t* pd = s->st_pos;
  float* dd = s->st_dir;
  cudaError_t e = cudaMemcpyAsync(pd, pos_q, sizeof(int32_t) * n * d, cudaMemcpyDefault, s->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dd, dir, sizeof(float) * n * d, cudaMemcpyDefault, s->stream);
  // the search state follows the particles (by id): a state read with
  // vk_get_state and set again steps as fast as it would have
  if (e == cudaSuccess && s->b.S_hint && s->n_rep > 1)
    e = cudaMemcpyAsync(s->b.U_hint, s->b.S_hint, sizeof(float) * N, cudaMemcpyDeviceToDevice, s->stream);
  if (e == cudaSuccess) e = launch_hints_by_id(s->b, R.p0, R.n, s->stream);
  // every other replica keeps its state: S -> U, then overwrite this replica
  if (s->n_rep > 1) {
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->b.U_pos, s->b.S_pos, pv * N, cudaMemcpyDeviceToDevice, s->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->b.U_dir, s->b.S_dir, fv * N, cudaMemcpyDeviceToDevice, s->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(s->b.U_id, s->b.S_id, sizeof(int32_t) * N, cudaMemcpyDeviceToDevice, s->stream);
  }
  // the import flags positions outside the box (and wraps them into it, so
  // that the sort below stays in bounds) and non-finite headings; the status
  // is read once at the end
  if (e == cudaSuccess) e = launch_import_state(s->g, s->b, replica, R.p0, R.n, pd, dd, s->stream);
  if (e != cudaSuccess) return cuda_fail(s, e, "set_state");
  vk_status st;
  if ((st = sort_from_U(s, true))) return st;
  if (step >= 0) {
    s->step = step;
    VK_CUDA(s, cudaMemcpyAsync(s->b.d_step, &s->step, sizeof(int64_t), cudaMemcpyHostToDevice, s->stream));
    if ((st = clear_phi(s))) return st;
  }
  VK_CUDA(s, cudaStreamSynchronize(s->stream));
  return read_status(s);
}

const char* vk_last_error(const vk_sim* s) {
  if (!s) return g_init_error.c_str();
  return s->err.c_str();
}

const char* vk_status_string(int32_t st) {
  switch (st) {
    case VK_OK: return "ok";
    case VK_ERR_ARG: return "invalid argument";
    case VK_ERR_CUDA: return "CUDA error";
    case VK_ERR_OOM: return "out of device memory";
    case VK_ERR_CAPACITY: return "capacity exceeded";
    case VK_ERR_RANGE: return "value out of range";
    case VK_ERR_DEGENERATE: return "degenerate input (coincident points)";
    case VK_ERR_TIMEOUT: return "device wait timed out";
    case VK_ERR_STATE: return "invalid state";
    default: return "unknown status";
  }
}

void vk_destroy(vk_sim* s) {
  if (!s) return;
  if (s->stream) cudaStreamSynchronize(s->stream);
  drop_graph(s);
  for (int p = 0; p < kPhases; ++p)
    for (auto& pr : s->ev[p]) {
      cudaEventDestroy(pr.first);
      cudaEventDestroy(pr.second);
    }
  void* bufs[] = {s->b.S_pos, s->b.S_dir, s->b.S_id, s->b.U_pos, s->b.U_dir, s->b.U_id, s->b.U_rank,
                  s->b.counts, s->b.offsets, s->b.bsum, s->b.phi_acc, s->b.d_step, s->b.d_status,
                  s->b.ovf_list, s->b.ovf_count, s->reps_d, s->tasks_d, s->b.sub_s, s->b.sub_base,
                  s->b.sub_count, s->b.sub_off, s->b.bsum2, s->d_stats, s->b.bounds,
                  s->st_pos, s->st_dir, s->st_theta, s->b.S_hint, s->b.U_hint, s->b.vor_seed,
                  s->b.vor_seed_n, s->b.slot_of, s->tis.nb_n, s->tis.nb_slot, s->tis.nb_off, s->tis.area,
                  s->tis.perim, s->tis_out};
  for (void* p : bufs)
    if (p) cudaFree(p);
  if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
  delete s;
}

vk_status vk_set_graph_steps(vk_sim* s, int32_t steps_per_graph) {
  if (!s || steps_per_graph < 0) return fail(s, VK_ERR_ARG, "bad arguments");
  s->graph_steps = steps_per_graph;
  drop_graph(s);
  return VK_OK;
}

vk_status vk_set_profiling(vk_sim* s, int32_t enable) {
  if (!s) return fail(s, VK_ERR_ARG, "sim is NULL");
  s->prof = enable != 0;
  s->prof_counters = enable >= 2;
  drop_graph(s);  // the captured launches carry the tracing switch
  if (s->prof) {
    cudaStreamSynchronize(s->stream);
    VK_CUDA(s, cudaMemsetAsync(s->d_stats, 0, kCounters * sizeof(unsigned long long), s->stream));
    for (int p = 0; p < kPhases; ++p) {
      for (auto& pr : s->ev[p]) {
        cudaEventDestroy(pr.first);
        cudaEventDestroy(pr.second);
      }
      s->ev[p].clear();
      s->prof_ms[p] = 0.0;
      s->prof_launches[p] = 0;
    }
  }
  return VK_OK;
}

vk_status vk_get_profile(vk_sim* s, double* ms, int64_t* launches, int32_t max_phases, int32_t* n_phases) {
  if (!s) return fail(s, VK_ERR_ARG, "sim is NULL");
  VK_CUDA(s, cudaStreamSynchronize(s->stream));
  for (int p = 0; p < kPhases; ++p) {
    for (auto& pr : s->ev[p]) {
      float t = 0.f;
      VK_CUDA(s, cudaEventElapsedTime(&t, pr.first, pr.second));
      s->prof_ms[p] += t;
      cudaEventDestroy(pr.first);
      cudaEventDestroy(pr.second);
    }
    s->ev[p].clear();
  }
  const int np = std::min<int>(kPhases, std::max<int>(0, max_phases));
  for (int p = 0; p < np; ++p) {
    if (ms) ms[p] = s->prof_ms[p];
    if (launches) launches[p] = s->prof_launches[p];
  }
  if (n_phases) *n_phases = kPhases;
  return VK_OK;
}

vk_status vk_get_search_stats(vk_sim* s, double* mean_candidates, double* mean_runs, int64_t* max_candidates,
                              double* split_fraction) {
  if (!s) return fail(s, VK_ERR_ARG, "sim is NULL");
  unsigned long long h[6] = {0, 0, 0, 0, 0, 0};
  VK_CUDA(s, cudaMemcpyAsync(h, s->d_stats, sizeof(h), cudaMemcpyDeviceToHost, s->stream));
  VK_CUDA(s, cudaStreamSynchronize(s->stream));
  const double n = h[3] ? (double)h[3] : 1.0;
  if (mean_candidates) *mean_candidates = (double)h[0] / n;
  if (mean_runs) *mean_runs = (double)h[1] / n;
  if (max_candidates) *max_candidates = (int64_t)h[2];
  if (split_fraction) *split_fraction = h[3] ? (double)h[4] / (double)h[3] : 0.0;
  return VK_OK;
}

vk_status vk_get_search_counters(vk_sim* s, int64_t* values, int32_t max_values, int32_t* n) {
  if (!s || (max_values > 0 && !values)) return fail(s, VK_ERR_ARG, "bad arguments");
  unsigned long long h[kCounters] = {};
  VK_CUDA(s, cudaMemcpyAsync(h, s->d_stats, sizeof(h), cudaMemcpyDeviceToHost, s->stream));
  VK_CUDA(s, cudaStreamSynchronize(s->stream));
  for (int i = 0; i < std::min<int>(kCounters, std::max<int>(0, max_values)); ++i) values[i] = (int64_t)h[i];
  if (n) *n = kCounters;
  return VK_OK;
}

const char* vk_phase_name(int32_t phase) {
  if (phase < 0 || phase >= kPhases) return "";
  return kPhaseNames[phase];
}

vk_status vk_get_info(vk_sim* s, vk_info* out) {
  if (!s || !out) return fail(s, VK_ERR_ARG, "bad arguments");
  out->n_total = s->n_total;
  out->n_rep = s->n_rep;
  out->dim = s->dim;
  out->n_cells = s->n_cells;
  out->step = s->step;
  out->kernels_per_step = 8 + search_launches(s);
  out->rule = s->prm.rule;
  out->k = s->prm.k;
  return VK_OK;
}

vk_status vk_autotune(vk_sim* s, const float* candidates, int32_t n_candidates, int32_t trial_steps, float* best) {
  if (!s || !candidates || n_candidates < 1 || trial_steps < 1) return fail(s, VK_ERR_ARG, "bad arguments");
  for (int i = 0; i < n_candidates; ++i)
    if (!(candidates[i] > 0.f)) return fail(s, VK_ERR_ARG, "occupancy candidates must be positive");
  const size_t N = (size_t)s->n_total;
  const size_t pv = s->dim == 2 ? sizeof(int2) : sizeof(int4);
  const size_t fv = s->dim == 2 ? sizeof(float2) : sizeof(float4);
  // snapshot of the sorted state, the step and the order-parameter ring
  void* snap_pos = nullptr;
  void* snap_dir = nullptr;
  int32_t* snap_id = nullptr;
  PhiAcc* snap_phi = nullptr;
  const size_t phin = 3 * (size_t)s->phi_cap * s->n_rep;
  cudaError_t e = cudaMalloc(&snap_pos, pv * N);
  if (e == cudaSuccess) e = cudaMalloc(&snap_dir, fv * N);
  if (e == cudaSuccess) e = dalloc(&snap_id, N);
  if (e == cudaSuccess) e = dalloc(&snap_phi, phin);
  auto cleanup = [&]() {
    cudaFree(snap_pos);
    cudaFree(snap_dir);
    cudaFree(snap_id);
    cudaFree(snap_phi);
  };
  if (e != cudaSuccess) {
    cleanup();
    return cuda_fail(s, e, "autotune snapshot");
  }
  e = cudaMemcpyAsync(snap_pos, s->b.S_pos, pv * N, cudaMemcpyDeviceToDevice, s->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(snap_dir, s->b.S_dir, fv * N, cudaMemcpyDeviceToDevice, s->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(snap_id, s->b.S_id, sizeof(int32_t) * N, cudaMemcpyDeviceToDevice, s->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(snap_phi, s->b.phi_acc, sizeof(PhiAcc) * phin, cudaMemcpyDeviceToDevice, s->stream);
  const int64_t step0 = s->step, phi_first0 = s->phi_first;
  const bool prof0 = s->prof;
  s->prof = false;
  drop_graph(s);
  auto restore_and_sort = [&](float occ) -> vk_status {
    plan_cells(s, occ);
    vk_status st = ensure_cells_capacity(s);
    if (st) return st;
    if ((st = upload_reps(s))) return st;
    VK_CUDA(s, cudaMemcpyAsync(s->b.U_pos, snap_pos, pv * N, cudaMemcpyDeviceToDevice, s->stream));
    VK_CUDA(s, cudaMemcpyAsync(s->b.U_dir, snap_dir, fv * N, cudaMemcpyDeviceToDevice, s->stream));
    VK_CUDA(s, cudaMemcpyAsync(s->b.U_id, snap_id, sizeof(int32_t) * N, cudaMemcpyDeviceToDevice, s->stream));
    VK_CUDA(s, cudaMemcpyAsync(s->b.d_step, &step0, sizeof(int64_t), cudaMemcpyHostToDevice, s->stream));
    VK_CUDA(s, cudaMemcpyAsync(s->b.phi_acc, snap_phi, sizeof(PhiAcc) * phin, cudaMemcpyDeviceToDevice, s->stream));
    if ((st = sort_from_U(s))) return st;
    VK_CUDA(s, cudaStreamSynchronize(s->stream));
    s->step = step0;
    s->phi_first = phi_first0;
    return VK_OK;
  };
  vk_status st = e == cudaSuccess ? VK_OK : cuda_fail(s, e, "autotune snapshot copies");
  float best_occ = s->occupancy;
  float best_ms = 3.0e38f;
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  if (st == VK_OK && (cudaEventCreate(&t0) != cudaSuccess || cudaEventCreate(&t1) != cudaSuccess))
    st = fail(s, VK_ERR_CUDA, "cudaEventCreate");
  for (int i = 0; i < n_candidates && st == VK_OK; ++i) {
    if ((st = restore_and_sort(candidates[i]))) break;
    if ((st = enqueue_step(s))) break;  // warm-up
    cudaEventRecord(t0, s->stream);
    for (int j = 0; j < trial_steps && st == VK_OK; ++j) st = enqueue_step(s);
    cudaEventRecord(t1, s->stream);
    if (cudaEventSynchronize(t1) != cudaSuccess) st = fail(s, VK_ERR_CUDA, "autotune timing");
    float ms = 0.f;
    cudaEventElapsedTime(&ms, t0, t1);
    if (st == VK_OK && (st = read_status(s)) == VK_OK && ms < best_ms) {
      best_ms = ms;
      best_occ = candidates[i];
    }
  }
  if (t0) cudaEventDestroy(t0);
  if (t1) cudaEventDestroy(t1);
  vk_status st2 = restore_and_sort(best_occ);
  cleanup();
  s->prof = prof0;
  if (st) return st;
  if (st2) return st2;
  s->occupancy = best_occ;
  if (best) *best = best_occ;
  {
    std::lock_guard<std::mutex> lock(g_tuned_mu);
    g_tuned[tune_key(s->prm, s->dim, s->n_total, s->n_rep)] = best_occ;
  }
  return read_status(s);
}

void vk_autotune_forget(void) {
  std::lock_guard<std::mutex> lock(g_tuned_mu);
  g_tuned.clear();
}

}  // extern "C"
