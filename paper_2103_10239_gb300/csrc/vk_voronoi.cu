// vk_voronoi.cu -- Voronoi-neighbor rule (Sec. "Computational tools: Voronoi
// neighbor lists": the Voronoi cell is the region closer to a particle than to
// any other; Voronoi and Delaunay neighbors are dual, and the relation is
// reciprocal) fused with the Vicsek update of Eq. (1) and Eq. (2).
//
// Instead of a global (serial) triangulation, every particle builds its own
// Voronoi cell by half-plane clipping, which is embarrassingly parallel:
//   * the cell starts as the square bounded by the particle's own periodic
//     images (+-L_x, 0), (0, +-L_y);
//   * candidates arrive ring by ring from the cell grid; each one clips the
//     convex polygon by its bisector.  The polygon is a cyclic list of the
//     sites that define its edges; a vertex is the circumcenter of the particle
//     (at the origin) and two consecutive sites.  "Vertex beyond the bisector
//     of m" is exactly incircle(0, a, b, m) > 0, i.e. 2 m.V > |m|^2: decided
//     from an FP32 estimate of V with a rigorous error bound, else by an FP32
//     filter of the incircle determinant, else exactly in int128;
//   * a site can still cut the cell only inside the union of the disks
//     through the particle centred at the vertices (the disk of V holds the
//     points closer to V than the particle is); its bounding box, the
//     relevance box, only shrinks.  The walk skips rows and cells that miss
//     it and stops once the scanned block holds it;
//   * a cell that outgrows 32 edges or needs more than kHeavy candidates
//     (a particle bordering a void) is finished by the overflow kernel, one
//     warp per cell: the lanes test 32 candidates at a time against the
//     current cell and one lane applies the few that cut it;
//   * neighbors are the sites of edges with positive length (an edge between
//     two coincident vertices, i.e. four cocircular points, is dropped);
//   * coincident particles form one site (see Poly).
// Exact predicates need |relative coordinates| < 1.5 * 2^30, hence L_q <= 2^30.
#include "vk_voronoi.cuh"

namespace vk {

namespace {

// the Vicsek update of one particle from its finished cell
template <int CAP>
__device__ __forceinline__ void voronoi_update(const Rep& R, const StepParams& Pm, int64_t step, int64_t s,
                                               const Poly<CAP>& P, const int32_t* pi, const float* ni,
                                               int32_t id, const float2* __restrict__ S_dir,
                                               int2* __restrict__ U_pos, float2* __restrict__ U_dir,
                                               int32_t* __restrict__ U_id, uint32_t* __restrict__ counts,
                                               float* nnew, int32_t* __restrict__ seed_out,
                                               int32_t* __restrict__ seed_n_out, bool heavy_next,
                                               uint32_t seen) {
  int32_t nid[CAP + Poly<CAP>::TW], nslot[CAP + Poly<CAP>::TW];
  const int cnt = voronoi_neighbors(P, id, nid, nslot);
  if (seed_out) {
    // the next step's seeds (any subset of sites would do)
    const int ns = min(cnt, kVorSeed);
    for (int j = 0; j < ns; ++j) seed_out[j] = nid[j];
    *seed_n_out = ns | (heavy_next ? kSeedHeavy : 0) | (cost_bucket(seen) << kSeedCostShift);
  }
  HeadSum<2> H;
  H.init();
  if (Pm.include_self) H.add(ni, Pm.sum_mode);
  for (int j = 0; j < cnt; ++j) {
    const float2 d = S_dir[nslot[j]];
    const float v[2] = {d.x, d.y};
    H.add(v, Pm.sum_mode);
  }
  int32_t pout[3] = {0, 0, 0};
  align_advect<2>(R, Pm, (uint32_t)step, id, ni, H, cnt + (Pm.include_self ? 1 : 0), pi, pout, nnew);
  U_pos[s] = make_int2(pout[0], pout[1]);
  U_dir[s] = make_float2(nnew[0], nnew[1]);
  U_id[s] = id;
  atomicAdd(counts + linear_cell<2>(R, pout), 1u);
}

// The visiting order of the main kernel.  Each particle carries the cost
// bucket of its last build in its seed word; the particles of every replica
// are grouped by bucket (stably: sorted order inside a bucket), so that a
// warp's lanes build cells of similar cost and the few expensive cells
// share warps instead of holding back 31 cheap ones each.  Three passes:
// bucket counts per block task, offsets per replica (one warp per replica,
// one lane per bucket), and the stable scatter.
__device__ __forceinline__ int order_bucket(const Rep& R, int li, const int32_t* __restrict__ S_id,
                                            const int32_t* __restrict__ vor_seed_n) {
  if (li >= R.n) return kVorBuckets;  // no particle: a bucket of its own, never counted
  const int32_t w = vor_seed_n[R.p0 + S_id[R.p0 + li]];
  return (w >> kSeedCostShift) & (kVorBuckets - 1);
}

__global__ void __launch_bounds__(kBlock) order_count_kernel(const Rep* __restrict__ reps,
                                                             const BlockTask* __restrict__ tasks,
                                                             const int32_t* __restrict__ S_id,
                                                             const int32_t* __restrict__ vor_seed_n,
                                                             uint32_t* __restrict__ table) {
  __shared__ uint32_t cnt[kVorBuckets];
  if (threadIdx.x < kVorBuckets) cnt[threadIdx.x] = 0;
  __syncthreads();
  const BlockTask t = tasks[blockIdx.x];
  const Rep R = reps[t.rep];
  const int b = order_bucket(R, t.first + (int)threadIdx.x, S_id, vor_seed_n);
  if (b < kVorBuckets) atomicAdd(&cnt[b], 1u);
  __syncthreads();
  if (threadIdx.x < kVorBuckets) table[(size_t)blockIdx.x * kVorBuckets + threadIdx.x] = cnt[threadIdx.x];
}

// one warp per replica: lane b < kVorBuckets turns the counts of bucket b in
// the replica's block tasks into write offsets (slot indices)
__global__ void __launch_bounds__(32) order_offset_kernel(const Rep* __restrict__ reps,
                                                          const int32_t* __restrict__ rep_task0,
                                                          uint32_t* __restrict__ table) {
  const int r = blockIdx.x;
  const int lane = (int)threadIdx.x;
  const int t0 = rep_task0[r], t1 = rep_task0[r + 1];
  uint32_t total = 0;
  if (lane < kVorBuckets)
    for (int t = t0; t < t1; ++t) total += table[(size_t)t * kVorBuckets + lane];
  // exclusive scan of the bucket totals across the lanes
  uint32_t base = total;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t v = __shfl_up_sync(0xffffffffu, base, o);
    if (lane >= o) base += v;
  }
  base -= total;
  if (lane < kVorBuckets) {
    uint32_t run = (uint32_t)reps[r].p0 + base;
    for (int t = t0; t < t1; ++t) {
      const uint32_t c = table[(size_t)t * kVorBuckets + lane];
      table[(size_t)t * kVorBuckets + lane] = run;
      run += c;
    }
  }
}

__global__ void __launch_bounds__(kBlock) order_scatter_kernel(const Rep* __restrict__ reps,
                                                               const BlockTask* __restrict__ tasks,
                                                               const int32_t* __restrict__ S_id,
                                                               const int32_t* __restrict__ vor_seed_n,
                                                               const uint32_t* __restrict__ table,
                                                               int32_t* __restrict__ order) {
  __shared__ uint32_t wcnt[kBlock / 32][kVorBuckets + 1];  // per warp and bucket
  for (int i = (int)threadIdx.x; i < (kBlock / 32) * (kVorBuckets + 1); i += kBlock) (&wcnt[0][0])[i] = 0u;
  __syncthreads();
  const BlockTask t = tasks[blockIdx.x];
  const Rep R = reps[t.rep];
  const int li = t.first + (int)threadIdx.x;
  const int b = order_bucket(R, li, S_id, vor_seed_n);
  const int lane = (int)(threadIdx.x & 31), wid = (int)(threadIdx.x >> 5);
  // rank among the warp's lanes of the same bucket (lane order)
  const unsigned same = __match_any_sync(0xffffffffu, b);
  const uint32_t rank_w = (uint32_t)__popc(same & ((1u << lane) - 1u));
  if (lane == __ffs(same) - 1) wcnt[wid][b] = (uint32_t)__popc(same);
  __syncthreads();
  if (b < kVorBuckets) {
    uint32_t before = 0;  // earlier warps of the block, same bucket
    for (int w2 = 0; w2 < wid; ++w2) before += wcnt[w2][b];
    order[table[(size_t)blockIdx.x * kVorBuckets + b] + before + rank_w] = (int32_t)(R.p0 + li);
  }
}

// 1: visit each replica's particles grouped by last step's cost (needs the seeds)
#ifndef VK_VOR_ORDER
#define VK_VOR_ORDER 1
#endif

// Heavy-cell hint: a cell that needed more than kHeavyHint candidates in the
// main kernel, or more than kHeavyKeep in the warp kernel, is flagged in its
// seed word, and the next step sends it to the warp kernel at once (particles
// on the rim of a void stay there for many steps).  Speed only.
#ifndef VK_VOR_HEAVY_HINT
#define VK_VOR_HEAVY_HINT 320
#endif
constexpr uint32_t kHeavyHint = VK_VOR_HEAVY_HINT > 0 ? VK_VOR_HEAVY_HINT : 0xFFFFFFFFu;
constexpr uint32_t kHeavyKeep = VK_VOR_HEAVY_HINT > 0 ? VK_VOR_HEAVY_HINT / 2 : 0xFFFFFFFFu;

// Main kernel: cells of up to kFastCap edges.  Particles whose cell outgrows
// it are appended to the overflow list and finished by the overflow kernel.
// resident 256-thread blocks per SM the main kernel is compiled for
#ifndef VK_VOR_MIN_BLOCKS
#define VK_VOR_MIN_BLOCKS 2
#endif
// threads per block of the main kernel: each 256-particle block task is
// split into kBlock / VK_VOR_BLOCK blocks, so that the few slow cells (void
// rims) hold back smaller blocks and the SMs stay evenly loaded
#ifndef VK_VOR_BLOCK
#define VK_VOR_BLOCK 256
#endif
constexpr int kVorBlock = VK_VOR_BLOCK;
constexpr int kVorSplit = kBlock / kVorBlock;

__global__ void __launch_bounds__(kVorBlock, VK_VOR_MIN_BLOCKS * kVorSplit) voronoi_step_kernel(
    const Rep* __restrict__ reps, const BlockTask* __restrict__ tasks, const int2* __restrict__ S_pos,
    const float2* __restrict__ S_dir, const int32_t* __restrict__ S_id, GridView G,
    int2* __restrict__ U_pos, float2* __restrict__ U_dir, int32_t* __restrict__ U_id,
    uint32_t* __restrict__ counts, PhiAcc* __restrict__ phi_acc, const int64_t* __restrict__ d_step, StepParams Pm,
    int2* __restrict__ ovf_list, int32_t* __restrict__ ovf_count, int32_t* status, int32_t* __restrict__ vor_seed,
    int32_t* __restrict__ vor_seed_n, const int32_t* __restrict__ slot_of, const int32_t* __restrict__ order) {
  __shared__ PhiShared phs;
  phi_block_begin(phs);
  const BlockTask t = tasks[blockIdx.x / kVorSplit];
  const Rep R = reps[t.rep];
  const int li = t.first + (int)(blockIdx.x % kVorSplit) * kVorBlock + (int)threadIdx.x;
  const int64_t step = *d_step;
  float nnew[3] = {0.f, 0.f, 0.f};
  uint32_t n_cand = 0, n_runs = 0;
  if (li < R.n) {
    // the replica's particles in the cost-grouped order (sorted order without seeds)
    const int64_t s = order ? (int64_t)order[R.p0 + li] : R.p0 + li;
    const int2 p = S_pos[s];
    const float2 nv = S_dir[s];
    const int32_t pi[3] = {p.x, p.y, 0};
    const float ni[3] = {nv.x, nv.y, 0.f};
    const int32_t id = S_id[s];
    const int64_t gi = R.p0 + id;
    const int32_t sw = vor_seed ? vor_seed_n[gi] : 0;
    const Seeds sd{vor_seed ? vor_seed + gi * kVorSeed : nullptr, sw & kSeedCount, slot_of};
    Poly<kFastCap> P;
    uint32_t seen = 0;
    // a cell that was heavy at the last step goes straight to the warp kernel
    const bool ok = !(sw & kSeedHeavy) &&
                    (Pm.stats ? voronoi_cell(R, s, pi, id, S_pos, S_id, G, P, status, kHeavy, sd, &seen, &n_cand,
                                             &n_runs)
                              : voronoi_cell(R, s, pi, id, S_pos, S_id, G, P, status, kHeavy, sd, &seen));
    if (ok) {
      voronoi_update(R, Pm, step, s, P, pi, ni, id, S_dir, U_pos, U_dir, U_id, counts, nnew,
                     vor_seed ? vor_seed + gi * kVorSeed : nullptr, vor_seed_n + gi, seen > kHeavyHint, seen);
    } else {
      const int q = atomicAdd(ovf_count, 1);
      ovf_list[q] = make_int2((int)s, t.rep);
    }
  }
  record_search_stats(Pm.stats, li < R.n, n_cand, n_runs);
  phi_block_end<2>(phs, nnew, phi_acc + ((size_t)(step % Pm.phi_cap) * (size_t)Pm.n_rep + (size_t)t.rep) * 3);
}

// Overflow kernel: the few particles whose cell outgrew the main kernel's
// polygon (a particle bordering a void can have dozens of Voronoi
// neighbors) or needed more than kHeavy candidates; one warp per particle.
constexpr int kOvfWarps = 4;

__global__ void __launch_bounds__(32 * kOvfWarps) voronoi_overflow_kernel(
    const Rep* __restrict__ reps, const int2* __restrict__ S_pos, const float2* __restrict__ S_dir,
    const int32_t* __restrict__ S_id, GridView G, int2* __restrict__ U_pos,
    float2* __restrict__ U_dir, int32_t* __restrict__ U_id,
    uint32_t* __restrict__ counts, PhiAcc* __restrict__ phi_acc, const int64_t* __restrict__ d_step, StepParams Pm,
    const int2* __restrict__ ovf_list, const int32_t* __restrict__ ovf_count, int32_t* status,
    int32_t* __restrict__ vor_seed, int32_t* __restrict__ vor_seed_n, const int32_t* __restrict__ slot_of) {
  __shared__ Poly<kSlowCap> poly[kOvfWarps];
  Poly<kSlowCap>& P = poly[threadIdx.x >> 5];
  const int total = *ovf_count;
  const int64_t step = *d_step;
  const int nwarps = gridDim.x * kOvfWarps;
  for (int q = blockIdx.x * kOvfWarps + (int)(threadIdx.x >> 5); q < total; q += nwarps) {
    const int2 e = ovf_list[q];
    const Rep R = reps[e.y];
    const int64_t s = e.x;
    const int2 p = S_pos[s];
    const int32_t pi[3] = {p.x, p.y, 0};
    const int32_t id = S_id[s];
    const int64_t gi = R.p0 + id;
    const Seeds sd{vor_seed ? vor_seed + gi * kVorSeed : nullptr, vor_seed ? vor_seed_n[gi] & kSeedCount : 0,
                   slot_of};
    uint32_t seen = 0;
    const bool ok = voronoi_cell_warp(R, s, pi, id, S_pos, S_id, G, P, status, sd, &seen);
    if ((threadIdx.x & 31) == 0) {
      if (!ok) {
        set_status(status, kStCapacity);
      } else {
        const float2 nv = S_dir[s];
        const float ni[3] = {nv.x, nv.y, 0.f};
        float nnew[3] = {0.f, 0.f, 0.f};
        voronoi_update(R, Pm, step, s, P, pi, ni, id, S_dir, U_pos, U_dir, U_id, counts, nnew,
                       vor_seed ? vor_seed + gi * kVorSeed : nullptr, vor_seed_n + gi, seen > kHeavyKeep, seen);
        PhiAcc* acc = phi_acc + ((size_t)(step % Pm.phi_cap) * (size_t)Pm.n_rep + (size_t)e.y) * 3;
        atomicAdd(acc + 0, (PhiAcc)phi_fixed(nnew[0]));
        atomicAdd(acc + 1, (PhiAcc)phi_fixed(nnew[1]));
      }
    }
    __syncwarp();
  }
}

// Export (not on the hot path): pass 0 writes the degree of every particle
// (by id), pass 1 writes the sorted ids at out_off[id].
__global__ void __launch_bounds__(64) voronoi_export_kernel(const Rep* __restrict__ reps, int rep,
                                                            const int2* __restrict__ S_pos,
                                                            const int32_t* __restrict__ S_id,
                                                            GridView G, int pass,
                                                            int32_t* __restrict__ deg,
                                                            const int64_t* __restrict__ out_off,
                                                            int32_t* __restrict__ out_ids, int32_t* status,
                                                            const int32_t* __restrict__ vor_seed,
                                                            const int32_t* __restrict__ vor_seed_n,
                                                            const int32_t* __restrict__ slot_of) {
  const Rep R = reps[rep];
  for (int li = blockIdx.x * blockDim.x + threadIdx.x; li < R.n; li += gridDim.x * blockDim.x) {
    const int64_t s = R.p0 + li;
    const int2 p = S_pos[s];
    const int32_t pi[3] = {p.x, p.y, 0};
    const int32_t id = S_id[s];
    const int64_t gi = R.p0 + id;
    const Seeds sd{vor_seed ? vor_seed + gi * kVorSeed : nullptr, vor_seed ? vor_seed_n[gi] & kSeedCount : 0,
                   slot_of};
    Poly<kSlowCap> P;
    if (!voronoi_cell(R, s, pi, id, S_pos, S_id, G, P, status, 0u, sd, nullptr)) {
      set_status(status, kStCapacity);
      if (pass == 0) deg[id] = 0;
      continue;
    }
    int32_t nid[kSlowCap + Poly<kSlowCap>::TW], nslot[kSlowCap + Poly<kSlowCap>::TW];
    const int cnt = voronoi_neighbors(P, id, nid, nslot);
    if (pass == 0) {
      deg[id] = cnt;
    } else {
      const int64_t o = out_off[id];
      for (int j = 0; j < cnt; ++j) out_ids[o + j] = nid[j];
    }
  }
}

}  // namespace

static GridView grid_view(const Buffers& b) {
  GridView G;
  G.off = b.offsets;
  G.sub_s = b.sub_s;
  G.sub_base = b.sub_base;
  G.sub_off = b.sub_off;
  return G;
}

cudaError_t launch_voronoi_step(const Geometry& g, const Buffers& b, const StepParams& P, cudaStream_t st) {
  const GridView G = grid_view(b);
  const bool ordered = VK_VOR_ORDER && b.vor_order != nullptr;
  if (ordered) {
    order_count_kernel<<<g.n_tasks, kBlock, 0, st>>>(g.reps, g.tasks, b.S_id, b.vor_seed_n, b.vor_bucket);
    order_offset_kernel<<<g.n_rep, 32, 0, st>>>(g.reps, b.rep_task0, b.vor_bucket);
    order_scatter_kernel<<<g.n_tasks, kBlock, 0, st>>>(g.reps, g.tasks, b.S_id, b.vor_seed_n, b.vor_bucket,
                                                       b.vor_order);
  }
  voronoi_step_kernel<<<g.n_tasks * kVorSplit, kVorBlock, 0, st>>>(
      g.reps, g.tasks, (const int2*)b.S_pos, (const float2*)b.S_dir, b.S_id, G, (int2*)b.U_pos, (float2*)b.U_dir,
      b.U_id, b.counts, b.phi_acc, b.d_step, P, b.ovf_list, b.ovf_count, b.d_status, b.vor_seed, b.vor_seed_n,
      b.slot_of, ordered ? b.vor_order : nullptr);
  voronoi_overflow_kernel<<<device_sm_count(), 32 * kOvfWarps, 0, st>>>(
      g.reps, (const int2*)b.S_pos, (const float2*)b.S_dir, b.S_id, G, (int2*)b.U_pos, (float2*)b.U_dir, b.U_id,
      b.counts, b.phi_acc, b.d_step, P, b.ovf_list, b.ovf_count, b.d_status, b.vor_seed, b.vor_seed_n, b.slot_of);
  return cudaGetLastError();
}

int voronoi_step_launches(const Buffers& b) { return (VK_VOR_ORDER && b.vor_order != nullptr) ? 5 : 2; }

cudaError_t launch_voronoi_export(const Geometry& g, const Buffers& b, int rep, int n, int pass, int32_t* deg,
                                  const int64_t* out_off, int32_t* out_ids, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  const int nb = std::min((n + 63) / 64, device_sm_count() * 8);
  voronoi_export_kernel<<<nb, 64, 0, st>>>(g.reps, rep, (const int2*)b.S_pos, b.S_id, grid_view(b), pass, deg,
                                           out_off, out_ids, b.d_status, b.vor_seed, b.vor_seed_n, b.slot_of);
  return cudaGetLastError();
}

}  // namespace vk
