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
                                               int32_t* __restrict__ seed_n_out, bool heavy_next) {
  int32_t nid[CAP + Poly<CAP>::TW], nslot[CAP + Poly<CAP>::TW];
  const int cnt = voronoi_neighbors(P, id, nid, nslot);
  if (seed_out) {
    // the next step's seeds (any subset of sites would do)
    const int ns = min(cnt, kVorSeed);
    for (int j = 0; j < ns; ++j) seed_out[j] = nid[j];
    *seed_n_out = ns | (heavy_next ? kSeedHeavy : 0);
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
    int32_t* __restrict__ vor_seed_n, const int32_t* __restrict__ slot_of) {
  __shared__ PhiShared phs;
  phi_block_begin(phs);
  const BlockTask t = tasks[blockIdx.x / kVorSplit];
  const Rep R = reps[t.rep];
  const int li = t.first + (int)(blockIdx.x % kVorSplit) * kVorBlock + (int)threadIdx.x;
  const int64_t step = *d_step;
  float nnew[3] = {0.f, 0.f, 0.f};
  uint32_t n_cand = 0, n_runs = 0;
  if (li < R.n) {
    const int64_t s = R.p0 + li;
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
                     vor_seed ? vor_seed + gi * kVorSeed : nullptr, vor_seed_n + gi, seen > kHeavyHint);
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
                       vor_seed ? vor_seed + gi * kVorSeed : nullptr, vor_seed_n + gi, seen > kHeavyKeep);
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
  voronoi_step_kernel<<<g.n_tasks * kVorSplit, kVorBlock, 0, st>>>(g.reps, g.tasks, (const int2*)b.S_pos, (const float2*)b.S_dir,
                                                    b.S_id, G, (int2*)b.U_pos, (float2*)b.U_dir, b.U_id,
                                                    b.counts, b.phi_acc, b.d_step, P, b.ovf_list,
                                                    b.ovf_count, b.d_status, b.vor_seed, b.vor_seed_n,
                                                    b.slot_of);
  voronoi_overflow_kernel<<<device_sm_count(), 32 * kOvfWarps, 0, st>>>(g.reps, (const int2*)b.S_pos, (const float2*)b.S_dir, b.S_id,
                                              G, (int2*)b.U_pos, (float2*)b.U_dir, b.U_id,
                                              b.counts, b.phi_acc, b.d_step, P, b.ovf_list, b.ovf_count,
                                              b.d_status, b.vor_seed, b.vor_seed_n, b.slot_of);
  return cudaGetLastError();
}

cudaError_t launch_voronoi_export(const Geometry& g, const Buffers& b, int rep, int n, int pass, int32_t* deg,
                                  const int64_t* out_off, int32_t* out_ids, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  const int nb = std::min((n + 63) / 64, device_sm_count() * 8);
  voronoi_export_kernel<<<nb, 64, 0, st>>>(g.reps, rep, (const int2*)b.S_pos, b.S_id, grid_view(b), pass, deg,
                                           out_off, out_ids, b.d_status, b.vor_seed, b.vor_seed_n, b.slot_of);
  return cudaGetLastError();
}

}  // namespace vk
