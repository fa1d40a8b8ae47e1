// vk_knn.cu -- k-nearest-neighbor rule (Sec. "Metric and topological flocking
// models": each particle aligns with its k nearest neighbors, at any distance,
// so the relation is not reciprocal) fused with the Vicsek update of Eq. (1)
// and Eq. (2), in 3D (the 2D rule, the benchmark's, is in vk_knn2d.cu).
//
// One thread per particle, in cell-sorted order.  The search walks rings of
// cells around the particle's cell; each row segment of a ring is one
// contiguous run of the sorted arrays.  The k best (exact int64 squared
// distance, id) pairs live in registers, sorted.  After ring r the search
// stops once the k-th best distance is below the exact integer distance from
// the particle to the boundary of the scanned (2r+1)^d block.
#include <climits>

#include "vk_internal.cuh"

namespace vk {

namespace {

// Top-k list of KC register slots.  For k < KC the first KC-k slots hold
// sentinels that order before every real candidate, so the threshold is
// always slot KC-1 and no register array is indexed dynamically.
template <int KC>
struct TopK {
  uint64_t d[KC];
  int32_t id[KC];
  int32_t slot[KC];
};

template <int KC>
__device__ __forceinline__ void topk_init(TopK<KC>& T, int k) {
#pragma unroll
  for (int s = 0; s < KC; ++s) {
    const bool sentinel = s < KC - k;
    T.d[s] = sentinel ? 0ull : ~0ull;
    T.id[s] = sentinel ? INT_MIN : INT_MAX;
    T.slot[s] = -1;
  }
}

template <int KC>
__device__ __forceinline__ void topk_insert(TopK<KC>& T, uint64_t D, int32_t idj, int32_t q) {
  bool placed = false;
#pragma unroll
  for (int s = KC - 1; s > 0; --s) {
    const bool before = (D < T.d[s - 1]) || (D == T.d[s - 1] && idj < T.id[s - 1]);
    if (!placed) {
      if (before) {
        T.d[s] = T.d[s - 1];
        T.id[s] = T.id[s - 1];
        T.slot[s] = T.slot[s - 1];
      } else {
        T.d[s] = D;
        T.id[s] = idj;
        T.slot[s] = q;
        placed = true;
      }
    }
  }
  if (!placed) {
    T.d[0] = D;
    T.id[0] = idj;
    T.slot[0] = q;
  }
}

template <int DIM, int KC>
__device__ __forceinline__ void knn_search(const Rep& R, int64_t self, const int32_t* pi,
                                           const typename Vec<DIM>::P* __restrict__ pos,
                                           const int32_t* __restrict__ ids, const GridView& G, TopK<KC>& T,
                                           uint32_t* n_cand = nullptr, uint32_t* n_runs = nullptr) {
  auto run = [&](uint32_t qb, uint32_t qe) {
    if (n_cand) {
      *n_cand += qe - qb;
      *n_runs += 1;
    }
    for (uint32_t q = qb; q < qe; ++q) {
      if ((int64_t)q == self) continue;
      int32_t pj[3];
      unpack(pos[q], pj);
      uint64_t D = 0;
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        const int64_t d = min_image((int64_t)pj[a] - (int64_t)pi[a], (int64_t)R.L[a]);
        D += (uint64_t)(d * d);
      }
      if (D <= T.d[KC - 1]) {
        const int32_t idj = ids[q];
        if (D < T.d[KC - 1] || idj < T.id[KC - 1]) topk_insert<KC>(T, D, idj, (int32_t)q);
      }
    }
  };
  // every unscanned particle is at squared distance >= B2: stop once the
  // k-th best is strictly closer (an equal distance could still win on id)
  auto stop = [&](uint64_t B2) { return T.d[KC - 1] < B2; };
  static_assert(DIM == 3, "the 2D rule is vk_knn2d.cu");
  grid_walk3(R, pi, G, run, stop);
}

// ---------------------------------------------------------------------------
// Radius first (3D): each particle scans the cube [p - a, p + a]^3, a a
// little above its k-th neighbor distance at the previous step, as the
// x-row segments of the cells it meets (each a contiguous run of the sorted
// arrays, with the periodic image it lies in).  Every candidate with exact
// squared distance D <= tau = (a+1)^2 - 1 goes into the register top-k by
// (D, id); nothing outside the cube is that close, so once the k-th best is
// <= tau the list is exact, ties included.  Otherwise one larger cube, then
// the ring walk.
// ---------------------------------------------------------------------------

// unwrapped cell index of an unwrapped coordinate, -L <= x < 2L
__device__ __forceinline__ int ucell3(int64_t x, int n, const uint32_t* __restrict__ bnd, float inv_w, int64_t L) {
  if (x < 0) return cell_of_tab((uint32_t)(x + L), n, bnd, inv_w) - n;
  if (x >= L) return cell_of_tab((uint32_t)(x - L), n, bnd, inv_w) + n;
  return cell_of_tab((uint32_t)x, n, bnd, inv_w);
}

// the coordinate of the particle shifted into the image an unwrapped cell
// index u lies in: offsets x_j - that are exact in wrapping 32-bit arithmetic
__device__ __forceinline__ uint32_t image_ref(uint32_t p, int u, int n, uint32_t L) {
  return u < 0 ? p + L : (u >= n ? p - L : p);
}

// the k nearest from the cube of half-width a; true when they are exact
template <int KC>
__device__ __forceinline__ bool cube_search(const Rep& R, const uint32_t* __restrict__ bounds, const GridView& G,
                                            const int4* __restrict__ pos, const int32_t* __restrict__ ids,
                                            int64_t self, const int32_t* pi, int64_t a, TopK<KC>& T,
                                            uint32_t* n_cand, uint32_t* n_runs) {
  int lo[3], hi[3];
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) {
    const int64_t L = R.L[ax];
    if (2 * (2 * a + 1) >= L) return false;
    const uint32_t* bnd = bounds + R.bnd[ax];
    lo[ax] = ucell3((int64_t)pi[ax] - a, R.nc[ax], bnd, R.inv_w[ax], L);
    hi[ax] = ucell3((int64_t)pi[ax] + a, R.nc[ax], bnd, R.inv_w[ax], L);
    if (hi[ax] - lo[ax] + 1 > R.nc[ax]) return false;
  }
  const uint64_t tau = (uint64_t)(a + 1) * (uint64_t)(a + 1) - 1;
  const int nx = R.nc[0], ny = R.nc[1], nz = R.nc[2];
  for (int uz = lo[2]; uz <= hi[2]; ++uz) {
    const int cz = uz < 0 ? uz + nz : (uz >= nz ? uz - nz : uz);
    const uint32_t oz = image_ref((uint32_t)pi[2], uz, nz, R.L[2]);
    for (int uy = lo[1]; uy <= hi[1]; ++uy) {
      const int cy = uy < 0 ? uy + ny : (uy >= ny ? uy - ny : uy);
      const uint32_t oy = image_ref((uint32_t)pi[1], uy, ny, R.L[1]);
      const int64_t row = R.c0 + ((int64_t)cz * ny + cy) * nx;
      // the x range splits at the period into up to three segments
      for (int seg = 0; seg < 3; ++seg) {
        int xs = seg == 0 ? lo[0] : (seg == 1 ? max(lo[0], 0) : max(lo[0], nx));
        int xe = seg == 0 ? min(hi[0], -1) : (seg == 1 ? min(hi[0], nx - 1) : hi[0]);
        if (xs > xe) continue;
        const uint32_t ox = image_ref((uint32_t)pi[0], xs, nx, R.L[0]);
        const int wxs = xs < 0 ? xs + nx : (xs >= nx ? xs - nx : xs);
        const uint32_t qb = __ldg(G.off + row + wxs), qe = __ldg(G.off + row + wxs + (xe - xs) + 1);
        if (n_cand) {
          *n_cand += qe - qb;
          *n_runs += 1;
        }
        for (uint32_t q = qb; q < qe; ++q) {
          const int4 pj = __ldg(pos + q);
          const int32_t dx = (int32_t)((uint32_t)pj.x - ox), dy = (int32_t)((uint32_t)pj.y - oy),
                        dz = (int32_t)((uint32_t)pj.z - oz);
          const uint64_t D = (uint64_t)((int64_t)dx * dx) + (uint64_t)((int64_t)dy * dy) +
                             (uint64_t)((int64_t)dz * dz);
          if (D <= tau && D <= T.d[KC - 1] && (int64_t)q != self) {
            const int32_t idj = __ldg(ids + q);
            if (D < T.d[KC - 1] || idj < T.id[KC - 1]) topk_insert<KC>(T, D, idj, (int32_t)q);
          }
        }
      }
    }
  }
  return T.d[KC - 1] <= tau;
}

// search radius without a hint: from the density of the particle's own cell
__device__ __forceinline__ float cube_radius_estimate(const Rep& R, const uint32_t* __restrict__ bounds,
                                                      const GridView& G, const int32_t* pi, int k) {
  int c[3];
  float vol = 1.f;
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) {
    const uint32_t* bnd = bounds + R.bnd[ax];
    c[ax] = cell_of_tab((uint32_t)pi[ax], R.nc[ax], bnd, R.inv_w[ax]);
    vol *= (float)(__ldg(bnd + c[ax] + 1) - __ldg(bnd + c[ax]));
  }
  const int64_t gc = R.c0 + ((int64_t)c[2] * R.nc[1] + c[1]) * R.nc[0] + c[0];
  const float m = (float)max(__ldg(G.off + gc + 1) - __ldg(G.off + gc), 1u);
  return 1.3f * cbrtf(3.f * (float)k * vol / (4.f * 3.14159265f * m));
}

template <int DIM, int KC>
__global__ void __launch_bounds__(kBlock) knn_step_kernel(
    const Rep* __restrict__ reps, const BlockTask* __restrict__ tasks,
    const typename Vec<DIM>::P* __restrict__ S_pos, const typename Vec<DIM>::F* __restrict__ S_dir,
    const int32_t* __restrict__ S_id, GridView G, typename Vec<DIM>::P* __restrict__ U_pos,
    typename Vec<DIM>::F* __restrict__ U_dir, int32_t* __restrict__ U_id,
    uint32_t* __restrict__ counts, PhiAcc* __restrict__ phi_acc, const int64_t* __restrict__ d_step, StepParams P,
    const uint32_t* __restrict__ bounds, const float* __restrict__ S_hint, float* __restrict__ U_hint) {
  using PV = typename Vec<DIM>::P;
  using FV = typename Vec<DIM>::F;
  const BlockTask t = tasks[blockIdx.x];
  const Rep R = reps[t.rep];
  const int li = t.first + (int)threadIdx.x;
  const int64_t step = *d_step;
  float nnew[3] = {0.f, 0.f, 0.f};
  uint32_t n_cand = 0, n_runs = 0;
  if (li < R.n) {
    const int64_t s = R.p0 + li;
    int32_t pi[3] = {0, 0, 0};
    float ni[3] = {0.f, 0.f, 0.f};
    unpack(S_pos[s], pi);
    unpack(S_dir[s], ni);
    const int32_t id = S_id[s];
    TopK<KC> T;
    bool done = false;
    if (S_hint && P.knn_search == 0) {
      // radius first: the hinted cube, then one larger
      const float hint = S_hint[s];
      float r = hint > 0.f ? P.halo_alpha * hint : cube_radius_estimate(R, bounds, G, pi, P.k);
      for (int tr = 0; tr < 2 && !done; ++tr) {
        topk_init<KC>(T, P.k);
        done = cube_search<KC>(R, bounds, G, S_pos, S_id, s, pi, (int64_t)ceilf(fminf(r, 1.0e9f)), T,
                               P.stats ? &n_cand : nullptr, &n_runs);
        r *= 1.6f;
      }
    }
    if (!done) {
      topk_init<KC>(T, P.k);
      if (P.stats) knn_search<DIM, KC>(R, s, pi, S_pos, S_id, G, T, &n_cand, &n_runs);
      else knn_search<DIM, KC>(R, s, pi, S_pos, S_id, G, T);
    }
    if (U_hint) U_hint[s] = sqrtf((float)T.d[KC - 1]) * 1.0001f + 1.f;
    HeadSum<DIM> H;
    H.init();
    if (P.include_self) H.add(ni, P.sum_mode);
#pragma unroll
    for (int j = 0; j < KC; ++j) {
      if (j >= KC - P.k) {
        float v[3];
        unpack(S_dir[T.slot[j]], v);
        H.add(v, P.sum_mode);
      }
    }
    int32_t pout[3] = {0, 0, 0};
    align_advect<DIM>(R, P, (uint32_t)step, id, ni, H, P.k + (P.include_self ? 1 : 0), pi, pout, nnew);
    U_pos[s] = make_p(pout, (PV*)nullptr);
    U_dir[s] = make_f(nnew, (FV*)nullptr);
    U_id[s] = id;
    atomicAdd(counts + linear_cell<DIM>(R, pout), 1u);
  }
  record_search_stats(P.stats, li < R.n, n_cand, n_runs);
  block_phi_accumulate<DIM>(nnew, phi_acc + ((size_t)(step % P.phi_cap) * (size_t)P.n_rep + (size_t)t.rep) * 3);
}

// neighbor lists of the current positions of one replica, written by id
template <int DIM, int KC>
__global__ void __launch_bounds__(kBlock) knn_export_kernel(const Rep* __restrict__ reps, int rep,
                                                            const typename Vec<DIM>::P* __restrict__ S_pos,
                                                            const int32_t* __restrict__ S_id, GridView G,
                                                            int k, int32_t* __restrict__ out) {
  const Rep R = reps[rep];
  const int li = blockIdx.x * kBlock + (int)threadIdx.x;
  if (li >= R.n) return;
  const int64_t s = R.p0 + li;
  int32_t pi[3] = {0, 0, 0};
  unpack(S_pos[s], pi);
  const int32_t id = S_id[s];
  TopK<KC> T;
  topk_init<KC>(T, k);
  knn_search<DIM, KC>(R, s, pi, S_pos, S_id, G, T);
#pragma unroll
  for (int j = 0; j < KC; ++j)
    if (j >= KC - k) out[(int64_t)id * k + (j - (KC - k))] = T.id[j];
}

GridView grid_view(const Buffers& b) {
  GridView G;
  G.off = b.offsets;
  G.sub_s = b.sub_s;
  G.sub_base = b.sub_base;
  G.sub_off = b.sub_off;
  return G;
}

template <int DIM, int KC>
cudaError_t step_dispatch(const Geometry& g, const Buffers& b, const StepParams& P, cudaStream_t st) {
  using PV = typename Vec<DIM>::P;
  using FV = typename Vec<DIM>::F;
  knn_step_kernel<DIM, KC><<<g.n_tasks, kBlock, 0, st>>>(
      g.reps, g.tasks, (const PV*)b.S_pos, (const FV*)b.S_dir, b.S_id, grid_view(b), (PV*)b.U_pos,
      (FV*)b.U_dir, b.U_id, b.counts, b.phi_acc, b.d_step, P, b.bounds, b.S_hint, b.U_hint);
  return cudaGetLastError();
}

template <int DIM, int KC>
cudaError_t export_dispatch(const Geometry& g, const Buffers& b, int k, int rep, int n, int32_t* out,
                            cudaStream_t st) {
  using PV = typename Vec<DIM>::P;
  const int nb = (n + kBlock - 1) / kBlock;
  if (nb == 0) return cudaSuccess;
  knn_export_kernel<DIM, KC><<<nb, kBlock, 0, st>>>(g.reps, rep, (const PV*)b.S_pos, b.S_id, grid_view(b), k, out);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_knn_step(const Geometry& g, const Buffers& b, const StepParams& P, cudaStream_t st) {
  if (g.dim != 3) return cudaErrorInvalidValue;  // 2D: launch_knn2_step
  if (P.k <= 8) return step_dispatch<3, 8>(g, b, P, st);
  if (P.k <= 16) return step_dispatch<3, 16>(g, b, P, st);
  return step_dispatch<3, 32>(g, b, P, st);
}

cudaError_t launch_knn_export(const Geometry& g, const Buffers& b, int k, int rep, int n, int32_t* out,
                              cudaStream_t st) {
  if (g.dim != 3) return cudaErrorInvalidValue;  // 2D: launch_knn2_export
  if (k <= 8) return export_dispatch<3, 8>(g, b, k, rep, n, out, st);
  if (k <= 16) return export_dispatch<3, 16>(g, b, k, rep, n, out, st);
  return export_dispatch<3, 32>(g, b, k, rep, n, out, st);
}

}  // namespace vk
