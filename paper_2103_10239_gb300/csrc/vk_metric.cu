// vk_metric.cu -- the metric rule (Sec. "Metric and topological flocking
// models": each particle aligns with every particle within the interaction
// radius r0, the original Vicsek rule; Eq. 1 and Eq. 2), 2D and 3D.
//
// One thread per particle, in cell-sorted order.  2D: the square
// [p - r0q, p + r0q] is walked as contiguous runs of the sorted arrays
// (vk_box2d.cuh); 3D: rings of cells until the scanned block holds the ball.
// A candidate is a neighbor iff its exact int64 squared minimum-image
// distance is <= r0q^2.  The neighbor count has no bound, so nothing is
// buffered: the headings are summed as they are found, each component
// rounded to 2^-32 and added in int64.  Integer addition is associative, so
// the sum does not depend on the visiting order (which the atomic ranks of
// the cell sort leave free) and a step is bit-identical run to run; the
// rounding errs by at most 2^-33 per neighbor.  The sum is converted to
// FP64 for the update.
#include <algorithm>

#include "vk_box2d.cuh"

namespace vk {

namespace {

// slot runs one listing buffers per thread (shared memory)
struct MetricRuns {
  static constexpr int kRuns = VK_KNN2_BOX_RUNS;
  uint2 run[kRuns][kBlock];
};

// heading sum and count of the neighbors found so far
template <int DIM>
struct MetricSum {
  long long s[DIM];
  int m;
  __device__ __forceinline__ void init() {
#pragma unroll
    for (int a = 0; a < DIM; ++a) s[a] = 0;
    m = 0;
  }
  __device__ __forceinline__ void add(const float* v) {
#pragma unroll
    for (int a = 0; a < DIM; ++a) s[a] += phi_fixed(v[a]);
    ++m;
  }
};

// 2D visitor of the square walk: neighbors by the exact distance test
struct MetricVisit2 {
  const Ctx& C;
  const float2* __restrict__ dir;
  uint64_t r2;
  MetricSum<2>& S;
  __device__ __forceinline__ void group(uint32_t q, uint32_t n, const int2* pj, uint32_t ox, uint32_t oy) {
#pragma unroll
    for (int u = 0; u < kGroup; ++u) {
      const int32_t dx = (int32_t)((uint32_t)pj[u].x - ox), dy = (int32_t)((uint32_t)pj[u].y - oy);
      const uint64_t D = (uint64_t)((int64_t)dx * dx) + (uint64_t)((int64_t)dy * dy);
      if ((uint32_t)u < n && D <= r2 && (int64_t)(q + (uint32_t)u) != C.self) {
        const float2 d = __ldg(dir + q + u);
        const float v[2] = {d.x, d.y};
        S.add(v);
      }
    }
  }
};

// Every neighbor of slot s (2D), found by the square walk, or by a scan of
// the whole replica when the square is too wide for it (r0 near a quarter of
// the box, or a coarse grid too small for the square).  Calls f(q) for each.
struct MetricList2 {
  const Ctx& C;
  uint64_t r2;
  int32_t* out;
  int w;
  __device__ __forceinline__ void group(uint32_t q, uint32_t n, const int2* pj, uint32_t ox, uint32_t oy) {
#pragma unroll
    for (int u = 0; u < kGroup; ++u) {
      const int32_t dx = (int32_t)((uint32_t)pj[u].x - ox), dy = (int32_t)((uint32_t)pj[u].y - oy);
      const uint64_t D = (uint64_t)((int64_t)dx * dx) + (uint64_t)((int64_t)dy * dy);
      if ((uint32_t)u < n && D <= r2 && (int64_t)(q + (uint32_t)u) != C.self) {
        if (out) out[w] = (int32_t)(q + (uint32_t)u);
        ++w;
      }
    }
  }
};

// the whole replica, one candidate at a time (the fallback of the 2D walk)
template <class V>
__device__ __forceinline__ void metric_scan_all2(const Rep& R, const int2* __restrict__ pos, const Ctx& C, V& v) {
  for (int64_t q = R.p0; q < R.p0 + R.n; ++q) {
    int32_t dx, dy;
    box_offset(C, __ldg(pos + q), dx, dy);
    // offsets relative to the particle itself: ox = x_i - 0 in the same image
    const int2 pj = make_int2((int32_t)((uint32_t)C.px + (uint32_t)dx), (int32_t)((uint32_t)C.py + (uint32_t)dy));
    int2 g[kGroup] = {pj, pj, pj, pj};
    v.group((uint32_t)q, 1u, g, C.px, C.py);
  }
}

// Eq. (2) alignment + noise and Eq. (1) advection from the exact sum
template <int DIM>
__device__ __forceinline__ void metric_update(const Rep& R, const StepParams& P, uint32_t step, int32_t id,
                                              const float* ni, MetricSum<DIM>& S, const int32_t* pi,
                                              int32_t* pout, float* nout) {
  if (P.include_self) S.add(ni);
  HeadSum<DIM> H;
  H.init();
#pragma unroll
  for (int a = 0; a < DIM; ++a) H.d[a] = ldexp((double)S.s[a], -32);
  align_advect_mode<DIM>(R, P, 2, step, id, ni, H, S.m, pi, pout, nout);
}

__global__ void __launch_bounds__(kBlock) metric2_step_kernel(
    const Rep* __restrict__ reps, const BlockTask* __restrict__ tasks, const uint32_t* __restrict__ bounds,
    const int2* __restrict__ S_pos, const float2* __restrict__ S_dir, const int32_t* __restrict__ S_id, GridView G,
    int2* __restrict__ U_pos, float2* __restrict__ U_dir, int32_t* __restrict__ U_id, uint32_t* __restrict__ counts,
    PhiAcc* __restrict__ phi_acc, const int64_t* __restrict__ d_step, StepParams P) {
  __shared__ MetricRuns H;
  __shared__ PhiShared phs;
  phi_block_begin(phs);
  const BlockTask t = tasks[blockIdx.x];
  const Rep R = reps[t.rep];
  const int li = t.first + (int)threadIdx.x;
  const int64_t step = *d_step;
  float nnew[3] = {0.f, 0.f, 0.f};
  BoxCount bc;
  if (li < R.n) {
    const int64_t s = R.p0 + li;
    const int2 p = S_pos[s];
    const float2 nv = S_dir[s];
    const int32_t id = S_id[s];
    Ctx C;
    init_ctx(C, R, s, p);
    MetricSum<2> S;
    S.init();
    MetricVisit2 v{C, S_dir, (uint64_t)R.r0q * (uint64_t)R.r0q, S};
    if (!box_walk(H, R, bounds, G, S_pos, C, (int64_t)R.r0q, bc, v)) {
      metric_scan_all2(R, S_pos, C, v);
      bc.cand += (uint32_t)R.n;
      bc.why = 1u;
    }
    const float ni[3] = {nv.x, nv.y, 0.f};
    const int32_t pi[3] = {p.x, p.y, 0};
    int32_t pout[3] = {0, 0, 0};
    metric_update<2>(R, P, (uint32_t)step, id, ni, S, pi, pout, nnew);
    U_pos[s] = make_int2(pout[0], pout[1]);
    U_dir[s] = make_float2(nnew[0], nnew[1]);
    U_id[s] = id;
    const int ncx = cell_of_tab((uint32_t)pout[0], R.nc[0], bounds + R.bnd[0], R.inv_w[0]);
    const int ncy = cell_of_tab((uint32_t)pout[1], R.nc[1], bounds + R.bnd[1], R.inv_w[1]);
    atomicAdd(counts + R.c0 + (int64_t)ncy * R.nc[0] + ncx, 1u);
  }
  record_search_stats(P.stats, li < R.n, bc.cand, bc.runs, bc.why != 0u);
  phi_block_end<2>(phs, nnew, phi_acc + ((size_t)(step % P.phi_cap) * (size_t)P.n_rep + (size_t)t.rep) * 3);
}

// 3D: rings of cells until every unscanned particle is farther than r0q
template <class F>
__device__ __forceinline__ void metric_walk3(const Rep& R, int64_t self, const int32_t* pi,
                                             const int4* __restrict__ pos, const GridView& G, uint64_t r2,
                                             uint32_t* n_cand, uint32_t* n_runs, F& f) {
  auto run = [&](uint32_t qb, uint32_t qe) {
    *n_cand += qe - qb;
    *n_runs += 1;
    for (uint32_t q = qb; q < qe; ++q) {
      if ((int64_t)q == self) continue;
      const int4 pj = __ldg(pos + q);
      const int32_t pjv[3] = {pj.x, pj.y, pj.z};
      uint64_t D = 0;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const int64_t d = min_image((int64_t)pjv[a] - (int64_t)pi[a], (int64_t)R.L[a]);
        D += (uint64_t)(d * d);
      }
      if (D <= r2) f(q);
    }
  };
  auto stop = [&](uint64_t B2) { return B2 > r2; };
  grid_walk3(R, pi, G, run, stop);
}

__global__ void __launch_bounds__(kBlock) metric3_step_kernel(
    const Rep* __restrict__ reps, const BlockTask* __restrict__ tasks, const int4* __restrict__ S_pos,
    const float4* __restrict__ S_dir, const int32_t* __restrict__ S_id, GridView G, int4* __restrict__ U_pos,
    float4* __restrict__ U_dir, int32_t* __restrict__ U_id, uint32_t* __restrict__ counts,
    PhiAcc* __restrict__ phi_acc, const int64_t* __restrict__ d_step, StepParams P) {
  const BlockTask t = tasks[blockIdx.x];
  const Rep R = reps[t.rep];
  const int li = t.first + (int)threadIdx.x;
  const int64_t step = *d_step;
  float nnew[3] = {0.f, 0.f, 0.f};
  uint32_t n_cand = 0, n_runs = 0;
  if (li < R.n) {
    const int64_t s = R.p0 + li;
    int32_t pi[3];
    float ni[3];
    unpack(S_pos[s], pi);
    unpack(S_dir[s], ni);
    const int32_t id = S_id[s];
    MetricSum<3> S;
    S.init();
    auto add = [&](uint32_t q) {
      float v[3];
      unpack(__ldg(S_dir + q), v);
      S.add(v);
    };
    metric_walk3(R, s, pi, S_pos, G, (uint64_t)R.r0q * (uint64_t)R.r0q, &n_cand, &n_runs, add);
    int32_t pout[3] = {0, 0, 0};
    metric_update<3>(R, P, (uint32_t)step, id, ni, S, pi, pout, nnew);
    U_pos[s] = make_int4(pout[0], pout[1], pout[2], 0);
    U_dir[s] = make_float4(nnew[0], nnew[1], nnew[2], 0.f);
    U_id[s] = id;
    atomicAdd(counts + linear_cell<3>(R, pout), 1u);
  }
  record_search_stats(P.stats, li < R.n, n_cand, n_runs);
  block_phi_accumulate<3>(nnew, phi_acc + ((size_t)(step % P.phi_cap) * (size_t)P.n_rep + (size_t)t.rep) * 3);
}

// sort row [b, e) of ids in place (insertion sort: rows are short, and the
// export is off the step path)
__device__ __forceinline__ void sort_row(int32_t* __restrict__ ids, int64_t b, int64_t e) {
  for (int64_t i = b + 1; i < e; ++i) {
    const int32_t x = ids[i];
    int64_t j = i;
    while (j > b && ids[j - 1] > x) {
      ids[j] = ids[j - 1];
      --j;
    }
    ids[j] = x;
  }
}

// Neighbor lists of one replica by id.  Pass 0: deg[id] = count.  Pass 1:
// the neighbor ids of row id at out_off[id] (the slots are collected in
// out_ids first, then mapped to ids and sorted).
__global__ void __launch_bounds__(kBlock) metric2_export_kernel(const Rep* __restrict__ reps, int rep,
                                                                const uint32_t* __restrict__ bounds,
                                                                const int2* __restrict__ S_pos,
                                                                const int32_t* __restrict__ S_id, GridView G,
                                                                int pass, int32_t* __restrict__ deg,
                                                                const int64_t* __restrict__ out_off,
                                                                int32_t* __restrict__ out_ids) {
  __shared__ MetricRuns H;
  const Rep R = reps[rep];
  const int li = blockIdx.x * kBlock + (int)threadIdx.x;
  // no early return: every thread of the block reaches the end together
  if (li < R.n) {
    const int64_t s = R.p0 + li;
    const int32_t id = S_id[s];
    Ctx C;
    init_ctx(C, R, s, S_pos[s]);
    int32_t* row = pass == 1 ? out_ids + out_off[id] : nullptr;
    MetricList2 v{C, (uint64_t)R.r0q * (uint64_t)R.r0q, row, 0};
    BoxCount bc;
    if (!box_walk(H, R, bounds, G, S_pos, C, (int64_t)R.r0q, bc, v)) {
      v.w = 0;
      metric_scan_all2(R, S_pos, C, v);
    }
    if (pass == 0) {
      deg[id] = v.w;
    } else {
      for (int j = 0; j < v.w; ++j) row[j] = __ldg(S_id + row[j]);
      sort_row(row, 0, v.w);
    }
  }
}

__global__ void __launch_bounds__(kBlock) metric3_export_kernel(const Rep* __restrict__ reps, int rep,
                                                                const int4* __restrict__ S_pos,
                                                                const int32_t* __restrict__ S_id, GridView G,
                                                                int pass, int32_t* __restrict__ deg,
                                                                const int64_t* __restrict__ out_off,
                                                                int32_t* __restrict__ out_ids) {
  const Rep R = reps[rep];
  const int li = blockIdx.x * kBlock + (int)threadIdx.x;
  if (li >= R.n) return;
  const int64_t s = R.p0 + li;
  const int32_t id = S_id[s];
  int32_t pi[3];
  unpack(S_pos[s], pi);
  int32_t* row = pass == 1 ? out_ids + out_off[id] : nullptr;
  int w = 0;
  auto put = [&](uint32_t q) {
    if (row) row[w] = __ldg(S_id + q);
    ++w;
  };
  uint32_t n_cand = 0, n_runs = 0;
  metric_walk3(R, s, pi, S_pos, G, (uint64_t)R.r0q * (uint64_t)R.r0q, &n_cand, &n_runs, put);
  if (pass == 0) deg[id] = w;
  else sort_row(row, 0, w);
}

GridView metric_view(const Buffers& b) {
  GridView G;
  G.off = b.offsets;
  G.sub_s = b.sub_s;
  G.sub_base = b.sub_base;
  G.sub_off = b.sub_off;
  return G;
}

}  // namespace

cudaError_t launch_metric_step(const Geometry& g, const Buffers& b, const StepParams& P, cudaStream_t st) {
  if (g.dim == 2) {
    metric2_step_kernel<<<g.n_tasks, kBlock, 0, st>>>(g.reps, g.tasks, b.bounds, (const int2*)b.S_pos,
                                                      (const float2*)b.S_dir, b.S_id, metric_view(b),
                                                      (int2*)b.U_pos, (float2*)b.U_dir, b.U_id, b.counts,
                                                      b.phi_acc, b.d_step, P);
  } else {
    metric3_step_kernel<<<g.n_tasks, kBlock, 0, st>>>(g.reps, g.tasks, (const int4*)b.S_pos,
                                                      (const float4*)b.S_dir, b.S_id, metric_view(b),
                                                      (int4*)b.U_pos, (float4*)b.U_dir, b.U_id, b.counts,
                                                      b.phi_acc, b.d_step, P);
  }
  return cudaGetLastError();
}

cudaError_t launch_metric_export(const Geometry& g, const Buffers& b, int rep, int n, int pass, int32_t* deg,
                                 const int64_t* out_off, int32_t* out_ids, cudaStream_t st) {
  const int nb = (n + kBlock - 1) / kBlock;
  if (nb == 0) return cudaSuccess;
  if (g.dim == 2) {
    metric2_export_kernel<<<nb, kBlock, 0, st>>>(g.reps, rep, b.bounds, (const int2*)b.S_pos, b.S_id,
                                                 metric_view(b), pass, deg, out_off, out_ids);
  } else {
    metric3_export_kernel<<<nb, kBlock, 0, st>>>(g.reps, rep, (const int4*)b.S_pos, b.S_id, metric_view(b), pass,
                                                 deg, out_off, out_ids);
  }
  return cudaGetLastError();
}

}  // namespace vk
