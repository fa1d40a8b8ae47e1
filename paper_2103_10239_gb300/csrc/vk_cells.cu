// vk_cells.cu -- the cell-list build of the search grid (Sec. "Introduction":
// partition the domain into cells so that only nearby cells are searched;
// stenciled or hierarchical structures for large density disparities):
//   coarse histogram (atomic, fused into the search+update kernel) ->
//   coarse scan, which also picks every coarse cell's sub-grid side ->
//   sub-cell histogram (atomic; the particle's rank in its sub-cell) ->
//   sub-cell scan -> scatter of the state into (coarse, sub-cell) order.
// Also the import/export of user arrays (id order) to and from that layout.
#include "vk_internal.cuh"

namespace vk {

namespace {

// user arrays (row-major, concatenated over replicas) -> U, with validation
template <int DIM>
__global__ void __launch_bounds__(kBlock) load_kernel(const Rep* __restrict__ reps,
                                                      const BlockTask* __restrict__ tasks,
                                                      const int32_t* __restrict__ pos_in,
                                                      const float* __restrict__ head_in, int heading_kind,
                                                      typename Vec<DIM>::P* __restrict__ U_pos,
                                                      typename Vec<DIM>::F* __restrict__ U_dir,
                                                      int32_t* __restrict__ U_id, int32_t* status) {
  using P = typename Vec<DIM>::P;
  using F = typename Vec<DIM>::F;
  const BlockTask t = tasks[blockIdx.x];
  const Rep R = reps[t.rep];
  const int li = t.first + (int)threadIdx.x;
  if (li >= R.n) return;
  const int64_t s = R.p0 + li;
  int32_t p[3] = {0, 0, 0};
  float h[3] = {0.f, 0.f, 0.f};
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    p[a] = pos_in[s * DIM + a];
    if (p[a] < 0 || (uint32_t)p[a] >= R.L[a]) set_status(status, kStRange);
  }
  if (heading_kind == 1) {
    const float th = head_in[s];
    if (!isfinite(th)) set_status(status, kStArg);
    sincosf(th, &h[1], &h[0]);
  } else {
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      h[a] = head_in[s * DIM + a];
      if (!isfinite(h[a])) set_status(status, kStArg);
    }
  }
  U_pos[s] = make_p(p, (P*)nullptr);
  U_dir[s] = make_f(h, (F*)nullptr);
  U_id[s] = li;
}

// coarse histogram of U (the search+update kernel does this for every step)
template <int DIM>
__global__ void __launch_bounds__(kBlock) count_kernel(const Rep* __restrict__ reps,
                                                       const BlockTask* __restrict__ tasks,
                                                       const typename Vec<DIM>::P* __restrict__ U_pos,
                                                       const uint32_t* __restrict__ bounds,
                                                       uint32_t* __restrict__ counts) {
  const BlockTask t = tasks[blockIdx.x];
  const Rep R = reps[t.rep];
  const int li = t.first + (int)threadIdx.x;
  if (li >= R.n) return;
  const int64_t s = R.p0 + li;
  int32_t p[3];
  unpack(U_pos[s], p);
  int c[3] = {0, 0, 0};
#pragma unroll
  for (int a = 0; a < DIM; ++a) c[a] = cell_of_tab((uint32_t)p[a], R.nc[a], bounds + R.bnd[a], R.inv_w[a]);
  int64_t lin = 0;
#pragma unroll
  for (int a = DIM - 1; a >= 0; --a) lin = lin * R.nc[a] + c[a];
  atomicAdd(counts + R.c0 + lin, 1u);
}

// sub-cell histogram of U: the rank of every particle inside its sub-cell
template <int DIM>
__global__ void __launch_bounds__(kBlock) sub_count_kernel(const Rep* __restrict__ reps,
                                                           const BlockTask* __restrict__ tasks,
                                                           const typename Vec<DIM>::P* __restrict__ U_pos,
                                                           const uint32_t* __restrict__ bounds, GridView G,
                                                           uint32_t* __restrict__ sub_count,
                                                           uint32_t* __restrict__ U_rank) {
  const BlockTask t = tasks[blockIdx.x];
  const Rep R = reps[t.rep];
  const int li = t.first + (int)threadIdx.x;
  if (li >= R.n) return;
  const int64_t s = R.p0 + li;
  int32_t p[3];
  unpack(U_pos[s], p);
  int64_t gc, g;
  locate_tab<DIM>(R, G, bounds, p, &gc, &g);
  U_rank[s] = atomicAdd(sub_count + g, 1u);
}

constexpr int kScanItems = 8;
constexpr int kScanTile = kBlock * kScanItems;

__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* total) {
  __shared__ uint32_t warp_tot[kBlock / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[wid] = x;
  __syncthreads();
  if (wid == 0) {
    uint32_t w = lane < kBlock / 32 ? warp_tot[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < kBlock / 32) warp_tot[lane] = w;  // inclusive warp prefix
  }
  __syncthreads();
  const uint32_t before = (wid > 0 ? warp_tot[wid - 1] : 0u) + x - v;
  *total = warp_tot[kBlock / 32 - 1];
  __syncthreads();
  return before;
}

__global__ void __launch_bounds__(kBlock) scan_reduce_kernel(const uint32_t* __restrict__ counts, int64_t n,
                                                             uint32_t* __restrict__ bsum) {
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  uint32_t v = 0;
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) {
    const int64_t c = base + (int64_t)j * kBlock + threadIdx.x;
    if (c < n) v += counts[c];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __shared__ uint32_t w[kBlock / 32];
  if ((threadIdx.x & 31) == 0) w[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t t = 0;
    for (int i = 0; i < kBlock / 32; ++i) t += w[i];
    bsum[blockIdx.x] = t;
  }
}

// one block: exclusive scan of the block sums in place; writes the grand total
__global__ void __launch_bounds__(kBlock) scan_bsum_kernel(uint32_t* __restrict__ bsum, int nb,
                                                           uint32_t* __restrict__ offsets, int64_t n) {
  uint32_t carry = 0;
  for (int base = 0; base < nb; base += kBlock) {
    const int i = base + (int)threadIdx.x;
    const uint32_t v = i < nb ? bsum[i] : 0u;
    uint32_t tot;
    const uint32_t ex = block_exclusive_scan(v, &tot);
    if (i < nb) bsum[i] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0) offsets[n] = carry;
}

// offsets[c] = exclusive prefix of counts; counts are cleared for the next step
__global__ void __launch_bounds__(kBlock) scan_apply_kernel(uint32_t* __restrict__ counts, int64_t n,
                                                            const uint32_t* __restrict__ bsum,
                                                            uint32_t* __restrict__ offsets) {
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  uint32_t v[kScanItems];
  uint32_t tsum = 0;
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) {
    const int64_t c = base + j;
    v[j] = c < n ? counts[c] : 0u;
    tsum += v[j];
  }
  uint32_t tot;
  uint32_t run = bsum[blockIdx.x] + block_exclusive_scan(tsum, &tot);
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) {
    const int64_t c = base + j;
    if (c < n) {
      offsets[c] = run;
      counts[c] = 0u;
    }
    run += v[j];
  }
}

// ---- coarse scan: (count, s^2) pairs -> offsets, sub-grid sides, sub bases
__device__ __forceinline__ uint32_t sub_cells(uint32_t count, int dim) {
  const int s = dim == 2 ? sub_side(count) : 1;
  return (uint32_t)(s * s);
}

__global__ void __launch_bounds__(kBlock) pair_reduce_kernel(const uint32_t* __restrict__ counts, int64_t n,
                                                             int dim, uint2* __restrict__ bsum) {
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  uint32_t v = 0, w = 0;
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) {
    const int64_t c = base + (int64_t)j * kBlock + threadIdx.x;
    if (c < n) {
      const uint32_t m = counts[c];
      v += m;
      w += sub_cells(m, dim);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v += __shfl_xor_sync(0xffffffffu, v, o);
    w += __shfl_xor_sync(0xffffffffu, w, o);
  }
  __shared__ uint2 sw[kBlock / 32];
  if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = make_uint2(v, w);
  __syncthreads();
  if (threadIdx.x == 0) {
    uint2 t = make_uint2(0, 0);
    for (int i = 0; i < kBlock / 32; ++i) {
      t.x += sw[i].x;
      t.y += sw[i].y;
    }
    bsum[blockIdx.x] = t;
  }
}

__global__ void __launch_bounds__(kBlock) pair_bsum_kernel(uint2* __restrict__ bsum, int nb,
                                                           uint32_t* __restrict__ offsets,
                                                           uint32_t* __restrict__ sub_base, int64_t n) {
  uint32_t cv = 0, cw = 0;
  for (int base = 0; base < nb; base += kBlock) {
    const int i = base + (int)threadIdx.x;
    const uint2 v = i < nb ? bsum[i] : make_uint2(0, 0);
    uint32_t tv, tw;
    const uint32_t ev = block_exclusive_scan(v.x, &tv);
    const uint32_t ew = block_exclusive_scan(v.y, &tw);
    if (i < nb) bsum[i] = make_uint2(cv + ev, cw + ew);
    cv += tv;
    cw += tw;
  }
  if (threadIdx.x == 0) {
    offsets[n] = cv;
    sub_base[n] = cw;
  }
}

__global__ void __launch_bounds__(kBlock) pair_apply_kernel(uint32_t* __restrict__ counts, int64_t n, int dim,
                                                            const uint2* __restrict__ bsum,
                                                            uint32_t* __restrict__ offsets,
                                                            uint8_t* __restrict__ sub_s,
                                                            uint32_t* __restrict__ sub_base) {
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  uint32_t v[kScanItems], w[kScanItems];
  uint32_t tv = 0, tw = 0;
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) {
    const int64_t c = base + j;
    v[j] = c < n ? counts[c] : 0u;
    w[j] = c < n ? sub_cells(v[j], dim) : 0u;
    tv += v[j];
    tw += w[j];
  }
  uint32_t totv, totw;
  uint32_t rv = bsum[blockIdx.x].x + block_exclusive_scan(tv, &totv);
  uint32_t rw = bsum[blockIdx.x].y + block_exclusive_scan(tw, &totw);
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) {
    const int64_t c = base + j;
    if (c < n) {
      offsets[c] = rv;
      sub_base[c] = rw;
      sub_s[c] = (uint8_t)(dim == 2 ? sub_side(v[j]) : 1);
      counts[c] = 0u;
    }
    rv += v[j];
    rw += w[j];
  }
}

template <int DIM>
__global__ void __launch_bounds__(kBlock) scatter_kernel(const Rep* __restrict__ reps,
                                                         const BlockTask* __restrict__ tasks,
                                                         const typename Vec<DIM>::P* __restrict__ U_pos,
                                                         const typename Vec<DIM>::F* __restrict__ U_dir,
                                                         const int32_t* __restrict__ U_id,
                                                         const uint32_t* __restrict__ U_rank,
                                                         const uint32_t* __restrict__ bounds, GridView G,
                                                         typename Vec<DIM>::P* __restrict__ S_pos,
                                                         typename Vec<DIM>::F* __restrict__ S_dir,
                                                         int32_t* __restrict__ S_id,
                                                         const float* __restrict__ U_hint,
                                                         float* __restrict__ S_hint,
                                                         int32_t* __restrict__ slot_of, int advance_step,
                                                         int64_t* d_step, PhiAcc* phi_acc, int n_rep,
                                                         int phi_cap, int32_t* ovf_count) {
  const BlockTask t = tasks[blockIdx.x];
  const Rep R = reps[t.rep];
  const int li = t.first + (int)threadIdx.x;
  if (advance_step && blockIdx.x == 0) {
    // clear the order-parameter slot of the next step, then advance the step
    const int64_t nxt = *d_step + 1;
    PhiAcc* slot = phi_acc + (size_t)(nxt % phi_cap) * (size_t)n_rep * 3;
    for (int i = threadIdx.x; i < n_rep * 3; i += blockDim.x) slot[i] = 0ull;
    __syncthreads();
    if (threadIdx.x == 0) {
      *d_step = nxt;
      ovf_count[0] = 0;  // the lists of this step (Voronoi overflow, kNN deferred and walk) are consumed
      ovf_count[1] = 0;
    }
  }
  if (li >= R.n) return;
  const int64_t s = R.p0 + li;
  const typename Vec<DIM>::P pv = U_pos[s];
  int32_t p[3];
  unpack(pv, p);
  int64_t gc, g;
  locate_tab<DIM>(R, G, bounds, p, &gc, &g);
  const uint32_t dst = G.sub_off[g] + U_rank[s];
  S_pos[dst] = pv;
  S_dir[dst] = U_dir[s];
  const int32_t id = U_id[s];
  S_id[dst] = id;
  if (S_hint) S_hint[dst] = U_hint[s];
  if (slot_of) slot_of[R.p0 + id] = (int32_t)dst;
}

template <int DIM>
__global__ void __launch_bounds__(kBlock) export_state_kernel(
    const typename Vec<DIM>::P* __restrict__ S_pos, const typename Vec<DIM>::F* __restrict__ S_dir,
    const int32_t* __restrict__ S_id, int64_t p0, int32_t n, int32_t* __restrict__ pos_out,
    float* __restrict__ dir_out, float* __restrict__ theta_out) {
  const int li = blockIdx.x * kBlock + (int)threadIdx.x;
  if (li >= n) return;
  const int64_t s = p0 + li;
  const int32_t id = S_id[s];
  int32_t p[3];
  float h[3];
  unpack(S_pos[s], p);
  unpack(S_dir[s], h);
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    if (pos_out) pos_out[(int64_t)id * DIM + a] = p[a];
    if (dir_out) dir_out[(int64_t)id * DIM + a] = h[a];
  }
  if (DIM == 2 && theta_out) {
    const float two_pi = 6.28318530717958647692f;
    float th = atan2f(h[1], h[0]);
    if (th < 0.f) th += two_pi;
    if (th >= two_pi) th = 0.f;
    theta_out[id] = th;
  }
}

// user arrays of one replica (id order) -> U slots of that replica
template <int DIM>
__global__ void __launch_bounds__(kBlock) import_state_kernel(
    const int32_t* __restrict__ pos_in, const float* __restrict__ dir_in, int64_t p0, int32_t n,
    const uint32_t* L, typename Vec<DIM>::P* __restrict__ U_pos, typename Vec<DIM>::F* __restrict__ U_dir,
    int32_t* __restrict__ U_id, int32_t* status) {
  using P = typename Vec<DIM>::P;
  using F = typename Vec<DIM>::F;
  const int li = blockIdx.x * kBlock + (int)threadIdx.x;
  if (li >= n) return;
  int32_t p[3] = {0, 0, 0};
  float h[3] = {0.f, 0.f, 0.f};
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    p[a] = pos_in[(int64_t)li * DIM + a];
    h[a] = dir_in[(int64_t)li * DIM + a];
    if (p[a] < 0 || (uint32_t)p[a] >= L[a]) {
      set_status(status, kStRange);
      p[a] = wrap_add(p[a], 0, L[a]);  // keeps the following sort in bounds; the call reports the error
    }
    if (!isfinite(h[a])) set_status(status, kStArg);
  }
  U_pos[p0 + li] = make_p(p, (P*)nullptr);
  U_dir[p0 + li] = make_f(h, (F*)nullptr);
  U_id[p0 + li] = li;
}

// the search hints of one replica, from sorted order into id order (the
// order vk_set_state imports a state in), so that they follow their
// particles through the re-sort
__global__ void __launch_bounds__(kBlock) hints_by_id_kernel(const int32_t* __restrict__ S_id,
                                                             const float* __restrict__ S_hint, int64_t p0, int32_t n,
                                                             float* __restrict__ U_hint) {
  const int li = blockIdx.x * kBlock + (int)threadIdx.x;
  if (li >= n) return;
  const int64_t s = p0 + li;
  U_hint[p0 + S_id[s]] = S_hint[s];
}

}  // namespace

cudaError_t launch_load(const Geometry& g, const Buffers& b, const int32_t* pos_in, const float* head_in,
                        int heading_kind, cudaStream_t st) {
  if (g.dim == 2)
    load_kernel<2><<<g.n_tasks, kBlock, 0, st>>>(g.reps, g.tasks, pos_in, head_in, heading_kind,
                                                  (int2*)b.U_pos, (float2*)b.U_dir, b.U_id, b.d_status);
  else
    load_kernel<3><<<g.n_tasks, kBlock, 0, st>>>(g.reps, g.tasks, pos_in, head_in, heading_kind,
                                                  (int4*)b.U_pos, (float4*)b.U_dir, b.U_id, b.d_status);
  return cudaGetLastError();
}

static GridView grid_view(const Buffers& b) {
  GridView G;
  G.off = b.offsets;
  G.sub_s = b.sub_s;
  G.sub_base = b.sub_base;
  G.sub_off = b.sub_off;
  return G;
}

cudaError_t launch_count(const Geometry& g, const Buffers& b, cudaStream_t st) {
  if (g.dim == 2)
    count_kernel<2><<<g.n_tasks, kBlock, 0, st>>>(g.reps, g.tasks, (const int2*)b.U_pos, b.bounds, b.counts);
  else
    count_kernel<3><<<g.n_tasks, kBlock, 0, st>>>(g.reps, g.tasks, (const int4*)b.U_pos, b.bounds, b.counts);
  return cudaGetLastError();
}

cudaError_t launch_build(const Geometry& g, const Buffers& b, cudaStream_t st) {
  const int nb = (int)((g.n_cells + kScanTile - 1) / kScanTile);
  pair_reduce_kernel<<<nb, kBlock, 0, st>>>(b.counts, g.n_cells, g.dim, (uint2*)b.bsum);
  pair_bsum_kernel<<<1, kBlock, 0, st>>>((uint2*)b.bsum, nb, b.offsets, b.sub_base, g.n_cells);
  pair_apply_kernel<<<nb, kBlock, 0, st>>>(b.counts, g.n_cells, g.dim, (const uint2*)b.bsum, b.offsets, b.sub_s,
                                           b.sub_base);
  const GridView G = grid_view(b);
  if (g.dim == 2)
    sub_count_kernel<2><<<g.n_tasks, kBlock, 0, st>>>(g.reps, g.tasks, (const int2*)b.U_pos, b.bounds, G, b.sub_count,
                                                       b.U_rank);
  else
    sub_count_kernel<3><<<g.n_tasks, kBlock, 0, st>>>(g.reps, g.tasks, (const int4*)b.U_pos, b.bounds, G, b.sub_count,
                                                       b.U_rank);
  const int nb2 = (int)((g.n_sub_max + kScanTile - 1) / kScanTile);
  scan_reduce_kernel<<<nb2, kBlock, 0, st>>>(b.sub_count, g.n_sub_max, b.bsum2);
  scan_bsum_kernel<<<1, kBlock, 0, st>>>(b.bsum2, nb2, b.sub_off, g.n_sub_max);
  scan_apply_kernel<<<nb2, kBlock, 0, st>>>(b.sub_count, g.n_sub_max, b.bsum2, b.sub_off);
  return cudaGetLastError();
}

cudaError_t launch_scatter(const Geometry& g, const Buffers& b, const StepParams& P, int advance_step,
                           cudaStream_t st) {
  const GridView G = grid_view(b);
  if (g.dim == 2)
    scatter_kernel<2><<<g.n_tasks, kBlock, 0, st>>>(
        g.reps, g.tasks, (const int2*)b.U_pos, (const float2*)b.U_dir, b.U_id, b.U_rank, b.bounds, G,
        (int2*)b.S_pos, (float2*)b.S_dir, b.S_id, b.U_hint, b.S_hint, b.slot_of, advance_step, b.d_step, b.phi_acc,
        P.n_rep, P.phi_cap, b.ovf_count);
  else
    scatter_kernel<3><<<g.n_tasks, kBlock, 0, st>>>(
        g.reps, g.tasks, (const int4*)b.U_pos, (const float4*)b.U_dir, b.U_id, b.U_rank, b.bounds, G,
        (int4*)b.S_pos, (float4*)b.S_dir, b.S_id, b.U_hint, b.S_hint, nullptr, advance_step, b.d_step, b.phi_acc,
        P.n_rep, P.phi_cap, b.ovf_count);
  return cudaGetLastError();
}

cudaError_t launch_export_state(const Geometry& g, const Buffers& b, int rep, int64_t p0, int32_t n,
                                int32_t* pos_out, float* dir_out, float* theta_out, cudaStream_t st) {
  (void)rep;
  const int nb = (n + kBlock - 1) / kBlock;
  if (nb == 0) return cudaSuccess;
  if (g.dim == 2)
    export_state_kernel<2><<<nb, kBlock, 0, st>>>((const int2*)b.S_pos, (const float2*)b.S_dir, b.S_id, p0, n,
                                                   pos_out, dir_out, theta_out);
  else
    export_state_kernel<3><<<nb, kBlock, 0, st>>>((const int4*)b.S_pos, (const float4*)b.S_dir, b.S_id, p0, n,
                                                   pos_out, dir_out, theta_out);
  return cudaGetLastError();
}

cudaError_t launch_import_state(const Geometry& g, const Buffers& b, int rep, int64_t p0, int32_t n,
                                const int32_t* pos_in, const float* dir_in, cudaStream_t st) {
  const int nb = (n + kBlock - 1) / kBlock;
  if (nb == 0) return cudaSuccess;
  const uint32_t* L = reinterpret_cast<const uint32_t*>(reinterpret_cast<const char*>(g.reps + rep) +
                                                        offsetof(Rep, L));
  if (g.dim == 2)
    import_state_kernel<2><<<nb, kBlock, 0, st>>>(pos_in, dir_in, p0, n, L, (int2*)b.U_pos, (float2*)b.U_dir,
                                                   b.U_id, b.d_status);
  else
    import_state_kernel<3><<<nb, kBlock, 0, st>>>(pos_in, dir_in, p0, n, L, (int4*)b.U_pos, (float4*)b.U_dir,
                                                   b.U_id, b.d_status);
  return cudaGetLastError();
}

cudaError_t launch_hints_by_id(const Buffers& b, int64_t p0, int32_t n, cudaStream_t st) {
  if (!b.S_hint || n == 0) return cudaSuccess;
  hints_by_id_kernel<<<(n + kBlock - 1) / kBlock, kBlock, 0, st>>>(b.S_id, b.S_hint, p0, n, b.U_hint);
  return cudaGetLastError();
}

}  // namespace vk
