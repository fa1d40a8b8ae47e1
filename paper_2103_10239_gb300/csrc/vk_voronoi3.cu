// vk_voronoi3.cu -- Voronoi-neighbor rule in 3D (Sec. "Computational tools:
// Voronoi neighbor lists": neighbors are the particles whose Voronoi cells
// share a face; the relation is reciprocal) fused with the Vicsek update of
// Eq. (1) and Eq. (2) (vectorial noise, as every 3D rule here).
//
// The cell starts as the box bounded by the particle's own periodic images
// and is clipped by the bisector planes of the candidates that the ring walk
// of the uniform 3D grid delivers (vk_voronoi3.cuh: exact predicates, dual
// triangulation).  A site at offset d can cut the cell only if |d| < 2R, R the
// distance of the farthest vertex, so the walk stops once the scanned block
// holds that ball.  When 2R reaches a quarter of the box, non-minimum images
// of other particles can cut too: the cell is then finished against every
// image of every particle within 2R.  Neighbors are the sites of faces of
// positive area, in id order.  Coincident particles latch VK_ERR_DEGENERATE
// (no cell separates them).
//
// Two kernels build the cells, with the same results:
//   * voronoi3_step_kernel (the default): one thread per particle, in
//     cell-sorted order, the cell in thread-local memory;
//   * voronoi3_warp_kernel: one warp per particle, the cell in shared memory,
//     vertex tests and vertex solves spread over the lanes.
// Cells whose intermediate polytope outgrows either are rebuilt by
// voronoi3_overflow_kernel with room for 128 faces and 256 vertices.
#include <algorithm>

#include "vk_internal.cuh"
#include "vk_voronoi3.cuh"
#include "vk_voronoi3_api.cuh"

namespace vk {

namespace {

// the main kernel's cells (about 15.5 faces and 27 vertices on average for
// uniform points) and the overflow kernel's, for the rare cell whose
// intermediate polytope outgrows the first
using CellS = v3::Cell<64, 128>;
using CellL = v3::Cell<128, 256>;

constexpr int kMaxImages = 64;

// the cell of the particle at sorted slot `self` (replica R); false when
// the build failed (C.status says why)
template <class Cell>
__device__ bool voronoi3_cell(const Rep& R, int64_t self, const int32_t* pi, const int4* __restrict__ S_pos,
                              const GridView& G, Cell& C, int8_t* sg, uint32_t* n_cand) {
  v3::cell_init(C, R.L, sg);
  auto clip = [&](int64_t q, const int32_t* d) {
    if (d[0] == 0 && d[1] == 0 && d[2] == 0) {
      C.status = v3::kCoincident;
      return;
    }
    v3::cell_clip(C, d, (int32_t)q, sg);
  };
  auto run = [&](uint32_t qb, uint32_t qe) {
    if (C.status != v3::kOk) return;
    *n_cand += qe - qb;
    for (uint32_t q = qb; q < qe && C.status == v3::kOk; ++q) {
      if ((int64_t)q == self) continue;
      const int4 pj = __ldg(S_pos + q);
      const int32_t d[3] = {(int32_t)min_image((int64_t)pj.x - pi[0], (int64_t)R.L[0]),
                            (int32_t)min_image((int64_t)pj.y - pi[1], (int64_t)R.L[1]),
                            (int32_t)min_image((int64_t)pj.z - pi[2], (int64_t)R.L[2])};
      clip(q, d);
    }
  };
  // every unscanned site is at squared distance >= B2; none can cut once
  // B2 >= 4 R^2 (the FP32 B2 is lowered by 2^-22 to stay below the exact value)
  auto stop = [&](uint64_t B2) { return C.status != v3::kOk || (float)B2 * 0.99999976f >= 4.f * C.r2; };
  grid_walk3(R, pi, G, run, stop);
  if (C.status != v3::kOk) return false;
  // other images lie at >= L_min / 2: they matter only when 2R > L_min / 2
  const float Lmin = (float)min(R.L[0], min(R.L[1], R.L[2]));
  if (16.f * C.r2 > Lmin * Lmin) {
    for (int32_t lj = 0; lj < R.n && C.status == v3::kOk; ++lj) {
      const int64_t q = R.p0 + lj;
      if (q == self) continue;
      const int4 pj = __ldg(S_pos + q);
      const int64_t d0[3] = {min_image((int64_t)pj.x - pi[0], (int64_t)R.L[0]),
                             min_image((int64_t)pj.y - pi[1], (int64_t)R.L[1]),
                             min_image((int64_t)pj.z - pi[2], (int64_t)R.L[2])};
      const float Rr = sqrtf(C.r2);
      int K[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const float k = floorf((2.f * Rr + 0.5f * (float)R.L[a]) / (float)R.L[a]) + 1.f;
        // more than kMaxImages images per axis (a box far longer than wide
        // holding a handful of particles) is outside the supported range
        if (!(k <= (float)kMaxImages)) {
          C.status = v3::kCapacity;
          return false;
        }
        K[a] = (int)k;
      }
      for (int kx = -K[0]; kx <= K[0]; ++kx)
        for (int ky = -K[1]; ky <= K[1]; ++ky)
          for (int kz = -K[2]; kz <= K[2] && C.status == v3::kOk; ++kz) {
            const int32_t d[3] = {(int32_t)(d0[0] + (int64_t)kx * R.L[0]), (int32_t)(d0[1] + (int64_t)ky * R.L[1]),
                                  (int32_t)(d0[2] + (int64_t)kz * R.L[2])};
            clip(q, d);
          }
    }
  }
  return C.status == v3::kOk;
}

__device__ __forceinline__ int32_t status_of(int st) {
  return st == v3::kCoincident ? kStDegenerate : kStCapacity;
}

// neighbor ids (sorted, each once) and their slots; returns the count.
// is_face(p): the face of live site plane p has positive area
template <class Cell, class IsFace>
__device__ int voronoi3_neighbors(const Cell& C, const int32_t* __restrict__ S_id, int32_t* nid, int32_t* nslot,
                                  IsFace is_face) {
  int cnt = 0;
  for (int p = 0; p < C.np; ++p) {
    if (C.pref[p] == 0 || C.pslot[p] < 0 || !is_face(p)) continue;
    const int32_t id = __ldg(S_id + C.pslot[p]);
    int j = cnt;
    while (j > 0 && nid[j - 1] > id) {
      nid[j] = nid[j - 1];
      nslot[j] = nslot[j - 1];
      --j;
    }
    if (j > 0 && nid[j - 1] == id) {  // another image of a site already listed
      for (int t = j; t < cnt; ++t) {
        nid[t] = nid[t + 1];
        nslot[t] = nslot[t + 1];
      }
      continue;
    }
    nid[j] = id;
    nslot[j] = C.pslot[p];
    ++cnt;
  }
  return cnt;
}

constexpr int kV3Block = 128;
constexpr int kV3Split = kBlock / kV3Block;

// Eq. (2) + Eq. (1) for one particle from its finished cell; writes the next
// state and counts its new grid cell
template <class Cell, class IsFace>
__device__ __forceinline__ void voronoi3_update(const Rep& R, const StepParams& Pm, int64_t step, int64_t s,
                                                const Cell& C, const int32_t* pi, const float* ni, int32_t id,
                                                const int32_t* __restrict__ S_id, const float4* __restrict__ S_dir,
                                                int4* __restrict__ U_pos, float4* __restrict__ U_dir,
                                                int32_t* __restrict__ U_id, uint32_t* __restrict__ counts,
                                                float* nnew, IsFace is_face) {
  int32_t nid[Cell::P], nslot[Cell::P];
  const int cnt = voronoi3_neighbors(C, S_id, nid, nslot, is_face);
  HeadSum<3> H;
  H.init();
  if (Pm.include_self) H.add(ni, Pm.sum_mode);
  for (int j = 0; j < cnt; ++j) {
    const float4 d = __ldg(S_dir + nslot[j]);
    const float v[3] = {d.x, d.y, d.z};
    H.add(v, Pm.sum_mode);
  }
  int32_t pout[3];
  align_advect<3>(R, Pm, (uint32_t)step, id, ni, H, cnt + (Pm.include_self ? 1 : 0), pi, pout, nnew);
  U_pos[s] = make_int4(pout[0], pout[1], pout[2], 0);
  U_dir[s] = make_float4(nnew[0], nnew[1], nnew[2], 0.f);
  U_id[s] = id;
  atomicAdd(counts + linear_cell<3>(R, pout), 1u);
}

// a particle whose cell could not be built: the state is carried over
// unchanged and the status latched (the host reports it)
__device__ __forceinline__ void voronoi3_keep(const Rep& R, int64_t s, const int32_t* pi, const float* ni,
                                              int32_t id, int st, int32_t* status, int4* __restrict__ U_pos,
                                              float4* __restrict__ U_dir, int32_t* __restrict__ U_id,
                                              uint32_t* __restrict__ counts, float* nnew) {
  set_status(status, status_of(st));
  nnew[0] = ni[0];
  nnew[1] = ni[1];
  nnew[2] = ni[2];
  U_pos[s] = make_int4(pi[0], pi[1], pi[2], 0);
  U_dir[s] = make_float4(ni[0], ni[1], ni[2], 0.f);
  U_id[s] = id;
  atomicAdd(counts + linear_cell<3>(R, pi), 1u);
}

__global__ void __launch_bounds__(kV3Block) voronoi3_step_kernel(
    const Rep* __restrict__ reps, const BlockTask* __restrict__ tasks, const int4* __restrict__ S_pos,
    const float4* __restrict__ S_dir, const int32_t* __restrict__ S_id, GridView G, int4* __restrict__ U_pos,
    float4* __restrict__ U_dir, int32_t* __restrict__ U_id, uint32_t* __restrict__ counts,
    PhiAcc* __restrict__ phi_acc, const int64_t* __restrict__ d_step, StepParams Pm, int32_t* status,
    int2* __restrict__ ovf_list, int32_t* __restrict__ ovf_count) {
  __shared__ PhiShared phs;
  phi_block_begin(phs);
  const BlockTask t = tasks[blockIdx.x / kV3Split];
  const Rep R = reps[t.rep];
  const int li = t.first + (int)(blockIdx.x % kV3Split) * kV3Block + (int)threadIdx.x;
  const int64_t step = *d_step;
  float nnew[3] = {0.f, 0.f, 0.f};
  uint32_t n_cand = 0;
  if (li < R.n) {
    const int64_t s = R.p0 + li;
    const int4 p = S_pos[s];
    const float4 nv = S_dir[s];
    const int32_t pi[3] = {p.x, p.y, p.z};
    const float ni[3] = {nv.x, nv.y, nv.z};
    const int32_t id = S_id[s];
    CellS C;
    int8_t sg[CellS::T];
    if (voronoi3_cell(R, s, pi, S_pos, G, C, sg, &n_cand)) {
      voronoi3_update(R, Pm, step, s, C, pi, ni, id, S_id, S_dir, U_pos, U_dir, U_id, counts, nnew,
                      [&](int p) { return v3::face_positive(C, p); });
    } else if (C.status == v3::kCapacity) {
      // finished by the overflow kernel (its heading enters phi there)
      const int q = atomicAdd(ovf_count, 1);
      ovf_list[q] = make_int2((int)s, t.rep);
    } else {
      voronoi3_keep(R, s, pi, ni, id, C.status, status, U_pos, U_dir, U_id, counts, nnew);
    }
  }
  record_search_stats(Pm.stats, li < R.n, n_cand, 0);
  phi_block_end<3>(phs, nnew, phi_acc + ((size_t)(step % Pm.phi_cap) * (size_t)Pm.n_rep + (size_t)t.rep) * 3);
}

// Overflow kernel: the particles whose intermediate cell outgrew CellS, one
// thread each with the larger cell.
constexpr int kV3OvfBlock = 64;

__global__ void __launch_bounds__(kV3OvfBlock) voronoi3_overflow_kernel(
    const Rep* __restrict__ reps, const int4* __restrict__ S_pos, const float4* __restrict__ S_dir,
    const int32_t* __restrict__ S_id, GridView G, int4* __restrict__ U_pos, float4* __restrict__ U_dir,
    int32_t* __restrict__ U_id, uint32_t* __restrict__ counts, PhiAcc* __restrict__ phi_acc,
    const int64_t* __restrict__ d_step, StepParams Pm, int32_t* status, const int2* __restrict__ ovf_list,
    const int32_t* __restrict__ ovf_count) {
  const int total = *ovf_count;
  const int64_t step = *d_step;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < total; q += gridDim.x * blockDim.x) {
    const int2 e = ovf_list[q];
    const Rep R = reps[e.y];
    const int64_t s = e.x;
    const int4 p = S_pos[s];
    const float4 nv = S_dir[s];
    const int32_t pi[3] = {p.x, p.y, p.z};
    const float ni[3] = {nv.x, nv.y, nv.z};
    const int32_t id = S_id[s];
    CellL C;
    int8_t sg[CellL::T];
    uint32_t n_cand = 0;
    float nnew[3];
    if (voronoi3_cell(R, s, pi, S_pos, G, C, sg, &n_cand))
      voronoi3_update(R, Pm, step, s, C, pi, ni, id, S_id, S_dir, U_pos, U_dir, U_id, counts, nnew,
                      [&](int p) { return v3::face_positive(C, p); });
    else
      voronoi3_keep(R, s, pi, ni, id, C.status, status, U_pos, U_dir, U_id, counts, nnew);
    PhiAcc* acc = phi_acc + ((size_t)(step % Pm.phi_cap) * (size_t)Pm.n_rep + (size_t)e.y) * 3;
#pragma unroll
    for (int a = 0; a < 3; ++a) atomicAdd(acc + a, (PhiAcc)phi_fixed(nnew[a]));
  }
}

// ---------------------------------------------------------------------------
// One warp per cell.  The cell lives in shared memory; the lanes test the
// vertices against a candidate plane in parallel and solve the new vertices
// of a clip in parallel, while lane 0 rewires the triangulation (the cheap
// part, clip_topology).  Candidates arrive from the same ring walk, 32 at a
// time, one load per lane.  Warps take particles from a work counter, so the
// slow cells of void rims do not hold back a block.  Results are the same as
// the one-thread-per-cell kernel's: the same exact predicates decide, and
// the neighbors do not depend on the order of the clips.
// ---------------------------------------------------------------------------
constexpr int kV3WarpsPerBlock = 4;

struct WarpCell {
  CellS C;
  int8_t sg[CellS::T];
  uint8_t bt[CellS::B];
  uint8_t face[CellS::P];
  int nb;
};

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// clip W.C by the plane at offset d (site slot `slot`); every lane calls it
__device__ void warp_clip(WarpCell& W, const int32_t* d, int32_t slot, int lane) {
  CellS& C = W.C;
  const int64_t w = v3::norm2(d);
  const float wf = (float)w;
  if (wf >= 4.f * C.r2) return;  // |d| / 2 beyond every vertex: cannot cut
  const float band = v3::side_band(C, wf);
  bool any = false;
  for (int t = lane; t < C.nt; t += 32) {
    if (C.ty[t][3] == 0.f) continue;
    const bool out = v3::side_of(C, t, d, wf, band) > 0;
    W.sg[t] = (int8_t)out;
    any = any || out;
  }
  if (!__any_sync(0xffffffffu, any)) return;
  __syncwarp();
  if (lane == 0) {
    int nb = 0;
    v3::clip_topology(C, d, slot, W.sg, W.bt, &nb);
    W.nb = nb;
  }
  __syncwarp();
  if (C.status != v3::kOk) return;
  for (int j = lane; j < W.nb; j += 32) v3::vertex_of(C, W.bt[j]);
  __syncwarp();
  float m = 0.f;
  for (int t = lane; t < C.nt; t += 32) {
    if (C.ty[t][3] == 0.f) continue;
    m = fmaxf(m, C.ty[t][0] * C.ty[t][0] + C.ty[t][1] * C.ty[t][1] + C.ty[t][2] * C.ty[t][2]);
  }
  m = warp_max(m);
  if (lane == 0) {  // as refresh_radius
    C.r2 = 0.25f * m * (1.f + 3.8147e-6f) + 1.f;
    C.ymax = sqrtf(m) * (1.f + 3.8147e-6f) + 1.f;
  }
  __syncwarp();
}

// the cell of the particle at sorted slot `self`, built by the whole warp;
// the same walk and the same small-box pass as voronoi3_cell
__device__ bool voronoi3_cell_warp(const Rep& R, int64_t self, const int32_t* pi, const int4* __restrict__ S_pos,
                                   const GridView& G, WarpCell& W, int lane, uint32_t* n_cand) {
  CellS& C = W.C;
  if (lane == 0) v3::cell_init(C, R.L, W.sg);
  __syncwarp();
  auto run = [&](uint32_t qb, uint32_t qe) {
    *n_cand += qe - qb;
    for (uint32_t base = qb; base < qe; base += 32) {
      if (C.status != v3::kOk) return;
      const uint32_t q = base + (uint32_t)lane;
      const bool valid = q < qe && (int64_t)q != self;
      int32_t d[3] = {0, 0, 0};
      if (valid) {
        const int4 pj = __ldg(S_pos + q);
        d[0] = (int32_t)min_image((int64_t)pj.x - pi[0], (int64_t)R.L[0]);
        d[1] = (int32_t)min_image((int64_t)pj.y - pi[1], (int64_t)R.L[1]);
        d[2] = (int32_t)min_image((int64_t)pj.z - pi[2], (int64_t)R.L[2]);
      }
      if (__any_sync(0xffffffffu, valid && d[0] == 0 && d[1] == 0 && d[2] == 0)) {
        if (lane == 0) C.status = v3::kCoincident;
        __syncwarp();
        return;
      }
      unsigned mask = __ballot_sync(0xffffffffu, valid);
      while (mask) {
        const int src = __ffs(mask) - 1;
        mask &= mask - 1u;
        const int32_t dd[3] = {__shfl_sync(0xffffffffu, d[0], src), __shfl_sync(0xffffffffu, d[1], src),
                               __shfl_sync(0xffffffffu, d[2], src)};
        warp_clip(W, dd, (int32_t)(base + (uint32_t)src), lane);
        if (C.status != v3::kOk) return;
      }
    }
  };
  auto stop = [&](uint64_t B2) { return C.status != v3::kOk || (float)B2 * 0.99999976f >= 4.f * C.r2; };
  grid_walk3(R, pi, G, run, stop);
  if (C.status != v3::kOk) return false;
  const float Lmin = (float)min(R.L[0], min(R.L[1], R.L[2]));
  if (16.f * C.r2 > Lmin * Lmin) {
    // tiny systems: lane 0 finishes the cell against every image within 2R
    if (lane == 0) {
      for (int32_t lj = 0; lj < R.n && C.status == v3::kOk; ++lj) {
        const int64_t q = R.p0 + lj;
        if (q == self) continue;
        const int4 pj = __ldg(S_pos + q);
        const int64_t d0[3] = {min_image((int64_t)pj.x - pi[0], (int64_t)R.L[0]),
                               min_image((int64_t)pj.y - pi[1], (int64_t)R.L[1]),
                               min_image((int64_t)pj.z - pi[2], (int64_t)R.L[2])};
        const float Rr = sqrtf(C.r2);
        int K[3];
        bool too_many = false;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          const float k = floorf((2.f * Rr + 0.5f * (float)R.L[a]) / (float)R.L[a]) + 1.f;
          too_many = too_many || !(k <= (float)kMaxImages);
          K[a] = too_many ? 0 : (int)k;
        }
        if (too_many) {
          C.status = v3::kCapacity;
          break;
        }
        for (int kx = -K[0]; kx <= K[0]; ++kx)
          for (int ky = -K[1]; ky <= K[1]; ++ky)
            for (int kz = -K[2]; kz <= K[2] && C.status == v3::kOk; ++kz) {
              const int32_t d[3] = {(int32_t)(d0[0] + (int64_t)kx * R.L[0]),
                                    (int32_t)(d0[1] + (int64_t)ky * R.L[1]),
                                    (int32_t)(d0[2] + (int64_t)kz * R.L[2])};
              if (d[0] == 0 && d[1] == 0 && d[2] == 0) C.status = v3::kCoincident;
              else v3::cell_clip(C, d, (int32_t)q, W.sg);
            }
      }
    }
    __syncwarp();
  }
  return C.status == v3::kOk;
}

__global__ void __launch_bounds__(32 * kV3WarpsPerBlock, 6) voronoi3_warp_kernel(
    const Rep* __restrict__ reps, const BlockTask* __restrict__ tasks, int n_items, const int4* __restrict__ S_pos,
    const float4* __restrict__ S_dir, const int32_t* __restrict__ S_id, GridView G, int4* __restrict__ U_pos,
    float4* __restrict__ U_dir, int32_t* __restrict__ U_id, uint32_t* __restrict__ counts,
    PhiAcc* __restrict__ phi_acc, const int64_t* __restrict__ d_step, StepParams Pm, int32_t* status,
    int2* __restrict__ ovf_list, int32_t* __restrict__ ovf_count, int32_t* __restrict__ work) {
  __shared__ WarpCell cells[kV3WarpsPerBlock];
  WarpCell& W = cells[threadIdx.x >> 5];
  const int lane = (int)(threadIdx.x & 31);
  const int64_t step = *d_step;
  for (;;) {
    int item = 0;
    if (lane == 0) item = atomicAdd(work, 1);
    item = __shfl_sync(0xffffffffu, item, 0);
    if (item >= n_items) break;
    const BlockTask t = tasks[item / kBlock];
    const Rep R = reps[t.rep];
    const int li = t.first + item % kBlock;
    if (li >= R.n) continue;
    const int64_t s = R.p0 + li;
    const int4 p = S_pos[s];
    const int32_t pi[3] = {p.x, p.y, p.z};
    uint32_t n_cand = 0;
    const bool ok = voronoi3_cell_warp(R, s, pi, S_pos, G, W, lane, &n_cand);
    if (ok) {
      for (int q = lane; q < W.C.np; q += 32)
        W.face[q] = (uint8_t)(W.C.pref[q] > 0 && W.C.pslot[q] >= 0 && v3::face_positive(W.C, q));
      __syncwarp();
    }
    if (lane == 0) {
      const float4 nv = S_dir[s];
      const float ni[3] = {nv.x, nv.y, nv.z};
      const int32_t id = S_id[s];
      float nnew[3];
      if (ok) {
        voronoi3_update(R, Pm, step, s, W.C, pi, ni, id, S_id, S_dir, U_pos, U_dir, U_id, counts, nnew,
                        [&](int q) { return W.face[q] != 0; });
      } else if (W.C.status == v3::kCapacity) {
        const int q = atomicAdd(ovf_count, 1);  // the overflow kernel adds its heading to phi
        ovf_list[q] = make_int2((int)s, t.rep);
      } else {
        voronoi3_keep(R, s, pi, ni, id, W.C.status, status, U_pos, U_dir, U_id, counts, nnew);
      }
      if (ok || W.C.status != v3::kCapacity) {
        PhiAcc* acc = phi_acc + ((size_t)(step % Pm.phi_cap) * (size_t)Pm.n_rep + (size_t)t.rep) * 3;
#pragma unroll
        for (int a = 0; a < 3; ++a) atomicAdd(acc + a, (PhiAcc)phi_fixed(nnew[a]));
      }
    }
    if (Pm.stats && lane == 0) {
      atomicAdd(Pm.stats + 0, (unsigned long long)n_cand);
      atomicMax(Pm.stats + 2, (unsigned long long)n_cand);
      atomicAdd(Pm.stats + 3, 1ull);
    }
    __syncwarp();
  }
}

// Export (not on the hot path): pass 0 writes the degree of every particle
// (by id), pass 1 the sorted ids at out_off[id].
__global__ void __launch_bounds__(kV3Block) voronoi3_export_kernel(
    const Rep* __restrict__ reps, int rep, const int4* __restrict__ S_pos, const int32_t* __restrict__ S_id,
    GridView G, int pass, int32_t* __restrict__ deg, const int64_t* __restrict__ out_off,
    int32_t* __restrict__ out_ids, int32_t* status) {
  const Rep R = reps[rep];
  for (int li = blockIdx.x * blockDim.x + threadIdx.x; li < R.n; li += gridDim.x * blockDim.x) {
    const int64_t s = R.p0 + li;
    const int4 p = S_pos[s];
    const int32_t pi[3] = {p.x, p.y, p.z};
    const int32_t id = S_id[s];
    CellL C;
    int8_t sg[CellL::T];
    uint32_t n_cand = 0;
    if (!voronoi3_cell(R, s, pi, S_pos, G, C, sg, &n_cand)) {
      set_status(status, status_of(C.status));
      if (pass == 0) deg[id] = 0;
      continue;
    }
    int32_t nid[CellL::P], nslot[CellL::P];
    const int cnt = voronoi3_neighbors(C, S_id, nid, nslot, [&](int p) { return v3::face_positive(C, p); });
    if (pass == 0) {
      deg[id] = cnt;
    } else {
      const int64_t o = out_off[id];
      for (int j = 0; j < cnt; ++j) out_ids[o + j] = nid[j];
    }
  }
}

GridView grid_view3(const Buffers& b) {
  GridView G;
  G.off = b.offsets;
  G.sub_s = b.sub_s;
  G.sub_base = b.sub_base;
  G.sub_off = b.sub_off;
  return G;
}

}  // namespace

cudaError_t launch_voronoi3_step(const Geometry& g, const Buffers& b, const StepParams& P, int warp,
                                 cudaStream_t st) {
  if (warp) {
    // persistent: as many blocks as fit at once; warps take particles from
    // the work counter (ovf_count[1], cleared by every scatter)
    // (initialised once, thread-safely; one block per SM if the query fails)
    static const int per_sm = [] {
      int blocks = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, voronoi3_warp_kernel, 32 * kV3WarpsPerBlock, 0) !=
          cudaSuccess)
        blocks = 1;
      return std::max(blocks, 1);
    }();
    voronoi3_warp_kernel<<<device_sm_count() * per_sm, 32 * kV3WarpsPerBlock, 0, st>>>(
        g.reps, g.tasks, g.n_tasks * kBlock, (const int4*)b.S_pos, (const float4*)b.S_dir, b.S_id, grid_view3(b),
        (int4*)b.U_pos, (float4*)b.U_dir, b.U_id, b.counts, b.phi_acc, b.d_step, P, b.d_status, b.ovf_list,
        b.ovf_count, b.ovf_count + 1);
  } else {
  voronoi3_step_kernel<<<g.n_tasks * kV3Split, kV3Block, 0, st>>>(
      g.reps, g.tasks, (const int4*)b.S_pos, (const float4*)b.S_dir, b.S_id, grid_view3(b), (int4*)b.U_pos,
      (float4*)b.U_dir, b.U_id, b.counts, b.phi_acc, b.d_step, P, b.d_status, b.ovf_list, b.ovf_count);
  }
  voronoi3_overflow_kernel<<<device_sm_count(), kV3OvfBlock, 0, st>>>(
      g.reps, (const int4*)b.S_pos, (const float4*)b.S_dir, b.S_id, grid_view3(b), (int4*)b.U_pos,
      (float4*)b.U_dir, b.U_id, b.counts, b.phi_acc, b.d_step, P, b.d_status, b.ovf_list, b.ovf_count);
  return cudaGetLastError();
}

cudaError_t launch_voronoi3_export(const Geometry& g, const Buffers& b, int rep, int n, int pass, int32_t* deg,
                                   const int64_t* out_off, int32_t* out_ids, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  const int nb = std::min((n + kV3Block - 1) / kV3Block, device_sm_count() * 8);
  voronoi3_export_kernel<<<nb, kV3Block, 0, st>>>(g.reps, rep, (const int4*)b.S_pos, b.S_id, grid_view3(b), pass,
                                                  deg, out_off, out_ids, b.d_status);
  return cudaGetLastError();
}

}  // namespace vk
