// vk_internal.cuh -- device-side building blocks shared by the libvk_nm kernels.
//
// Data layout (HBM, all replicas concatenated):
//   * particle state in cell-sorted order (the "S" buffers): position as
//     int2 (2D) / int4 (3D, w unused), heading as float2 / float4, replica-local
//     id as int32;
//   * the "U" buffers hold the next state in the order of S (written by the
//     search+update kernel), plus the rank of each particle inside its new cell;
//   * counts[c] / offsets[c] over the concatenated cells of all replicas; an
//     exclusive scan of the counts gives global slot offsets directly;
//   * a per-replica table (Rep) and a per-block task table (BlockTask), so a
//     256-thread block never straddles two replicas.
#pragma once
#include <cstdint>
#include <climits>
#include <cuda_runtime.h>

namespace vk {

constexpr int kBlock = 256;
constexpr int kMaxK = 32;

// device status codes (same values as vk_status)
enum : int32_t {
  kStOk = 0,
  kStCapacity = 4,
  kStRange = 5,
  kStDegenerate = 6,
  kStArg = 1,
};

struct Rep {
  int64_t p0;      // first slot of the replica in the particle arrays
  int64_t c0;      // first cell of the replica in counts / offsets
  int32_t n;       // particles
  int32_t nc[3];   // cells per axis
  uint32_t L[3];   // box edge per axis (grid units)
  float eta;       // noise strength
  float s;         // grid units per unit heading and step: fl32(v0*dt) * 2^F
  uint32_t replica;
  int32_t bnd[3];  // offset of the axis' cell-boundary table in the bounds array
  float inv_w[3];  // nc / L (estimate of the cell index; corrected exactly)
  uint32_t r0q;    // metric rule: interaction radius in grid units, rint(r0 * 2^F)
};

struct BlockTask {
  int32_t rep;
  int32_t first;  // replica-local index of the block's first particle
};

constexpr int32_t kViewAll = INT_MIN;  // fov_cq of the full circle (the plain kNN rule)

struct StepParams {
  int32_t k;
  int32_t noise;         // 0 angular, 1 vectorial
  int32_t include_self;
  int32_t advect_new;
  int32_t sum_mode;      // 0 plain, 1 compensated, 2 fp64
  uint32_t seed_lo, seed_hi;
  int32_t n_rep;
  int32_t phi_cap;
  // 2D kNN search: 0 = radius first (per-particle walk as the last resort),
  // 1 = per-particle walk only
  int32_t knn_search;
  // radius-first search square: halo_alpha * (the particle's k-th distance at
  // the previous step) + halo_beta * (grid step per unit heading)
  float halo_alpha, halo_beta;
  // 2D kNN field of view: the cosine of the half-angle in 2^-24 units, or
  // INT_MIN for the full circle (the plain rule)
  int32_t fov_cq;
  // tracing only (NULL = off): [candidates, runs or squares, max candidates,
  // particles, particles whose own coarse cell is split (walk) or that fell
  // back to the walk (radius first), then radius first only: squares, runs,
  // candidates, coarse cells, hits]
  unsigned long long* stats;
};

// Tracing: add one particle's search counters to the global totals.
__device__ __forceinline__ void record_search_stats(unsigned long long* stats, bool valid, uint32_t cand,
                                                    uint32_t runs, bool split = false) {
  if (!stats) return;
  unsigned long long c = valid ? cand : 0, r = valid ? runs : 0, n = valid ? 1 : 0;
  unsigned long long mx = c, sp = (valid && split) ? 1 : 0;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    c += __shfl_xor_sync(0xffffffffu, c, o);
    r += __shfl_xor_sync(0xffffffffu, r, o);
    n += __shfl_xor_sync(0xffffffffu, n, o);
    sp += __shfl_xor_sync(0xffffffffu, sp, o);
    mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  }
  if ((threadIdx.x & 31) == 0 && n) {
    atomicAdd(stats + 0, c);
    atomicAdd(stats + 1, r);
    atomicMax(stats + 2, mx);
    atomicAdd(stats + 3, n);
    atomicAdd(stats + 4, sp);
  }
}

template <int DIM> struct Vec;
template <> struct Vec<2> { using P = int2; using F = float2; };
template <> struct Vec<3> { using P = int4; using F = float4; };

template <int DIM> __device__ __forceinline__ int32_t comp(const typename Vec<DIM>::P& p, int a) {
  return a == 0 ? p.x : (a == 1 ? p.y : reinterpret_cast<const int4&>(p).z);
}

__device__ __forceinline__ int2 make_p(const int32_t* v, int2*) { return make_int2(v[0], v[1]); }
__device__ __forceinline__ int4 make_p(const int32_t* v, int4*) { return make_int4(v[0], v[1], v[2], 0); }
__device__ __forceinline__ float2 make_f(const float* v, float2*) { return make_float2(v[0], v[1]); }
__device__ __forceinline__ float4 make_f(const float* v, float4*) { return make_float4(v[0], v[1], v[2], 0.f); }
__device__ __forceinline__ void unpack(const int2& p, int32_t* v) { v[0] = p.x; v[1] = p.y; }
__device__ __forceinline__ void unpack(const int4& p, int32_t* v) { v[0] = p.x; v[1] = p.y; v[2] = p.z; }
__device__ __forceinline__ void unpack(const float2& p, float* v) { v[0] = p.x; v[1] = p.y; }
__device__ __forceinline__ void unpack(const float4& p, float* v) { v[0] = p.x; v[1] = p.y; v[2] = p.z; }

// --------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11), written for the device.
// --------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k.x += 0x9E3779B9u;
      k.y += 0xBB67AE85u;
    }
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

__device__ __forceinline__ float unit24(uint32_t w) {
  return (float)(w >> 8) * 5.9604644775390625e-08f;  // exact: 24-bit integer * 2^-24
}

// --------------------------------------------------------------------------
// Periodic integer geometry
// --------------------------------------------------------------------------

// cell index along one axis of a coordinate p in [0, L): floor(p * n / L)
__device__ __forceinline__ int32_t cell_of(int32_t p, int32_t n, uint32_t L) {
  return (int32_t)(((uint64_t)(uint32_t)p * (uint64_t)n) / (uint64_t)L);
}

// smallest unwrapped coordinate whose (unwrapped) cell index is >= b
__device__ __forceinline__ int64_t cell_lo(int64_t b, int32_t n, int64_t L) {
  int64_t q = b >= 0 ? b / n : -((-b + n - 1) / n);
  int64_t r = b - q * n;
  return q * L + (r * L + n - 1) / n;
}

// difference mapped into (-L/2, L/2]
__device__ __forceinline__ int64_t min_image(int64_t d, int64_t L) {
  if (2 * d > L) d -= L;
  if (2 * d <= -L) d += L;
  return d;
}

// ring r of the search block covers offsets [ring_lo, ring_hi] along an axis
// of n cells, clamped so that no cell is visited twice
__device__ __forceinline__ int ring_lo(int r, int n) { return -min(r, (n - 1) / 2); }
__device__ __forceinline__ int ring_hi(int r, int n) { return min(r, n / 2); }

// --------------------------------------------------------------------------
// Eq. (1): exact grid step round-half-even(s * h) for |s| <= 2^22, |h| <= 1.
// p = fl(s*h) and e = s*h - p (exact, from an FMA) decide the rounding of the
// exact product; only a half-way p needs e.
// --------------------------------------------------------------------------
__device__ __forceinline__ int32_t grid_step(float s, float h) {
  const float p = __fmul_rn(s, h);
  const float e = __fmaf_rn(s, h, -p);
  float r = rintf(p);
  if (fabsf(__fsub_rn(p, r)) == 0.5f) {
    if (e > 0.f) r = __fadd_rn(p, 0.5f);
    else if (e < 0.f) r = __fsub_rn(p, 0.5f);
  }
  return (int32_t)r;
}

// Cell geometry from the per-replica boundary tables: bnd[b] is the first
// grid coordinate of cell b (b = 0..n), so no division is needed.
__device__ __forceinline__ int cell_of_tab(uint32_t p, int n, const uint32_t* __restrict__ bnd, float inv_w) {
  int c = min((int)((float)p * inv_w), n - 1);
  while (c > 0 && p < __ldg(bnd + c)) --c;
  while (c < n - 1 && p >= __ldg(bnd + c + 1)) ++c;
  return c;
}

// first (unwrapped) coordinate of unwrapped cell b, -n <= b < 2n
__device__ __forceinline__ int64_t cell_lo_tab(int b, int n, const uint32_t* __restrict__ bnd, int64_t L) {
  if (b < 0) return (int64_t)__ldg(bnd + b + n) - L;
  if (b >= n) return (int64_t)__ldg(bnd + b - n) + L;
  return (int64_t)__ldg(bnd + b);
}

// global cell index of a position in replica R (x fastest)
template <int DIM>
__device__ __forceinline__ int64_t linear_cell(const Rep& R, const int32_t* p) {
  int64_t c = 0;
#pragma unroll
  for (int a = DIM - 1; a >= 0; --a) c = c * R.nc[a] + cell_of(p[a], R.nc[a], R.L[a]);
  return R.c0 + c;
}

__device__ __forceinline__ int wrap_index(int x, int n) {
  x %= n;
  return x < 0 ? x + n : x;
}

__device__ __forceinline__ int32_t wrap_add(int32_t p, int32_t d, uint32_t L) {
  int64_t q = ((int64_t)p + (int64_t)d) % (int64_t)L;
  if (q < 0) q += (int64_t)L;
  return (int32_t)q;
}

// --------------------------------------------------------------------------
// Two-level search grid.  The coarse grid is uniform per replica; coarse
// cell c holding m particles is split into s x s sub-cells, s = sub_side(m)
// (2D; 3D keeps s = 1).  Particles are sorted by (coarse cell, sub-cell
// row-major), so every row of sub-cells, and every row of coarse cells, is a
// contiguous run of the sorted arrays.
// --------------------------------------------------------------------------
#ifndef VK_SUB_MAX
#define VK_SUB_MAX 64
#endif
constexpr int kSubMax = VK_SUB_MAX;  // largest sub-grid side (sub_s is 8 bits: at most 255)
#ifndef VK_SUB_TARGET
#define VK_SUB_TARGET 2
#endif
constexpr int kSubTarget = VK_SUB_TARGET;  // target particles per sub-cell

__device__ __host__ __forceinline__ int sub_side(uint32_t m) {
  int s = 1;
  while (s < kSubMax && (uint32_t)((s + 1) * (s + 1) * kSubTarget) <= m) ++s;
  return s;
}

struct GridView {
  const uint32_t* __restrict__ off;       // coarse cell -> first slot (n_cells + 1)
  const uint8_t* __restrict__ sub_s;      // coarse cell -> s
  const uint32_t* __restrict__ sub_base;  // coarse cell -> first sub-cell (n_cells + 1)
  const uint32_t* __restrict__ sub_off;   // sub-cell -> first slot
};

// sub-cell (sx, sy) of a point at in-cell offset u in a cell of width w
__device__ __forceinline__ int sub_index(int64_t u, int64_t w, int s) {
  return (int)((u * s) / w);
}

// global sub-cell index of a position (2D), given its coarse cell
template <int DIM>
__device__ __forceinline__ int64_t sub_cell_of(const Rep& R, const GridView& G, const int32_t* p, int64_t gcell) {
  const int s = G.sub_s[gcell];
  int64_t j = 0;
  if (DIM == 2 && s > 1) {
    const int cx = cell_of(p[0], R.nc[0], R.L[0]), cy = cell_of(p[1], R.nc[1], R.L[1]);
    const int64_t x0 = cell_lo(cx, R.nc[0], R.L[0]), y0 = cell_lo(cy, R.nc[1], R.L[1]);
    const int64_t wx = cell_lo(cx + 1, R.nc[0], R.L[0]) - x0, wy = cell_lo(cy + 1, R.nc[1], R.L[1]) - y0;
    j = (int64_t)sub_index(p[1] - y0, wy, s) * s + sub_index(p[0] - x0, wx, s);
  }
  return (int64_t)G.sub_base[gcell] + j;
}

// sub-cell index of offset u (0 <= u < w) in a cell of width w split s ways:
// floor(u*s/w), from a float estimate corrected with exact products
__device__ __forceinline__ int sub_idx(int64_t u, int64_t w, int s) {
  int j = min(max((int)((float)u * ((float)s / (float)w)), 0), s - 1);
  const int64_t us = u * s;
  while (j > 0 && us < (int64_t)j * w) --j;
  while (j < s - 1 && us >= (int64_t)(j + 1) * w) ++j;
  return j;
}

// Coarse cell and sub-cell (global indices) of a position, from the
// per-replica boundary tables (no 64-bit division); the same cells as
// linear_cell / sub_cell_of.
template <int DIM>
__device__ __forceinline__ void locate_tab(const Rep& R, const GridView& G, const uint32_t* __restrict__ bounds,
                                           const int32_t* p, int64_t* gcell, int64_t* gsub) {
  int c[3] = {0, 0, 0};
#pragma unroll
  for (int a = 0; a < DIM; ++a) c[a] = cell_of_tab((uint32_t)p[a], R.nc[a], bounds + R.bnd[a], R.inv_w[a]);
  int64_t lin = 0;
#pragma unroll
  for (int a = DIM - 1; a >= 0; --a) lin = lin * R.nc[a] + c[a];
  *gcell = R.c0 + lin;
  const int s = G.sub_s[*gcell];
  int64_t j = 0;
  if (DIM == 2 && s > 1) {
    const uint32_t* bx = bounds + R.bnd[0];
    const uint32_t* by = bounds + R.bnd[1];
    const int64_t x0 = __ldg(bx + c[0]), wx = (int64_t)__ldg(bx + c[0] + 1) - x0;
    const int64_t y0 = __ldg(by + c[1]), wy = (int64_t)__ldg(by + c[1] + 1) - y0;
    j = (int64_t)sub_idx(p[1] - y0, wy, s) * s + sub_idx(p[0] - x0, wx, s);
  }
  *gsub = (int64_t)G.sub_base[*gcell] + j;
}

// upper bound (integer) of the square root of r2; r2 may be ~0ull (infinite)
__device__ __forceinline__ int64_t radius_upper(uint64_t r2) {
  if (r2 >= (1ull << 62)) return INT64_MAX / 4;
  const float f = sqrtf((float)r2) * 1.0000005f;
  int64_t r = (int64_t)f + 1;
  while ((uint64_t)r * (uint64_t)r < r2) ++r;
  return r;
}

// Walk the 3D grid around the particle at pi (3D coarse cells are never
// split into sub-cells).  run(qb, qe) receives runs of sorted slots (a row
// segment of coarse cells along x is one run); stop(B2) is asked after each
// ring of cells, B2 being the exact squared distance from the particle to the
// nearest point outside the scanned block.  Rings are clamped so that no cell
// is visited twice; every candidate is measured by its minimum image.
// Returns true iff the whole box was scanned.
template <class RunFn, class StopFn>
__device__ __forceinline__ bool grid_walk3(const Rep& R, const int32_t* pi, const GridView& G, RunFn& run,
                                           StopFn& stop) {
  int c[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) c[a] = cell_of(pi[a], R.nc[a], R.L[a]);
  // cells x-offsets [a, b] of the row whose first cell is rowbase: one run
  // per wrap-free segment
  auto visit_row = [&](int a, int b, int64_t rowbase) {
    if (a > b) return;
    const int nx = R.nc[0];
    uint32_t pend_b = 0, pend_e = 0;
    bool pend = false;
    for (int ox = a; ox <= b; ++ox) {
      const int64_t g = rowbase + wrap_index(c[0] + ox, nx);
      const uint32_t qb = G.off[g], qe = G.off[g + 1];
      if (pend && qb == pend_e) {
        pend_e = qe;
      } else {
        if (pend) run(pend_b, pend_e);
        pend = true;
        pend_b = qb;
        pend_e = qe;
      }
    }
    if (pend) run(pend_b, pend_e);
  };
  for (int r = 0;; ++r) {
    int lo[3], hi[3], plo[3], phi[3];
    bool full_all = true, any_new = (r == 0);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      lo[a] = ring_lo(r, R.nc[a]);
      hi[a] = ring_hi(r, R.nc[a]);
      plo[a] = r ? ring_lo(r - 1, R.nc[a]) : 1;
      phi[a] = r ? ring_hi(r - 1, R.nc[a]) : 0;
      full_all = full_all && (hi[a] - lo[a] + 1 == R.nc[a]);
      any_new = any_new || lo[a] < plo[a] || hi[a] > phi[a];
    }
    if (!any_new) return true;
    for (int oz = lo[2]; oz <= hi[2]; ++oz) {
      const int64_t zb = (int64_t)wrap_index(c[2] + oz, R.nc[2]) * R.nc[1];
      const bool oldz = !(oz < plo[2] || oz > phi[2]);
      for (int oy = lo[1]; oy <= hi[1]; ++oy) {
        const int64_t rowbase = R.c0 + (zb + wrap_index(c[1] + oy, R.nc[1])) * R.nc[0];
        if (!oldz || oy < plo[1] || oy > phi[1]) {
          visit_row(lo[0], hi[0], rowbase);
        } else {
          visit_row(lo[0], plo[0] - 1, rowbase);
          visit_row(phi[0] + 1, hi[0], rowbase);
        }
      }
    }
    if (full_all) return true;
    int64_t B = INT64_MAX;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (hi[a] - lo[a] + 1 == R.nc[a]) continue;
      const int64_t bl = (int64_t)pi[a] - cell_lo((int64_t)c[a] - r, R.nc[a], R.L[a]) + 1;
      const int64_t bh = cell_lo((int64_t)c[a] + r + 1, R.nc[a], R.L[a]) - (int64_t)pi[a];
      B = min(B, min(bl, bh));
    }
    if (stop((uint64_t)B * (uint64_t)B)) return false;
  }
}

// --------------------------------------------------------------------------
// Heading sums in the canonical neighbor order (plain / Neumaier / FP64)
// --------------------------------------------------------------------------
template <int DIM>
struct HeadSum {
  float s[DIM];
  float c[DIM];
  double d[DIM];
  __device__ __forceinline__ void init() {
#pragma unroll
    for (int a = 0; a < DIM; ++a) { s[a] = 0.f; c[a] = 0.f; d[a] = 0.0; }
  }
  __device__ __forceinline__ void add(const float* v, int mode) {
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      if (mode == 2) {
        d[a] += (double)v[a];
      } else if (mode == 1) {
        const float t = __fadd_rn(s[a], v[a]);
        if (fabsf(s[a]) >= fabsf(v[a])) c[a] = __fadd_rn(c[a], __fadd_rn(__fsub_rn(s[a], t), v[a]));
        else c[a] = __fadd_rn(c[a], __fadd_rn(__fsub_rn(v[a], t), s[a]));
        s[a] = t;
      } else {
        s[a] = __fadd_rn(s[a], v[a]);
      }
    }
  }
};

// --------------------------------------------------------------------------
// Eq. (2) alignment + noise and Eq. (1) advection for one particle.
// --------------------------------------------------------------------------
// sum_mode selects which of H's sums is the total (2: H.d, FP64).
template <int DIM>
__device__ __forceinline__ void align_advect_mode(const Rep& R, const StepParams& P, int sum_mode, uint32_t step,
                                                  int32_t id, const float* ni, const HeadSum<DIM>& H, int m,
                                                  const int32_t* pi, int32_t* pout, float* nout) {
  const uint4 w = philox4x32_10(make_uint4((uint32_t)id, step, R.replica, 0u),
                                make_uint2(P.seed_lo, P.seed_hi));
  const float u = unit24(w.x);
  if (sum_mode == 2) {
    double S[DIM];
#pragma unroll
    for (int a = 0; a < DIM; ++a) S[a] = H.d[a];
    if (P.noise == 0) {
      double th = (S[0] == 0.0 && S[1] == 0.0) ? atan2((double)ni[1], (double)ni[0]) : atan2(S[1], S[0]);
      th += (double)R.eta * ((double)u - 0.5);
      double sn, cs;
      sincos(th, &sn, &cs);
      nout[0] = (float)cs;
      nout[1] = (float)sn;
    } else {
      double xi[3];
      double sx, cx;
      sincospi(2.0 * (double)u, &sx, &cx);
      if (DIM == 2) {
        xi[0] = cx; xi[1] = sx; xi[2] = 0.0;
      } else {
        const double z = 2.0 * (double)unit24(w.y) - 1.0, r = sqrt(fmax(0.0, 1.0 - z * z));
        xi[0] = r * cx; xi[1] = r * sx; xi[2] = z;
      }
      double v[DIM], n2 = 0.0;
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        v[a] = (double)R.eta * xi[a] + (m > 0 ? S[a] / (double)m : 0.0);
        n2 += v[a] * v[a];
      }
      if (n2 == 0.0) {
#pragma unroll
        for (int a = 0; a < DIM; ++a) nout[a] = ni[a];
      } else {
        const double inv = 1.0 / sqrt(n2);
#pragma unroll
        for (int a = 0; a < DIM; ++a) nout[a] = (float)(v[a] * inv);
      }
    }
  } else {
    float S[DIM];
#pragma unroll
    for (int a = 0; a < DIM; ++a) S[a] = (sum_mode == 1) ? __fadd_rn(H.s[a], H.c[a]) : H.s[a];
    if (P.noise == 0) {
      float th = (S[0] == 0.f && S[1] == 0.f) ? atan2f(ni[1], ni[0]) : atan2f(S[1], S[0]);
      th = th + R.eta * (u - 0.5f);
      float sn, cs;
      sincosf(th, &sn, &cs);
      nout[0] = cs;
      nout[1] = sn;
    } else {
      float xi[3];
      float sx, cx;
      sincospif(2.0f * u, &sx, &cx);
      if (DIM == 2) {
        xi[0] = cx; xi[1] = sx; xi[2] = 0.f;
      } else {
        const float z = 2.0f * unit24(w.y) - 1.0f, r = sqrtf(fmaxf(0.f, 1.0f - z * z));
        xi[0] = r * cx; xi[1] = r * sx; xi[2] = z;
      }
      float v[DIM], n2 = 0.f;
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        v[a] = R.eta * xi[a] + (m > 0 ? S[a] / (float)m : 0.f);
        n2 += v[a] * v[a];
      }
      if (n2 == 0.f) {
#pragma unroll
        for (int a = 0; a < DIM; ++a) nout[a] = ni[a];
      } else {
        const float nrm = sqrtf(n2);
#pragma unroll
        for (int a = 0; a < DIM; ++a) nout[a] = v[a] / nrm;
      }
    }
  }
  const float* h = P.advect_new ? nout : ni;
#pragma unroll
  for (int a = 0; a < DIM; ++a) pout[a] = wrap_add(pi[a], grid_step(R.s, h[a]), R.L[a]);
}

template <int DIM>
__device__ __forceinline__ void align_advect(const Rep& R, const StepParams& P, uint32_t step,
                                             int32_t id, const float* ni, const HeadSum<DIM>& H,
                                             int m, const int32_t* pi, int32_t* pout, float* nout) {
  align_advect_mode<DIM>(R, P, P.sum_mode, step, id, ni, H, m, pi, pout, nout);
}

// --------------------------------------------------------------------------
// Order parameter: compensated FP32 block partials -> FP64 atomics
// --------------------------------------------------------------------------
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Order parameter accumulators.  Every heading component is rounded to a
// fixed point of 2^-32 (exact scaling of the FP32 value, then round to the
// nearest integer) and summed in int64: integer addition is exact and
// associative, so the sums, and phi, are bit-identical from run to run
// whatever order the particles are visited in (the order inside a cell of
// the sorted state comes from atomic ranks).  The rounding errs by at most
// 2^-33 per particle, about 1e-10 of phi.  N <= 2^31 keeps the sums below
// 2^63.  The FP64 conversion happens when phi is read.
using PhiAcc = unsigned long long;
constexpr float kPhiScale = 4294967296.0f;  // 2^32

__device__ __forceinline__ long long phi_fixed(float v) { return __float2ll_rn(v * kPhiScale); }

__device__ __forceinline__ long long warp_sum_ll(long long x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// Block-wide sum of v[0..DIM) without a block barrier at the end: every warp
// reduces its lanes and parks the partial in shared memory; the last warp of
// the block to arrive adds the block total into acc[0..DIM).
// phi_block_begin() must be called by all threads first.
struct PhiShared {
  long long s[kBlock / 32][3];
  unsigned int arrived;
};

__device__ __forceinline__ void phi_block_begin(PhiShared& sh) {
  if (threadIdx.x == 0) sh.arrived = 0;
  __syncthreads();
}

template <int DIM>
__device__ __forceinline__ void phi_block_end(PhiShared& sh, const float* v, PhiAcc* acc) {
  long long s[DIM];
#pragma unroll
  for (int a = 0; a < DIM; ++a) s[a] = warp_sum_ll(phi_fixed(v[a]));
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
#pragma unroll
    for (int a = 0; a < DIM; ++a) ((volatile long long*)sh.s[wid])[a] = s[a];
    __threadfence_block();
    const unsigned int before = atomicAdd(&sh.arrived, 1u);
    if (before == blockDim.x / 32 - 1) {
      __threadfence_block();
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        long long t = 0;
        for (int w2 = 0; w2 < (int)(blockDim.x / 32); ++w2) t += ((volatile long long*)sh.s[w2])[a];
        atomicAdd(acc + a, (PhiAcc)t);
      }
    }
  }
}

// (for kernels whose warps finish together: both halves at the end)
template <int DIM>
__device__ __forceinline__ void block_phi_accumulate(const float* v, PhiAcc* acc) {
  __shared__ PhiShared sh;
  phi_block_begin(sh);
  phi_block_end<DIM>(sh, v, acc);
}

// Warp-wide add of the headings of the active lanes, each to its own
// replica's accumulators step_acc + 3 * rep (lanes of one replica are summed
// first, then one lane adds the total).  All lanes of the warp must call it.
template <int DIM>
__device__ __forceinline__ void phi_add_warp(PhiAcc* step_acc, int rep, const float* v, bool active) {
  const int lane = threadIdx.x & 31;
  unsigned rem = __ballot_sync(0xffffffffu, active);
  while (rem) {
    const int leader = __ffs(rem) - 1;
    const int r = __shfl_sync(0xffffffffu, rep, leader);
    const bool in = active && rep == r;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      const long long t = warp_sum_ll(in ? phi_fixed(v[a]) : 0ll);
      if (lane == leader) atomicAdd(step_acc + (size_t)r * 3 + a, (PhiAcc)t);
    }
    rem &= ~__ballot_sync(0xffffffffu, in);
  }
}

__device__ __forceinline__ void set_status(int32_t* status, int32_t code) {
  atomicCAS(status, 0, code);
}

}  // namespace vk

// host-side launchers (defined in the .cu files)
namespace vk {

// streaming multiprocessors of the current device (for fixed-size grids)
inline int device_sm_count() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      sms <= 0)
    return 1;
  return sms;
}

struct Buffers {
  // sorted current state
  void* S_pos;
  void* S_dir;
  int32_t* S_id;
  // next state in S order + rank in the new cell
  void* U_pos;
  void* U_dir;
  int32_t* U_id;
  uint32_t* U_rank;
  uint32_t* counts;   // n_cells
  uint32_t* offsets;  // n_cells + 1
  uint32_t* bsum;     // scan block sums (coarse)
  uint8_t* sub_s;     // n_cells: sub-grid side per coarse cell
  uint32_t* sub_base; // n_cells + 1: first sub-cell of every coarse cell
  uint32_t* sub_count;  // n_sub_max
  uint32_t* sub_off;    // n_sub_max + 1
  uint32_t* bsum2;      // scan block sums (sub-cells)
  uint32_t* bounds;     // per replica and axis: first coordinate of every cell (nc + 1 entries)
  PhiAcc* phi_acc;    // phi_cap * n_rep * 3 fixed-point heading sums (see PhiAcc)
  int64_t* d_step;
  int32_t* d_status;
  int2* ovf_list;      // 2 N entries of (slot, replica): Voronoi cells too large for the main kernel;
                       // 2D kNN: deferred particles (first half) and particles for the walk (second)
  int32_t* ovf_count;  // 2 counters for those lists, cleared by the scatter of every step
  // 2D kNN: each particle's k-th neighbor distance (grid units) found at the
  // previous step, in S order, and the one found now in U order (0 = unknown);
  // only a search hint, results never depend on it (NULL for other rules)
  float* S_hint;
  float* U_hint;
  // Voronoi rule (Sec. "Computational tools: Voronoi neighbor lists": last
  // step's triangulation is re-checked rather than rebuilt): every
  // particle's neighbor ids of the last step, indexed by (replica's first
  // slot + id), up to kVorSeed each (count in vor_seed_n), and the sorted
  // slot of every particle by the same index (written by the scatter).  A
  // cell is clipped by these sites first; only the order of the work
  // depends on them, never the result (NULL: build every cell from scratch).
  int32_t* vor_seed;
  int32_t* vor_seed_n;
  int32_t* slot_of;
};

constexpr int kVorSeed = 12;

struct Geometry {
  int dim;
  int rule;
  int n_rep;
  int64_t n_total;
  int64_t n_cells;
  int64_t n_sub_max;  // bound of the number of sub-cells: n_cells + n_total / kSubTarget
  int n_tasks;
  const Rep* reps;
  const BlockTask* tasks;
};

// vk_cells.cu
cudaError_t launch_load(const Geometry& g, const Buffers& b, const int32_t* pos_in, const float* head_in,
                        int heading_kind, cudaStream_t st);
cudaError_t launch_count(const Geometry& g, const Buffers& b, cudaStream_t st);
// coarse counts -> offsets, sub-grid sides and sub-cell bases; sub-cell
// histogram of U (ranks); sub-cell scan
cudaError_t launch_build(const Geometry& g, const Buffers& b, cudaStream_t st);
cudaError_t launch_scatter(const Geometry& g, const Buffers& b, const StepParams& P, int advance_step,
                           cudaStream_t st);
cudaError_t launch_export_state(const Geometry& g, const Buffers& b, int rep, int64_t p0, int32_t n,
                                int32_t* pos_out, float* dir_out, float* theta_out, cudaStream_t st);
// 2D kNN: the search hints of one replica into id order in U (before an import)
cudaError_t launch_hints_by_id(const Buffers& b, int64_t p0, int32_t n, cudaStream_t st);
cudaError_t launch_import_state(const Geometry& g, const Buffers& b, int rep, int64_t p0, int32_t n,
                                const int32_t* pos_in, const float* dir_in, cudaStream_t st);

// vk_knn.cu (3D)
cudaError_t launch_knn_step(const Geometry& g, const Buffers& b, const StepParams& P, cudaStream_t st);
cudaError_t launch_knn_export(const Geometry& g, const Buffers& b, int k, int rep, int n, int32_t* out,
                              cudaStream_t st);

// vk_knn2d.cu (the 2D kNN hot path)
// search + update of every particle (radius first: those it can serve; the
// rest is listed) ...
cudaError_t launch_knn2_step(const Geometry& g, const Buffers& b, const StepParams& P, cudaStream_t st);
// ... and of the listed particles (deferred squares, then the walk); no-op for the walk-only search
cudaError_t launch_knn2_finish(const Geometry& g, const Buffers& b, const StepParams& P, cudaStream_t st);
cudaError_t launch_knn2_export(const Geometry& g, const Buffers& b, int k, int rep, int n, int32_t* out,
                               cudaStream_t st, const StepParams& P);
// one-time kernel attributes (shared memory of the radius-first search)
cudaError_t prepare_knn2();

// vk_metric.cu (metric rule, 2D and 3D)
cudaError_t launch_metric_step(const Geometry& g, const Buffers& b, const StepParams& P, cudaStream_t st);
// pass 0: deg[id] = neighbor count; pass 1: the ids of row id at out_off[id], sorted by id
cudaError_t launch_metric_export(const Geometry& g, const Buffers& b, int rep, int n, int pass, int32_t* deg,
                                 const int64_t* out_off, int32_t* out_ids, cudaStream_t st);

// vk_tissue.cu (Voronoi tissue model): per-slot scratch of the cells pass
constexpr int kTissueCap = 32;  // edges per cell kept for the force pass
struct TissueScratch {
  int32_t* nb_n;     // edges of every cell (0: failed, status latched)
  int32_t* nb_slot;  // kTissueCap per slot: edge sites, counter-clockwise
  int2* nb_off;      // ... and their exact offsets from the particle
  double* area;      // per slot, length units
  double* perim;
};
// cells, forces (by id) and energy of one replica; any output may be NULL
cudaError_t launch_tissue(const Geometry& g, const Buffers& b, int rep, int n, double KA, double KP, double A0,
                          double P0, double unit, TissueScratch w, double* area_out, double* perim_out,
                          double* force_out, double* energy_out, cudaStream_t st);

// vk_voronoi.cu
cudaError_t launch_voronoi_step(const Geometry& g, const Buffers& b, const StepParams& P, cudaStream_t st);
cudaError_t launch_voronoi_export(const Geometry& g, const Buffers& b, int rep, int n, int pass, int32_t* deg,
                                  const int64_t* out_off, int32_t* out_ids, cudaStream_t st);
// largest Voronoi cell (edges) handled; larger cells latch VK_ERR_CAPACITY
constexpr int kVoronoiMaxDeg = 256;

}  // namespace vk
