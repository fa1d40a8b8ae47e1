// vk_box2d.cuh -- the square walk of the 2D two-level search grid, shared
// by the radius-first k-nearest search (vk_knn2d.cu) and the metric rule
// (vk_metric.cu): every particle of the square [p - a, p + a] around a
// particle, listed as contiguous runs of the cell-sorted arrays, with exact
// minimum-image offsets.  Also the particle's search context and the exact
// field-of-view test of the kNN rule.
#pragma once
#include <climits>

#include "vk_internal.cuh"

// slot runs one square listing may buffer per thread
#ifndef VK_KNN2_BOX_RUNS
#define VK_KNN2_BOX_RUNS 16
#endif

namespace vk {

// The field of view of the kNN rule (reading of Sec. "Metric and topological
// flocking models": the k nearest neighbors within an angular field of
// view): offset d is in view iff d.nq >= cq |d|, with the heading and the
// cosine of the half-angle rounded to 2^-24 (nq = rint(n 2^24), cq =
// rint(c 2^24), round half to even), compared exactly through squares in
// 128-bit integers; d = 0 is in view, and everything is when c <= -1.
struct View {
  int32_t nxq, nyq, cq;
};

__device__ __forceinline__ View make_view(float2 n, int32_t cq) {
  View w;
  w.nxq = (int32_t)__float2ll_rn(n.x * 16777216.0f);
  w.nyq = (int32_t)__float2ll_rn(n.y * 16777216.0f);
  w.cq = cq;
  return w;
}

__device__ __forceinline__ bool in_view(const View& w, int32_t dx, int32_t dy, uint64_t D) {
  if (w.cq <= -(1 << 24)) return true;  // a full circle
  const long long sdot = (long long)dx * w.nxq + (long long)dy * w.nyq;
  const __int128 lhs = (__int128)sdot * sdot;
  const __int128 rhs = (__int128)((long long)w.cq * w.cq) * (__int128)D;
  if (w.cq >= 0) return sdot >= 0 && lhs >= rhs;
  return sdot >= 0 || lhs <= rhs;
}


struct Ctx {
  int64_t self;
  uint32_t px, py;
  uint32_t Lx, Ly;
  int32_t hix, lox, hiy, loy;  // minimum image: d > hi -> d - L, d <= lo -> d + L
  uint32_t n_cand, n_runs;
  bool split;  // the particle's own coarse cell is split (tracing)
  View view;  // field of view of the kNN rule (everything when view.cq <= -2^24)
};

__device__ __forceinline__ void init_ctx(Ctx& C, const Rep& R, int64_t self, int2 p) {
  C.self = self;
  C.px = (uint32_t)p.x;
  C.py = (uint32_t)p.y;
  C.Lx = R.L[0];
  C.Ly = R.L[1];
  C.hix = (int32_t)(R.L[0] / 2);
  C.lox = -(int32_t)((R.L[0] + 1) / 2);
  C.hiy = (int32_t)(R.L[1] / 2);
  C.loy = -(int32_t)((R.L[1] + 1) / 2);
  C.n_cand = 0;
  C.n_runs = 0;
  C.split = false;
  C.view.nxq = 0;
  C.view.nyq = 0;
  C.view.cq = kViewAll;
}

// tracing counters of the radius-first search
struct BoxCount {
  uint32_t cand = 0;   // candidates examined
  uint32_t tries = 0;  // squares scanned
  uint32_t runs = 0;   // contiguous slot runs read
  uint32_t hits = 0;   // hits merged
  uint32_t cells = 0;  // coarse cells visited
  uint32_t why = 0;    // fallback reason: 0 none, 1 square too wide (or too many runs), 2 too few hits, 3 tie
};

// unwrapped coarse-cell index of an unwrapped coordinate x, -L <= x < 2L
__device__ __forceinline__ int box_ucell(int64_t x, int n, const uint32_t* __restrict__ bnd, float inv_w, int64_t L) {
  if (x < 0) return cell_of_tab((uint32_t)(x + L), n, bnd, inv_w) - n;
  if (x >= L) return cell_of_tab((uint32_t)(x - L), n, bnd, inv_w) + n;
  return cell_of_tab((uint32_t)x, n, bnd, inv_w);
}

// exact minimum-image offset and squared distance of pj from the particle
__device__ __forceinline__ uint64_t box_offset(const Ctx& C, int2 pj, int32_t& dx, int32_t& dy) {
  dx = (int32_t)((uint32_t)pj.x - C.px);
  dy = (int32_t)((uint32_t)pj.y - C.py);
  if (dx > C.hix) dx = (int32_t)((uint32_t)dx - C.Lx);
  else if (dx <= C.lox) dx = (int32_t)((uint32_t)dx + C.Lx);
  if (dy > C.hiy) dy = (int32_t)((uint32_t)dy - C.Ly);
  else if (dy <= C.loy) dy = (int32_t)((uint32_t)dy + C.Ly);
  return (uint64_t)((int64_t)dx * dx) + (uint64_t)((int64_t)dy * dy);
}

__device__ __forceinline__ uint64_t box_dist2(const Ctx& C, int2 pj) {
  int32_t dx, dy;
  return box_offset(C, pj, dx, dy);
}

// Walk the slot runs of the square [p - a, p + a] (the sub-cell rows of the
// coarse cells it meets), each with the periodic image its cell lies in.
// Runs are listed up to HB::kRuns at a time into the thread's column of
// H.run (uint2 run[kRuns][kBlock]); one
// flat loop walks each batch, so that threads of a warp whose squares split
// into different numbers of runs still scan candidates together.  The
// visitor gets the candidates four at a time (their loads are independent,
// so they are in flight together; a group never crosses a run):
// v.group(q, n, pj, ox, oy) for slots q..q+n-1 at positions pj[0..n), whose
// exact offsets from the particle are pj - (ox, oy) in wrapping 32-bit
// arithmetic.  False when the square is too wide for the minimum image or
// meets a coarse cell through two periodic images (nothing was visited).
constexpr int kGroup = 4;

template <class HB, class V>
__device__ __forceinline__ bool box_walk(HB& H, const Rep& R, const uint32_t* __restrict__ bounds,
                                         const GridView& G, const int2* __restrict__ pos, const Ctx& C, int64_t a,
                                         BoxCount& bc, V& v) {
  const int64_t Lx = C.Lx, Ly = C.Ly;
  if (2 * (2 * a + 1) >= Lx || 2 * (2 * a + 1) >= Ly) return false;
  const int nx = R.nc[0], ny = R.nc[1];
  const uint32_t* bx = bounds + R.bnd[0];
  const uint32_t* by = bounds + R.bnd[1];
  const int64_t qx0 = (int64_t)C.px - a, qx1 = (int64_t)C.px + a;
  const int64_t qy0 = (int64_t)C.py - a, qy1 = (int64_t)C.py + a;
  const int ucx0 = box_ucell(qx0, nx, bx, R.inv_w[0], Lx), ucx1 = box_ucell(qx1, nx, bx, R.inv_w[0], Lx);
  const int ucy0 = box_ucell(qy0, ny, by, R.inv_w[1], Ly), ucy1 = box_ucell(qy1, ny, by, R.inv_w[1], Ly);
  if (ucx1 - ucx0 + 1 > nx || ucy1 - ucy0 + 1 > ny) return false;
  bc.tries += 1;
  // enumeration cursor over (coarse cell, row of sub-cells): runs are listed
  // kRuns at a time, each batch is scanned, then listing resumes
  int ucx = ucx0, ucy = ucy0;
  int row = 0, row_end = -1;  // rows of the current cell still to list
  int64_t gc = 0;
  uint32_t sb0 = 0, code = 0;
  int s = 1, sx0 = 0, sx1 = 0;
  bool split = false, listed_all = false;
  while (!listed_all) {
    int nrun = 0;
    while (nrun < HB::kRuns) {
      if (row > row_end) {  // next coarse cell
        if (ucx > ucx1) {
          ucx = ucx0;
          ++ucy;
        }
        if (ucy > ucy1) {
          listed_all = true;
          break;
        }
        const int cy = ucy < 0 ? ucy + ny : (ucy >= ny ? ucy - ny : ucy);
        const int cx = ucx < 0 ? ucx + nx : (ucx >= nx ? ucx - nx : ucx);
        // shift code per axis: 0 same image, 1 the image at -L, 2 at +L
        code = (ucx < 0 ? 1u : (ucx >= nx ? 2u : 0u)) << 2 | (ucy < 0 ? 1u : (ucy >= ny ? 2u : 0u));
        gc = R.c0 + (int64_t)cy * nx + cx;
        sb0 = __ldg(G.sub_base + gc);
        split = __ldg(G.sub_base + gc + 1) - sb0 > 1;
        bc.cells += 1;
        row = 0;
        row_end = 0;
        if (split) {
          const int64_t y0c = cell_lo_tab(ucy, ny, by, Ly);
          const int64_t wy = cell_lo_tab(ucy + 1, ny, by, Ly) - y0c;
          const int64_t x0c = cell_lo_tab(ucx, nx, bx, Lx);
          const int64_t wx = cell_lo_tab(ucx + 1, nx, bx, Lx) - x0c;
          s = __ldg(G.sub_s + gc);
          sx0 = sub_idx(max(qx0 - x0c, (int64_t)0), wx, s);
          sx1 = sub_idx(min(qx1 - x0c, wx - 1), wx, s);
          row = sub_idx(max(qy0 - y0c, (int64_t)0), wy, s);
          row_end = sub_idx(min(qy1 - y0c, wy - 1), wy, s);
        }
        ++ucx;
      }
      uint32_t qb, qe;
      if (split) {
        const uint32_t rb = sb0 + (uint32_t)row * (uint32_t)s;
        qb = __ldg(G.sub_off + rb + sx0);
        qe = __ldg(G.sub_off + rb + sx1 + 1);
      } else {
        qb = __ldg(G.off + gc);
        qe = __ldg(G.off + gc + 1);
      }
      ++row;
      if (qe > qb) H.run[nrun++][threadIdx.x] = make_uint2(qb, (qe - qb) << 4 | code);
    }
    bc.runs += (uint32_t)nrun;
    int r = -1;
    uint32_t q = 0, qe = 0, ox = 0, oy = 0;
    for (;;) {
      if (q == qe) {
        if (++r == nrun) break;
        const uint2 e = H.run[r][threadIdx.x];
        q = e.x;
        qe = e.x + (e.y >> 4);
        // reference shifted into the run's periodic image: dx = x_j - ox exactly
        const uint32_t cxd = (e.y >> 2) & 3u, cyd = e.y & 3u;
        ox = C.px + (cxd == 1u ? (uint32_t)C.Lx : 0u) - (cxd == 2u ? (uint32_t)C.Lx : 0u);
        oy = C.py + (cyd == 1u ? (uint32_t)C.Ly : 0u) - (cyd == 2u ? (uint32_t)C.Ly : 0u);
        bc.cand += qe - q;
      }
      const uint32_t n = min(qe - q, (uint32_t)kGroup);
      int2 pj[kGroup];
#pragma unroll
      for (int u = 0; u < kGroup; ++u) pj[u] = __ldg(pos + q + min((uint32_t)u, n - 1));
      v.group(q, n, pj, ox, oy);
      q += n;
    }
  }
  return true;
}

}  // namespace vk
