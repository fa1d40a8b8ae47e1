// vk_knn2d.cu -- the 2D k-nearest-neighbor rule fused with the Vicsek update
// (Sec. "Metric and topological flocking models": each particle aligns with
// its k nearest neighbors at any distance; Eq. 1 and Eq. 2).  This is the
// benchmark's hot kernel, written for issue efficiency:
//   * cell indices and cell boundaries come from per-replica tables (no
//     64-bit division on the search path);
//   * a row segment of coarse cells without sub-grids is one run of the
//     sorted arrays (detected from the sub-cell bases, no per-cell branch);
//   * minimum-image differences in int32, exact int64 squared distances, a
//     register top-k ordered by (D, id);
//   * the block's order-parameter partials are combined by the last warp to
//     finish (no barrier that would hold finished warps).
// The search is the two-level walk documented in vk_internal.cuh.
#include <algorithm>
#include <climits>

#include "vk_box2d.cuh"

// resident 256-thread blocks per SM the step kernels are compiled for
// (register budget): the per-particle walk, and the radius-first search
#ifndef VK_KNN2_MIN_BLOCKS
#define VK_KNN2_MIN_BLOCKS 4
#endif
#ifndef VK_KNN2_BOX_BLOCKS
#define VK_KNN2_BOX_BLOCKS 3
#endif
// ... and the deferred-particle kernel (a few larger squares per particle)
#ifndef VK_KNN2_DEFER_BLOCKS
#define VK_KNN2_DEFER_BLOCKS 2
#endif

namespace vk {

namespace {

// Top-k in registers: exact squared distances and sorted slots, ordered by
// (D, id).  For k < KC the first KC-k entries are sentinels (D = 0, slot -1)
// that order before every real candidate, so the threshold is always entry
// KC-1 and no register array is indexed dynamically.  Ids are only read to
// break an exact distance tie.
template <int KC>
struct Top {
  uint64_t d[KC];
  int32_t slot[KC];
};

template <int KC>
__device__ __forceinline__ void top_init(Top<KC>& T, int k) {
#pragma unroll
  for (int s = 0; s < KC; ++s) {
    T.d[s] = s < KC - k ? 0ull : ~0ull;
    T.slot[s] = -1;
  }
}

// insert candidate slot q at squared distance D, known to order before the
// current last entry; an exact distance tie is decided by the ids (a real
// candidate never orders before a sentinel)
template <int KC>
__device__ __forceinline__ void top_insert(Top<KC>& T, uint64_t D, int32_t q, const int32_t* __restrict__ ids) {
  bool placed = false;
#pragma unroll
  for (int s = KC - 1; s > 0; --s) {
    if (!placed) {
      bool before = D < T.d[s - 1];
      if (D == T.d[s - 1]) before = T.slot[s - 1] >= 0 && __ldg(ids + q) < __ldg(ids + T.slot[s - 1]);
      if (before) {
        T.d[s] = T.d[s - 1];
        T.slot[s] = T.slot[s - 1];
      } else {
        T.d[s] = D;
        T.slot[s] = q;
        placed = true;
      }
    }
  }
  if (!placed) {
    T.d[0] = D;
    T.slot[0] = q;
  }
}

template <int KC>
__device__ __forceinline__ void scan_run(Ctx& C, const int2* __restrict__ pos, const int32_t* __restrict__ ids,
                                         uint32_t qb, uint32_t qe, Top<KC>& T) {
  C.n_cand += qe - qb;
  C.n_runs += 1;
  for (uint32_t q = qb; q < qe; ++q) {
    const int2 pj = __ldg(pos + q);
    int32_t dx = (int32_t)((uint32_t)pj.x - C.px);
    int32_t dy = (int32_t)((uint32_t)pj.y - C.py);
    if (dx > C.hix) dx = (int32_t)((uint32_t)dx - C.Lx);
    else if (dx <= C.lox) dx = (int32_t)((uint32_t)dx + C.Lx);
    if (dy > C.hiy) dy = (int32_t)((uint32_t)dy - C.Ly);
    else if (dy <= C.loy) dy = (int32_t)((uint32_t)dy + C.Ly);
    const uint64_t D = (uint64_t)((int64_t)dx * dx) + (uint64_t)((int64_t)dy * dy);
    if (D <= T.d[KC - 1] && (int64_t)q != C.self && in_view(C.view, dx, dy, D)) {
      // an exact tie with the current k-th best is decided by the ids
      if (D < T.d[KC - 1] || (T.slot[KC - 1] >= 0 && __ldg(ids + q) < __ldg(ids + T.slot[KC - 1])))
        top_insert<KC>(T, D, (int32_t)q, ids);
    }
  }
}

// first offset of sub-cell b: ceil(b*w/s)
__device__ __forceinline__ int64_t sub_lo(int b, int64_t w, int s) {
  const int64_t bw = (int64_t)b * w;
  int64_t q = (int64_t)((float)bw / (float)s);
  while (q * s < bw) ++q;
  while (q > 0 && (q - 1) * s >= bw) --q;
  return q;
}

// Resumable generator of the slot runs of the two-level walk, so that the
// candidate loop exists once in the kernel (instruction-cache footprint).
// Phase 1: rings of sub-cells in the own coarse cell (when it is split).
// Phase 2: rings of coarse cells; a row segment without sub-grids is one run,
// a split cell contributes the rows of its sub-cells that meet the box
// [p - rad, p + rad], rad^2 >= the current k-th best distance.
struct RunGen {
  // fixed
  const Rep* R;
  const uint32_t* __restrict__ bx;
  const uint32_t* __restrict__ by;
  GridView G;
  int64_t px, py;
  int nx, ny, cx, cy;
  int64_t own;
  // phase 1 geometry
  int s1, sx, sy;
  uint32_t ob0;
  int64_t cx0, wx1, cy0, wy1;
  // cursor
  int phase, r;
  int bx0, bx1, by0, by1, px0, px1, py0, py1;  // phase 1 block (current and previous ring)
  int yy, seg;                                  // phase 1 row / segment
  int lox, hix, loy, hiy, plox, phix, ploy, phiy;
  int oy;                                       // phase 2 row offset
  int part, nparts;                             // phase 2 parts of the row
  int pa[4], pb[4], pu[4];                      // part x0, x1, unwrapped x of x0
  int64_t rowbase;
  int ucy;
  int x;                                        // current cell in a per-cell part (-1: part not started)
  bool fast;
  int sr, sr1, sx0r, sx1r;                      // rows of the current split-cell rectangle
  uint32_t sbase;
  int sstride;
  bool in_rect;
  bool own_done;
  // the box [p - rad, p + rad] stays within every ring's representative cell
  // offsets (so a cell meets it at its visited offset only) while rad < safe
  int64_t safe;
  int64_t prad;  // radius used to skip rows and cells of the current part (-1: none)
  // split cells met while the search radius was still unknown, revisited at
  // the end of the ring (when it usually is known)
  int ndef;
  int64_t def_g[4];
  int def_ucx[4], def_ucy[4];
};

enum { kRun = 0, kRingEnd = 1, kDone = 2 };

__device__ __forceinline__ void gen_row_parts(RunGen& g) {
  // parts of row offset g.oy of ring g.r: up to 2 segments, each split by the wrap
  g.nparts = 0;
  const int ay = g.ucy < 0 ? g.ucy + g.ny : (g.ucy >= g.ny ? g.ucy - g.ny : g.ucy);
  g.rowbase = g.R->c0 + (int64_t)ay * g.nx;
  int sa[2], sb[2], ns = 0;
  if (g.oy < g.ploy || g.oy > g.phiy) {
    sa[0] = g.lox; sb[0] = g.hix; ns = 1;
  } else {
    if (g.lox <= g.plox - 1) { sa[ns] = g.lox; sb[ns] = g.plox - 1; ++ns; }
    if (g.phix + 1 <= g.hix) { sa[ns] = g.phix + 1; sb[ns] = g.hix; ++ns; }
  }
  for (int q = 0; q < ns; ++q) {
    const int ua = g.cx + sa[q];
    const int start = ua < 0 ? ua + g.nx : (ua >= g.nx ? ua - g.nx : ua);
    const int len = sb[q] - sa[q] + 1;
    if (start + len <= g.nx) {
      g.pa[g.nparts] = start; g.pb[g.nparts] = start + len - 1; g.pu[g.nparts] = ua; ++g.nparts;
    } else {
      g.pa[g.nparts] = start; g.pb[g.nparts] = g.nx - 1; g.pu[g.nparts] = ua; ++g.nparts;
      g.pa[g.nparts] = 0; g.pb[g.nparts] = start + len - g.nx - 1; g.pu[g.nparts] = ua + (g.nx - start);
      ++g.nparts;
    }
  }
  g.part = 0;
  g.x = -1;
}

// sub-cell rectangle of split cell gc (unwrapped indices ucx, ucy) meeting
// the box [p - rad, p + rad]; false if it misses the cell
__device__ __forceinline__ bool gen_rect(RunGen& g, int64_t gc, int ucx, int ucy, uint64_t r2) {
  const GridView& G = g.G;
  const Rep& R = *g.R;
  const int s = __ldg(G.sub_s + gc);
  g.sbase = __ldg(G.sub_base + gc);
  g.sstride = s;
  if (r2 == ~0ull) {
    g.sx0r = 0; g.sx1r = s - 1; g.sr = 0; g.sr1 = s - 1;
    g.in_rect = true;
    return true;
  }
  const int64_t rad = radius_upper(r2);
  // Rings visit every cell once, at its offset in [-(n-1)/2, n/2].  If the
  // box [p - rad, p + rad] reaches past that range (few cells per axis, or a
  // large radius), the cell can meet the box through another periodic image:
  // then all of it is scanned (every candidate is measured by its minimum
  // image, so scanning more is always correct).
  if (rad >= g.safe) {
    g.sx0r = 0; g.sx1r = s - 1; g.sr = 0; g.sr1 = s - 1;
    g.in_rect = true;
    return true;
  }
  const int64_t cx0 = cell_lo_tab(ucx, g.nx, g.bx, R.L[0]);
  const int64_t wx = cell_lo_tab(ucx + 1, g.nx, g.bx, R.L[0]) - cx0;
  const int64_t cy0 = cell_lo_tab(ucy, g.ny, g.by, R.L[1]);
  const int64_t wy = cell_lo_tab(ucy + 1, g.ny, g.by, R.L[1]) - cy0;
  const int64_t lx = g.px - rad - cx0, hx = g.px + rad - cx0;
  const int64_t ly = g.py - rad - cy0, hy = g.py + rad - cy0;
  if (hx < 0 || lx >= wx || hy < 0 || ly >= wy) return false;
  g.sx0r = lx <= 0 ? 0 : sub_idx(lx, wx, s);
  g.sx1r = hx >= wx ? s - 1 : sub_idx(hx, wx, s);
  g.sr = ly <= 0 ? 0 : sub_idx(ly, wy, s);
  g.sr1 = hy >= wy ? s - 1 : sub_idx(hy, wy, s);
  g.in_rect = true;
  return true;
}

__device__ __forceinline__ void gen_ring2(RunGen& g) {
  const int r = g.r;
  g.lox = -min(r, (g.nx - 1) / 2); g.hix = min(r, g.nx / 2);
  g.loy = -min(r, (g.ny - 1) / 2); g.hiy = min(r, g.ny / 2);
  g.plox = r ? -min(r - 1, (g.nx - 1) / 2) : 1; g.phix = r ? min(r - 1, g.nx / 2) : 0;
  g.ploy = r ? -min(r - 1, (g.ny - 1) / 2) : 1; g.phiy = r ? min(r - 1, g.ny / 2) : 0;
  g.oy = g.loy;
  g.ucy = g.cy + g.oy;
  gen_row_parts(g);
}

__device__ __forceinline__ void gen_ring1(RunGen& g) {
  const int r = g.r, s = g.s1;
  g.bx0 = max(g.sx - r, 0); g.bx1 = min(g.sx + r, s - 1);
  g.by0 = max(g.sy - r, 0); g.by1 = min(g.sy + r, s - 1);
  g.px0 = r ? max(g.sx - r + 1, 0) : 1; g.px1 = r ? min(g.sx + r - 1, s - 1) : 0;
  g.py0 = r ? max(g.sy - r + 1, 0) : 1; g.py1 = r ? min(g.sy + r - 1, s - 1) : 0;
  g.yy = g.by0;
  g.seg = 0;
}

__device__ __forceinline__ void gen_init(RunGen& g, const Rep& R, const uint32_t* __restrict__ bounds,
                                         const GridView& G, uint32_t px, uint32_t py, int k) {
  g.R = &R;
  g.bx = bounds + R.bnd[0];
  g.by = bounds + R.bnd[1];
  g.G = G;
  g.px = px;
  g.py = py;
  g.nx = R.nc[0];
  g.ny = R.nc[1];
  g.cx = cell_of_tab(px, g.nx, g.bx, R.inv_w[0]);
  g.cy = cell_of_tab(py, g.ny, g.by, R.inv_w[1]);
  g.own = R.c0 + (int64_t)g.cy * g.nx + g.cx;
  g.safe = min(min((int64_t)px - cell_lo_tab(g.cx - (g.nx - 1) / 2, g.nx, g.bx, R.L[0]),
                   cell_lo_tab(g.cx + g.nx / 2 + 1, g.nx, g.bx, R.L[0]) - (int64_t)px),
               min((int64_t)py - cell_lo_tab(g.cy - (g.ny - 1) / 2, g.ny, g.by, R.L[1]),
                   cell_lo_tab(g.cy + g.ny / 2 + 1, g.ny, g.by, R.L[1]) - (int64_t)py));
  g.prad = -1;
  g.own_done = false;
  g.in_rect = false;
  g.ndef = 0;
  g.ob0 = __ldg(G.sub_base + g.own);
  const uint32_t ob1 = __ldg(G.sub_base + g.own + 1);
  g.r = 0;
  // phase 1 (sub-cell rings inside the own cell) bounds the rest of the own
  // cell by its distance to the scanned sub-block, which needs the own cell
  // to be narrower than half a period: at least 3 cells per axis
  if (ob1 - g.ob0 > 1 && g.nx >= 3 && g.ny >= 3) {
    g.phase = 1;
    g.s1 = __ldg(G.sub_s + g.own);
    g.cx0 = __ldg(g.bx + g.cx);
    g.wx1 = (int64_t)__ldg(g.bx + g.cx + 1) - g.cx0;
    g.cy0 = __ldg(g.by + g.cy);
    g.wy1 = (int64_t)__ldg(g.by + g.cy + 1) - g.cy0;
    g.sx = sub_idx(px - g.cx0, g.wx1, g.s1);
    g.sy = sub_idx(py - g.cy0, g.wy1, g.s1);
    // Start with the 3 x 3 block of sub-cells, scanned as whole rows, rather
    // than the own sub-cell and a ring around it: the own sub-cell (about 2
    // particles) rarely holds and certifies the k nearest.  Only a very dense
    // own sub-cell (more than 16 k particles, where the 64 x 64 cap of the
    // sub-grid leaves dense cluster cores) starts alone.
    const uint32_t os = g.ob0 + (uint32_t)(g.sy * g.s1 + g.sx);
    if (__ldg(G.sub_off + os + 1) - __ldg(G.sub_off + os) <= (uint32_t)(16 * k)) {
      g.r = 1;
      gen_ring1(g);
      g.px0 = 1;
      g.px1 = 0;
    } else {
      gen_ring1(g);
    }
  } else {
    g.phase = 2;
    gen_ring2(g);
  }
}

// squared distance bound of the current ring's block (call at kRingEnd);
// returns ~0ull when the phase has covered everything it can
__device__ __forceinline__ uint64_t gen_ring_bound(const RunGen& g) {
  int64_t B = INT64_MAX;
  if (g.phase == 1) {
    const int s = g.s1;
    if (g.bx0 == 0 && g.by0 == 0 && g.bx1 == s - 1 && g.by1 == s - 1) return ~0ull;
    if (g.bx0 > 0) B = min(B, g.px - (g.cx0 + sub_lo(g.bx0, g.wx1, s)) + 1);
    if (g.bx1 < s - 1) B = min(B, g.cx0 + sub_lo(g.bx1 + 1, g.wx1, s) - g.px);
    if (g.by0 > 0) B = min(B, g.py - (g.cy0 + sub_lo(g.by0, g.wy1, s)) + 1);
    if (g.by1 < s - 1) B = min(B, g.cy0 + sub_lo(g.by1 + 1, g.wy1, s) - g.py);
  } else {
    const bool fullx = g.hix - g.lox + 1 == g.nx, fully = g.hiy - g.loy + 1 == g.ny;
    if (fullx && fully) return ~0ull;
    const int r = g.r;
    if (!fullx) {
      B = min(B, g.px - cell_lo_tab(g.cx - r, g.nx, g.bx, g.R->L[0]) + 1);
      B = min(B, cell_lo_tab(g.cx + r + 1, g.nx, g.bx, g.R->L[0]) - g.px);
    }
    if (!fully) {
      B = min(B, g.py - cell_lo_tab(g.cy - r, g.ny, g.by, g.R->L[1]) + 1);
      B = min(B, cell_lo_tab(g.cy + r + 1, g.ny, g.by, g.R->L[1]) - g.py);
    }
  }
  return (uint64_t)B * (uint64_t)B;
}

// after kRingEnd: move to the next ring (stop=false) or end the phase (stop=true)
__device__ __forceinline__ bool gen_advance(RunGen& g, bool stop) {
  if (g.phase == 1) {
    g.own_done = true;
    if (!stop) {
      ++g.r;
      gen_ring1(g);
      return true;
    }
    g.phase = 2;
    g.r = 0;
    gen_ring2(g);
    return true;
  }
  if (stop) return false;
  ++g.r;
  const int lox = -min(g.r, (g.nx - 1) / 2), hix = min(g.r, g.nx / 2);
  const int loy = -min(g.r, (g.ny - 1) / 2), hiy = min(g.r, g.ny / 2);
  if (lox == g.lox && hix == g.hix && loy == g.loy && hiy == g.hiy) return false;  // nothing new
  gen_ring2(g);
  return true;
}

// next run [qb, qe) of the current ring, or kRingEnd
__device__ __forceinline__ int gen_next(RunGen& g, uint64_t r2, uint32_t& qb, uint32_t& qe) {
  const GridView& G = g.G;
  if (g.phase == 1) {
    for (;;) {
      if (g.yy > g.by1) return kRingEnd;
      const uint32_t rb = g.ob0 + (uint32_t)g.yy * g.s1;
      const bool oldrow = !(g.yy < g.py0 || g.yy > g.py1 || g.px0 > g.px1);
      int a, b;
      if (!oldrow) {
        a = g.bx0; b = g.bx1;
        ++g.yy;
      } else if (g.seg == 0) {
        a = g.bx0; b = g.px0 - 1;
        g.seg = 1;
      } else {
        a = g.px1 + 1; b = g.bx1;
        g.seg = 0;
        ++g.yy;
      }
      if (a > b) continue;
      qb = __ldg(G.sub_off + rb + a);
      qe = __ldg(G.sub_off + rb + b + 1);
      return kRun;
    }
  }
  for (;;) {
    if (g.in_rect) {  // rows of a split cell's rectangle
      if (g.sr > g.sr1) {
        g.in_rect = false;
        continue;
      }
      const uint32_t rb = g.sbase + (uint32_t)g.sr * g.sstride;
      ++g.sr;
      qb = __ldg(G.sub_off + rb + g.sx0r);
      qe = __ldg(G.sub_off + rb + g.sx1r + 1);
      return kRun;
    }
    if (g.part >= g.nparts) {  // next row
      if (g.oy + 1 > g.hiy) {
        if (g.ndef > 0) {  // deferred split cells, now with the current radius
          --g.ndef;
          gen_rect(g, g.def_g[g.ndef], g.def_ucx[g.ndef], g.def_ucy[g.ndef], r2);
          continue;
        }
        return kRingEnd;
      }
      ++g.oy;
      g.ucy = g.cy + g.oy;
      gen_row_parts(g);
      continue;
    }
    const int x0 = g.pa[g.part], x1 = g.pb[g.part];
    if (g.x < 0) {  // start of a part: one run when no cell in it is split
      // once the radius is known, a row that misses the box is skipped, and
      // so are (below) its cells that miss it
      g.prad = -1;
      if (r2 != ~0ull) {
        const int64_t rad = radius_upper(r2);
        if (rad < g.safe) {
          if (cell_lo_tab(g.ucy, g.ny, g.by, g.R->L[1]) > g.py + rad ||
              cell_lo_tab(g.ucy + 1, g.ny, g.by, g.R->L[1]) <= g.py - rad) {
            ++g.part;
            continue;
          }
          g.prad = rad;
        }
      }
      const uint32_t sb0 = __ldg(G.sub_base + g.rowbase + x0), sb1 = __ldg(G.sub_base + g.rowbase + x1 + 1);
      if (sb1 - sb0 == (uint32_t)(x1 - x0 + 1)) {
        ++g.part;
        qb = __ldg(G.off + g.rowbase + x0);
        qe = __ldg(G.off + g.rowbase + x1 + 1);
        return kRun;
      }
      g.x = x0;
    }
    if (g.x > x1) {
      ++g.part;
      g.x = -1;
      continue;
    }
    if (g.prad >= 0) {
      const int ucx = g.pu[g.part] + (g.x - x0);
      if (cell_lo_tab(ucx, g.nx, g.bx, g.R->L[0]) > g.px + g.prad ||
          cell_lo_tab(ucx + 1, g.nx, g.bx, g.R->L[0]) <= g.px - g.prad) {
        ++g.x;
        continue;
      }
    }
    // per cell: a maximal run of unsplit cells, or one split cell
    const int64_t gc = g.rowbase + g.x;
    uint32_t b0 = __ldg(G.sub_base + gc), b1 = __ldg(G.sub_base + gc + 1);
    if (b1 - b0 == 1) {
      const int xs = g.x;
      while (g.x + 1 <= x1) {
        const uint32_t c1 = __ldg(G.sub_base + gc + (g.x - xs) + 2);
        if (c1 - b1 != 1) break;
        b1 = c1;
        ++g.x;
      }
      qb = __ldg(G.off + g.rowbase + xs);
      qe = __ldg(G.off + g.rowbase + g.x + 1);
      ++g.x;
      return kRun;
    }
    const int xc = g.x;
    ++g.x;
    if (gc == g.own && g.own_done) continue;
    const int ucx = g.pu[g.part] + (xc - x0);
    if (r2 == ~0ull && g.ndef < 4) {
      g.def_g[g.ndef] = gc;
      g.def_ucx[g.ndef] = ucx;
      g.def_ucy[g.ndef] = g.ucy;
      ++g.ndef;
      continue;
    }
    gen_rect(g, gc, ucx, g.ucy, r2);
  }
}

template <int KC>
__device__ __forceinline__ void knn2_search(Ctx& C, const Rep& R, const uint32_t* __restrict__ bounds,
                                            const GridView& G, const int2* __restrict__ pos,
                                            const int32_t* __restrict__ ids, Top<KC>& T, int k) {
  RunGen g;
  gen_init(g, R, bounds, G, C.px, C.py, k);
  C.split = g.phase == 1;
  for (;;) {
    uint32_t qb = 0, qe = 0;
    const int ev = gen_next(g, T.d[KC - 1], qb, qe);
    if (ev == kRun) {
      scan_run<KC>(C, pos, ids, qb, qe, T);  // the only copy of the candidate loop
      continue;
    }
    // ring end: every unscanned particle (of the phase's region) is at
    // squared distance >= B2; an equal distance could still win on id
    const uint64_t B2 = gen_ring_bound(g);
    const bool stop = (B2 == ~0ull) || (T.d[KC - 1] < B2);
    if (!gen_advance(g, stop)) break;
  }
}

// the general update (vectorial noise, FP64 sums), kept out of line
__device__ __noinline__ void align_advect_general(const Rep& R, const StepParams& P, uint32_t step, int32_t id,
                                                  const float* ni, const HeadSum<2>& H, int m, const int32_t* pi,
                                                  int32_t* pout, float* nout) {
  align_advect<2>(R, P, step, id, ni, H, m, pi, pout, nout);
}

// Eq. (2) alignment + noise and Eq. (1) advection of one particle from its
// finished top-k; writes the next state and counts the new coarse cell.
template <int KC, bool FOV = true>
__device__ __forceinline__ void knn2_update(const Rep& R, const StepParams& P, int64_t step, int64_t s, int2 p,
                                            float2 nv, int32_t id, const Top<KC>& T,
                                            const uint32_t* __restrict__ bounds, const float2* __restrict__ S_dir,
                                            int2* __restrict__ U_pos, float2* __restrict__ U_dir,
                                            int32_t* __restrict__ U_id, uint32_t* __restrict__ counts, float* nnew) {
  // Eq. (2): neighbor headings in (D, id) order; with a field of view the
  // list may be shorter than k (unfilled entries have slot -1)
  HeadSum<2> H;
  H.init();
  const float ni[3] = {nv.x, nv.y, 0.f};
  int m = P.include_self ? 1 : 0;
  if (P.include_self) H.add(ni, P.sum_mode);
#pragma unroll
  for (int j = 0; j < KC; ++j) {
    if (j >= KC - P.k && (!FOV || T.slot[j] >= 0)) {
      const float2 d = __ldg(S_dir + T.slot[j]);
      const float v[2] = {d.x, d.y};
      H.add(v, P.sum_mode);
      ++m;
    }
  }
  const int32_t pi[3] = {p.x, p.y, 0};
  int32_t pout[3] = {0, 0, 0};
  if (P.noise == 0 && P.sum_mode != 2) {
    // angular noise, FP32 sums (the default) inline
    const uint4 w = philox4x32_10(make_uint4((uint32_t)id, (uint32_t)step, R.replica, 0u),
                                  make_uint2(P.seed_lo, P.seed_hi));
    const float u = unit24(w.x);
    const float Sx = P.sum_mode == 1 ? __fadd_rn(H.s[0], H.c[0]) : H.s[0];
    const float Sy = P.sum_mode == 1 ? __fadd_rn(H.s[1], H.c[1]) : H.s[1];
    // Eq. (2) with angular noise: the direction of S (the own heading when
    // S = 0) turned by eta (u - 1/2), as a rotation of the unit vector
    float ex = nv.x, ey = nv.y;
    if (Sx != 0.f || Sy != 0.f) {
      const float inv = rsqrtf(Sx * Sx + Sy * Sy);
      ex = Sx * inv;
      ey = Sy * inv;
    }
    float sn, cs;
    sincosf(R.eta * (u - 0.5f), &sn, &cs);
    nnew[0] = cs * ex - sn * ey;
    nnew[1] = sn * ex + cs * ey;
    const float hx = P.advect_new ? nnew[0] : nv.x, hy = P.advect_new ? nnew[1] : nv.y;
    int64_t qx = (int64_t)p.x + grid_step(R.s, hx), qy = (int64_t)p.y + grid_step(R.s, hy);
    if (qx < 0 || qx >= (int64_t)R.L[0]) {
      qx %= (int64_t)R.L[0];
      if (qx < 0) qx += R.L[0];
    }
    if (qy < 0 || qy >= (int64_t)R.L[1]) {
      qy %= (int64_t)R.L[1];
      if (qy < 0) qy += R.L[1];
    }
    pout[0] = (int32_t)qx;
    pout[1] = (int32_t)qy;
  } else {
    align_advect_general(R, P, (uint32_t)step, id, ni, H, m, pi, pout, nnew);
  }
  U_pos[s] = make_int2(pout[0], pout[1]);
  U_dir[s] = make_float2(nnew[0], nnew[1]);
  U_id[s] = id;
  const uint32_t* bx = bounds + R.bnd[0];
  const uint32_t* by = bounds + R.bnd[1];
  const int ncx = cell_of_tab((uint32_t)pout[0], R.nc[0], bx, R.inv_w[0]);
  const int ncy = cell_of_tab((uint32_t)pout[1], R.nc[1], by, R.inv_w[1]);
  atomicAdd(counts + R.c0 + (int64_t)ncy * R.nc[0] + ncx, 1u);
}

// thread-per-particle search + update (the walk of RunGen for every particle)
template <int KC>
__global__ void __launch_bounds__(kBlock, VK_KNN2_MIN_BLOCKS) knn2_step_kernel(
    const Rep* __restrict__ reps, const BlockTask* __restrict__ tasks, const uint32_t* __restrict__ bounds,
    const int2* __restrict__ S_pos, const float2* __restrict__ S_dir, const int32_t* __restrict__ S_id, GridView G,
    int2* __restrict__ U_pos, float2* __restrict__ U_dir, int32_t* __restrict__ U_id, uint32_t* __restrict__ counts,
    PhiAcc* __restrict__ phi_acc, const int64_t* __restrict__ d_step, StepParams P) {
  __shared__ PhiShared phs;
  phi_block_begin(phs);
  const BlockTask t = tasks[blockIdx.x];
  const Rep R = reps[t.rep];
  const int li = t.first + (int)threadIdx.x;
  const int64_t step = *d_step;
  float nnew[3] = {0.f, 0.f, 0.f};
  Ctx C;
  C.n_cand = 0;
  C.n_runs = 0;
  C.split = false;
  if (li < R.n) {
    const int64_t s = R.p0 + li;
    const int2 p = S_pos[s];
    const float2 nv = S_dir[s];
    const int32_t id = S_id[s];
    init_ctx(C, R, s, p);
    if (P.fov_cq != kViewAll) C.view = make_view(nv, P.fov_cq);
    Top<KC> T;
    top_init<KC>(T, P.k);
    knn2_search<KC>(C, R, bounds, G, S_pos, S_id, T, P.k);
    knn2_update<KC>(R, P, step, s, p, nv, id, T, bounds, S_dir, U_pos, U_dir, U_id, counts, nnew);
  }
  record_search_stats(P.stats, li < R.n, C.n_cand, C.n_runs, C.split);
  phi_block_end<2>(phs, nnew, phi_acc + ((size_t)(step % P.phi_cap) * (size_t)P.n_rep + (size_t)t.rep) * 3);
}

// row id of the export table: the ids of T in (D, id) order, -1 past the
// count found (a field of view may hold fewer than k)
template <int KC>
__device__ __forceinline__ void write_row(const Top<KC>& T, const int32_t* __restrict__ S_id, int32_t id, int k,
                                          int32_t* __restrict__ out) {
#pragma unroll
  for (int j = 0; j < KC; ++j)
    if (j >= KC - k) out[(int64_t)id * k + (j - (KC - k))] = T.slot[j] >= 0 ? __ldg(S_id + T.slot[j]) : -1;
}

template <int KC>
__global__ void __launch_bounds__(kBlock, 2) knn2_export_kernel(const Rep* __restrict__ reps, int rep,
                                                                const uint32_t* __restrict__ bounds,
                                                                const int2* __restrict__ S_pos,
                                                                const float2* __restrict__ S_dir,
                                                                const int32_t* __restrict__ S_id, GridView G, int k,
                                                                int32_t cq, int32_t* __restrict__ out) {
  const Rep R = reps[rep];
  const int li = blockIdx.x * kBlock + (int)threadIdx.x;
  if (li >= R.n) return;
  const int64_t s = R.p0 + li;
  Ctx C;
  init_ctx(C, R, s, S_pos[s]);
  if (cq != kViewAll) C.view = make_view(S_dir[s], cq);
  Top<KC> T;
  top_init<KC>(T, k);
  knn2_search<KC>(C, R, bounds, G, S_pos, S_id, T, k);
  write_row<KC>(T, S_id, S_id[s], k, out);
}

// ---------------------------------------------------------------------------
// Radius-first search (the default).  Each particle knows roughly how far
// its k-th neighbor is: its k-th distance at the previous step, kept as a
// per-particle hint in the state (particles move by at most v0 dt per step,
// and neighbors mostly move together).  So it scans, once, every particle of
// the square [p - a, p + a], a a little above that distance: the sub-cell
// rows of the one to four coarse cells that overlap the square, each a
// contiguous run of the sorted arrays.  A candidate whose exact int64
// squared distance D is <= tau = (a+1)^2 - 1 goes to the particle's short
// hit list in shared memory; nothing outside the square is that close, so
// with at least k hits the k best hits by (D, id) are exactly the k nearest.
// The hits are merged into the register top-k by a branch-free insertion on
// D.  With fewer than k hits the square doubles and the scan repeats.  Equal
// distances (the ids must decide), a full hit list, or a square wider than
// half the period hand the particle to the per-particle walk, which runs in
// a separate kernel over a device list so that its code and registers stay
// out of this one; so do particles that need a second square, so that a
// warp never waits for one particle's rescan.
// ---------------------------------------------------------------------------
constexpr int kBoxTries = 4;  // square sizes tried before the walk takes over


template <int KC>
struct BoxHits {
  static constexpr int kCap = KC + 16;  // buffered hits per particle (merged when full)
  static constexpr int kRuns = VK_KNN2_BOX_RUNS;  // slot runs of one square
  int32_t slot[kCap][kBlock];           // one column per thread
  uint2 run[kRuns][kBlock];             // (first slot, length << 4 | image shift codes)
};

// Merge the thread's hits into T by a branch-free insertion on D and return
// how many of them count: the particle itself is skipped, and so is a hit
// outside the field of view (the view test runs here, per hit, not per
// candidate in the scan).  Sets *tie if two counted candidates at the same
// distance met (their order, or which of them is kept, needs the ids: the
// caller falls back to the walk).
template <int KC>
__device__ __forceinline__ int box_merge(const BoxHits<KC>& H, int cnt, const Ctx& C, const int2* __restrict__ pos,
                                         Top<KC>& T, bool* tie) {
  bool t = false;
  int got = 0;
  for (int b = 0; b < cnt; ++b) {
    const int32_t q = H.slot[b][threadIdx.x];
    if ((int64_t)q == C.self) continue;  // the particle is a hit of its own square
    int32_t dx, dy;
    const uint64_t D = box_offset(C, __ldg(pos + q), dx, dy);
    if (!in_view(C.view, dx, dy, D)) continue;
    ++got;
    t |= D == T.d[KC - 1];
    if (D < T.d[KC - 1]) {
      bool lt_hi = true;
#pragma unroll
      for (int s = KC - 1; s > 0; --s) {
        const bool lt_lo = D < T.d[s - 1];
        t |= D == T.d[s - 1];
        const uint64_t nd = lt_lo ? T.d[s - 1] : (lt_hi ? D : T.d[s]);
        const int32_t ns = lt_lo ? T.slot[s - 1] : (lt_hi ? q : T.slot[s]);
        T.d[s] = nd;
        T.slot[s] = ns;
        lt_hi = lt_lo;
      }
      if (lt_hi) {
        T.d[0] = D;
        T.slot[0] = q;
      }
    }
  }
  *tie = *tie || t;
  return got;
}

// kNN visitor of the square walk: candidates with D <= tau go to the hit
// list, which is merged into T when nearly full (tau then shrinks to T's
// k-th distance) and by the caller at the end.  AHEAD (a view of at most a
// half-plane, cq >= 0): a candidate behind the particle (d.nq < 0, exact in
// int64) is out of view and is not buffered; the merge decides the rest.
template <int KC, bool AHEAD>
struct KnnVisit {
  BoxHits<KC>& H;
  const Ctx& C;
  const int2* __restrict__ pos;
  Top<KC>& T;
  bool* tie;
  uint64_t tau;
  int cnt, got;
  __device__ __forceinline__ void group(uint32_t q, uint32_t n, const int2* pj, uint32_t ox, uint32_t oy) {
    // branch-free append: every candidate is written at the next free slot,
    // and the slot advances only for a hit
#pragma unroll
    for (int u = 0; u < kGroup; ++u) {
      const int32_t dx = (int32_t)((uint32_t)pj[u].x - ox), dy = (int32_t)((uint32_t)pj[u].y - oy);
      const uint64_t D = (uint64_t)((int64_t)dx * dx) + (uint64_t)((int64_t)dy * dy);
      bool hit = (uint32_t)u < n && D <= tau;
      if (AHEAD) hit = hit && (long long)dx * C.view.nxq + (long long)dy * C.view.nyq >= 0;
      H.slot[cnt][threadIdx.x] = (int32_t)(q + (uint32_t)u);
      cnt += hit ? 1 : 0;
    }
    if (cnt > BoxHits<KC>::kCap - kGroup) {  // rare: a nearly full buffer is merged on the spot
      got += box_merge<KC>(H, cnt, C, pos, T, tie);
      cnt = 0;
      if (T.d[KC - 1] < tau) tau = T.d[KC - 1];
    }
  }
};

// Scan the square [p - a, p + a] into T (initialised by the caller): every
// slot with D <= tau = (a+1)^2 - 1 is a hit.  Nothing outside the square is
// that close.  Hits are buffered and merged into T at the end (and, rarely,
// when the buffer fills, after which tau shrinks to T's k-th distance).
// Returns the number of hits that count (other particles, in view), >= k
// exactly when T is full, or -1 when the square is too wide for the minimum
// image or meets a coarse cell through two periodic images.
template <int KC, bool AHEAD>
__device__ __forceinline__ int box_scan_v(BoxHits<KC>& H, const Rep& R, const uint32_t* __restrict__ bounds,
                                          const GridView& G, const int2* __restrict__ pos, const Ctx& C, int64_t a,
                                          Top<KC>& T, bool* tie, BoxCount& bc) {
  KnnVisit<KC, AHEAD> v{H, C, pos, T, tie, (uint64_t)(a + 1) * (uint64_t)(a + 1) - 1, 0, 0};
  if (!box_walk(H, R, bounds, G, pos, C, a, bc, v)) return -1;
  // after the loop, where the threads have reconverged
  return v.got + box_merge<KC>(H, v.cnt, C, pos, T, tie);
}

// the view is the same for every particle: the branch is warp-uniform, and
// only one copy of the scan loop runs in a given simulation
template <int KC>
__device__ __forceinline__ int box_scan(BoxHits<KC>& H, const Rep& R, const uint32_t* __restrict__ bounds,
                                        const GridView& G, const int2* __restrict__ pos, const Ctx& C, int64_t a,
                                        Top<KC>& T, bool* tie, BoxCount& bc) {
  if (C.view.cq >= 0) return box_scan_v<KC, true>(H, R, bounds, G, pos, C, a, T, tie, bc);
  return box_scan_v<KC, false>(H, R, bounds, G, pos, C, a, T, tie, bc);
}

// search radius without a hint: a multiple of the k-th distance expected
// from the density of the particle's own sub-cell
__device__ __forceinline__ float box_radius_estimate(const Rep& R, const uint32_t* __restrict__ bounds,
                                                     const GridView& G, int2 p, int k) {
  const uint32_t* bx = bounds + R.bnd[0];
  const uint32_t* by = bounds + R.bnd[1];
  const int cx = cell_of_tab((uint32_t)p.x, R.nc[0], bx, R.inv_w[0]);
  const int cy = cell_of_tab((uint32_t)p.y, R.nc[1], by, R.inv_w[1]);
  const int64_t gc = R.c0 + (int64_t)cy * R.nc[0] + cx;
  const uint32_t sb0 = __ldg(G.sub_base + gc), sb1 = __ldg(G.sub_base + gc + 1);
  const int64_t x0 = __ldg(bx + cx), wx = (int64_t)__ldg(bx + cx + 1) - x0;
  const int64_t y0 = __ldg(by + cy), wy = (int64_t)__ldg(by + cy + 1) - y0;
  int s = 1;
  uint32_t cnt;
  if (sb1 - sb0 > 1) {
    s = __ldg(G.sub_s + gc);
    const uint32_t sub = sb0 + (uint32_t)(sub_idx((int64_t)p.y - y0, wy, s) * s + sub_idx((int64_t)p.x - x0, wx, s));
    cnt = __ldg(G.sub_off + sub + 1) - __ldg(G.sub_off + sub);
  } else {
    cnt = __ldg(G.off + gc + 1) - __ldg(G.off + gc);
  }
  const float area = (float)wx * (float)wy / ((float)s * (float)s);
  return 1.6f * sqrtf((float)k * area / (3.14159265f * (float)max(cnt, 1u)));
}

// The radius-first search of one particle with a first radius r: up to
// `tries` squares.  A square with fewer than k hits is followed by one with
// the radius scaled up towards about 1.5 k expected hits (hits grow with the
// area, the square of the radius).
// Returns true when T holds the exact top-k; otherwise *r_next is the radius
// to try next, or -1 when only the walk can serve the particle (a square
// too wide for the box, or two candidates at the same distance).
template <int KC>
__device__ __forceinline__ bool box_search(BoxHits<KC>& H, const Rep& R, const uint32_t* __restrict__ bounds,
                                           const GridView& G, const int2* __restrict__ pos, const Ctx& C, float r,
                                           int k, int tries, Top<KC>& T, BoxCount& bc, float* r_next) {
  for (int tr = 0; tr < tries; ++tr) {
    const int64_t a = (int64_t)ceilf(fminf(r, 2.0e9f));
    bool tie = false;
    top_init<KC>(T, k);
    const int hits = box_scan<KC>(H, R, bounds, G, pos, C, a, T, &tie, bc);
    if (hits < 0) {
      bc.why = 1u;
      *r_next = -1.f;
      return false;
    }
    if (hits >= k) {
      bc.hits += (uint32_t)hits;
      if (!tie) return true;
      bc.why = 3u;
      *r_next = -1.f;
      return false;
    }
    const float want = 1.5f * (float)k + 1.f;
    const float f = hits > 0 ? sqrtf(want / (float)hits) : 2.f;
    r = (float)a * fminf(f, 2.f);
  }
  bc.why = 2u;
  *r_next = r;
  return false;
}

// Tracing: totals of the radius-first counters (stats[5..13]).
__device__ __forceinline__ void record_box_stats(unsigned long long* stats, const BoxCount& bc) {
  if (!stats) return;
  unsigned long long v[9] = {bc.tries, bc.runs, bc.cand, bc.cells, bc.hits, bc.why == 1u, bc.why == 2u,
                              bc.why == 3u, bc.why == 4u};
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int i = 0; i < 9; ++i) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
  if ((threadIdx.x & 31) == 0)
#pragma unroll
    for (int i = 0; i < 9; ++i) atomicAdd(stats + 5 + i, v[i]);
}

// Append (slot, replica) to a device list, one atomic per warp: the
// warp's entries land next to each other, so the kernel that consumes the
// list reads spatially close particles in one warp.  Every lane of the warp
// must call it.
__device__ __forceinline__ void warp_append(bool put, int2 e, int2* __restrict__ list, int32_t* __restrict__ count) {
  const unsigned m = __ballot_sync(0xffffffffu, put);
  if (m == 0u) return;
  const int lane = (int)(threadIdx.x & 31);
  int base = 0;
  if (lane == __ffs(m) - 1) base = atomicAdd(count, __popc(m));
  base = __shfl_sync(0xffffffffu, base, __ffs(m) - 1);
  if (put) list[base + __popc(m & ((1u << lane) - 1u))] = e;
}

// Search + update, radius first, one square per particle.  Particles it
// cannot serve go on the deferred list (slot, replica) with the radius to
// try next in U_hint (-1: walk), and knn2_deferred_kernel finishes them: a
// warp here never waits for one particle's second square.
template <int KC, bool FOV>
__global__ void __launch_bounds__(kBlock, VK_KNN2_BOX_BLOCKS) knn2_box_step_kernel(
    const Rep* __restrict__ reps, const BlockTask* __restrict__ tasks, const uint32_t* __restrict__ bounds,
    const int2* __restrict__ S_pos, const float2* __restrict__ S_dir, const int32_t* __restrict__ S_id,
    const float* __restrict__ S_hint, GridView G, int2* __restrict__ U_pos, float2* __restrict__ U_dir,
    int32_t* __restrict__ U_id, float* __restrict__ U_hint, uint32_t* __restrict__ counts,
    PhiAcc* __restrict__ phi_acc, const int64_t* __restrict__ d_step, StepParams P, int2* __restrict__ defer_list,
    int32_t* __restrict__ defer_count) {
  extern __shared__ __align__(16) unsigned char box_smem[];
  BoxHits<KC>& H = *reinterpret_cast<BoxHits<KC>*>(box_smem);
  __shared__ PhiShared phs;
  phi_block_begin(phs);
  const BlockTask t = tasks[blockIdx.x];
  const Rep R = reps[t.rep];
  const int li = t.first + (int)threadIdx.x;
  const bool valid = li < R.n;
  const int64_t step = *d_step;
  float nnew[3] = {0.f, 0.f, 0.f};
  BoxCount bc;
  bool served = false;
  if (valid) {
    const int64_t s = R.p0 + li;
    const int2 p = S_pos[s];
    const float hint = S_hint[s];
    Ctx C;
    init_ctx(C, R, s, p);
    if (FOV) C.view = make_view(S_dir[s], P.fov_cq);
    Top<KC> T;
    const float r =
        hint > 0.f ? P.halo_alpha * hint + P.halo_beta * fabsf(R.s) : box_radius_estimate(R, bounds, G, p, P.k);
    float r_next = -1.f;
    served = box_search<KC>(H, R, bounds, G, S_pos, C, r, P.k, 1, T, bc, &r_next);
    if (served) {
      knn2_update<KC, FOV>(R, P, step, s, p, S_dir[s], S_id[s], T, bounds, S_dir, U_pos, U_dir, U_id, counts, nnew);
      U_hint[s] = sqrtf((float)T.d[KC - 1]) * 1.0001f + 1.f;
    } else {
      U_hint[s] = r_next;
    }
  }
  warp_append(valid && !served, make_int2((int)(R.p0 + li), t.rep), defer_list, defer_count);
  record_search_stats(P.stats, served, bc.cand, bc.tries, false);
  record_box_stats(P.stats, bc);
  phi_block_end<2>(phs, nnew, phi_acc + ((size_t)(step % P.phi_cap) * (size_t)P.n_rep + (size_t)t.rep) * 3);
}

// Search + update of the deferred particles: more squares from the radius
// the step kernel left in U_hint.  A grid of one thread per particle covers
// a list of any length (the length is read on the device, so the launch can
// sit in a CUDA graph); particles that still cannot be served go on the walk
// list.
template <int KC, bool FOV>
__global__ void __launch_bounds__(kBlock, VK_KNN2_DEFER_BLOCKS) knn2_deferred_kernel(
    const Rep* __restrict__ reps, const uint32_t* __restrict__ bounds, const int2* __restrict__ S_pos,
    const float2* __restrict__ S_dir, const int32_t* __restrict__ S_id, GridView G, int2* __restrict__ U_pos,
    float2* __restrict__ U_dir, int32_t* __restrict__ U_id, float* __restrict__ U_hint,
    uint32_t* __restrict__ counts, PhiAcc* __restrict__ phi_acc, const int64_t* __restrict__ d_step, StepParams P,
    const int2* __restrict__ defer_list, const int32_t* __restrict__ defer_count, int2* __restrict__ walk_list,
    int32_t* __restrict__ walk_count) {
  extern __shared__ __align__(16) unsigned char box_smem[];
  BoxHits<KC>& H = *reinterpret_cast<BoxHits<KC>*>(box_smem);
  const int total = *defer_count;
  if ((int)(blockIdx.x * kBlock) >= total) return;  // whole block past the list
  const int i = blockIdx.x * kBlock + (int)threadIdx.x;
  const int64_t step = *d_step;
  float nnew[3] = {0.f, 0.f, 0.f};
  bool served = false;
  int rep = 0;
  BoxCount bc;
  int2 e = make_int2(0, 0);
  if (i < total) {
    e = defer_list[i];
    const int64_t s = e.x;
    rep = e.y;
    const Rep R = reps[e.y];
    const int2 p = S_pos[s];
    Ctx C;
    init_ctx(C, R, s, p);
    if (FOV) C.view = make_view(S_dir[s], P.fov_cq);
    Top<KC> T;
    const float r = U_hint[s];
    float r_next = -1.f;
    served = r > 0.f && box_search<KC>(H, R, bounds, G, S_pos, C, r, P.k, kBoxTries, T, bc, &r_next);
    if (served) {
      knn2_update<KC, FOV>(R, P, step, s, p, S_dir[s], S_id[s], T, bounds, S_dir, U_pos, U_dir, U_id, counts, nnew);
      U_hint[s] = sqrtf((float)T.d[KC - 1]) * 1.0001f + 1.f;
    }
  }
  warp_append(i < total && !served, e, walk_list, walk_count);
  phi_add_warp<2>(phi_acc + (size_t)(step % P.phi_cap) * (size_t)P.n_rep * 3, rep, nnew, served);
  if (P.stats && served) {
    atomicAdd(P.stats + 0, (unsigned long long)bc.cand);
    atomicAdd(P.stats + 1, (unsigned long long)bc.tries);
    atomicMax(P.stats + 2, (unsigned long long)bc.cand);
    atomicAdd(P.stats + 3, 1ull);
  }
}

// Per-particle walk + update for the particles the radius-first kernels
// could not serve (squares wider than the box allows, equal distances, no
// fitting square).  A small fixed grid strides over the (short) list; the
// stride loop is warp-uniform so that the order-parameter add is too.
template <int KC>
__global__ void __launch_bounds__(kBlock, 2) knn2_walk_list_kernel(
    const Rep* __restrict__ reps, const uint32_t* __restrict__ bounds, const int2* __restrict__ S_pos,
    const float2* __restrict__ S_dir, const int32_t* __restrict__ S_id, GridView G, int2* __restrict__ U_pos,
    float2* __restrict__ U_dir, int32_t* __restrict__ U_id, float* __restrict__ U_hint,
    uint32_t* __restrict__ counts, PhiAcc* __restrict__ phi_acc, const int64_t* __restrict__ d_step, StepParams P,
    const int2* __restrict__ walk_list, const int32_t* __restrict__ walk_count) {
  const int total = *walk_count;
  const int64_t step = *d_step;
  PhiAcc* step_acc = phi_acc + (size_t)(step % P.phi_cap) * (size_t)P.n_rep * 3;
  for (int base = blockIdx.x * kBlock; base < total; base += gridDim.x * kBlock) {
    const int i = base + (int)threadIdx.x;
    float nnew[3] = {0.f, 0.f, 0.f};
    int rep = 0;
    const bool active = i < total;
    if (active) {
      const int2 e = walk_list[i];
      const int64_t s = e.x;
      rep = e.y;
      const Rep R = reps[e.y];
      const int2 p = S_pos[s];
      Ctx C;
      init_ctx(C, R, s, p);
      if (P.fov_cq != kViewAll) C.view = make_view(S_dir[s], P.fov_cq);
      Top<KC> T;
      top_init<KC>(T, P.k);
      knn2_search<KC>(C, R, bounds, G, S_pos, S_id, T, P.k);
      knn2_update<KC>(R, P, step, s, p, S_dir[s], S_id[s], T, bounds, S_dir, U_pos, U_dir, U_id, counts, nnew);
      U_hint[s] = sqrtf((float)T.d[KC - 1]) * 1.0001f + 1.f;
      if (P.stats) {
        atomicAdd(P.stats + 0, (unsigned long long)C.n_cand);
        atomicAdd(P.stats + 1, (unsigned long long)C.n_runs);
        atomicMax(P.stats + 2, (unsigned long long)C.n_cand);
        atomicAdd(P.stats + 3, 1ull);
        atomicAdd(P.stats + 4, 1ull);
      }
    }
    phi_add_warp<2>(step_acc, rep, nnew, active);
  }
}

template <int KC>
__global__ void __launch_bounds__(kBlock, 3) knn2_box_export_kernel(
    const Rep* __restrict__ reps, int rep, const uint32_t* __restrict__ bounds, const int2* __restrict__ S_pos,
    const float2* __restrict__ S_dir, const int32_t* __restrict__ S_id, const float* __restrict__ S_hint, GridView G,
    int k, int32_t cq, float alpha, float beta, int32_t* __restrict__ out, int2* __restrict__ walk_list,
    int32_t* __restrict__ walk_count) {
  extern __shared__ __align__(16) unsigned char box_smem[];
  BoxHits<KC>& H = *reinterpret_cast<BoxHits<KC>*>(box_smem);
  const Rep R = reps[rep];
  const int li = blockIdx.x * kBlock + (int)threadIdx.x;
  if (li >= R.n) return;
  const int64_t s = R.p0 + li;
  const int2 p = S_pos[s];
  Ctx C;
  init_ctx(C, R, s, p);
  if (cq != kViewAll) C.view = make_view(S_dir[s], cq);
  Top<KC> T;
  BoxCount bc;
  const float hint = S_hint ? S_hint[s] : 0.f;
  const float r = hint > 0.f ? alpha * hint + beta * fabsf(R.s) : box_radius_estimate(R, bounds, G, p, k);
  float r_next = -1.f;
  if (!box_search<KC>(H, R, bounds, G, S_pos, C, r, k, kBoxTries, T, bc, &r_next)) {
    walk_list[atomicAdd(walk_count, 1)] = make_int2((int)s, rep);
    return;
  }
  write_row<KC>(T, S_id, S_id[s], k, out);
}

// the per-particle walk for the listed particles of an export
template <int KC>
__global__ void __launch_bounds__(kBlock, 2) knn2_walk_export_list_kernel(
    const Rep* __restrict__ reps, const uint32_t* __restrict__ bounds, const int2* __restrict__ S_pos,
    const float2* __restrict__ S_dir, const int32_t* __restrict__ S_id, GridView G, int k, int32_t cq,
    int32_t* __restrict__ out, const int2* __restrict__ walk_list, const int32_t* __restrict__ walk_count) {
  const int total = *walk_count;
  for (int i = blockIdx.x * kBlock + (int)threadIdx.x; i < total; i += gridDim.x * kBlock) {
    const int2 e = walk_list[i];
    const int64_t s = e.x;
    const Rep R = reps[e.y];
    Ctx C;
    init_ctx(C, R, s, S_pos[s]);
    if (cq != kViewAll) C.view = make_view(S_dir[s], cq);
    Top<KC> T;
    top_init<KC>(T, k);
    knn2_search<KC>(C, R, bounds, G, S_pos, S_id, T, k);
    write_row<KC>(T, S_id, S_id[s], k, out);
  }
}

GridView view_of(const Buffers& b) {
  GridView G;
  G.off = b.offsets;
  G.sub_s = b.sub_s;
  G.sub_base = b.sub_base;
  G.sub_off = b.sub_off;
  return G;
}

template <int KC>
constexpr size_t box_smem_bytes() {
  return sizeof(BoxHits<KC>);
}

// blocks of the deferred-particle kernel: enough threads for a list of every
// particle (the length is known only on the device; threads past it exit at
// once), so a long list never queues on a few threads
int walk_blocks(const Geometry& g) { return (int)std::max<int64_t>(1, (g.n_total + kBlock - 1) / kBlock); }

// blocks of the walk-list kernels: a small fixed grid striding over the
// (short) list
int walk_list_blocks(const Geometry& g) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((g.n_total + kBlock - 1) / kBlock, device_sm_count()));
}

template <int KC>
cudaError_t step2(const Geometry& g, const Buffers& b, const StepParams& P, cudaStream_t st) {
  if (P.knn_search == 1 || !b.S_hint) {
    knn2_step_kernel<KC><<<g.n_tasks, kBlock, 0, st>>>(g.reps, g.tasks, b.bounds, (const int2*)b.S_pos,
                                                       (const float2*)b.S_dir, b.S_id, view_of(b), (int2*)b.U_pos,
                                                       (float2*)b.U_dir, b.U_id, b.counts, b.phi_acc, b.d_step, P);
    if (b.U_hint) cudaMemsetAsync(b.U_hint, 0, sizeof(float) * (size_t)g.n_total, st);
  } else {
    // the lists are empty here: the previous scatter (or init) cleared them
    // a field of view gets its own instantiation, so that the plain rule
    // carries no view code (registers)
    auto k = P.fov_cq != kViewAll ? knn2_box_step_kernel<KC, true> : knn2_box_step_kernel<KC, false>;
    k<<<g.n_tasks, kBlock, box_smem_bytes<KC>(), st>>>(
        g.reps, g.tasks, b.bounds, (const int2*)b.S_pos, (const float2*)b.S_dir, b.S_id, b.S_hint, view_of(b),
        (int2*)b.U_pos, (float2*)b.U_dir, b.U_id, b.U_hint, b.counts, b.phi_acc, b.d_step, P, b.ovf_list,
        b.ovf_count);
  }
  return cudaGetLastError();
}

template <int KC>
cudaError_t finish2(const Geometry& g, const Buffers& b, const StepParams& P, cudaStream_t st) {
  if (P.knn_search == 0 && b.S_hint) {
    // the deferred list lives in the first half of ovf_list, the walk list in the second
    auto k = P.fov_cq != kViewAll ? knn2_deferred_kernel<KC, true> : knn2_deferred_kernel<KC, false>;
    k<<<walk_blocks(g), kBlock, box_smem_bytes<KC>(), st>>>(
        g.reps, b.bounds, (const int2*)b.S_pos, (const float2*)b.S_dir, b.S_id, view_of(b), (int2*)b.U_pos,
        (float2*)b.U_dir, b.U_id, b.U_hint, b.counts, b.phi_acc, b.d_step, P, b.ovf_list, b.ovf_count,
        b.ovf_list + g.n_total, b.ovf_count + 1);
    knn2_walk_list_kernel<KC><<<walk_list_blocks(g), kBlock, 0, st>>>(
        g.reps, b.bounds, (const int2*)b.S_pos, (const float2*)b.S_dir, b.S_id, view_of(b), (int2*)b.U_pos,
        (float2*)b.U_dir, b.U_id, b.U_hint, b.counts, b.phi_acc, b.d_step, P, b.ovf_list + g.n_total,
        b.ovf_count + 1);
  }
  return cudaGetLastError();
}

template <int KC>
cudaError_t export2(const Geometry& g, const Buffers& b, int k, int rep, int n, int32_t* out, cudaStream_t st,
                    const StepParams& P) {
  const int nb = (n + kBlock - 1) / kBlock;
  if (nb == 0) return cudaSuccess;
  if (P.knn_search == 1 || !b.S_hint) {
    knn2_export_kernel<KC><<<nb, kBlock, 0, st>>>(g.reps, rep, b.bounds, (const int2*)b.S_pos,
                                                  (const float2*)b.S_dir, b.S_id, view_of(b), k, P.fov_cq, out);
  } else {
    cudaError_t e = cudaMemsetAsync(b.ovf_count, 0, sizeof(int32_t), st);
    if (e != cudaSuccess) return e;
    knn2_box_export_kernel<KC><<<nb, kBlock, box_smem_bytes<KC>(), st>>>(
        g.reps, rep, b.bounds, (const int2*)b.S_pos, (const float2*)b.S_dir, b.S_id, b.S_hint, view_of(b), k,
        P.fov_cq, P.halo_alpha, P.halo_beta, out, b.ovf_list, b.ovf_count);
    knn2_walk_export_list_kernel<KC><<<walk_list_blocks(g), kBlock, 0, st>>>(
        g.reps, b.bounds, (const int2*)b.S_pos, (const float2*)b.S_dir, b.S_id, view_of(b), k, P.fov_cq, out,
        b.ovf_list, b.ovf_count);
    // leave the list empty for the next step
    e = cudaMemsetAsync(b.ovf_count, 0, sizeof(int32_t), st);
    if (e != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

template <int KC>
cudaError_t prepare2() {
  cudaError_t e = cudaFuncSetAttribute(knn2_box_step_kernel<KC, false>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)box_smem_bytes<KC>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(knn2_box_step_kernel<KC, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)box_smem_bytes<KC>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(knn2_box_export_kernel<KC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)box_smem_bytes<KC>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(knn2_deferred_kernel<KC, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)box_smem_bytes<KC>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(knn2_deferred_kernel<KC, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)box_smem_bytes<KC>());
  return e;
}

}  // namespace

cudaError_t prepare_knn2() {
  cudaError_t e = prepare2<8>();
  if (e == cudaSuccess) e = prepare2<16>();
  if (e == cudaSuccess) e = prepare2<32>();
  return e;
}

cudaError_t launch_knn2_step(const Geometry& g, const Buffers& b, const StepParams& P, cudaStream_t st) {
  if (P.k <= 8) return step2<8>(g, b, P, st);
  if (P.k <= 16) return step2<16>(g, b, P, st);
  return step2<32>(g, b, P, st);
}

cudaError_t launch_knn2_finish(const Geometry& g, const Buffers& b, const StepParams& P, cudaStream_t st) {
  if (P.k <= 8) return finish2<8>(g, b, P, st);
  if (P.k <= 16) return finish2<16>(g, b, P, st);
  return finish2<32>(g, b, P, st);
}

cudaError_t launch_knn2_export(const Geometry& g, const Buffers& b, int k, int rep, int n, int32_t* out,
                               cudaStream_t st, const StepParams& P) {
  if (k <= 8) return export2<8>(g, b, k, rep, n, out, st, P);
  if (k <= 16) return export2<16>(g, b, k, rep, n, out, st, P);
  return export2<32>(g, b, k, rep, n, out, st, P);
}

}  // namespace vk
