// vk_voronoi.cuh -- the per-particle Voronoi cell builder (Sec.
// "Computational tools: Voronoi neighbor lists"), shared by the Voronoi rule
// (vk_voronoi.cu) and the Voronoi tissue model (vk_tissue.cu): half-plane
// clipping of the cell by the bisectors of candidate sites from the
// two-level grid, with exact predicates; see vk_voronoi.cu for the method.
// Exact predicates need |relative coordinates| < 1.5 * 2^30, hence L_q <= 2^30.
#pragma once
#include <algorithm>
#include <climits>

#include "vk_internal.cuh"

namespace vk {

namespace {

constexpr int kFastCap = 32;    // polygon capacity of the main kernel
constexpr int kSlowCap = kVoronoiMaxDeg;  // capacity of the overflow kernel and the export
constexpr uint32_t kHeavy = 384;  // candidates after which the main kernel hands a cell to the overflow kernel

__device__ __noinline__ int vertex_cut_exact(int32_t ax, int32_t ay, int32_t bx, int32_t by, int32_t mx,
                                             int32_t my);

// sign of incircle(0, a, b, m): > 0 iff m lies strictly inside the circle
// through the origin, a and b (with (0, a, b) counter-clockwise), i.e. iff
// the vertex defined by a and b is strictly closer to m than to the origin.
__device__ __forceinline__ int vertex_cut_sign(int32_t ax, int32_t ay, int32_t bx, int32_t by, int32_t mx,
                                               int32_t my) {
  // det3 = | ax ay al ; bx by bl ; mx my ml | = -incircle(0, a, b, m)
  const float fax = (float)ax, fay = (float)ay, fbx = (float)bx, fby = (float)by, fmx = (float)mx,
              fmy = (float)my;
  const float fal = fax * fax + fay * fay, fbl = fbx * fbx + fby * fby, fml = fmx * fmx + fmy * fmy;
  const float t1 = fby * fml, t2 = fbl * fmy, t3 = fbx * fml, t4 = fbl * fmx, t5 = fbx * fmy, t6 = fby * fmx;
  const float det = fax * (t1 - t2) - fay * (t3 - t4) + fal * (t5 - t6);
  const float perm = fabsf(fax) * (fabsf(t1) + fabsf(t2)) + fabsf(fay) * (fabsf(t3) + fabsf(t4)) +
                     fal * (fabsf(t5) + fabsf(t6));
  const float bound = perm * 1.9073486328125e-06f;  // 2^-19: 32 ulps of the permanent
  if (det > bound) return -1;
  if (det < -bound) return 1;
  return vertex_cut_exact(ax, ay, bx, by, mx, my);
}

// the exact incircle sign (int128), kept out of line: it is rarely needed,
// and a small hot loop keeps divergent warps in the instruction cache
__device__ __noinline__ int vertex_cut_exact(int32_t ax, int32_t ay, int32_t bx, int32_t by, int32_t mx,
                                             int32_t my) {
  const int64_t al = (int64_t)ax * ax + (int64_t)ay * ay;
  const int64_t bl = (int64_t)bx * bx + (int64_t)by * by;
  const int64_t ml = (int64_t)mx * mx + (int64_t)my * my;
  const __int128 A = (__int128)by * ml - (__int128)bl * my;
  const __int128 Bt = (__int128)bx * ml - (__int128)bl * mx;
  const __int128 C = (__int128)bx * my - (__int128)by * mx;
  const __int128 d = (__int128)ax * A - (__int128)ay * Bt + (__int128)al * C;
  return d > 0 ? -1 : (d < 0 ? 1 : 0);
}

// Vertex V = circumcenter of (0, a, b) (consecutive edge sites, so that
// ax*by - ay*bx > 0): FP32 estimate (vx, vy) with |vx - Vx|, |vy - Vy| <= e,
// and a rigorous FP32 upper bound of |V|^2 (returned).
__device__ __noinline__ float vertex_geom(int32_t ax, int32_t ay, int32_t bx, int32_t by, float* vx, float* vy,
                                          float* e, bool* bad) {
  const int64_t dh = (int64_t)ax * by - (int64_t)ay * bx;  // exact
  if (dh <= 0) {
    *bad = true;
    *vx = *vy = 0.f;
    *e = 3.0e38f;
    return 3.0e38f;
  }
  const float fax = (float)ax, fay = (float)ay, fbx = (float)bx, fby = (float)by;
  const float al = fax * fax + fay * fay, bl = fbx * fbx + fby * fby;
  const float p1 = fby * al, p2 = fay * bl, p3 = fax * bl, p4 = fbx * al;
  // numerator errors: 16 ulps of the magnitudes (inputs, squares, products, difference)
  const float ex = (fabsf(p1) + fabsf(p2)) * 9.5367431640625e-07f;
  const float ey = (fabsf(p3) + fabsf(p4)) * 9.5367431640625e-07f;
  const float d2 = 2.0f * (float)dh * (1.0f - 2.384185791015625e-07f);  // rounded down
  const float ax_ = (fabsf(p1 - p2) + ex) / d2;  // bounds of |Vx|, |Vy|
  const float ay_ = (fabsf(p3 - p4) + ey) / d2;
  const float r2 = (ax_ * ax_ + ay_ * ay_) * (1.0f + 9.5367431640625e-07f);
  const float q = 2.0f * (float)dh;
  *vx = (p1 - p2) / q;
  *vy = (p3 - p4) / q;
  // numerator error / denominator, plus the relative rounding of the quotient
  const float e0 = (fmaxf(ex, ey) / d2 + fmaxf(ax_, ay_) * 4.76837158203125e-07f) * 1.5f;
  *e = isfinite(e0) ? e0 : 3.0e38f;
  return isfinite(r2) ? r2 : 3.0e38f;
}

// Fast decision of "site m cuts vertex V", i.e. |m - V| < |V|, i.e.
// t = 2 m.V - |m|^2 > 0, from the FP32 estimate of V: returns +1 (cut), -1
// (not cut, not on the circle) or 0 (undecided: use the exact predicate).
__device__ __forceinline__ int vertex_cut_fast(float vx, float vy, float e, int32_t mx, int32_t my) {
  const float fmx = (float)mx, fmy = (float)my;
  const float a = 2.0f * fmx * vx, b = 2.0f * fmy * vy, c = fmx * fmx + fmy * fmy;
  const float t = (a + b) - c;
  // error of V (2 |m| e) plus 16 ulps of the magnitudes (inputs, products, sums)
  const float tol = (2.0f * (fabsf(fmx) + fabsf(fmy)) * e + (fabsf(a) + fabsf(b) + c) * 9.5367431640625e-07f) * 1.5f;
  if (!(tol < 1.0e37f)) return 0;
  if (t > tol) return 1;
  if (t < -tol) return -1;
  return 0;
}

// Coincident particles form one Voronoi site: they are each other's
// neighbors and share the site's neighbors.  A candidate at exactly the
// position of an edge site (or of the particle itself) clips nothing; it is
// kept in the twin list and joins the neighbors if that edge survives.
template <int CAP>
struct Poly {
  static constexpr int TW = CAP / 4;
  int32_t qx[CAP], qy[CAP];  // relative coordinates of the edge sites
  int32_t id[CAP];           // replica-local id of the site
  int32_t slot[CAP];         // sorted slot of the site (-1: an image of the particle itself)
  float vr2[CAP];            // vertex a (between edges a and a+1): upper bound of |V|^2
  float vx[CAP], vy[CAP];    // ... its FP32 estimate ...
  float ve[CAP];             // ... and the error bound of each coordinate
  int32_t tw_slot[TW];       // coincident twins: their sorted slot ...
  int32_t tw_id[TW];         // ... their id ...
  int32_t tw_of[TW];         // ... and the slot of the site they sit on (-2: the particle itself)
  int m;
  int nt;
  float max_r2;
  // relevance box (offsets from the particle, inclusive): every site that can
  // still cut the cell lies in the union of the disks through the particle
  // centred at the vertices, hence in this box; it only shrinks
  int64_t bx0, bx1, by0, by1;
};

__device__ __forceinline__ int64_t box_floor(float x) {
  if (!(x > -4.0e18f)) return -(int64_t)4e18;
  if (x > 4.0e18f) return (int64_t)4e18;
  return (int64_t)floorf(x) - 2;
}

__device__ __forceinline__ int64_t box_ceil(float x) {
  if (!(x < 4.0e18f)) return (int64_t)4e18;
  if (x < -4.0e18f) return -(int64_t)4e18;
  return (int64_t)ceilf(x) + 2;
}

template <int CAP>
__device__ __forceinline__ void poly_refresh_max(Poly<CAP>& P) {
  float mx = 0.f;
  for (int a = 0; a < P.m; ++a) mx = fmaxf(mx, P.vr2[a]);
  P.max_r2 = mx;
}

// recompute the relevance box; between calls it is stale but still valid,
// since the cell only shrinks
template <int CAP>
__device__ __noinline__ void poly_refresh_box(Poly<CAP>& P) {
  float x0 = 3.0e38f, x1 = -3.0e38f, y0 = 3.0e38f, y1 = -3.0e38f;
  for (int a = 0; a < P.m; ++a) {
    const float r = __fadd_ru(__fsqrt_ru(P.vr2[a]), P.ve[a]);
    x0 = fminf(x0, __fsub_rd(P.vx[a], r));
    x1 = fmaxf(x1, __fadd_ru(P.vx[a], r));
    y0 = fminf(y0, __fsub_rd(P.vy[a], r));
    y1 = fmaxf(y1, __fadd_ru(P.vy[a], r));
  }
  P.bx0 = box_floor(x0);
  P.bx1 = box_ceil(x1);
  P.by0 = box_floor(y0);
  P.by1 = box_ceil(y1);
}

template <int CAP>
__device__ __forceinline__ void poly_init(Poly<CAP>& P, int32_t self_id, uint32_t Lx, uint32_t Ly, bool* bad) {
  const int32_t X = (int32_t)Lx, Y = (int32_t)Ly;
  const int32_t sx[4] = {X, 0, -X, 0}, sy[4] = {0, Y, 0, -Y};
  P.m = 4;
  P.nt = 0;
  for (int a = 0; a < 4; ++a) {
    P.qx[a] = sx[a];
    P.qy[a] = sy[a];
    P.id[a] = self_id;
    P.slot[a] = -1;
  }
  for (int a = 0; a < 4; ++a)
    P.vr2[a] = vertex_geom(P.qx[a], P.qy[a], P.qx[(a + 1) & 3], P.qy[(a + 1) & 3], &P.vx[a], &P.vy[a], &P.ve[a],
                           bad);
  poly_refresh_max(P);
  poly_refresh_box(P);
}

// replace the cut vertices [s, s + c) (cyclic) by site m; returns false if
// the polygon would outgrow CAP.  Out of line: only actual cuts run it.
template <int CAP>
__device__ __noinline__ bool poly_apply_cut(Poly<CAP>& P, int s, int c, int32_t mx, int32_t my, int32_t mid,
                                            int32_t mslot, bool* bad) {
  const int m = P.m;
  const int t = (s + c - 1) % m;
  const int newm = m - c + 2;
  if (newm > CAP) return false;
  int mpos;
  if (s <= t) {
    // keep e_0..e_s, insert m, keep e_{t+1}..e_{m-1}
    const int delta = s + 2 - (t + 1);  // <= 1
    if (delta < 0) {
      for (int a = t + 1; a < m; ++a) {
        P.qx[a + delta] = P.qx[a]; P.qy[a + delta] = P.qy[a]; P.id[a + delta] = P.id[a];
        P.slot[a + delta] = P.slot[a]; P.vr2[a + delta] = P.vr2[a];
        P.vx[a + delta] = P.vx[a]; P.vy[a + delta] = P.vy[a]; P.ve[a + delta] = P.ve[a];
      }
    } else if (delta > 0) {
      for (int a = m - 1; a >= t + 1; --a) {
        P.qx[a + delta] = P.qx[a]; P.qy[a + delta] = P.qy[a]; P.id[a + delta] = P.id[a];
        P.slot[a + delta] = P.slot[a]; P.vr2[a + delta] = P.vr2[a];
        P.vx[a + delta] = P.vx[a]; P.vy[a + delta] = P.vy[a]; P.ve[a + delta] = P.ve[a];
      }
    }
    mpos = s + 1;
  } else {
    // the run wraps: keep e_{t+1}..e_s (contiguous), then m
    const int sh = t + 1;
    for (int a = sh; a <= s; ++a) {
      P.qx[a - sh] = P.qx[a]; P.qy[a - sh] = P.qy[a]; P.id[a - sh] = P.id[a];
      P.slot[a - sh] = P.slot[a]; P.vr2[a - sh] = P.vr2[a];
      P.vx[a - sh] = P.vx[a]; P.vy[a - sh] = P.vy[a]; P.ve[a - sh] = P.ve[a];
    }
    mpos = s - sh + 1;
  }
  P.qx[mpos] = mx;
  P.qy[mpos] = my;
  P.id[mpos] = mid;
  P.slot[mpos] = mslot;
  P.m = newm;
  const int before = (mpos == 0) ? newm - 1 : mpos - 1;
  const int after = (mpos + 1 == newm) ? 0 : mpos + 1;
  P.vr2[before] = vertex_geom(P.qx[before], P.qy[before], mx, my, &P.vx[before], &P.vy[before], &P.ve[before], bad);
  P.vr2[mpos] = vertex_geom(mx, my, P.qx[after], P.qy[after], &P.vx[mpos], &P.vy[mpos], &P.ve[mpos], bad);
  poly_refresh_max(P);
  return true;
}

// The vertex of the cell farthest in the direction of m.  Vertex a lies
// between the edges of sites q_a and q_a+1, whose outward normals point at
// those sites, so it maximises V.m for every m whose direction lies in the
// sector from q_a to q_a+1 (counter-clockwise).  The sites run counter-
// clockwise around the particle: a binary search over their directions,
// with exact int64 cross and dot products, finds the sector of m.  Since
// "m cuts V" (2 m.V > |m|^2) is linear in V, m cuts or touches some vertex
// only if it cuts or touches this one.
template <int CAP>
__device__ __forceinline__ int support_vertex(const Poly<CAP>& P, int32_t mx, int32_t my) {
  const int64_t rx = P.qx[0], ry = P.qy[0];
  // half-turn of a direction counted from q_0: 0 for [0, pi), 1 for [pi, 2 pi)
  auto half = [&](int64_t x, int64_t y) {
    const int64_t c = rx * y - ry * x;
    return (c < 0 || (c == 0 && rx * x + ry * y < 0)) ? 1 : 0;
  };
  const int hm = half(mx, my);
  int lo = 0, hi = P.m - 1;  // the last site at or before m's direction, counted from q_0
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    const int64_t x = P.qx[mid], y = P.qy[mid];
    const int hq = half(x, y);
    if (hq < hm || (hq == hm && x * (int64_t)my - y * (int64_t)mx >= 0)) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// cells of at least this many edges test a candidate's support vertex first
#ifndef VK_VOR_SUPPORT_MIN
#define VK_VOR_SUPPORT_MIN 3
#endif

// true when site m (with Dm <= |m|^2) certainly neither cuts nor touches
// the cell: its support vertex is farther than |m|/2 ... or decided by the
// FP32 bound to lie strictly on the particle's side of the bisector
template <int CAP>
__device__ __forceinline__ bool site_misses(const Poly<CAP>& P, int32_t mx, int32_t my, float Dm) {
  const int a = support_vertex(P, mx, my);
  return Dm > 4.0f * P.vr2[a] || vertex_cut_fast(P.vx[a], P.vy[a], P.ve[a], mx, my) < 0;
}

// clip the cell by the bisector of site (mx, my); returns false on overflow
template <int CAP>
__device__ __forceinline__ bool poly_clip(Poly<CAP>& P, int32_t mx, int32_t my, int32_t mid, int32_t mslot,
                                          float Dm, bool* bad, bool* touch) {
  const int m = P.m;
  *touch = false;
  // large cells: the common case (no cut) in O(log m)
  if (m >= VK_VOR_SUPPORT_MIN && site_misses(P, mx, my, Dm)) return true;
  // the vertices strictly beyond the bisector form one cyclic run [s, s+c)
  int c = 0, s = -1;
  bool first_cut = false, prev_cut = false;
  for (int a = 0; a < m; ++a) {
    bool cut = false;
    if (!(Dm > 4.0f * P.vr2[a])) {  // a vertex closer than |m|/2 cannot be cut
      const int f = vertex_cut_fast(P.vx[a], P.vy[a], P.ve[a], mx, my);
      if (f != 0) {
        cut = f > 0;
      } else {
        const int b = (a + 1 == m) ? 0 : a + 1;
        const int sg = vertex_cut_sign(P.qx[a], P.qy[a], P.qx[b], P.qy[b], mx, my);
        cut = sg > 0;
        *touch = *touch || sg == 0;
      }
    }
    if (a == 0) first_cut = cut;
    if (cut) {
      if (a > 0 && !prev_cut) {
        if (s >= 0) {  // a second run: cannot happen with exact predicates
          *bad = true;
          return true;
        }
        s = a;
      }
      ++c;
    }
    prev_cut = cut;
  }
  if (c == 0) return true;  // *touch: some vertex lies exactly on the bisector
  *touch = false;
  if (first_cut) {
    if (!prev_cut) {
      if (s >= 0) {
        *bad = true;
        return true;
      }
      s = 0;  // the run starts at vertex 0
    } else if (s < 0) {
      *bad = true;  // every vertex cut: impossible, the particle keeps its own side
      return true;
    }
    // else: the run wraps from s through m-1 into 0
  }
  if (s < 0 || c >= m) {
    *bad = true;
    return true;
  }
  return poly_apply_cut(P, s, c, mx, my, mid, mslot, bad);
}

// Walk of the cell grid for one Voronoi cell: rings of sub-cells inside the
// particle's own coarse cell when it is split, then rings of coarse cells.
// box(b) gives the cell's current relevance box b = {x0, x1, y0, y1}
// (offsets from the particle, inclusive), which only shrinks.  Rows and
// cells that miss it are skipped, a split cell contributes only the
// sub-cells that meet it, and the walk stops once the scanned block holds
// it.  run(qb, qe) receives runs of sorted slots.  Returns true if the whole
// grid was visited.
__device__ __forceinline__ int unwrapped_cell(int64_t X, int n, int64_t L) {
  // X within one period of [0, L)
  if (X < 0) return cell_of((int32_t)(X + L), n, (uint32_t)L) - n;
  if (X >= L) return cell_of((int32_t)(X - L), n, (uint32_t)L) + n;
  return cell_of((int32_t)X, n, (uint32_t)L);
}

// the box holds only minimum images (offsets strictly inside half a period),
// so that visiting every site once, at its minimum image, is enough
__device__ __forceinline__ bool within_half(const int64_t* b, int64_t Lx, int64_t Ly) {
  return b[0] > 1 - Lx / 2 && b[1] < Lx / 2 - 1 && b[2] > 1 - Ly / 2 && b[3] < Ly / 2 - 1;
}

template <class RunFn, class BoxFn>
__device__ bool voronoi_walk(const Rep& R, const int32_t* pi, const GridView& G, RunFn& run, BoxFn& box) {
  const int nx = R.nc[0], ny = R.nc[1];
  const int64_t Lx = R.L[0], Ly = R.L[1];
  const int64_t px = pi[0], py = pi[1];
  const int cx = cell_of(pi[0], nx, R.L[0]), cy = cell_of(pi[1], ny, R.L[1]);
  const int64_t own = R.c0 + (int64_t)cy * nx + cx;
  const int s_own = G.sub_s[own];
  int64_t b[4];
  bool own_done = false;
  if (s_own > 1) {
    // ---- rings of sub-cells inside the own coarse cell
    const int s = s_own;
    const int64_t x0 = cell_lo(cx, nx, Lx), y0 = cell_lo(cy, ny, Ly);
    const int64_t wx = cell_lo(cx + 1, nx, Lx) - x0, wy = cell_lo(cy + 1, ny, Ly) - y0;
    const int sx = sub_index(px - x0, wx, s), sy = sub_index(py - y0, wy, s);
    const uint32_t base = G.sub_base[own];
    for (int r = 0;; ++r) {
      const int bx0 = max(sx - r, 0), bx1 = min(sx + r, s - 1), by0 = max(sy - r, 0), by1 = min(sy + r, s - 1);
      const int px0 = r ? max(sx - r + 1, 0) : 1, px1 = r ? min(sx + r - 1, s - 1) : 0;
      const int py0 = r ? max(sy - r + 1, 0) : 1, py1 = r ? min(sy + r - 1, s - 1) : 0;
      for (int yy = by0; yy <= by1; ++yy) {
        const uint32_t rb = base + (uint32_t)yy * s;
        if (yy < py0 || yy > py1 || px0 > px1) {
          run(G.sub_off[rb + bx0], G.sub_off[rb + bx1 + 1]);
        } else {
          if (bx0 < px0) run(G.sub_off[rb + bx0], G.sub_off[rb + px0]);
          if (bx1 > px1) run(G.sub_off[rb + px1 + 1], G.sub_off[rb + bx1 + 1]);
        }
      }
      // the scanned sub-block, as offsets from the particle
      const int64_t xlo = x0 + (bx0 * wx + s - 1) / s - px, xhi = x0 + ((bx1 + 1) * wx + s - 1) / s - 1 - px;
      const int64_t ylo = y0 + (by0 * wy + s - 1) / s - py, yhi = y0 + ((by1 + 1) * wy + s - 1) / s - 1 - py;
      box(b);
      if (b[0] >= xlo && b[1] <= xhi && b[2] >= ylo && b[3] <= yhi && within_half(b, Lx, Ly)) return false;
      if (bx0 == 0 && by0 == 0 && bx1 == s - 1 && by1 == s - 1) break;
    }
    own_done = true;
  }
  // ---- rings of coarse cells
  for (int r = 0;; ++r) {
    const int lox = ring_lo(r, nx), hix = ring_hi(r, nx), loy = ring_lo(r, ny), hiy = ring_hi(r, ny);
    const int plox = r ? ring_lo(r - 1, nx) : 1, phix = r ? ring_hi(r - 1, nx) : 0;
    const int ploy = r ? ring_lo(r - 1, ny) : 1, phiy = r ? ring_hi(r - 1, ny) : 0;
    const bool fullx = hix - lox + 1 == nx, fully = hiy - loy + 1 == ny;
    if (r > 0 && lox == plox && hix == phix && loy == ploy && hiy == phiy) return true;
    box(b);
    // Cell offsets of the box.  A ring visits every cell once, at its
    // representative offset in [-(n-1)/2, n/2]; clipping to the box is exact
    // only when the box's offsets lie in that range (otherwise a cell could
    // meet the box through another periodic image): then nothing is clipped
    // and split cells are visited whole.
    int ox0 = -(nx - 1) / 2, ox1 = nx / 2, oy0 = -(ny - 1) / 2, oy1 = ny / 2;
    bool clx = false, cly = false;
    if (b[0] > -Lx && b[1] < Lx) {
      const int a0 = unwrapped_cell(px + b[0], nx, Lx) - cx, a1 = unwrapped_cell(px + b[1], nx, Lx) - cx;
      if (a0 >= ox0 && a1 <= ox1) {
        clx = true;
        ox0 = a0;
        ox1 = a1;
      }
    }
    if (b[2] > -Ly && b[3] < Ly) {
      const int a0 = unwrapped_cell(py + b[2], ny, Ly) - cy, a1 = unwrapped_cell(py + b[3], ny, Ly) - cy;
      if (a0 >= oy0 && a1 <= oy1) {
        cly = true;
        oy0 = a0;
        oy1 = a1;
      }
    }
    auto visit_row = [&](int a, int e, int oy) {
      a = max(a, ox0);
      e = min(e, ox1);
      if (a > e) return;
      const int64_t ucy = (int64_t)cy + oy;
      const int64_t rowbase = R.c0 + (int64_t)wrap_index(cy + oy, ny) * nx;
      uint32_t pend_b = 0, pend_e = 0;
      bool pend = false;
      for (int ox = a; ox <= e; ++ox) {
        const int64_t g = rowbase + wrap_index(cx + ox, nx);
        const int s = G.sub_s[g];
        if ((g == own && own_done) || s > 1) {
          if (pend) run(pend_b, pend_e);
          pend = false;
          if (g == own && own_done) continue;
          if (!(clx && cly)) {
            run(G.off[g], G.off[g + 1]);
            continue;
          }
          // split cell: the sub-cells meeting the box
          const int64_t ucx = (int64_t)cx + ox;
          const int64_t x0 = cell_lo(ucx, nx, Lx), y0 = cell_lo(ucy, ny, Ly);
          const int64_t wx = cell_lo(ucx + 1, nx, Lx) - x0, wy = cell_lo(ucy + 1, ny, Ly) - y0;
          const int64_t lx = px + b[0] - x0, hx = px + b[1] - x0;
          const int64_t ly = py + b[2] - y0, hy = py + b[3] - y0;
          if (hx < 0 || lx >= wx || hy < 0 || ly >= wy) continue;
          const int sx0 = lx <= 0 ? 0 : sub_index(lx, wx, s), sx1 = hx >= wx ? s - 1 : sub_index(hx, wx, s);
          const int sy0 = ly <= 0 ? 0 : sub_index(ly, wy, s), sy1 = hy >= wy ? s - 1 : sub_index(hy, wy, s);
          const uint32_t base = G.sub_base[g];
          for (int yy = sy0; yy <= sy1; ++yy) {
            const uint32_t rb = base + (uint32_t)yy * s;
            run(G.sub_off[rb + sx0], G.sub_off[rb + sx1 + 1]);
          }
        } else {
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
      }
      if (pend) run(pend_b, pend_e);
    };
    for (int oy = max(loy, oy0); oy <= min(hiy, oy1); ++oy) {
      if (oy < ploy || oy > phiy) {
        visit_row(lox, hix, oy);
      } else {
        visit_row(lox, plox - 1, oy);
        visit_row(phix + 1, hix, oy);
      }
    }
    if (fullx && fully) return true;
    // stop once the scanned block holds the (current) box
    box(b);
    const bool inx = fullx || (b[0] >= cell_lo((int64_t)cx - r, nx, Lx) - px &&
                               b[1] <= cell_lo((int64_t)cx + r + 1, nx, Lx) - 1 - px);
    const bool iny = fully || (b[2] >= cell_lo((int64_t)cy - r, ny, Ly) - py &&
                               b[3] <= cell_lo((int64_t)cy + r + 1, ny, Ly) - 1 - py);
    if (inx && iny && within_half(b, Lx, Ly)) return false;
  }
}

// tiny boxes: visit the eight non-minimum periodic images of every other
// particle (out of line: small systems only)
template <class VisitFn>
__device__ __noinline__ void far_images(const Rep& R, int64_t self, const int32_t* pi, const int2* __restrict__ pos,
                                        const int32_t* __restrict__ ids, VisitFn& visit) {
  const int64_t Lx = R.L[0], Ly = R.L[1];
  for (int64_t q = R.p0; q < R.p0 + R.n; ++q) {
    if (q == self) continue;
    const int2 pj = pos[q];
    const int32_t qx0 = (int32_t)min_image((int64_t)pj.x - pi[0], Lx);
    const int32_t qy0 = (int32_t)min_image((int64_t)pj.y - pi[1], Ly);
    for (int sy = -1; sy <= 1; ++sy)
      for (int sx = -1; sx <= 1; ++sx) {
        if (sx == 0 && sy == 0) continue;
        const int64_t X = (int64_t)qx0 + sx * Lx, Y = (int64_t)qy0 + sy * Ly;
        visit((int32_t)X, (int32_t)Y, ids[q], (int32_t)q);
      }
  }
}

// Voronoi cell of the particle at slot `self`.  Status codes are latched on
// internal inconsistencies (kStRange); capacity overflow is returned.
// Returns false (and leaves the cell unusable) if the polygon or the twin list
// outgrew its capacity.
//
// Seeds (last step's neighbors, the lazy re-check of Sec. "Computational
// tools: Voronoi neighbor lists"): when given, the cell is first clipped by
// those sites, so it starts close to its final shape and with a tight
// relevance box; the walk then checks every site that could still cut it
// (a site inside a vertex disk is a site inside the circumcircle of one of
// the old Delaunay triangles) and clips by it, which repairs the cell where
// the triangulation changed.  The half-plane intersection does not depend
// on the order of the sites, so the cell is the same as without seeds.
struct Seeds {
  const int32_t* ids;      // replica-local ids of last step's neighbors (NULL: none)
  int n;
  const int32_t* slot_of;  // sorted slot by (replica's first slot + id)
};

// a particle's seed word: the number of seeds in the low byte, and a flag
// for a cell that needed many candidates at the last step (a particle on the
// rim of a void), which goes straight to the warp-cooperative kernel
constexpr int32_t kSeedCount = 0xFF;
constexpr int32_t kSeedHeavy = 0x100;

// flags of one cell build
struct CellFlags {
  bool bad;       // an internal inconsistency (latched as kStRange)
  bool overflow;  // the polygon or the twin list outgrew its capacity
};

template <int CAP>
__device__ __forceinline__ void cell_add_twin(Poly<CAP>& P, CellFlags& F, int32_t slot, int32_t jid, int32_t of) {
  for (int t = 0; t < P.nt; ++t)
    if (P.tw_slot[t] == slot) return;  // met again (a seed is visited twice)
  if (P.nt == Poly<CAP>::TW) {
    F.overflow = true;
    return;
  }
  P.tw_slot[P.nt] = slot;
  P.tw_id[P.nt] = jid;
  P.tw_of[P.nt] = of;
  ++P.nt;
}

// one candidate site at offset (qx, qy) from the particle
template <int CAP>
__device__ __forceinline__ void cell_visit(Poly<CAP>& P, CellFlags& F, int32_t qx, int32_t qy, int32_t jid,
                                           int32_t slot) {
  if (F.overflow) return;
  const uint64_t D = (uint64_t)((int64_t)qx * qx) + (uint64_t)((int64_t)qy * qy);
  if (D == 0) {
    cell_add_twin(P, F, slot, jid, -2);  // coincident with the particle itself
    return;
  }
  const float Df = (float)D * (1.0f - 2.384185791015625e-07f);  // rounded down
  if (Df > 4.0f * P.max_r2) return;
  if (qx < P.bx0 || qx > P.bx1 || qy < P.by0 || qy > P.by1) return;  // outside the relevance box
  bool touch = false;
  if (!poly_clip(P, qx, qy, jid, slot, Df, &F.bad, &touch)) {
    F.overflow = true;
    return;
  }
  if (touch) {
    // no vertex cut but some vertex on the bisector: a twin of an edge site?
    for (int a = 0; a < P.m; ++a)
      if (P.qx[a] == qx && P.qy[a] == qy && P.slot[a] >= 0) {
        if (P.slot[a] != slot) cell_add_twin(P, F, slot, jid, P.slot[a]);  // not the edge site itself, met again
        break;
      }
  }
}

// The candidates of slots [qb, qe), or of the slots list[qb..qe), at their
// minimum image.  Out of line, so that the candidate loop and the clipping
// exist once in the kernel whichever part of the walk (or the seeds) feeds
// them: divergent warps then share one stretch of instruction cache.
template <int CAP>
__device__ __noinline__ void cell_visit_slots(Poly<CAP>& P, CellFlags& F, const int2* __restrict__ pos,
                                              const int32_t* __restrict__ ids, int64_t self, int32_t px,
                                              int32_t py, int64_t Lx, int64_t Ly, const int32_t* list,
                                              uint32_t qb, uint32_t qe) {
  for (uint32_t j = qb; j < qe; ++j) {
    const int32_t q = list ? list[j] : (int32_t)j;
    if ((int64_t)q == self) continue;
    const int2 pj = pos[q];
    cell_visit(P, F, (int32_t)min_image((int64_t)pj.x - px, Lx), (int32_t)min_image((int64_t)pj.y - py, Ly),
               ids[q], q);
  }
}

// the same for one candidate at an explicit offset (far periodic images)
template <int CAP>
__device__ __noinline__ void cell_visit_one(Poly<CAP>& P, CellFlags& F, int32_t qx, int32_t qy, int32_t jid,
                                            int32_t slot) {
  cell_visit(P, F, qx, qy, jid, slot);
}

template <int CAP>
__device__ bool voronoi_cell(const Rep& R, int64_t self, const int32_t* pi, int32_t self_id,
                             const int2* __restrict__ pos, const int32_t* __restrict__ ids,
                             const GridView& G, Poly<CAP>& P, int32_t* status, uint32_t budget, const Seeds& sd,
                             uint32_t* seen_out, uint32_t* n_cand = nullptr, uint32_t* n_runs = nullptr) {
  CellFlags F{false, false};
  uint32_t seen = 0;
  poly_init(P, self_id, R.L[0], R.L[1], &F.bad);
  const int64_t Lx = R.L[0], Ly = R.L[1];
  // the seeds first: their slots, then one pass of the candidate loop
  if (sd.n > 0) {
    int32_t ss[kVorSeed];
    const int n = min(sd.n, kVorSeed);
    for (int j = 0; j < n; ++j) ss[j] = sd.slot_of[R.p0 + sd.ids[j]];
    cell_visit_slots(P, F, pos, ids, self, pi[0], pi[1], Lx, Ly, ss, 0u, (uint32_t)n);
  }
  auto run = [&](uint32_t qb, uint32_t qe) {
    if (n_cand) {
      *n_cand += qe - qb;
      *n_runs += 1;
    }
    seen += qe - qb;
    if (budget && seen > budget) F.overflow = true;  // a heavy cell: left to the warp-cooperative kernel
    if (!F.overflow) cell_visit_slots(P, F, pos, ids, self, pi[0], pi[1], Lx, Ly, nullptr, qb, qe);
  };
  auto box = [&](int64_t* b) {
    poly_refresh_box(P);
    // after an overflow nothing more is needed: an empty box ends the walk
    b[0] = F.overflow ? 0 : P.bx0;
    b[1] = F.overflow ? 0 : P.bx1;
    b[2] = F.overflow ? 0 : P.by0;
    b[3] = F.overflow ? 0 : P.by1;
  };
  const bool all = voronoi_walk(R, pi, G, run, box);
  if (all && !F.overflow) {
    // tiny boxes: other periodic images than the minimum one can still shape
    // the cell when the relevance box reaches half a period
    poly_refresh_box(P);
    const int64_t b[4] = {P.bx0, P.bx1, P.by0, P.by1};
    auto visit = [&](int32_t qx, int32_t qy, int32_t jid, int32_t slot) { cell_visit_one(P, F, qx, qy, jid, slot); };
    if (!within_half(b, Lx, Ly)) far_images(R, self, pi, pos, ids, visit);
  }
  if (F.bad) set_status(status, kStRange);
  if (seen_out) *seen_out = seen;
  return !F.overflow;
}

// Effect of site m on the current cell: 1 if it cuts a vertex, 2 if some
// vertex lies exactly on its bisector, 0 otherwise -- and then it never
// will, since the cell only shrinks and stays on the same side.
template <int CAP>
__device__ __forceinline__ int site_effect(const Poly<CAP>& P, int32_t mx, int32_t my, float Dm) {
  if (site_misses(P, mx, my, Dm)) return 0;
  int r = 0;
  for (int a = 0; a < P.m; ++a) {
    if (Dm > 4.0f * P.vr2[a]) continue;
    const int f = vertex_cut_fast(P.vx[a], P.vy[a], P.ve[a], mx, my);
    if (f > 0) return 1;
    if (f == 0) {
      const int b = (a + 1 == P.m) ? 0 : a + 1;
      const int sg = vertex_cut_sign(P.qx[a], P.qy[a], P.qx[b], P.qy[b], mx, my);
      if (sg > 0) return 1;
      if (sg == 0) r = 2;
    }
  }
  return r;
}

// every lane: could the candidate at (qx, qy) cut or touch the current cell?
template <int CAP>
__device__ __forceinline__ bool site_matters(const Poly<CAP>& P, int32_t qx, int32_t qy) {
  const uint64_t D = (uint64_t)((int64_t)qx * qx) + (uint64_t)((int64_t)qy * qy);
  if (D == 0) return true;
  const float Df = (float)D * (1.0f - 2.384185791015625e-07f);
  if (Df > 4.0f * P.max_r2) return false;
  if (qx < P.bx0 || qx > P.bx1 || qy < P.by0 || qy > P.by1) return false;
  return site_effect(P, qx, qy, Df) != 0;
}

// the lanes whose candidate matters hand it to lane 0, which applies them in
// lane order; every lane leaves with lane 0's overflow flag
template <int CAP>
__device__ __forceinline__ void warp_apply(Poly<CAP>& P, CellFlags& F, bool flag, int32_t qx, int32_t qy,
                                           int32_t jid, int32_t slot) {
  const int lane = threadIdx.x & 31;
  unsigned mask = __ballot_sync(0xffffffffu, flag);
  while (mask) {
    const int src = __ffs(mask) - 1;
    mask &= mask - 1;
    const int32_t sx = __shfl_sync(0xffffffffu, qx, src), sy = __shfl_sync(0xffffffffu, qy, src);
    const int32_t sid = __shfl_sync(0xffffffffu, jid, src), ss = __shfl_sync(0xffffffffu, slot, src);
    if (lane == 0) cell_visit(P, F, sx, sy, sid, ss);
    __syncwarp();
  }
  F.overflow = __shfl_sync(0xffffffffu, F.overflow, 0);
}

// The warp's pass over slots [qb, qe): the lanes test 32 candidates at a
// time against the current cell (in shared memory), lane 0 applies the few
// that matter.  All lanes call it; out of line like cell_visit_slots.
template <int CAP>
__device__ __noinline__ void warp_visit_slots(Poly<CAP>& P, CellFlags& F, const int2* __restrict__ pos,
                                              const int32_t* __restrict__ ids, int64_t self, int32_t px,
                                              int32_t py, int64_t Lx, int64_t Ly, uint32_t qb, uint32_t qe) {
  const int lane = threadIdx.x & 31;
  for (uint32_t q0 = qb; q0 < qe && !F.overflow; q0 += 32) {
    const uint32_t q = q0 + (uint32_t)lane;
    bool flag = false;
    int32_t qx = 0, qy = 0, jid = 0;
    if (q < qe && (int64_t)q != self) {
      const int2 pj = pos[q];
      qx = (int32_t)min_image((int64_t)pj.x - px, Lx);
      qy = (int32_t)min_image((int64_t)pj.y - py, Ly);
      jid = ids[q];
      flag = site_matters(P, qx, qy);
    }
    warp_apply(P, F, flag, qx, qy, jid, (int32_t)q);
  }
}

// The same cell as voronoi_cell, built by a whole warp (all 32 lanes call
// it; P is the warp's polygon in shared memory).  The walk is the same; the
// lanes test 32 candidates at a time against the current cell, and lane 0
// applies, in candidate order, the few that cut it or touch it.  For the
// rare cells with many edges or many candidates (particles bordering voids).
template <int CAP>
__device__ bool voronoi_cell_warp(const Rep& R, int64_t self, const int32_t* pi, int32_t self_id,
                                  const int2* __restrict__ pos, const int32_t* __restrict__ ids, const GridView& G,
                                  Poly<CAP>& P, int32_t* status, const Seeds& sd, uint32_t* seen_out) {
  const int lane = threadIdx.x & 31;
  CellFlags F{false, false};  // lane 0's is authoritative, broadcast after every serial part
  if (lane == 0) poly_init(P, self_id, R.L[0], R.L[1], &F.bad);
  const int64_t Lx = R.L[0], Ly = R.L[1];
  if (lane == 0 && sd.n > 0) {
    int32_t ss[kVorSeed];
    const int n = min(sd.n, kVorSeed);
    for (int j = 0; j < n; ++j) ss[j] = sd.slot_of[R.p0 + sd.ids[j]];
    cell_visit_slots(P, F, pos, ids, self, pi[0], pi[1], Lx, Ly, ss, 0u, (uint32_t)n);
  }
  __syncwarp();
  F.overflow = __shfl_sync(0xffffffffu, F.overflow, 0);
  uint32_t seen = 0;
  auto run = [&](uint32_t qb, uint32_t qe) {
    seen += qe - qb;
    warp_visit_slots(P, F, pos, ids, self, pi[0], pi[1], Lx, Ly, qb, qe);
  };
  auto box = [&](int64_t* b) {
    if (lane == 0) poly_refresh_box(P);
    __syncwarp();
    b[0] = F.overflow ? 0 : P.bx0;
    b[1] = F.overflow ? 0 : P.bx1;
    b[2] = F.overflow ? 0 : P.by0;
    b[3] = F.overflow ? 0 : P.by1;
  };
  const bool all = voronoi_walk(R, pi, G, run, box);
  if (all && !F.overflow) {
    if (lane == 0) poly_refresh_box(P);
    __syncwarp();
    const int64_t b[4] = {P.bx0, P.bx1, P.by0, P.by1};
    if (!within_half(b, Lx, Ly)) {
      // tiny boxes: the other periodic images of every particle
      for (int64_t q0 = R.p0; q0 < R.p0 + R.n; q0 += 32) {
        const int64_t q = q0 + lane;
        const bool ok = q < R.p0 + R.n && q != self;
        int32_t qx0 = 0, qy0 = 0, jid = 0;
        if (ok) {
          const int2 pj = pos[q];
          qx0 = (int32_t)min_image((int64_t)pj.x - pi[0], Lx);
          qy0 = (int32_t)min_image((int64_t)pj.y - pi[1], Ly);
          jid = ids[q];
        }
        for (int sy = -1; sy <= 1; ++sy)
          for (int sx = -1; sx <= 1; ++sx) {
            if (sx == 0 && sy == 0) continue;
            const int32_t X = (int32_t)((int64_t)qx0 + sx * Lx), Y = (int32_t)((int64_t)qy0 + sy * Ly);
            warp_apply(P, F, ok && !F.overflow && site_matters(P, X, Y), X, Y, jid, (int32_t)q);
          }
      }
    }
  }
  F.bad = __shfl_sync(0xffffffffu, F.bad, 0);
  if (F.bad && lane == 0) set_status(status, kStRange);
  if (seen_out) *seen_out = seen;
  return !F.overflow;
}

// neighbors: sites of edges with positive length (never the particle's own
// images) plus the coincident twins of the particle and of those sites;
// sorted by id and de-duplicated; returns the count
template <int CAP>
__device__ __forceinline__ int voronoi_neighbors(const Poly<CAP>& P, int32_t self_id, int32_t* nid,
                                                 int32_t* nslot) {
  int cnt = 0;
  const int m = P.m;
  auto push = [&](int32_t v, int32_t sl) {
    for (int q = 0; q < cnt; ++q)
      if (nid[q] == v) return;
    int j = cnt;
    while (j > 0 && nid[j - 1] > v) {
      nid[j] = nid[j - 1];
      nslot[j] = nslot[j - 1];
      --j;
    }
    nid[j] = v;
    nslot[j] = sl;
    ++cnt;
  };
  for (int a = 0; a < m; ++a) {
    if (P.slot[a] < 0) continue;  // an image of the particle itself
    const int pa = (a == 0) ? m - 1 : a - 1, na = (a + 1 == m) ? 0 : a + 1;
    if (vertex_cut_sign(P.qx[pa], P.qy[pa], P.qx[a], P.qy[a], P.qx[na], P.qy[na]) == 0) continue;
    push(P.id[a], P.slot[a]);
    for (int t = 0; t < P.nt; ++t)
      if (P.tw_of[t] == P.slot[a]) push(P.tw_id[t], P.tw_slot[t]);
  }
  for (int t = 0; t < P.nt; ++t)
    if (P.tw_of[t] == -2 && P.tw_id[t] != self_id) push(P.tw_id[t], P.tw_slot[t]);
  return cnt;
}

}  // namespace

}  // namespace vk
