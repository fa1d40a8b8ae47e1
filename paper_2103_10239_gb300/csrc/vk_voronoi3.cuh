// vk_voronoi3.cuh -- the 3D Voronoi cell of one particle by exact half-space
// clipping (Sec. "Computational tools: Voronoi neighbor lists": the Voronoi
// cell of a particle holds the points closer to it than to any other particle,
// and two particles are neighbors when their cells share a face).
//
// The cell is the intersection of the half-spaces {x : d.x <= |d|^2 / 2}, one
// per site image at offset d from the particle.  It is kept in dual form: a
// triangulation of the sphere whose nodes are the planes (faces) of the cell
// and whose triangles are its vertices.  A triangle (a, b, c) is the point y/2
// with d_a.y = w_a, d_b.y = w_b, d_c.y = w_c (w = |d|^2), listed so that
// det(d_a, d_b, d_c) > 0, and it stores the three triangles across its edges.
// Clipping by a new plane e removes the triangles whose point lies strictly
// beyond it (d_e.y > w_e) and fans the boundary of the removed region to e,
// as in Bowyer-Watson insertion.
//
// Exactness.  Every decision is an integer sign:
//   * "beyond": the FP32 vertex estimate y (from exact int128 Cramer
//     numerators, relative error <= 2^-22 per coordinate) gives
//     s = d_e.y - w_e with |error| <= 2^-19 (|d_e| |y|_max + w_e); outside that
//     band the sign of s is the answer, inside it the exact 4x4 determinant
//     det[d_a w_a; d_b w_b; d_c w_c; d_e w_e] = det(M) (w_e - d_e.y) decides;
//   * a point exactly on the plane stays (it is inside the closed half-space).
//     This is the outcome of shifting every plane outward by an infinitesimal
//     that grows with its insertion order, so the structure always stays a
//     valid simple polytope, but a face may keep zero area;
//   * a face counts (its site is a neighbor) when it has positive area: two of
//     its edges of positive length are not parallel.  An edge between
//     triangles (p, q, r) and (q, p, s) has zero length iff the point of the
//     first lies on plane s; lines p^q and p^q' are parallel iff
//     det(d_p, d_q, d_q') = 0.
// Range: |d| < 2^24 for every clipped plane keeps every product below 2^125;
// with candidates limited to |d| < 2 R (R <= sqrt(3)/2 L) that is box edges up
// to 2^23 grid units.
//
// The builder is plain C++ usable on the host and the device.
#pragma once
#include <cmath>
#include <cstdint>

// V3_HD: small helpers, inlined.  V3_OUT: the large ones (int128 solves, the
// rewiring of a clip, the face test), kept out of line on the device so that
// one copy of each serves every call site: inlined copies made the kernels
// stall on instruction fetch.
#ifdef __CUDACC__
#define V3_HD __host__ __device__ __forceinline__
#define V3_OUT __host__ __device__ __noinline__
#else
#define V3_HD inline
#define V3_OUT inline
#endif

namespace vk {
namespace v3 {

typedef __int128 i128;


// build status
enum : int {
  kOk = 0,
  kCapacity = 1,  // more than P faces, T vertices or B boundary edges of one clip
  kInternal = 2,  // the removed region was not a disk (cannot happen with exact signs)
  kCoincident = 3,
};

// A cell of at most P live planes (faces) and T live triangles (vertices;
// 2F - 4 for F faces); indices are 8-bit, so P, T <= 256.
template <int PM, int TM>
struct Cell {
  static constexpr int P = PM, T = TM, B = TM / 2;
  static_assert(PM <= 256 && TM <= 256, "8-bit plane and triangle indices");
  // planes: offset d (grid units) and the site's slot (-1: own image)
  int32_t pd[PM][3];
  int32_t pslot[PM];
  int32_t pref[PM];  // live triangles on the plane (0: free)
  // triangles: y = 2x (FP32 estimate) and alive flag (w: 1 alive, 0 free)
  float ty[TM][4];
  uint8_t tp[TM][4];  // planes, det(d_a, d_b, d_c) > 0
  uint8_t tn[TM][4];  // tn[t][k]: triangle across edge (tp[t][k], tp[t][k+1])
  int np, nt;            // slots in use (planes, triangles; free slots inside are reused)
  float r2;              // upper bound of max |x|^2 over the vertices (grid units^2)
  float ymax;            // upper bound of max |y|
  int status;
};

V3_HD int clz64(uint64_t x) {
#ifdef __CUDA_ARCH__
  return __clzll((long long)x);
#else
  return __builtin_clzll(x);
#endif
}

// correctly rounded int128 -> float
V3_HD float i128_to_float(i128 v) {
  const bool neg = v < 0;
  const unsigned __int128 u = neg ? (unsigned __int128)0 - (unsigned __int128)v : (unsigned __int128)v;
  const uint64_t hi = (uint64_t)(u >> 64), lo = (uint64_t)u;
  float f;
  if (hi == 0) {
    f = (float)lo;
  } else {
    const int sh = 64 - clz64(hi);  // 1..63 for |v| < 2^127
    const uint64_t top = (uint64_t)(u >> sh) | (uint64_t)((lo & ((1ull << sh) - 1ull)) != 0ull);
    f = ldexpf((float)top, sh);
  }
  return neg ? -f : f;
}

V3_HD int64_t minor2(int32_t a0, int32_t a1, int32_t b0, int32_t b1) {
  return (int64_t)a0 * b1 - (int64_t)a1 * b0;
}

V3_HD i128 det3(const int32_t* a, const int32_t* b, const int32_t* c) {
  return (i128)a[0] * minor2(b[1], b[2], c[1], c[2]) - (i128)a[1] * minor2(b[0], b[2], c[0], c[2]) +
         (i128)a[2] * minor2(b[0], b[1], c[0], c[1]);
}

V3_HD int64_t norm2(const int32_t* d) {
  return (int64_t)d[0] * d[0] + (int64_t)d[1] * d[1] + (int64_t)d[2] * d[2];
}

V3_HD int sgn128(i128 v) { return (v > 0) - (v < 0); }

// exact side of the point of planes (a, b, c) with respect to plane e:
// +1 beyond (d_e.y > w_e), 0 on it, -1 inside
V3_OUT int side_exact(const int32_t* da, const int32_t* db, const int32_t* dc, const int32_t* de) {
  const i128 m = det3(da, db, dc);
  const i128 t = -(i128)norm2(da) * det3(db, dc, de) + (i128)norm2(db) * det3(da, dc, de) -
                 (i128)norm2(dc) * det3(da, db, de) + (i128)norm2(de) * m;
  return -sgn128(t) * sgn128(m);
}

// y = 2x of the point of planes (a, b, c) by Cramer's rule on exact integers
V3_OUT void vertex_y(const int32_t* da, const int32_t* db, const int32_t* dc, float* y) {
  const int32_t* M[3] = {da, db, dc};
  const int64_t w[3] = {norm2(da), norm2(db), norm2(dc)};
  int64_t cf[3][3];
  for (int r = 0; r < 3; ++r) {
    const int r1 = (r + 1) % 3, r2 = (r + 2) % 3;
    for (int k = 0; k < 3; ++k) {
      const int k1 = (k + 1) % 3, k2 = (k + 2) % 3;
      cf[r][k] = minor2(M[r1][k1], M[r1][k2], M[r2][k1], M[r2][k2]);
    }
  }
  const i128 det = (i128)M[0][0] * cf[0][0] + (i128)M[0][1] * cf[0][1] + (i128)M[0][2] * cf[0][2];
  const float fd = i128_to_float(det);
  for (int k = 0; k < 3; ++k) {
    const i128 num = (i128)w[0] * cf[0][k] + (i128)w[1] * cf[1][k] + (i128)w[2] * cf[2][k];
    y[k] = i128_to_float(num) / fd;
  }
}

// side of the point of triangle t with respect to the plane at offset d
// (w = |d|^2 as float): the FP32 estimate when it is outside the error band,
// else exact
template <class Cell>
V3_HD int side_of(const Cell& C, int t, const int32_t* d, float wf, float band) {
  const float s = fmaf((float)d[0], C.ty[t][0], fmaf((float)d[1], C.ty[t][1], fmaf((float)d[2], C.ty[t][2], -wf)));
  if (s > band) return 1;
  if (s < -band) return -1;
  return side_exact(C.pd[C.tp[t][0]], C.pd[C.tp[t][1]], C.pd[C.tp[t][2]], d);
}

// 2^-19 (|d| ymax + w): bound of the error of the FP32 side estimate for
// every vertex of the cell (the estimate of y errs by <= 2^-22 |y| per
// coordinate, the three FMAs and the rounding of w add < 2^-21 (|d||y| + w))
template <class Cell>
V3_HD float side_band(const Cell& C, float wf) {
  return 1.9073486e-6f * (sqrtf(wf) * 1.0001f * C.ymax + wf);
}

template <class Cell>
V3_HD void refresh_radius(Cell& C) {
  float m = 0.f;
  for (int t = 0; t < C.nt; ++t) {
    if (C.ty[t][3] == 0.f) continue;
    const float q = C.ty[t][0] * C.ty[t][0] + C.ty[t][1] * C.ty[t][1] + C.ty[t][2] * C.ty[t][2];
    m = fmaxf(m, q);
  }
  // |x| = |y| / 2; 2^-18 covers the estimate's and this sum's rounding
  C.r2 = 0.25f * m * (1.f + 3.8147e-6f) + 1.f;
  C.ymax = sqrtf(m) * (1.f + 3.8147e-6f) + 1.f;
}

template <class Cell>
V3_HD int new_plane(Cell& C, const int32_t* d, int32_t slot) {
  int p = -1;
  for (int q = 0; q < C.np; ++q)
    if (C.pref[q] == 0) {
      p = q;
      break;
    }
  if (p < 0) {
    if (C.np == Cell::P) return -1;
    p = C.np++;
  }
  C.pd[p][0] = d[0];
  C.pd[p][1] = d[1];
  C.pd[p][2] = d[2];
  C.pslot[p] = slot;
  C.pref[p] = 0;
  return p;
}

template <class Cell>
V3_HD void set_triangle(Cell& C, int t, int a, int b, int c) {
  C.tp[t][0] = (uint8_t)a;
  C.tp[t][1] = (uint8_t)b;
  C.tp[t][2] = (uint8_t)c;
  vertex_y(C.pd[a], C.pd[b], C.pd[c], C.ty[t]);
  C.ty[t][3] = 1.f;
  ++C.pref[a];
  ++C.pref[b];
  ++C.pref[c];
}

// the box bounded by the particle's own images at +-L per axis; clears the
// scratch sg (Cell::T entries) that cell_clip and clip_topology take
template <class Cell>
V3_HD void cell_init(Cell& C, const uint32_t* L, int8_t* sg) {
  C.np = 6;
  C.nt = 8;
  C.status = kOk;
  for (int t = 0; t < Cell::T; ++t) sg[t] = 0;
  for (int a = 0; a < 3; ++a)
    for (int s = 0; s < 2; ++s) {
      const int p = 2 * a + s;
      C.pd[p][0] = C.pd[p][1] = C.pd[p][2] = 0;
      C.pd[p][a] = s ? -(int32_t)L[a] : (int32_t)L[a];
      C.pslot[p] = -1;
      C.pref[p] = 0;
    }
  // octant t = (bit 0: -x, bit 1: -y, bit 2: -z); planes 0/1 = +x/-x, 2/3, 4/5
  for (int t = 0; t < 8; ++t) {
    const int px = (t & 1), py = 2 + ((t >> 1) & 1), pz = 4 + ((t >> 2) & 1);
    const int odd = ((t & 1) + ((t >> 1) & 1) + ((t >> 2) & 1)) & 1;  // det sign flips per minus
    if (odd) set_triangle(C, t, px, pz, py);
    else set_triangle(C, t, px, py, pz);
  }
  // adjacency by matching reversed edges
  for (int t = 0; t < 8; ++t)
    for (int k = 0; k < 3; ++k) {
      const int a = C.tp[t][k], b = C.tp[t][(k + 1) % 3];
      for (int u = 0; u < 8; ++u)
        for (int j = 0; j < 3; ++j)
          if (C.tp[u][j] == b && C.tp[u][(j + 1) % 3] == a) C.tn[t][k] = (uint8_t)u;
    }
  refresh_radius(C);
}

// The topology of a clip by the plane at offset d (slot: the site's sorted
// slot), given sg[t] = 1 for the triangles whose point lies strictly beyond
// it (0 for every other slot below C.nt; at least one is 1): a new plane,
// the boundary edges of the removed region, the removed triangles freed and
// the new ones (p, q, e) linked in their place.  The new triangles' slots go
// to bt[0..*nb); their points are NOT computed (vertex_of does that).
// Returns the new plane, or -1 on a failure (C.status set).  sg is left
// cleared.
template <class Cell>
V3_OUT int clip_topology(Cell& C, const int32_t* d, int32_t slot, int8_t* sg, uint8_t* bt, int* nb_out) {
  const int e = new_plane(C, d, slot);
  if (e < 0) {
    C.status = kCapacity;
    return -1;
  }
  // boundary edges (p -> q) of the removed region, with the kept triangle
  // across them
  uint8_t bp[Cell::B], bq[Cell::B], bo[Cell::B];
  int nb = 0;
  for (int t = 0; t < C.nt; ++t) {
    if (!sg[t]) continue;
    for (int k = 0; k < 3; ++k) {
      const int o = C.tn[t][k];
      if (sg[o]) continue;
      if (nb == Cell::B) {
        C.status = kCapacity;
        return -1;
      }
      bp[nb] = C.tp[t][k];
      bq[nb] = C.tp[t][(k + 1) % 3];
      bo[nb] = (uint8_t)o;
      ++nb;
    }
  }
  if (nb < 3) {
    C.status = kInternal;
    return -1;
  }
  // free the removed triangles; their slots are reused first
  for (int t = 0; t < C.nt; ++t) {
    if (!sg[t]) continue;
    sg[t] = 0;
    C.ty[t][3] = 0.f;
    --C.pref[C.tp[t][0]];
    --C.pref[C.tp[t][1]];
    --C.pref[C.tp[t][2]];
  }
  int scan = 0;
  for (int j = 0; j < nb; ++j) {
    while (scan < C.nt && C.ty[scan][3] != 0.f) ++scan;
    if (scan == C.nt) {
      if (C.nt == Cell::T) {
        C.status = kCapacity;
        return -1;
      }
      ++C.nt;
    }
    bt[j] = (uint8_t)scan;
    C.ty[scan][3] = 1.f;  // alive (its point follows)
    ++scan;
  }
  for (int j = 0; j < nb; ++j) {
    const int t = bt[j];
    C.tp[t][0] = bp[j];
    C.tp[t][1] = bq[j];
    C.tp[t][2] = (uint8_t)e;
    ++C.pref[bp[j]];
    ++C.pref[bq[j]];
    ++C.pref[e];
    // edge 0 (p, q): the kept triangle, which points back across (q, p)
    const int o = bo[j];
    C.tn[t][0] = (uint8_t)o;
    for (int k = 0; k < 3; ++k)
      if (C.tp[o][k] == bq[j] && C.tp[o][(k + 1) % 3] == bp[j]) C.tn[o][k] = (uint8_t)t;
    // edge 1 (q, e): the new triangle of the boundary edge leaving q;
    // edge 2 (e, p): the one arriving at p
    int nx = -1, pv = -1, cx = 0, cp = 0;
    for (int m = 0; m < nb; ++m) {
      if (bp[m] == bq[j]) nx = m, ++cx;
      if (bq[m] == bp[j]) pv = m, ++cp;
    }
    if (cx != 1 || cp != 1) {
      C.status = kInternal;
      return -1;
    }
    C.tn[t][1] = bt[nx];
    C.tn[t][2] = bt[pv];
  }
  while (C.nt > 0 && C.ty[C.nt - 1][3] == 0.f) --C.nt;
  *nb_out = nb;
  return e;
}

// the point of triangle t from its planes
template <class Cell>
V3_HD void vertex_of(Cell& C, int t) {
  vertex_y(C.pd[C.tp[t][0]], C.pd[C.tp[t][1]], C.pd[C.tp[t][2]], C.ty[t]);
}

// Clip by the plane of the site at offset d (slot: its sorted slot).
// Returns 1 when some vertex lay strictly beyond it, 0 when not, -1 on a
// failure (C.status set).  sg is scratch of Cell::T entries, all zero on
// entry and on return.
template <class Cell>
V3_OUT int cell_clip(Cell& C, const int32_t* d, int32_t slot, int8_t* sg) {
  const int64_t w = norm2(d);
  const float wf = (float)w;
  if (wf >= 4.f * C.r2) return 0;  // |d| / 2 beyond every vertex: cannot cut
  const float band = side_band(C, wf);
  int nout = 0;
  for (int t = 0; t < C.nt; ++t) {
    if (C.ty[t][3] == 0.f) continue;
    const int side = side_of(C, t, d, wf, band);
    sg[t] = (int8_t)(side > 0);
    nout += side > 0;
  }
  if (nout == 0) return 0;
  uint8_t bt[Cell::B];
  int nb = 0;
  if (clip_topology(C, d, slot, sg, bt, &nb) < 0) return -1;
  for (int j = 0; j < nb; ++j) vertex_of(C, bt[j]);
  refresh_radius(C);
  return 1;
}

// Does the face of plane p (live, C.pref[p] > 0) have positive area?
template <class Cell>
V3_OUT bool face_positive(const Cell& C, int p) {
  int t0 = -1, k0 = 0;
  for (int t = 0; t < C.nt && t0 < 0; ++t) {
    if (C.ty[t][3] == 0.f) continue;
    for (int k = 0; k < 3; ++k)
      if (C.tp[t][k] == p) {
        t0 = t;
        k0 = k;
        break;
      }
  }
  if (t0 < 0) return false;
  int t = t0, k = k0, qfirst = -1;
  for (int guard = 0; guard < Cell::T; ++guard) {
    // t = (p, q, r) in cyclic order from p; the next triangle around p is
    // across the edge (p, q) and reads (q, p, s)
    const int q = C.tp[t][(k + 1) % 3];
    const int u = C.tn[t][k];
    int ku = 0;
    while (ku < 3 && C.tp[u][ku] != p) ++ku;
    if (ku == 3) return false;  // (not reached: adjacency is consistent)
    const int s = C.tp[u][(ku + 1) % 3];
    // the edge t -> u on line p^q has zero length iff t's point is on plane s
    const float ws = (float)norm2(C.pd[s]);
    const bool nonzero = side_of(C, t, C.pd[s], ws, side_band(C, ws)) != 0;
    if (nonzero) {
      if (qfirst < 0) qfirst = q;
      else if (det3(C.pd[p], C.pd[qfirst], C.pd[q]) != 0) return true;
    }
    t = u;
    k = ku;
    if (t == t0) break;
  }
  return false;
}

}  // namespace v3
}  // namespace vk
