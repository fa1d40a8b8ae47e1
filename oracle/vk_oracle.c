/*
 * vk_oracle.c -- plain, slow CPU oracle for the topological Vicsek hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call this code:
 * only the test suite, the package smoke check and the CPU-baseline leg of the
 * benchmark load it.  It shares no source, header, table or helper with the
 * CUDA implementation; both consume the same seeded integer inputs.
 *
 * What it computes (arxiv 2103.10239, "Non-metric interaction rules in models
 * of active matter"):
 *   - the k nearest neighbors of every particle in a periodic box, with no
 *     distance cutoff (Sec. "Metric and topological flocking models": each
 *     particle aligns with its k nearest neighbors regardless of distance),
 *     by brute force over all pairs (the naive O(N^2) evaluation of Sec.
 *     "Introduction");
 *   - the Voronoi neighbors of every particle (Sec. "Computational tools:
 *     Voronoi neighbor lists"): a Delaunay triangulation built by incremental
 *     Bowyer-Watson insertion with exact integer orient/incircle predicates
 *     (empty-circumcircle definition), from which an edge is kept iff its dual
 *     Voronoi edge has positive length; coincident particles form one site,
 *     are each other's neighbors and share the site's neighbors;
 *   - one Vicsek update: the position step of Eq. (1) and the alignment rule of
 *     Eq. (2), in FP64, with the noise drawn from Philox4x32-10 (Salmon, Moraes,
 *     Dror & Shaw, SC'11) keyed by (seed) and countered by (id, step, replica);
 *   - the polar order parameter |sum_i n_i| / N;
 *   - the k nearest neighbors inside a field of view and the metric (r0)
 *     neighbors (Sec. "Metric and topological flocking models");
 *   - the 3D Voronoi neighbors (same section): every cell built by exact
 *     clipping with the bisector half-spaces of the periodic images of the
 *     other particles, neighbors being the sites whose plane carries a face
 *     of positive area (insphere-type integer determinants decide every
 *     vertex); coincident particles are reported as degenerate;
 *   - the Voronoi tissue model (Sec. "Geometric models of dense tissue"):
 *     cell areas and perimeters, the energy of Eq. (vmEnergy) and the forces
 *     of Sec. "Voronoi model forces" by the chain rule through the vertices.
 *
 * Readings where the paper is silent (documented in the design notes):
 *   - minimum image maps a difference into (-L/2, L/2];
 *   - kNN order is (exact squared distance, id); self is excluded;
 *   - the default noise is angular: theta = atan2(S) + eta*(u - 1/2);
 *     Eq. (2)'s vectorial form is the alternative;
 *   - advection uses the heading before the update (Eq. 1 literally), the step
 *     s = fl32(v0*dt) * 2^F in grid units, rounded half-to-even to the grid.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef __int128 i128;
typedef unsigned __int128 u128;

/* Status codes returned by the oracle entry points. */
#define ORC_OK 0
#define ORC_ERR_ARG 1
#define ORC_ERR_OOM 2
#define ORC_ERR_DEGENERATE 3
#define ORC_ERR_INTERNAL 4

/* ======================================================================== */
/* Philox4x32-10 (Salmon et al., SC'11): ten rounds of two 32x32->64        */
/* multiplies with the published multipliers and Weyl key increments.        */
/* ======================================================================== */
void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += 0x9E3779B9u; /* golden ratio */
      k1 += 0xBB67AE85u; /* sqrt(3) - 1 */
    }
    uint64_t prod0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
    uint64_t prod1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
    uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Uniform in [0,1) from the top 24 bits of a 32-bit word. */
static double unit24(uint32_t w) { return (double)(w >> 8) * (1.0 / 16777216.0); }

/* ======================================================================== */
/* Periodic geometry on the integer grid                                     */
/* ======================================================================== */

/* Map a difference of two in-box coordinates into (-L/2, L/2]. */
static int64_t min_image(int64_t d, int64_t L) {
  if (2 * d > L) d -= L;
  if (2 * d <= -L) d += L;
  return d;
}

static uint64_t sqdist(int dim, const int32_t* a, const int32_t* b, const int64_t* box) {
  uint64_t D = 0;
  for (int ax = 0; ax < dim; ++ax) {
    int64_t d = min_image((int64_t)b[ax] - (int64_t)a[ax], box[ax]);
    D += (uint64_t)(d * d);
  }
  return D;
}

/* ======================================================================== */
/* k nearest neighbors by brute force                                        */
/* ======================================================================== */

/* For each query particle q (all particles if query == NULL) write its k
 * nearest other particles, ordered by (squared distance, id), into
 * out[q*k .. q*k+k).  Requires 1 <= k <= n-1. */
int orc_knn(int dim, int64_t n, const int32_t* pos, const int64_t* box, int k,
            const int64_t* query, int64_t nq, int32_t* out) {
  if (dim < 1 || dim > 3 || n < 2 || k < 1 || k > n - 1) return ORC_ERR_ARG;
  for (int ax = 0; ax < dim; ++ax)
    if (box[ax] < 1 || box[ax] > ((int64_t)1 << 31)) return ORC_ERR_ARG;
  if (query == NULL) nq = n;
  int bad = 0;
#pragma omp parallel
  {
    uint64_t* bd = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)k);
    int32_t* bi = (int32_t*)malloc(sizeof(int32_t) * (size_t)k);
    if (!bd || !bi) {
#pragma omp atomic write
      bad = 1;
    }
#pragma omp for schedule(dynamic, 16)
    for (int64_t qq = 0; qq < nq; ++qq) {
      if (!bd || !bi) continue;
      int64_t i = query ? query[qq] : qq;
      int filled = 0;
      for (int64_t j = 0; j < n; ++j) {
        if (j == i) continue;
        uint64_t D = sqdist(dim, pos + i * dim, pos + j * dim, box);
        /* keep the k smallest (D, j); j grows, so an equal D never displaces */
        if (filled == k && D >= bd[k - 1]) continue;
        int s = filled < k ? filled++ : k - 1;
        while (s > 0 && bd[s - 1] > D) {
          bd[s] = bd[s - 1];
          bi[s] = bi[s - 1];
          --s;
        }
        bd[s] = D;
        bi[s] = (int32_t)j;
      }
      for (int s = 0; s < k; ++s) out[qq * k + s] = bi[s];
    }
    free(bd);
    free(bi);
  }
  return bad ? ORC_ERR_OOM : ORC_OK;
}

/* ======================================================================== */
/* Exact predicates on integer points                                        */
/* ======================================================================== */

/* orient(a,b,c) = sign of (b-a) x (c-a); |coords| < 2^37 keeps it in i128. */
/* ------------------------------------------------------------------------
 * Metric rule (Sec. "Metric and topological flocking models": all pairs
 * within a distance r0 are neighbors).  Reading: j != i is a neighbor of i
 * iff the exact squared minimum-image distance D <= r0q^2, r0q being the
 * radius in grid units.  Rows sorted by id.  Two calls: offsets (and the
 * count) first with ids == NULL, then the ids.
 * ------------------------------------------------------------------------ */
int orc_metric(int dim, int64_t n, const int32_t* pos, const int64_t* box, int64_t r0q, int64_t* offsets,
               int32_t* ids, int64_t cap, int64_t* nnz) {
  if (dim < 1 || dim > 3 || n < 1 || r0q < 0 || r0q > ((int64_t)1 << 31)) return ORC_ERR_ARG;
  const uint64_t r2 = (uint64_t)r0q * (uint64_t)r0q;
  offsets[0] = 0;
  for (int64_t i = 0; i < n; ++i) {
    int64_t c = 0;
    for (int64_t j = 0; j < n; ++j)
      if (j != i && sqdist(dim, pos + i * dim, pos + j * dim, box) <= r2) ++c;
    offsets[i + 1] = offsets[i] + c;
  }
  *nnz = offsets[n];
  if (!ids) return ORC_OK;
  if (cap < offsets[n]) return ORC_ERR_ARG;
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t i = 0; i < n; ++i) {
    int64_t w = offsets[i];
    for (int64_t j = 0; j < n; ++j)
      if (j != i && sqdist(dim, pos + i * dim, pos + j * dim, box) <= r2) ids[w++] = (int32_t)j;
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------------
 * k nearest neighbors inside a field of view (Sec. "Metric and topological
 * flocking models": the k nearest neighbors within an angular field of
 * view).  Reading: j is in i's field of view iff its offset d = r_j - r_i
 * (minimum image) makes an angle of at most the half-angle with i's heading,
 * i.e. d.n >= c |d| with c the cosine of the half-angle.  To be decided
 * exactly, the heading and c are rounded to a fixed point of 2^-24:
 * nq = rint(n * 2^24), cq = rint(c * 2^24) (round half to even), and the
 * test is s = d.nq >= cq |d|, compared through squares in 128-bit integers.
 * Coincident particles (d = 0) are in view, and so is everyone when c <= -1
 * (a full circle).  Among the particles in view,
 * the k nearest by (D, id); out[qq*k + s] = -1 past the count found.
 * ------------------------------------------------------------------------ */
static int64_t fix24(double v) { return (int64_t)nearbyint(v * 16777216.0); }

static int in_view(int64_t dx, int64_t dy, int64_t nxq, int64_t nyq, int64_t cq) {
  if (cq <= -((int64_t)1 << 24)) return 1; /* a full circle: every particle is in view */
  const __int128 sdot = (__int128)dx * nxq + (__int128)dy * nyq;
  const __int128 D = (__int128)dx * dx + (__int128)dy * dy;
  const __int128 lhs = sdot * sdot, rhs = (__int128)cq * cq * D;
  if (cq >= 0) return sdot >= 0 && lhs >= rhs;
  return sdot >= 0 || lhs <= rhs;
}

int orc_knn_fov(int64_t n, const int32_t* pos, const float* dir, const int64_t* box, int k, float fov_cos,
                const int64_t* query, int64_t nq, int32_t* out, int32_t* count) {
  if (n < 2 || k < 1 || k > n - 1 || !(fov_cos >= -1.0f && fov_cos <= 1.0f)) return ORC_ERR_ARG;
  if (query == NULL) nq = n;
  const int64_t cq = fix24((double)fov_cos);
  int bad = 0;
#pragma omp parallel
  {
    uint64_t* bd = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)k);
    int32_t* bi = (int32_t*)malloc(sizeof(int32_t) * (size_t)k);
    if (!bd || !bi) {
#pragma omp atomic write
      bad = 1;
    }
#pragma omp for schedule(dynamic, 16)
    for (int64_t qq = 0; qq < nq; ++qq) {
      if (!bd || !bi) continue;
      int64_t i = query ? query[qq] : qq;
      const int64_t nxq = fix24((double)dir[2 * i]), nyq = fix24((double)dir[2 * i + 1]);
      int filled = 0;
      for (int64_t j = 0; j < n; ++j) {
        if (j == i) continue;
        const int64_t dx = min_image((int64_t)pos[2 * j] - pos[2 * i], box[0]);
        const int64_t dy = min_image((int64_t)pos[2 * j + 1] - pos[2 * i + 1], box[1]);
        if (!in_view(dx, dy, nxq, nyq, cq)) continue;
        const uint64_t D = (uint64_t)(dx * dx) + (uint64_t)(dy * dy);
        if (filled == k && D >= bd[k - 1]) continue;
        int s = filled < k ? filled++ : k - 1;
        while (s > 0 && bd[s - 1] > D) {
          bd[s] = bd[s - 1];
          bi[s] = bi[s - 1];
          --s;
        }
        bd[s] = D;
        bi[s] = (int32_t)j;
      }
      for (int s = 0; s < k; ++s) out[qq * k + s] = s < filled ? bi[s] : -1;
      count[qq] = filled;
    }
    free(bd);
    free(bi);
  }
  return bad ? ORC_ERR_OOM : ORC_OK;
}

static int orient2(int64_t ax, int64_t ay, int64_t bx, int64_t by, int64_t cx, int64_t cy) {
  i128 v = (i128)(bx - ax) * (i128)(cy - ay) - (i128)(by - ay) * (i128)(cx - ax);
  return (v > 0) - (v < 0);
}

/* Signed 256-bit integers, just enough for the incircle determinant. */
typedef struct { uint64_t w[4]; } i256; /* two's complement, w[0] least significant */

static i256 i256_zero(void) { i256 r = {{0, 0, 0, 0}}; return r; }

static i256 i256_add(i256 a, i256 b) {
  i256 r;
  u128 carry = 0;
  for (int t = 0; t < 4; ++t) {
    u128 s = (u128)a.w[t] + (u128)b.w[t] + carry;
    r.w[t] = (uint64_t)s;
    carry = s >> 64;
  }
  return r;
}

static i256 i256_neg(i256 a) {
  i256 r;
  for (int t = 0; t < 4; ++t) r.w[t] = ~a.w[t];
  i256 one = i256_zero();
  one.w[0] = 1;
  return i256_add(r, one);
}

/* Exact product of two signed 128-bit values with |a|,|b| < 2^127. */
static i256 i256_mul(i128 a, i128 b) {
  int neg = (a < 0) != (b < 0);
  u128 ua = a < 0 ? (u128)(-a) : (u128)a;
  u128 ub = b < 0 ? (u128)(-b) : (u128)b;
  uint64_t a0 = (uint64_t)ua, a1 = (uint64_t)(ua >> 64);
  uint64_t b0 = (uint64_t)ub, b1 = (uint64_t)(ub >> 64);
  u128 p00 = (u128)a0 * b0, p01 = (u128)a0 * b1, p10 = (u128)a1 * b0, p11 = (u128)a1 * b1;
  i256 r = i256_zero();
  r.w[0] = (uint64_t)p00;
  u128 mid = (p00 >> 64) + (uint64_t)p01 + (uint64_t)p10;
  r.w[1] = (uint64_t)mid;
  u128 hi = (mid >> 64) + (p01 >> 64) + (p10 >> 64) + (uint64_t)p11;
  r.w[2] = (uint64_t)hi;
  r.w[3] = (uint64_t)((hi >> 64) + (p11 >> 64));
  return neg ? i256_neg(r) : r;
}

static int i256_sign(i256 a) {
  if (a.w[3] >> 63) return -1;
  return (a.w[0] | a.w[1] | a.w[2] | a.w[3]) ? 1 : 0;
}

/* incircle(a,b,c,d) > 0 iff d lies strictly inside the circle through a,b,c
 * when a,b,c are counter-clockwise (the empty-circumcircle test). */
static int incircle(const int64_t* a, const int64_t* b, const int64_t* c, const int64_t* d) {
  i128 adx = a[0] - d[0], ady = a[1] - d[1];
  i128 bdx = b[0] - d[0], bdy = b[1] - d[1];
  i128 cdx = c[0] - d[0], cdy = c[1] - d[1];
  i128 al = adx * adx + ady * ady;
  i128 bl = bdx * bdx + bdy * bdy;
  i128 cl = cdx * cdx + cdy * cdy;
  i128 bc = bdx * cdy - bdy * cdx;
  i128 ca = cdx * ady - cdy * adx;
  i128 ab = adx * bdy - ady * bdx;
  i256 det = i256_add(i256_add(i256_mul(al, bc), i256_mul(bl, ca)), i256_mul(cl, ab));
  return i256_sign(det);
}

/* Exported for the tests: the same predicates on explicit points. */
int orc_orient2d(const int64_t* a, const int64_t* b, const int64_t* c) {
  return orient2(a[0], a[1], b[0], b[1], c[0], c[1]);
}
int orc_incircle(const int64_t* a, const int64_t* b, const int64_t* c, const int64_t* d) {
  return incircle(a, b, c, d);
}

/* ======================================================================== */
/* Bowyer-Watson Delaunay triangulation of a finite integer point set         */
/* ======================================================================== */

typedef struct {
  int32_t v[3];  /* vertices, counter-clockwise */
  int32_t nb[3]; /* nb[e] = triangle across the edge opposite v[e]; -1 = none */
  int32_t alive;
  int32_t mark;
} tri_t;

typedef struct {
  int64_t* xy;   /* 2 * npts coordinates, the last three are the super-triangle */
  int32_t npts;
  tri_t* t;
  int32_t nt, cap;
  int32_t* freelist;
  int32_t nfree;
  int32_t stamp;
  int32_t* stack;  /* scratch for the cavity search */
  int32_t* cav;
  int32_t scap;
} dt_t;

static int dt_newtri(dt_t* D) {
  if (D->nfree > 0) return D->freelist[--D->nfree];
  if (D->nt == D->cap) {
    int32_t nc = D->cap * 2;
    tri_t* nt = (tri_t*)realloc(D->t, sizeof(tri_t) * (size_t)nc);
    int32_t* nf = (int32_t*)realloc(D->freelist, sizeof(int32_t) * (size_t)nc);
    if (!nt || !nf) { if (nt) D->t = nt; if (nf) D->freelist = nf; return -1; }
    D->t = nt;
    D->freelist = nf;
    D->cap = nc;
  }
  return D->nt++;
}

static const int64_t* P(const dt_t* D, int32_t v) { return D->xy + 2 * (int64_t)v; }

static int tri_incircle(const dt_t* D, int32_t t, int32_t p) {
  const tri_t* T = &D->t[t];
  return incircle(P(D, T->v[0]), P(D, T->v[1]), P(D, T->v[2]), P(D, p));
}

static int grow_scratch(dt_t* D, int32_t need) {
  if (need <= D->scap) return 0;
  int32_t nc = D->scap * 2;
  while (nc < need) nc *= 2;
  int32_t* s = (int32_t*)realloc(D->stack, sizeof(int32_t) * (size_t)nc);
  if (!s) return -1;
  D->stack = s;
  int32_t* c = (int32_t*)realloc(D->cav, sizeof(int32_t) * (size_t)nc);
  if (!c) return -1;
  D->cav = c;
  D->scap = nc;
  return 0;
}

/* Insert point p.  *hint is a live triangle to start the walk from; on return
 * it holds one of the new triangles. */
static int dt_insert(dt_t* D, int32_t p, int32_t* hint) {
  const int64_t* q = P(D, p);
  /* 1. locate: straight visibility walk (terminates on a Delaunay mesh) */
  int32_t t = *hint;
  int64_t guard = 0;
  for (;;) {
    if (++guard > 4 * (int64_t)D->nt + 64) return ORC_ERR_INTERNAL;
    tri_t* T = &D->t[t];
    int moved = 0;
    for (int e = 0; e < 3; ++e) {
      const int64_t* a = P(D, T->v[(e + 1) % 3]);
      const int64_t* b = P(D, T->v[(e + 2) % 3]);
      if (orient2(a[0], a[1], b[0], b[1], q[0], q[1]) < 0) {
        if (T->nb[e] < 0) return ORC_ERR_INTERNAL; /* outside the super-triangle */
        t = T->nb[e];
        moved = 1;
        break;
      }
    }
    if (!moved) break;
  }
  for (int e = 0; e < 3; ++e) {
    const int64_t* a = P(D, D->t[t].v[e]);
    if (a[0] == q[0] && a[1] == q[1]) return ORC_ERR_DEGENERATE; /* coincident point */
  }
  /* 2. cavity: every triangle whose circumcircle strictly contains p,
   *    grown from the containing triangle across shared edges */
  D->stamp++;
  int32_t ncav = 0, sp = 0;
  if (grow_scratch(D, 16)) return ORC_ERR_OOM;
  D->stack[sp++] = t;
  D->t[t].mark = D->stamp;
  while (sp > 0) {
    int32_t c = D->stack[--sp];
    if (grow_scratch(D, ncav + sp + 8)) return ORC_ERR_OOM;
    D->cav[ncav++] = c;
    for (int e = 0; e < 3; ++e) {
      int32_t nb = D->t[c].nb[e];
      if (nb < 0 || D->t[nb].mark == D->stamp) continue;
      if (tri_incircle(D, nb, p) > 0) {
        D->t[nb].mark = D->stamp;
        D->stack[sp++] = nb;
      }
    }
  }
  /* 3. boundary edges (a -> b, counter-clockwise seen from inside) */
  int32_t nbd = 0;
  int32_t bcap = ncav + 2;
  int32_t* ba = (int32_t*)malloc(sizeof(int32_t) * (size_t)bcap * 3);
  if (!ba) return ORC_ERR_OOM;
  int32_t* bb = ba + bcap;
  int32_t* bo = bb + bcap;
  for (int32_t ci = 0; ci < ncav; ++ci) {
    tri_t* C = &D->t[D->cav[ci]];
    for (int e = 0; e < 3; ++e) {
      int32_t nb = C->nb[e];
      if (nb >= 0 && D->t[nb].mark == D->stamp) continue;
      if (nbd == bcap) { free(ba); return ORC_ERR_INTERNAL; }
      ba[nbd] = C->v[(e + 1) % 3];
      bb[nbd] = C->v[(e + 2) % 3];
      bo[nbd] = nb;
      ++nbd;
    }
  }
  if (nbd != ncav + 2) { free(ba); return ORC_ERR_INTERNAL; }
  /* 4. retriangulate the star-shaped cavity as a fan around p */
  for (int32_t ci = 0; ci < ncav; ++ci) {
    D->t[D->cav[ci]].alive = 0;
    D->freelist[D->nfree++] = D->cav[ci];
  }
  int32_t* nt = (int32_t*)malloc(sizeof(int32_t) * (size_t)nbd);
  if (!nt) { free(ba); return ORC_ERR_OOM; }
  for (int32_t k = 0; k < nbd; ++k) {
    int32_t id = dt_newtri(D);
    if (id < 0) { free(ba); free(nt); return ORC_ERR_OOM; }
    nt[k] = id;
    tri_t* T = &D->t[id];
    T->v[0] = p; T->v[1] = ba[k]; T->v[2] = bb[k];
    T->nb[0] = bo[k]; T->nb[1] = -1; T->nb[2] = -1;
    T->alive = 1;
    T->mark = 0;
    if (bo[k] >= 0) { /* re-point the outside neighbor at the new triangle */
      tri_t* O = &D->t[bo[k]];
      for (int e = 0; e < 3; ++e)
        if (O->v[(e + 1) % 3] == bb[k] && O->v[(e + 2) % 3] == ba[k]) O->nb[e] = id;
    }
  }
  for (int32_t k = 0; k < nbd; ++k) {
    tri_t* T = &D->t[nt[k]];
    for (int32_t m = 0; m < nbd; ++m) {
      if (ba[m] == T->v[2]) T->nb[1] = nt[m]; /* across edge (b, p) */
      if (bb[m] == T->v[1]) T->nb[2] = nt[m]; /* across edge (p, a) */
    }
  }
  *hint = nt[0];
  free(nt);
  free(ba);
  return ORC_OK;
}

static void dt_free(dt_t* D) {
  free(D->t); free(D->freelist); free(D->stack); free(D->cav);
}

/* Triangulate npts points (coords in xy[0 .. 2*npts), xy must have room for
 * three more points).  Insertion follows `order`. */
static int dt_build(dt_t* D, int64_t* xy, int32_t npts, const int32_t* order) {
  memset(D, 0, sizeof(*D));
  D->xy = xy;
  D->npts = npts;
  const int64_t T0 = (int64_t)1 << 34; /* encloses [-2^34, 2^34)^2 */
  xy[2 * (int64_t)npts + 0] = -T0;     xy[2 * (int64_t)npts + 1] = -T0;
  xy[2 * (int64_t)npts + 2] = 3 * T0;  xy[2 * (int64_t)npts + 3] = -T0;
  xy[2 * (int64_t)npts + 4] = -T0;     xy[2 * (int64_t)npts + 5] = 3 * T0;
  D->cap = 2 * npts + 64;
  D->t = (tri_t*)malloc(sizeof(tri_t) * (size_t)D->cap);
  D->freelist = (int32_t*)malloc(sizeof(int32_t) * (size_t)D->cap);
  D->scap = 64;
  D->stack = (int32_t*)malloc(sizeof(int32_t) * 64);
  D->cav = (int32_t*)malloc(sizeof(int32_t) * 64);
  if (!D->t || !D->freelist || !D->stack || !D->cav) return ORC_ERR_OOM;
  D->nt = 1;
  tri_t* S = &D->t[0];
  S->v[0] = npts; S->v[1] = npts + 1; S->v[2] = npts + 2;
  S->nb[0] = S->nb[1] = S->nb[2] = -1;
  S->alive = 1;
  S->mark = 0;
  int32_t hint = 0;
  for (int32_t k = 0; k < npts; ++k) {
    int rc = dt_insert(D, order[k], &hint);
    if (rc) return rc;
  }
  return ORC_OK;
}

/* ======================================================================== */
/* Periodic Voronoi neighbors                                                */
/* ======================================================================== */

typedef struct { int32_t a, b; } pair_t;

static int cmp_pair(const void* x, const void* y) {
  const pair_t* p = (const pair_t*)x;
  const pair_t* q = (const pair_t*)y;
  if (p->a != q->a) return p->a < q->a ? -1 : 1;
  if (p->b != q->b) return p->b < q->b ? -1 : 1;
  return 0;
}

/* Circumdisk of a triangle inside [xlo, xhi) x [ylo, yhi) (with a safety allowance)? */
static int disk_inside(const int64_t* a, const int64_t* b, const int64_t* c, double xlo, double xhi,
                       double ylo, double yhi) {
  long double bx = (long double)(b[0] - a[0]), by = (long double)(b[1] - a[1]);
  long double cx = (long double)(c[0] - a[0]), cy = (long double)(c[1] - a[1]);
  long double d = 2.0L * (bx * cy - by * cx);
  if (d == 0.0L) return 0;
  long double b2 = bx * bx + by * by, c2 = cx * cx + cy * cy;
  long double ux = (cy * b2 - by * c2) / d;
  long double uy = (bx * c2 - cx * b2) / d;
  long double R = sqrtl(ux * ux + uy * uy);
  long double ox = (long double)a[0] + ux, oy = (long double)a[1] + uy;
  long double tol = 1e-9L * (fabsl(ox) + fabsl(oy) + R) + 4.0L;
  return ox - R - tol >= xlo && ox + R + tol < xhi && oy - R - tol >= ylo && oy + R + tol < yhi;
}

typedef struct {
  int64_t* xy;
  int32_t* orig;  /* original id of every tiled point */
  int32_t npts;
  dt_t D;
  int built;
} vtess_t;

static void vtess_free(vtess_t* V) {
  if (V->built) dt_free(&V->D);
  free(V->xy);
  free(V->orig);
  memset(V, 0, sizeof(*V));
}

static uint64_t spread_bits(uint32_t v) { /* 16 -> 32 bit interleave helper */
  uint64_t x = v & 0xFFFFu;
  x = (x | (x << 8)) & 0x00FF00FFu;
  x = (x | (x << 4)) & 0x0F0F0F0Fu;
  x = (x | (x << 2)) & 0x33333333u;
  x = (x | (x << 1)) & 0x55555555u;
  return x;
}

typedef struct { uint64_t key; int32_t idx; } keyed_t;
static int cmp_keyed(const void* x, const void* y) {
  const keyed_t* p = (const keyed_t*)x;
  const keyed_t* q = (const keyed_t*)y;
  if (p->key != q->key) return p->key < q->key ? -1 : 1;
  return p->idx < q->idx ? -1 : (p->idx > q->idx);
}

/* Build the triangulation of the originals plus their periodic images within
 * `margin` of the box, and check that every triangle touching an original
 * point is a triangle of the periodic Delaunay triangulation.
 * Returns ORC_OK, a failure code, or -1 if the margin was too small. */
static int vtess_build(vtess_t* V, int64_t n, const int32_t* pos, const int64_t* box, int64_t margin) {
  memset(V, 0, sizeof(*V));
  int64_t Lx = box[0], Ly = box[1];
  /* a star circumdisk reaches at most sqrt(2) L from its point (the largest
   * empty circle of a periodic set has radius <= L/sqrt(2)), so margins up
   * to 2L (a 5x5 tiling) always suffice */
  int64_t mx = margin < 2 * Lx ? margin : 2 * Lx, my = margin < 2 * Ly ? margin : 2 * Ly;
  int64_t cap = 25 * n;
  V->xy = (int64_t*)malloc(sizeof(int64_t) * (size_t)(2 * cap + 6));
  V->orig = (int32_t*)malloc(sizeof(int32_t) * (size_t)cap);
  if (!V->xy || !V->orig) return ORC_ERR_OOM;
  int32_t m = 0;
  /* originals first (indices 0..n-1), then images */
  for (int pass = 0; pass < 2; ++pass)
    for (int sy = -2; sy <= 2; ++sy)
      for (int sx = -2; sx <= 2; ++sx) {
        int center = (sx == 0 && sy == 0);
        if ((pass == 0) != center) continue;
        for (int64_t i = 0; i < n; ++i) {
          int64_t x = (int64_t)pos[2 * i] + sx * Lx;
          int64_t y = (int64_t)pos[2 * i + 1] + sy * Ly;
          if (x < -mx || x >= Lx + mx || y < -my || y >= Ly + my) continue;
          V->xy[2 * (int64_t)m] = x;
          V->xy[2 * (int64_t)m + 1] = y;
          V->orig[m] = (int32_t)i;
          ++m;
        }
      }
  V->npts = m;
  /* spatially coherent insertion order (Morton order of a coarse grid) keeps
   * the point-location walks short */
  keyed_t* ks = (keyed_t*)malloc(sizeof(keyed_t) * (size_t)m);
  int32_t* order = (int32_t*)malloc(sizeof(int32_t) * (size_t)m);
  if (!ks || !order) { free(ks); free(order); return ORC_ERR_OOM; }
  long double spanx = (long double)(Lx + 2 * mx), spany = (long double)(Ly + 2 * my);
  for (int32_t i = 0; i < m; ++i) {
    uint32_t gx = (uint32_t)((long double)(V->xy[2 * (int64_t)i] + mx) / spanx * 65535.0L);
    uint32_t gy = (uint32_t)((long double)(V->xy[2 * (int64_t)i + 1] + my) / spany * 65535.0L);
    ks[i].key = spread_bits(gx) | (spread_bits(gy) << 1);
    ks[i].idx = i;
  }
  qsort(ks, (size_t)m, sizeof(keyed_t), cmp_keyed);
  for (int32_t i = 0; i < m; ++i) order[i] = ks[i].idx;
  free(ks);
  int rc = dt_build(&V->D, V->xy, m, order);
  free(order);
  V->built = 1;
  if (rc) return rc;
  /* verification of the stars of the originals */
  double xlo = (double)(-mx), xhi = (double)(Lx + mx), ylo = (double)(-my), yhi = (double)(Ly + my);
  for (int32_t t = 0; t < V->D.nt; ++t) {
    tri_t* T = &V->D.t[t];
    if (!T->alive) continue;
    int touches = 0, super = 0;
    for (int e = 0; e < 3; ++e) {
      if (T->v[e] < n) touches = 1;
      if (T->v[e] >= m) super = 1;
    }
    if (!touches) continue;
    if (super) return -1;
    if (!disk_inside(P(&V->D, T->v[0]), P(&V->D, T->v[1]), P(&V->D, T->v[2]), xlo, xhi, ylo, yhi))
      return -1;
  }
  return ORC_OK;
}

static int vtess_build_auto(vtess_t* V, int64_t n, const int32_t* pos, const int64_t* box) {
  int64_t L2 = 2 * (box[0] > box[1] ? box[0] : box[1]);
  double spacing = sqrt((double)box[0] * (double)box[1] / (double)n);
  int64_t margin = (int64_t)ceil(8.0 * spacing);
  for (;;) {
    if (margin > L2) margin = L2;
    int rc = vtess_build(V, n, pos, box, margin);
    if (rc == ORC_OK) return ORC_OK;
    vtess_free(V);
    if (rc > 0) return rc;
    if (margin == L2) return ORC_ERR_INTERNAL;
    margin *= 2;
  }
}

typedef struct { int32_t x, y, id; } pidx_t;
static int cmp_pidx(const void* a, const void* b) {
  const pidx_t* p = (const pidx_t*)a;
  const pidx_t* q = (const pidx_t*)b;
  if (p->x != q->x) return p->x < q->x ? -1 : 1;
  if (p->y != q->y) return p->y < q->y ? -1 : 1;
  return p->id < q->id ? -1 : (p->id > q->id);
}

/* Voronoi neighbors of every particle in a periodic rectangular box.
 * Coincident particles are one site: they are each other's neighbors and
 * share the neighbors of their site (the Voronoi cell of the site).  On
 * success offsets[0..n] is a CSR index into ids (sorted by id within a row).
 * With ids == NULL only *nnz is computed; if `cap` is too small, *nnz
 * receives the size needed and ORC_ERR_ARG is returned. */
int orc_voronoi(int64_t n, const int32_t* pos, const int64_t* box, int64_t* offsets,
                int32_t* ids, int64_t cap, int64_t* nnz) {
  if (n < 1 || box[0] < 2 || box[1] < 2 || box[0] > ((int64_t)1 << 31) || box[1] > ((int64_t)1 << 31))
    return ORC_ERR_ARG;
  for (int64_t i = 0; i < n; ++i)
    if (pos[2 * i] < 0 || pos[2 * i] >= box[0] || pos[2 * i + 1] < 0 || pos[2 * i + 1] >= box[1])
      return ORC_ERR_ARG;
  /* distinct sites: site_of[i], members of each site in id order */
  pidx_t* srt = (pidx_t*)malloc(sizeof(pidx_t) * (size_t)n);
  int32_t* site_of = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  int32_t* site_pos = (int32_t*)malloc(sizeof(int32_t) * 2 * (size_t)n);
  int64_t* site_beg = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
  int32_t* members = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  if (!srt || !site_of || !site_pos || !site_beg || !members) {
    free(srt); free(site_of); free(site_pos); free(site_beg); free(members);
    return ORC_ERR_OOM;
  }
  for (int64_t i = 0; i < n; ++i) { srt[i].x = pos[2 * i]; srt[i].y = pos[2 * i + 1]; srt[i].id = (int32_t)i; }
  qsort(srt, (size_t)n, sizeof(pidx_t), cmp_pidx);
  int64_t ns = 0;
  for (int64_t r = 0; r < n; ++r) {
    if (r == 0 || srt[r].x != srt[r - 1].x || srt[r].y != srt[r - 1].y) {
      site_beg[ns] = r;
      site_pos[2 * ns] = srt[r].x;
      site_pos[2 * ns + 1] = srt[r].y;
      ++ns;
    }
    site_of[srt[r].id] = (int32_t)(ns - 1);
    members[r] = srt[r].id;
  }
  site_beg[ns] = n;
  free(srt);
  int64_t npair = 0;
  pair_t* pr = NULL;
  int rc = ORC_OK;
  if (ns >= 1) {
    vtess_t V;
    rc = vtess_build_auto(&V, ns, site_pos, box);
    if (rc == ORC_OK) {
      dt_t* D = &V.D;
      int64_t pcap = 8 * ns + 64;
      pair_t* sp = (pair_t*)malloc(sizeof(pair_t) * (size_t)pcap);
      int64_t nsp = 0;
      if (!sp) rc = ORC_ERR_OOM;
      for (int32_t t = 0; t < D->nt && rc == ORC_OK; ++t) {
        tri_t* T = &D->t[t];
        if (!T->alive) continue;
        for (int e = 0; e < 3; ++e) {
          int32_t a = T->v[(e + 1) % 3], b = T->v[(e + 2) % 3];
          if (a >= ns) continue; /* only edges leaving an original site */
          int32_t u = T->nb[e];
          if (u < 0) { rc = ORC_ERR_INTERNAL; break; }
          int32_t w = -1;
          for (int f = 0; f < 3; ++f)
            if (D->t[u].v[f] != a && D->t[u].v[f] != b) w = D->t[u].v[f];
          /* the dual Voronoi edge has zero length iff the four points are cocircular */
          if (incircle(P(D, T->v[0]), P(D, T->v[1]), P(D, T->v[2]), P(D, w)) == 0) continue;
          int32_t jb = V.orig[b];
          if (jb == a) continue; /* an image of the site itself */
          if (nsp == pcap) {
            pcap *= 2;
            pair_t* q = (pair_t*)realloc(sp, sizeof(pair_t) * (size_t)pcap);
            if (!q) { rc = ORC_ERR_OOM; break; }
            sp = q;
          }
          sp[nsp].a = a;
          sp[nsp].b = jb;
          ++nsp;
        }
      }
      vtess_free(&V);
      /* expand site pairs to particle pairs, plus the coincident partners */
      int64_t tot = 0;
      for (int64_t q = 0; q < nsp && rc == ORC_OK; ++q)
        tot += (site_beg[sp[q].a + 1] - site_beg[sp[q].a]) * (site_beg[sp[q].b + 1] - site_beg[sp[q].b]);
      for (int64_t c = 0; c < ns; ++c) {
        int64_t m = site_beg[c + 1] - site_beg[c];
        tot += m * (m - 1);
      }
      if (rc == ORC_OK) {
        pr = (pair_t*)malloc(sizeof(pair_t) * (size_t)(tot > 0 ? tot : 1));
        if (!pr) rc = ORC_ERR_OOM;
      }
      for (int64_t q = 0; q < nsp && rc == ORC_OK; ++q)
        for (int64_t x = site_beg[sp[q].a]; x < site_beg[sp[q].a + 1]; ++x)
          for (int64_t y = site_beg[sp[q].b]; y < site_beg[sp[q].b + 1]; ++y) {
            pr[npair].a = members[x];
            pr[npair].b = members[y];
            ++npair;
          }
      for (int64_t c = 0; c < ns && rc == ORC_OK; ++c)
        for (int64_t x = site_beg[c]; x < site_beg[c + 1]; ++x)
          for (int64_t y = site_beg[c]; y < site_beg[c + 1]; ++y)
            if (x != y) {
              pr[npair].a = members[x];
              pr[npair].b = members[y];
              ++npair;
            }
      free(sp);
    }
  }
  free(site_of); free(site_pos); free(site_beg); free(members);
  if (rc != ORC_OK) { free(pr); return rc; }
  qsort(pr, (size_t)npair, sizeof(pair_t), cmp_pair);
  int64_t u = 0;
  for (int64_t s2 = 0; s2 < npair; ++s2)
    if (s2 == 0 || pr[s2].a != pr[s2 - 1].a || pr[s2].b != pr[s2 - 1].b) pr[u++] = pr[s2];
  *nnz = u;
  if (ids == NULL) { free(pr); return ORC_OK; } /* size query */
  if (u > cap) { free(pr); return ORC_ERR_ARG; }
  int64_t s = 0;
  for (int64_t i = 0; i < n; ++i) {
    offsets[i] = s;
    while (s < u && pr[s].a == i) { ids[s] = pr[s].b; ++s; }
  }
  offsets[n] = s;
  free(pr);
  return ORC_OK;
}

/* The triangles of the periodic Delaunay triangulation that touch an original
 * point, as tiled coordinates (6 int64 per triangle, counter-clockwise) and
 * original ids (3 per triangle).  For the empty-circumcircle checks. */
int orc_delaunay_star_triangles(int64_t n, const int32_t* pos, const int64_t* box,
                                int64_t* coords, int32_t* tids, int64_t cap, int64_t* ntri) {
  vtess_t V;
  int rc = vtess_build_auto(&V, n, pos, box);
  if (rc) return rc;
  int64_t c = 0;
  for (int32_t t = 0; t < V.D.nt; ++t) {
    tri_t* T = &V.D.t[t];
    if (!T->alive) continue;
    if (T->v[0] >= n && T->v[1] >= n && T->v[2] >= n) continue;
    if (c < cap) {
      for (int e = 0; e < 3; ++e) {
        coords[6 * c + 2 * e] = V.xy[2 * (int64_t)T->v[e]];
        coords[6 * c + 2 * e + 1] = V.xy[2 * (int64_t)T->v[e] + 1];
        tids[3 * c + e] = V.orig[T->v[e]];
      }
    }
    ++c;
  }
  *ntri = c;
  vtess_free(&V);
  return c > cap ? ORC_ERR_ARG : ORC_OK;
}

/* ======================================================================== */
/* Voronoi tissue model: cell areas, perimeters, energy and forces            */
/* ======================================================================== */

/* Circumcenter of (0, a, b) (a, b relative to the first point), FP64. */
static void circum_rel(double ax, double ay, double bx, double by, double* ux, double* uy) {
  const double D = 2.0 * (ax * by - ay * bx);
  const double a2 = ax * ax + ay * ay, b2 = bx * bx + by * by;
  *ux = (by * a2 - ay * b2) / D;
  *uy = (ax * b2 - bx * a2) / D;
}

/* Jacobian J[mu][lam] = d h_mu / d r_lam of the circumcenter h of the
 * triangle (r, r + a, r + b) with respect to its first point r: h = r + u(a, b)
 * with a = r_a - r, b = r_b - r, so dh/dr = I - du/da - du/db.  Obtained by
 * differentiating the closed form of circum_rel (quotient rule). */
static void circum_jac_first(double ax, double ay, double bx, double by, double J[2][2]) {
  const double D = 2.0 * (ax * by - ay * bx);
  const double a2 = ax * ax + ay * ay, b2 = bx * bx + by * by;
  const double Nx = by * a2 - ay * b2, Ny = ax * b2 - bx * a2;
  /* partial derivatives of Nx, Ny, D with respect to (ax, ay, bx, by) */
  const double dNx[4] = {2.0 * ax * by, 2.0 * ay * by - b2, -2.0 * bx * ay, a2 - 2.0 * by * ay};
  const double dNy[4] = {b2 - 2.0 * ax * bx, -2.0 * ay * bx, 2.0 * bx * ax - a2, 2.0 * by * ax};
  const double dD[4] = {2.0 * by, -2.0 * bx, -2.0 * ay, 2.0 * ax};
  double du[2][4];
  for (int v = 0; v < 4; ++v) {
    du[0][v] = (dNx[v] * D - Nx * dD[v]) / (D * D);
    du[1][v] = (dNy[v] * D - Ny * dD[v]) / (D * D);
  }
  for (int mu = 0; mu < 2; ++mu)
    for (int lam = 0; lam < 2; ++lam) J[mu][lam] = (mu == lam ? 1.0 : 0.0) - du[mu][lam] - du[mu][2 + lam];
}

/* dE_c/dh for the vertex h of cell c whose polygon neighbors (counter-
 * clockwise order) are prev and next, all relative to the same origin:
 * A = (1/2) sum cross(h_k, h_k+1) gives dA/dh = (1/2)(y_next - y_prev,
 * x_prev - x_next); P = sum |h_k+1 - h_k| gives dP/dh = (h - prev)/|h - prev|
 * + (h - next)/|h - next|. */
static int cell_grad(double hx, double hy, double px, double py, double nx, double ny, double gA, double gP,
                     double* gx, double* gy) {
  const double l1 = hypot(hx - px, hy - py), l2 = hypot(hx - nx, hy - ny);
  if (!(l1 > 0.0) || !(l2 > 0.0)) return ORC_ERR_DEGENERATE;
  *gx = gA * 0.5 * (ny - py) + gP * ((hx - px) / l1 + (hx - nx) / l2);
  *gy = gA * 0.5 * (px - nx) + gP * ((hy - py) / l1 + (hy - ny) / l2);
  return ORC_OK;
}

/* Voronoi tissue model (Sec. "Geometric models of dense tissue"): every
 * particle is the generator of its Voronoi cell, of area A_i and perimeter
 * P_i; the energy is Eq. (vmEnergy), E = sum_i KA (A_i - A0)^2 +
 * KP (P_i - P0)^2, and the force on particle i is F_i = -dE/dr_i (Sec.
 * "Voronoi model forces"): moving r_i moves the vertices of cell i, the
 * circumcenters h of the Delaunay triangles (i, a, b) around it, and each
 * such vertex is shared by the cells i, a and b, so
 *   F_i = - sum_{h of cell i} (dh/dr_i)^T (dE_i/dh + dE_a/dh + dE_b/dh).
 * Positions are grid units scaled by `unit` (the length of one grid unit)
 * into length units; everything is FP64.  Needs distinct particles and a
 * cell polygon without zero-length edges (no four cocircular particles),
 * else ORC_ERR_DEGENERATE.  force: 2 n doubles (may be NULL). */
int orc_tissue(int64_t n, const int32_t* pos, const int64_t* box, double unit, double KA, double KP, double A0,
               double P0, double* area, double* perim, double* force, double* energy) {
  if (n < 3 || box[0] < 2 || box[1] < 2 || !(unit > 0.0)) return ORC_ERR_ARG;
  /* distinct particles */
  {
    pidx_t* srt = (pidx_t*)malloc(sizeof(pidx_t) * (size_t)n);
    if (!srt) return ORC_ERR_OOM;
    for (int64_t i = 0; i < n; ++i) {
      srt[i].x = pos[2 * i];
      srt[i].y = pos[2 * i + 1];
      srt[i].id = (int32_t)i;
    }
    qsort(srt, (size_t)n, sizeof(pidx_t), cmp_pidx);
    int dup = 0;
    for (int64_t i = 1; i < n; ++i) dup |= srt[i].x == srt[i - 1].x && srt[i].y == srt[i - 1].y;
    free(srt);
    if (dup) return ORC_ERR_DEGENERATE;
  }
  vtess_t V;
  int rc = vtess_build_auto(&V, n, pos, box);
  if (rc) return rc;
  /* stars of the originals: triangles (i, a, b), counter-clockwise, i first */
  int64_t* beg = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  if (!beg) { vtess_free(&V); return ORC_ERR_OOM; }
  for (int32_t t = 0; t < V.D.nt; ++t) {
    const tri_t* T = &V.D.t[t];
    if (!T->alive) continue;
    for (int e = 0; e < 3; ++e)
      if (T->v[e] < n) beg[T->v[e] + 1] += 1;
  }
  for (int64_t i = 0; i < n; ++i) beg[i + 1] += beg[i];
  const int64_t ns = beg[n];
  int32_t* sa = (int32_t*)malloc(sizeof(int32_t) * (size_t)ns);
  int32_t* sb = (int32_t*)malloc(sizeof(int32_t) * (size_t)ns);
  int32_t* ord = (int32_t*)malloc(sizeof(int32_t) * (size_t)ns);  /* star entries in fan order */
  double* hx = (double*)malloc(sizeof(double) * (size_t)ns);     /* vertices relative to the owner */
  double* hy = (double*)malloc(sizeof(double) * (size_t)ns);
  int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
  if (!sa || !sb || !ord || !hx || !hy || !fill) {
    free(beg); free(sa); free(sb); free(ord); free(hx); free(hy); free(fill);
    vtess_free(&V);
    return ORC_ERR_OOM;
  }
  for (int64_t i = 0; i < n; ++i) fill[i] = beg[i];
  for (int32_t t = 0; t < V.D.nt; ++t) {
    const tri_t* T = &V.D.t[t];
    if (!T->alive) continue;
    for (int e = 0; e < 3; ++e)
      if (T->v[e] < n) {
        const int64_t w = fill[T->v[e]]++;
        sa[w] = T->v[(e + 1) % 3];
        sb[w] = T->v[(e + 2) % 3];
      }
  }
  rc = ORC_OK;
  /* chain every star into a fan: entry k is followed by the entry whose a is
   * its b; then the vertices (circumcenters) in counter-clockwise order */
  for (int64_t i = 0; i < n && rc == ORC_OK; ++i) {
    const int64_t b0 = beg[i], m = beg[i + 1] - beg[i];
    if (m < 3) { rc = ORC_ERR_DEGENERATE; break; }
    int64_t cur = b0;
    for (int64_t k = 0; k < m; ++k) {
      ord[b0 + k] = (int32_t)(cur - b0);
      int64_t nxt = -1;
      for (int64_t q = b0; q < b0 + m; ++q)
        if (sa[q] == sb[cur]) { nxt = q; break; }
      if (nxt < 0) { rc = ORC_ERR_INTERNAL; break; }
      cur = nxt;
    }
    if (rc == ORC_OK && cur != b0) rc = ORC_ERR_INTERNAL;  /* the fan must close after m triangles */
    const double xi = (double)V.xy[2 * i], yi = (double)V.xy[2 * i + 1];
    double A = 0.0, Pm = 0.0;
    for (int64_t k = 0; k < m && rc == ORC_OK; ++k) {
      const int64_t q = b0 + ord[b0 + k];
      circum_rel(((double)V.xy[2 * (int64_t)sa[q]] - xi) * unit, ((double)V.xy[2 * (int64_t)sa[q] + 1] - yi) * unit,
                 ((double)V.xy[2 * (int64_t)sb[q]] - xi) * unit, ((double)V.xy[2 * (int64_t)sb[q] + 1] - yi) * unit,
                 &hx[b0 + k], &hy[b0 + k]);
    }
    for (int64_t k = 0; k < m && rc == ORC_OK; ++k) {
      const int64_t k1 = (k + 1) % m;
      A += 0.5 * (hx[b0 + k] * hy[b0 + k1] - hx[b0 + k1] * hy[b0 + k]);
      Pm += hypot(hx[b0 + k1] - hx[b0 + k], hy[b0 + k1] - hy[b0 + k]);
    }
    area[i] = A;
    perim[i] = Pm;
  }
  double E = 0.0;
  for (int64_t i = 0; i < n && rc == ORC_OK; ++i)
    E += KA * (area[i] - A0) * (area[i] - A0) + KP * (perim[i] - P0) * (perim[i] - P0);
  if (rc == ORC_OK) *energy = E;
  /* forces: for vertex k of cell i (triangle (i, a, b)), the same vertex in
   * the fans of the originals of a and b is found by the integer offsets of
   * the triangle's other two points */
  for (int64_t i = 0; force && i < n && rc == ORC_OK; ++i) {
    const int64_t b0 = beg[i], m = beg[i + 1] - beg[i];
    const int64_t xi = V.xy[2 * i], yi = V.xy[2 * i + 1];
    double Fx = 0.0, Fy = 0.0;
    for (int64_t k = 0; k < m && rc == ORC_OK; ++k) {
      const int64_t q = b0 + ord[b0 + k];
      const int32_t va = sa[q], vb = sb[q];
      double gx = 0.0, gy = 0.0, cx, cy;
      /* cell i itself */
      const int64_t kp = (k + m - 1) % m, kn = (k + 1) % m;
      rc = cell_grad(hx[b0 + k], hy[b0 + k], hx[b0 + kp], hy[b0 + kp], hx[b0 + kn], hy[b0 + kn],
                     2.0 * KA * (area[i] - A0), 2.0 * KP * (perim[i] - P0), &cx, &cy);
      gx += cx;
      gy += cy;
      /* cells a and b: the triangle is (a, b, i) around a and (b, i, a) around b */
      for (int side = 0; side < 2 && rc == ORC_OK; ++side) {
        const int32_t vc = side == 0 ? va : vb;          /* the cell's point (tiled) */
        const int32_t v1 = side == 0 ? vb : (int32_t)i;  /* next point around it */
        const int32_t v2 = side == 0 ? (int32_t)i : va;
        const int32_t c = V.orig[vc];
        const int64_t d1x = V.xy[2 * (int64_t)v1] - V.xy[2 * (int64_t)vc], d1y = V.xy[2 * (int64_t)v1 + 1] - V.xy[2 * (int64_t)vc + 1];
        const int64_t d2x = V.xy[2 * (int64_t)v2] - V.xy[2 * (int64_t)vc], d2y = V.xy[2 * (int64_t)v2 + 1] - V.xy[2 * (int64_t)vc + 1];
        const int64_t cb = beg[c], cm = beg[c + 1] - beg[c];
        const int64_t cxo = V.xy[2 * (int64_t)c], cyo = V.xy[2 * (int64_t)c + 1];
        int64_t at = -1;
        for (int64_t kk = 0; kk < cm; ++kk) {
          const int64_t qq = cb + ord[cb + kk];
          if (V.xy[2 * (int64_t)sa[qq]] - cxo == d1x && V.xy[2 * (int64_t)sa[qq] + 1] - cyo == d1y &&
              V.xy[2 * (int64_t)sb[qq]] - cxo == d2x && V.xy[2 * (int64_t)sb[qq] + 1] - cyo == d2y) {
            at = kk;
            break;
          }
        }
        if (at < 0) { rc = ORC_ERR_INTERNAL; break; }
        const int64_t ap = (at + cm - 1) % cm, an = (at + 1) % cm;
        rc = cell_grad(hx[cb + at], hy[cb + at], hx[cb + ap], hy[cb + ap], hx[cb + an], hy[cb + an],
                       2.0 * KA * (area[c] - A0), 2.0 * KP * (perim[c] - P0), &cx, &cy);
        gx += cx;
        gy += cy;
      }
      if (rc != ORC_OK) break;
      double J[2][2];
      circum_jac_first(((double)(V.xy[2 * (int64_t)va] - xi)) * unit, ((double)(V.xy[2 * (int64_t)va + 1] - yi)) * unit,
                       ((double)(V.xy[2 * (int64_t)vb] - xi)) * unit, ((double)(V.xy[2 * (int64_t)vb + 1] - yi)) * unit, J);
      Fx -= gx * J[0][0] + gy * J[1][0];
      Fy -= gx * J[0][1] + gy * J[1][1];
    }
    force[2 * i] = Fx;
    force[2 * i + 1] = Fy;
  }
  free(beg); free(sa); free(sb); free(ord); free(hx); free(hy); free(fill);
  vtess_free(&V);
  return rc;
}

/* ======================================================================== */
/* 3D Voronoi neighbors (Sec. "Computational tools: Voronoi neighbor lists": */
/* the Voronoi cell of a particle holds the points closer to it than to any  */
/* other particle; two particles are neighbors when their cells share a      */
/* face).                                                                    */
/*                                                                          */
/* The cell is the intersection of the half-spaces {x : d.x <= |d|^2 / 2},   */
/* one for every periodic image d (offset from the particle) of every other  */
/* particle, and of the particle's own images.  It is built by clipping a    */
/* polytope held as faces (one per plane) with vertex loops.  A vertex is    */
/* the meeting point y/2 of three planes (d_a.y = w_a, d_b.y = w_b,          */
/* d_c.y = w_c with w = |d|^2); whether it lies beyond the plane of a site e */
/* is decided exactly: with M the 3x3 matrix of rows d_a, d_b, d_c,          */
/*   det [d_a w_a; d_b w_b; d_c w_c; d_e w_e] = det(M) (w_e - d_e.y),        */
/* so sign(d_e.y - w_e) = -sign(det4) sign(det M), both integer determinants */
/* (the 4x4 one is the insphere test of the particle, a, b, c and e).        */
/* Neighbors are the sites whose plane carries a face of positive area; a    */
/* plane that meets the cell in an edge or a vertex only (the diagonal       */
/* neighbors of a cubic lattice) does not count.  Coincident particles are   */
/* reported as degenerate.                                                   */
/* ======================================================================== */

typedef struct {
  int64_t d[3]; /* offset of the site image from the particle (grid units) */
  i128 w;       /* |d|^2 */
  int32_t id;   /* particle id of the site; -1 for an image of the particle itself */
} c3plane;

typedef struct {
  int32_t p[3]; /* the three planes defining the vertex */
  int32_t alive;
  double x[3];  /* approximate position (grid units): search radius and volume only */
} c3vert;

typedef struct {
  int32_t plane, alive, n, cap;
  int32_t* v;   /* vertex loop, counter-clockwise seen from outside the cell */
} c3face;

typedef struct {
  c3plane* pl; int32_t npl, cappl;
  c3vert* vt; int32_t nvt, capvt;
  c3face* fc; int32_t nfc, capfc;
  int8_t* sg; int32_t capsg;            /* side of every vertex for the current clip */
  int32_t* memo; int32_t nmemo, capmemo; /* crossing vertices of the current clip: (a, b, x) */
  int32_t* eg; int32_t neg, capeg;      /* boundary edges of the new face: (tail, head) */
  int32_t* tmp; int32_t captmp;
} c3cell;

static int c3_grow(void** p, int32_t* cap, int64_t need, size_t elem) {
  if (need <= *cap) return 0;
  int64_t nc = *cap ? *cap : 16;
  while (nc < need) nc *= 2;
  if (nc > INT32_MAX) return 1;
  void* q = realloc(*p, (size_t)nc * elem);
  if (!q) return 1;
  *p = q;
  *cap = (int32_t)nc;
  return 0;
}

static void c3_free(c3cell* C) {
  for (int32_t f = 0; f < C->capfc; ++f) free(C->fc[f].v);
  free(C->pl); free(C->vt); free(C->fc); free(C->sg); free(C->memo); free(C->eg); free(C->tmp);
  memset(C, 0, sizeof(*C));
}

static i128 det3_i(const int64_t* a, const int64_t* b, const int64_t* c) {
  return (i128)a[0] * ((i128)b[1] * c[2] - (i128)b[2] * c[1]) -
         (i128)a[1] * ((i128)b[0] * c[2] - (i128)b[2] * c[0]) +
         (i128)a[2] * ((i128)b[0] * c[1] - (i128)b[1] * c[0]);
}

static double i256_to_double(i256 a) {
  const int neg = (a.w[3] >> 63) != 0;
  if (neg) a = i256_neg(a);
  double r = 0.0;
  for (int t = 3; t >= 0; --t) r = r * 18446744073709551616.0 + (double)a.w[t];
  return neg ? -r : r;
}

/* Side of vertex v of the cell with respect to the plane of site e:
 * +1 strictly beyond it, 0 on it, -1 strictly inside. */
static int c3_side(const c3cell* C, int32_t v, int32_t e) {
  const c3plane* A = &C->pl[C->vt[v].p[0]];
  const c3plane* B = &C->pl[C->vt[v].p[1]];
  const c3plane* D = &C->pl[C->vt[v].p[2]];
  const c3plane* E = &C->pl[e];
  const i128 m = det3_i(A->d, B->d, D->d);
  /* det4 expanded along its last column (w) */
  i256 t = i256_mul(-A->w, det3_i(B->d, D->d, E->d));
  t = i256_add(t, i256_mul(B->w, det3_i(A->d, D->d, E->d)));
  t = i256_add(t, i256_mul(-D->w, det3_i(A->d, B->d, E->d)));
  t = i256_add(t, i256_mul(E->w, m));
  const int s4 = i256_sign(t), sm = (m > 0) - (m < 0);
  return -s4 * sm;
}

/* new vertex of planes (a, b, c); its approximate position by Cramer's rule
 * on the exact integer determinants */
static int32_t c3_new_vertex(c3cell* C, int32_t a, int32_t b, int32_t c) {
  if (c3_grow((void**)&C->vt, &C->capvt, (int64_t)C->nvt + 1, sizeof(c3vert))) return -1;
  c3vert* V = &C->vt[C->nvt];
  V->p[0] = a; V->p[1] = b; V->p[2] = c;
  V->alive = 1;
  const int64_t* M[3] = {C->pl[a].d, C->pl[b].d, C->pl[c].d};
  const i128 w[3] = {C->pl[a].w, C->pl[b].w, C->pl[c].w};
  /* cofactors of M: cyclic index form */
  i128 cf[3][3];
  for (int r = 0; r < 3; ++r)
    for (int k = 0; k < 3; ++k) {
      const int r0 = (r + 1) % 3, r1 = (r + 2) % 3, k0 = (k + 1) % 3, k1 = (k + 2) % 3;
      cf[r][k] = (i128)M[r0][k0] * M[r1][k1] - (i128)M[r0][k1] * M[r1][k0];
    }
  const i128 det = (i128)M[0][0] * cf[0][0] + (i128)M[0][1] * cf[0][1] + (i128)M[0][2] * cf[0][2];
  const double dd = (double)det;
  for (int k = 0; k < 3; ++k) {
    i256 num = i256_add(i256_add(i256_mul(w[0], cf[0][k]), i256_mul(w[1], cf[1][k])), i256_mul(w[2], cf[2][k]));
    V->x[k] = 0.5 * i256_to_double(num) / dd; /* x = y / 2 */
  }
  return C->nvt++;
}

static int32_t c3_add_plane(c3cell* C, const int64_t* d, int32_t id) {
  if (c3_grow((void**)&C->pl, &C->cappl, (int64_t)C->npl + 1, sizeof(c3plane))) return -1;
  c3plane* P = &C->pl[C->npl];
  for (int a = 0; a < 3; ++a) P->d[a] = d[a];
  P->w = (i128)d[0] * d[0] + (i128)d[1] * d[1] + (i128)d[2] * d[2];
  P->id = id;
  return C->npl++;
}

static int c3_face_push(c3face* F, int32_t v) {
  if (c3_grow((void**)&F->v, &F->cap, (int64_t)F->n + 1, sizeof(int32_t))) return 1;
  F->v[F->n++] = v;
  return 0;
}

static int32_t c3_new_face(c3cell* C, int32_t plane) {
  if (C->nfc == C->capfc) {
    const int32_t old = C->capfc;
    if (c3_grow((void**)&C->fc, &C->capfc, (int64_t)C->nfc + 1, sizeof(c3face))) return -1;
    for (int32_t f = old; f < C->capfc; ++f) {
      C->fc[f].v = NULL;
      C->fc[f].cap = 0;
    }
  }
  c3face* F = &C->fc[C->nfc];
  F->plane = plane;
  F->alive = 1;
  F->n = 0;
  return C->nfc++;
}

/* The cell bounded by the particle's own images at +-L along each axis: the
 * box-shaped cube (planes 0..5 = +x, -x, +y, -y, +z, -z). */
static int c3_init(c3cell* C, const int64_t* box) {
  C->npl = C->nvt = C->nfc = 0;
  for (int a = 0; a < 3; ++a)
    for (int sgn = 0; sgn < 2; ++sgn) {
      int64_t d[3] = {0, 0, 0};
      d[a] = sgn ? -box[a] : box[a];
      if (c3_add_plane(C, d, -1) < 0) return ORC_ERR_OOM;
    }
  /* vertex (sx, sy, sz) = bit 0, 1, 2 set for the + side */
  for (int v = 0; v < 8; ++v)
    if (c3_new_vertex(C, (v & 1) ? 0 : 1, (v & 2) ? 2 : 3, (v & 4) ? 4 : 5) < 0) return ORC_ERR_OOM;
  static const int loops[6][4] = {{1, 3, 7, 5}, {0, 4, 6, 2}, {2, 6, 7, 3},
                                  {0, 1, 5, 4}, {4, 5, 7, 6}, {0, 2, 3, 1}};
  for (int f = 0; f < 6; ++f) {
    const int32_t h = c3_new_face(C, f);
    if (h < 0) return ORC_ERR_OOM;
    for (int k = 0; k < 4; ++k)
      if (c3_face_push(&C->fc[h], loops[f][k])) return ORC_ERR_OOM;
  }
  return ORC_OK;
}

/* the vertex where the plane of site e crosses the edge a->b of face f
 * (one end strictly inside, the other strictly beyond); shared with the
 * edge's other face, which runs it as b->a */
static int32_t c3_cross(c3cell* C, int32_t f, int32_t a, int32_t b, int32_t e) {
  for (int32_t t = 0; t < C->nmemo; ++t) {
    const int32_t* m = C->memo + 3 * t;
    if ((m[0] == a && m[1] == b) || (m[0] == b && m[1] == a)) return m[2];
  }
  int32_t g = -1;
  for (int32_t h = 0; h < C->nfc && g < 0; ++h) {
    if (h == f || !C->fc[h].alive) continue;
    const c3face* F = &C->fc[h];
    for (int32_t k = 0; k < F->n; ++k)
      if (F->v[k] == b && F->v[(k + 1) % F->n] == a) {
        g = h;
        break;
      }
  }
  if (g < 0) return -2;
  const int32_t x = c3_new_vertex(C, C->fc[f].plane, C->fc[g].plane, e);
  if (x < 0) return -1;
  if (c3_grow((void**)&C->memo, &C->capmemo, 3 * ((int64_t)C->nmemo + 1), sizeof(int32_t))) return -1;
  C->memo[3 * C->nmemo] = a;
  C->memo[3 * C->nmemo + 1] = b;
  C->memo[3 * C->nmemo + 2] = x;
  ++C->nmemo;
  return x;
}

static int c3_edge(c3cell* C, int32_t tail, int32_t head) {
  if (c3_grow((void**)&C->eg, &C->capeg, 2 * ((int64_t)C->neg + 1), sizeof(int32_t))) return 1;
  C->eg[2 * C->neg] = tail;
  C->eg[2 * C->neg + 1] = head;
  ++C->neg;
  return 0;
}

/* Clip the cell by the half-space of plane e.  *cut = 1 when some vertex lay
 * strictly beyond it (the plane then carries a new face of positive area). */
static int c3_clip(c3cell* C, int32_t e, int* cut) {
  *cut = 0;
  const int32_t nv0 = C->nvt;
  if (c3_grow((void**)&C->sg, &C->capsg, nv0, sizeof(int8_t))) return ORC_ERR_OOM;
  int any_out = 0;
  for (int32_t v = 0; v < nv0; ++v) {
    C->sg[v] = C->vt[v].alive ? (int8_t)c3_side(C, v, e) : 0;
    any_out |= C->vt[v].alive && C->sg[v] > 0;
  }
  if (!any_out) return ORC_OK;
  *cut = 1;
  C->nmemo = 0;
  C->neg = 0;
  const int32_t nf0 = C->nfc;
  for (int32_t f = 0; f < nf0; ++f) {
    c3face* F = &C->fc[f];
    if (!F->alive) continue;
    int nin = 0, nout = 0;
    for (int32_t k = 0; k < F->n; ++k) {
      nin += C->sg[F->v[k]] < 0;
      nout += C->sg[F->v[k]] > 0;
    }
    if (!nout) {
      /* untouched; an edge lying in the plane bounds the new face */
      for (int32_t k = 0; k < F->n; ++k) {
        const int32_t u = F->v[k], v = F->v[(k + 1) % F->n];
        if (C->sg[u] == 0 && C->sg[v] == 0 && c3_edge(C, v, u)) return ORC_ERR_OOM;
      }
      continue;
    }
    if (!nin) {
      F->alive = 0; /* nothing of it is strictly inside: gone (or reduced to an edge or a vertex) */
      continue;
    }
    int32_t k0 = 0;
    while (C->sg[F->v[k0]] >= 0) ++k0;
    if (c3_grow((void**)&C->tmp, &C->captmp, (int64_t)F->n + 2, sizeof(int32_t))) return ORC_ERR_OOM;
    int32_t m = 0, A = -1, B = -1;
    for (int32_t t = 0; t < F->n; ++t) {
      const int32_t u = F->v[(k0 + t) % F->n], v = F->v[(k0 + t + 1) % F->n];
      const int su = C->sg[u], sv = C->sg[v];
      if (su <= 0) C->tmp[m++] = u;
      if (su < 0 && sv > 0) {
        const int32_t x = c3_cross(C, f, u, v, e);
        if (x < 0) return x == -1 ? ORC_ERR_OOM : ORC_ERR_INTERNAL;
        C->tmp[m++] = x;
        A = x;
      } else if (su == 0 && sv > 0) {
        A = u;
      } else if (su > 0 && sv < 0) {
        const int32_t x = c3_cross(C, f, u, v, e);
        if (x < 0) return x == -1 ? ORC_ERR_OOM : ORC_ERR_INTERNAL;
        C->tmp[m++] = x;
        B = x;
      } else if (su > 0 && sv == 0) {
        B = v;
      }
      if (c3_grow((void**)&C->tmp, &C->captmp, (int64_t)m + 2, sizeof(int32_t))) return ORC_ERR_OOM;
    }
    if (A < 0 || B < 0) return ORC_ERR_INTERNAL;
    F = &C->fc[f]; /* (no reallocation of fc happens above; kept for clarity) */
    F->n = 0;
    for (int32_t t = 0; t < m; ++t)
      if (c3_face_push(F, C->tmp[t])) return ORC_ERR_OOM;
    if (c3_edge(C, B, A)) return ORC_ERR_OOM;
  }
  for (int32_t v = 0; v < nv0; ++v)
    if (C->sg[v] > 0) C->vt[v].alive = 0;
  /* chain the boundary edges into the loop of the new face */
  const int32_t h = c3_new_face(C, e);
  if (h < 0) return ORC_ERR_OOM;
  if (C->neg < 3) return ORC_ERR_INTERNAL;
  const int32_t start = C->eg[0];
  int32_t cur = start, steps = 0;
  do {
    if (c3_face_push(&C->fc[h], cur)) return ORC_ERR_OOM;
    int32_t nxt = -1;
    for (int32_t t = 0; t < C->neg; ++t)
      if (C->eg[2 * t] == cur) {
        if (nxt >= 0) return ORC_ERR_INTERNAL; /* two edges leave one vertex */
        nxt = C->eg[2 * t + 1];
      }
    if (nxt < 0) return ORC_ERR_INTERNAL;
    cur = nxt;
    ++steps;
  } while (cur != start && steps <= C->neg);
  if (cur != start || steps != C->neg) return ORC_ERR_INTERNAL;
  return ORC_OK;
}

/* squared distance of the farthest vertex, rounded up generously */
static double c3_radius2(const c3cell* C) {
  double r2 = 0.0;
  for (int32_t v = 0; v < C->nvt; ++v) {
    if (!C->vt[v].alive) continue;
    const double* x = C->vt[v].x;
    const double q = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
    if (q > r2) r2 = q;
  }
  return r2 * (1.0 + 1e-9) + 1.0;
}

/* Euler's relation V - E + F = 2 of the finished cell: a self-check */
static int c3_check(const c3cell* C) {
  int64_t V = 0, E2 = 0, F = 0;
  for (int32_t v = 0; v < C->nvt; ++v) V += C->vt[v].alive;
  for (int32_t f = 0; f < C->nfc; ++f)
    if (C->fc[f].alive) {
      if (C->fc[f].n < 3) return ORC_ERR_INTERNAL;
      ++F;
      E2 += C->fc[f].n;
    }
  return (E2 % 2 == 0 && V - E2 / 2 + F == 2) ? ORC_OK : ORC_ERR_INTERNAL;
}

static double c3_volume(const c3cell* C) {
  double vol = 0.0;
  for (int32_t f = 0; f < C->nfc; ++f) {
    const c3face* F = &C->fc[f];
    if (!F->alive) continue;
    const double* a = C->vt[F->v[0]].x;
    for (int32_t k = 1; k + 1 < F->n; ++k) {
      const double* b = C->vt[F->v[k]].x;
      const double* c = C->vt[F->v[k + 1]].x;
      vol += a[0] * (b[1] * c[2] - b[2] * c[1]) - a[1] * (b[0] * c[2] - b[2] * c[0]) +
             a[2] * (b[0] * c[1] - b[1] * c[0]);
    }
  }
  return vol / 6.0;
}

typedef struct {
  uint64_t w;
  int32_t id;
  int64_t d[3];
} c3cand;

static int cmp_c3cand(const void* x, const void* y) {
  const c3cand* a = (const c3cand*)x;
  const c3cand* b = (const c3cand*)y;
  if (a->w != b->w) return a->w < b->w ? -1 : 1;
  if (a->id != b->id) return a->id < b->id ? -1 : 1;
  for (int t = 0; t < 3; ++t)
    if (a->d[t] != b->d[t]) return a->d[t] < b->d[t] ? -1 : 1;
  return 0;
}

/* clip the cube by every candidate in (w, id) order, skipping those that
 * lie too far to reach the cell */
static int c3_build(c3cell* C, const int64_t* box, const c3cand* cand, int64_t nc) {
  int rc = c3_init(C, box);
  if (rc) return rc;
  double r2 = c3_radius2(C);
  for (int64_t t = 0; t < nc; ++t) {
    if ((double)cand[t].w >= 4.0 * r2) break; /* |d|/2 >= every vertex's distance */
    const int32_t e = c3_add_plane(C, cand[t].d, cand[t].id);
    if (e < 0) return ORC_ERR_OOM;
    int cut = 0;
    if ((rc = c3_clip(C, e, &cut))) return rc;
    if (cut) r2 = c3_radius2(C);
    else --C->npl; /* the plane carries no face and no vertex: drop it */
  }
  return c3_check(C);
}

/* Cell of particle i.  Candidates are the minimum images of the other
 * particles within a growing radius T, until the cell is certified to lie
 * within sqrt(T)/2 of the particle; when the cell reaches a quarter of the
 * box, every periodic image within twice its radius is used instead. */
static int c3_particle(c3cell* C, int64_t n, const int32_t* pos, const int64_t* box, int64_t i, double T,
                       c3cand** buf, int64_t* cap) {
  int rc;
  const int64_t Lmin = box[0] < box[1] ? (box[0] < box[2] ? box[0] : box[2]) : (box[1] < box[2] ? box[1] : box[2]);
  for (;;) {
    int64_t nc = 0;
    for (int64_t j = 0; j < n; ++j) {
      if (j == i) continue;
      int64_t d[3];
      uint64_t w = 0;
      for (int a = 0; a < 3; ++a) {
        d[a] = min_image((int64_t)pos[3 * j + a] - (int64_t)pos[3 * i + a], box[a]);
        w += (uint64_t)(d[a] * d[a]);
      }
      if (w == 0) return ORC_ERR_DEGENERATE;
      if ((double)w > T) continue;
      if (nc == *cap) {
        const int64_t nc2 = *cap ? 2 * *cap : 1024;
        c3cand* q = (c3cand*)realloc(*buf, (size_t)nc2 * sizeof(c3cand));
        if (!q) return ORC_ERR_OOM;
        *buf = q;
        *cap = nc2;
      }
      c3cand* c = &(*buf)[nc++];
      c->w = w;
      c->id = (int32_t)j;
      for (int a = 0; a < 3; ++a) c->d[a] = d[a];
    }
    qsort(*buf, (size_t)nc, sizeof(c3cand), cmp_c3cand);
    if ((rc = c3_build(C, box, *buf, nc))) return rc;
    const double r2 = c3_radius2(C);
    const int all = (nc == n - 1);
    if (4.0 * r2 > T && !all) {
      T *= 4.0;
      continue;
    }
    /* a non-minimum image is at least Lmin/2 away: it cannot reach the cell
     * when 4 r2 <= (Lmin/2)^2 */
    if (16.0 * r2 <= (double)Lmin * (double)Lmin) return ORC_OK;
    /* small box: every image of every particle within 2 sqrt(r2) */
    const double R = sqrt(r2);
    int64_t K[3];
    for (int a = 0; a < 3; ++a) K[a] = (int64_t)floor((2.0 * R + 0.5 * (double)box[a]) / (double)box[a]) + 1;
    nc = 0;
    for (int64_t j = 0; j < n; ++j) {
      int64_t d0[3];
      for (int a = 0; a < 3; ++a) d0[a] = min_image((int64_t)pos[3 * j + a] - (int64_t)pos[3 * i + a], box[a]);
      for (int64_t kx = -K[0]; kx <= K[0]; ++kx)
        for (int64_t ky = -K[1]; ky <= K[1]; ++ky)
          for (int64_t kz = -K[2]; kz <= K[2]; ++kz) {
            if (j == i && kx == 0 && ky == 0 && kz == 0) continue;
            const int64_t d[3] = {d0[0] + kx * box[0], d0[1] + ky * box[1], d0[2] + kz * box[2]};
            const double wd = (double)d[0] * d[0] + (double)d[1] * d[1] + (double)d[2] * d[2];
            if (wd >= 4.0 * r2) continue;
            if (nc == *cap) {
              const int64_t nc2 = *cap ? 2 * *cap : 1024;
              c3cand* q = (c3cand*)realloc(*buf, (size_t)nc2 * sizeof(c3cand));
              if (!q) return ORC_ERR_OOM;
              *buf = q;
              *cap = nc2;
            }
            c3cand* c = &(*buf)[nc++];
            c->w = (uint64_t)(d[0] * d[0]) + (uint64_t)(d[1] * d[1]) + (uint64_t)(d[2] * d[2]);
            c->id = j == i ? -1 : (int32_t)j;
            for (int a = 0; a < 3; ++a) c->d[a] = d[a];
          }
    }
    qsort(*buf, (size_t)nc, sizeof(c3cand), cmp_c3cand);
    return c3_build(C, box, *buf, nc);
  }
}

static int cmp_i32(const void* x, const void* y) {
  const int32_t a = *(const int32_t*)x, b = *(const int32_t*)y;
  return (a > b) - (a < b);
}

/* Voronoi neighbors (sorted by id) and cell volumes (grid units^3) of the
 * query particles (all when query is NULL).  Rows hold up to maxdeg ids;
 * deg[q] is the true count, and a larger one returns ORC_ERR_ARG.  Box edges
 * up to 2^28. */
int orc_voronoi3(int64_t n, const int32_t* pos, const int64_t* box, const int64_t* query, int64_t nq,
                 int32_t maxdeg, int32_t* deg, int32_t* ids, double* volume) {
  if (n < 1 || nq < 0 || maxdeg < 0) return ORC_ERR_ARG;
  for (int a = 0; a < 3; ++a)
    if (box[a] < 1 || box[a] > (1ll << 28)) return ORC_ERR_ARG;
  for (int64_t j = 0; j < 3 * n; ++j)
    if (pos[j] < 0 || (int64_t)pos[j] >= box[j % 3]) return ORC_ERR_ARG;
  /* first radius: about 4.5 mean spacings */
  const double spacing = cbrt((double)box[0] * (double)box[1] * (double)box[2] / (double)n);
  const double T0 = 20.0 * spacing * spacing;
  int rc_all = ORC_OK;
#pragma omp parallel
  {
    c3cell C;
    memset(&C, 0, sizeof(C));
    c3cand* buf = NULL;
    int64_t cap = 0;
    int32_t* row = NULL;
    int32_t rowcap = 0;
#pragma omp for schedule(dynamic, 4)
    for (int64_t q = 0; q < nq; ++q) {
      const int64_t i = query ? query[q] : q;
      int rc = (i < 0 || i >= n) ? ORC_ERR_ARG : c3_particle(&C, n, pos, box, i, T0, &buf, &cap);
      int32_t cnt = 0;
      if (!rc) {
        for (int32_t f = 0; f < C.nfc && !rc; ++f) {
          if (!C.fc[f].alive || C.pl[C.fc[f].plane].id < 0) continue;
          if (c3_grow((void**)&row, &rowcap, (int64_t)cnt + 1, sizeof(int32_t))) rc = ORC_ERR_OOM;
          else row[cnt++] = C.pl[C.fc[f].plane].id;
        }
      }
      if (!rc) {
        qsort(row, (size_t)cnt, sizeof(int32_t), cmp_i32);
        int32_t u = 0;
        for (int32_t t = 0; t < cnt; ++t)
          if (u == 0 || row[t] != row[u - 1]) row[u++] = row[t];
        cnt = u;
        deg[q] = cnt;
        if (cnt > maxdeg) rc = ORC_ERR_ARG;
        else
          for (int32_t t = 0; t < cnt; ++t) ids[q * (int64_t)maxdeg + t] = row[t];
        if (volume) volume[q] = c3_volume(&C);
      }
      if (rc) {
#pragma omp critical
        if (rc_all == ORC_OK || rc == ORC_ERR_DEGENERATE) rc_all = rc;
      }
    }
    c3_free(&C);
    free(buf);
    free(row);
  }
  return rc_all;
}

/* The exact side test on explicit site offsets (for the tests): the sign of
 * d_e.y - |d_e|^2 at the point y where d_a.y = |d_a|^2, d_b.y = |d_b|^2 and
 * d_c.y = |d_c|^2 (0 when a, b, c do not meet in one point). */
int orc_voronoi3_side(const int64_t* da, const int64_t* db, const int64_t* dc, const int64_t* de) {
  c3cell C;
  memset(&C, 0, sizeof(C));
  int s = 0;
  if (c3_add_plane(&C, da, 0) >= 0 && c3_add_plane(&C, db, 1) >= 0 && c3_add_plane(&C, dc, 2) >= 0 &&
      c3_add_plane(&C, de, 3) >= 0 && det3_i(da, db, dc) != 0) {
    c3vert V;
    V.p[0] = 0; V.p[1] = 1; V.p[2] = 2; V.alive = 1;
    if (c3_grow((void**)&C.vt, &C.capvt, 1, sizeof(c3vert)) == 0) {
      C.vt[0] = V;
      C.nvt = 1;
      s = c3_side(&C, 0, 3);
    }
  }
  c3_free(&C);
  return s;
}

/* ======================================================================== */
/* One Vicsek update: Eq. (2) alignment + noise, Eq. (1) advection           */
/* ======================================================================== */

typedef struct {
  int32_t dim;
  int32_t frac_bits;
  int32_t noise;        /* 0 angular (2D), 1 vectorial (Eq. 2) */
  int32_t include_self; /* 0: sum over the neighbors only */
  int32_t advect_new;   /* 0: Eq. (1) with n_i(t); 1: with n_i(t+dt) */
  float v0, dt, eta;
  uint64_t seed;
} orc_params;

/* pos (n*dim int32) and dir (n*dim float32) hold the state at step `step`;
 * nb_off/nb_ids is the neighbor CSR in canonical order.  Writes the state at
 * step+1: positions (exact), headings in FP64, and (2D) angles in [0, 2pi). */
int orc_vicsek_step(const orc_params* prm, int64_t n, const int32_t* pos, const float* dir,
                    const int64_t* box, const int64_t* nb_off, const int32_t* nb_ids,
                    int64_t step, uint32_t replica, int32_t* pos_out, double* dir_out,
                    double* theta_out) {
  const int dim = prm->dim;
  if (dim < 2 || dim > 3 || n < 1) return ORC_ERR_ARG;
  if (dim == 3 && prm->noise == 0) return ORC_ERR_ARG;
  /* grid step per unit heading: fl32(v0*dt) scaled by 2^F (exact) */
  float vdt = prm->v0 * prm->dt;
  double s = ldexp((double)vdt, prm->frac_bits);
  const uint32_t key[2] = {(uint32_t)prm->seed, (uint32_t)(prm->seed >> 32)};
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    double S[3] = {0.0, 0.0, 0.0};
    int64_t m = 0;
    if (prm->include_self) {
      for (int a = 0; a < dim; ++a) S[a] += (double)dir[i * dim + a];
      ++m;
    }
    for (int64_t q = nb_off[i]; q < nb_off[i + 1]; ++q) {
      int64_t j = nb_ids[q];
      for (int a = 0; a < dim; ++a) S[a] += (double)dir[j * dim + a];
      ++m;
    }
    uint32_t ctr[4] = {(uint32_t)i, (uint32_t)step, replica, 0u}, w[4];
    orc_philox4x32_10(ctr, key, w);
    double u = unit24(w[0]), u1 = unit24(w[1]);
    double nn[3] = {0.0, 0.0, 0.0};
    if (prm->noise == 0) {
      double th;
      if (S[0] == 0.0 && S[1] == 0.0)
        th = atan2((double)dir[i * dim + 1], (double)dir[i * dim]);
      else
        th = atan2(S[1], S[0]);
      th += (double)prm->eta * (u - 0.5);
      nn[0] = cos(th);
      nn[1] = sin(th);
    } else {
      const double twopi = 6.283185307179586476925286766559;
      double xi[3];
      if (dim == 2) {
        xi[0] = cos(twopi * u);
        xi[1] = sin(twopi * u);
        xi[2] = 0.0;
      } else {
        double z = 2.0 * u1 - 1.0, r = sqrt(fmax(0.0, 1.0 - z * z));
        xi[0] = r * cos(twopi * u);
        xi[1] = r * sin(twopi * u);
        xi[2] = z;
      }
      double v[3], norm2 = 0.0;
      for (int a = 0; a < dim; ++a) {
        v[a] = (double)prm->eta * xi[a] + (m > 0 ? S[a] / (double)m : 0.0);
        norm2 += v[a] * v[a];
      }
      if (norm2 == 0.0) {
        for (int a = 0; a < dim; ++a) nn[a] = (double)dir[i * dim + a];
      } else {
        double inv = 1.0 / sqrt(norm2);
        for (int a = 0; a < dim; ++a) nn[a] = v[a] * inv;
      }
    }
    for (int a = 0; a < dim; ++a) {
      dir_out[i * dim + a] = nn[a];
      double h = prm->advect_new ? nn[a] : (double)dir[i * dim + a];
      /* s*h is exact in FP64 (two 24-bit significands); round half to even */
      double delta = nearbyint(s * h);
      int64_t L = box[a];
      int64_t p = ((int64_t)pos[i * dim + a] + (int64_t)delta) % L;
      if (p < 0) p += L;
      pos_out[i * dim + a] = (int32_t)p;
    }
    if (dim == 2 && theta_out) {
      const double twopi = 6.283185307179586476925286766559;
      double th = atan2(nn[1], nn[0]);
      if (th < 0.0) th += twopi;
      if (th >= twopi) th -= twopi;
      theta_out[i] = th;
    }
  }
  return ORC_OK;
}

/* Polar order parameter |sum_i n_i| / N in FP64. */
double orc_order_parameter_f32(int dim, int64_t n, const float* dir) {
  double S[3] = {0.0, 0.0, 0.0};
  for (int64_t i = 0; i < n; ++i)
    for (int a = 0; a < dim; ++a) S[a] += (double)dir[i * dim + a];
  double r = 0.0;
  for (int a = 0; a < dim; ++a) r += S[a] * S[a];
  return sqrt(r) / (double)n;
}

double orc_order_parameter_f64(int dim, int64_t n, const double* dir) {
  double S[3] = {0.0, 0.0, 0.0};
  for (int64_t i = 0; i < n; ++i)
    for (int a = 0; a < dim; ++a) S[a] += dir[i * dim + a];
  double r = 0.0;
  for (int a = 0; a < dim; ++a) r += S[a] * S[a];
  return sqrt(r) / (double)n;
}

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
