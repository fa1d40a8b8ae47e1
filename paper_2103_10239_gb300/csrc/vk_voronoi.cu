// vk_voronoi.cu -- Voronoi-neighbor rule (Sec. "Computational tools: Voronoi
// neighbor lists": the Voronoi cell is the region closer to a particle than to
// any other; Voronoi and Delaunay neighbors are dual, and the relation is
// reciprocal) fused with the Vicsek update of Eq. (1) and Eq. (2).
//
// Instead of a global (serial) triangulation, every particle builds its own
// Voronoi cell by half-plane clipping, which is embarrassingly parallel:
//   * the cell starts as the square bounded by the particle's own periodic
//     images (+-L_x, 0), (0, +-L_y);
//   * candidates arrive ring by ring from the cell grid; each one clips the
//     convex polygon by its bisector.  The polygon is a cyclic list of the
//     sites that define its edges; a vertex is the circumcenter of the particle
//     (at the origin) and two consecutive sites.  "Vertex beyond the bisector
//     of m" is exactly incircle(0, a, b, m) > 0, evaluated with an FP32 filter
//     and an exact int128 fallback on integer relative coordinates;
//   * the walk stops once every unscanned site is farther than twice the
//     largest vertex distance (the security radius), using a rigorous FP32
//     upper bound of the vertex distances;
//   * neighbors are the sites of edges with positive length (an edge between
//     two coincident vertices, i.e. four cocircular points, is dropped);
//   * coincident particles form one site (see Poly).
// Exact predicates need |relative coordinates| < 1.5 * 2^30, hence L_q <= 2^30.
#include <algorithm>
#include <climits>

#include "vk_internal.cuh"

namespace vk {

namespace {

constexpr int kFastCap = 32;    // polygon capacity of the main kernel
constexpr int kSlowCap = kVoronoiMaxDeg;  // capacity of the overflow kernel and the export

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
  // exact
  const int64_t al = (int64_t)ax * ax + (int64_t)ay * ay;
  const int64_t bl = (int64_t)bx * bx + (int64_t)by * by;
  const int64_t ml = (int64_t)mx * mx + (int64_t)my * my;
  const __int128 A = (__int128)by * ml - (__int128)bl * my;
  const __int128 Bt = (__int128)bx * ml - (__int128)bl * mx;
  const __int128 C = (__int128)bx * my - (__int128)by * mx;
  const __int128 d = (__int128)ax * A - (__int128)ay * Bt + (__int128)al * C;
  return d > 0 ? -1 : (d < 0 ? 1 : 0);
}

// rigorous FP32 upper bound of |V|^2, V = circumcenter of (0, a, b)
__device__ __forceinline__ float vertex_r2_upper(int32_t ax, int32_t ay, int32_t bx, int32_t by, bool* bad) {
  const int64_t dh = (int64_t)ax * by - (int64_t)ay * bx;  // exact; > 0 for consecutive edges
  if (dh <= 0) {
    *bad = true;
    return 3.0e38f;
  }
  const float fax = (float)ax, fay = (float)ay, fbx = (float)bx, fby = (float)by;
  const float al = fax * fax + fay * fay, bl = fbx * fbx + fby * fby;
  const float p1 = fby * al, p2 = fay * bl, p3 = fax * bl, p4 = fbx * al;
  const float ex = (fabsf(p1) + fabsf(p2)) * 9.5367431640625e-07f;  // 16 ulps
  const float ey = (fabsf(p3) + fabsf(p4)) * 9.5367431640625e-07f;
  const float d2 = 2.0f * (float)dh * (1.0f - 2.384185791015625e-07f);  // rounded down
  const float vx = (fabsf(p1 - p2) + ex) / d2;
  const float vy = (fabsf(p3 - p4) + ey) / d2;
  const float r2 = (vx * vx + vy * vy) * (1.0f + 9.5367431640625e-07f);
  return isfinite(r2) ? r2 : 3.0e38f;
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
  int32_t tw_slot[TW];       // coincident twins: their sorted slot ...
  int32_t tw_id[TW];         // ... their id ...
  int32_t tw_of[TW];         // ... and the slot of the site they sit on (-2: the particle itself)
  int m;
  int nt;
  float max_r2;
};

template <int CAP>
__device__ __forceinline__ void poly_refresh_max(Poly<CAP>& P) {
  float mx = 0.f;
  for (int a = 0; a < P.m; ++a) mx = fmaxf(mx, P.vr2[a]);
  P.max_r2 = mx;
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
    P.vr2[a] = vertex_r2_upper(P.qx[a], P.qy[a], P.qx[(a + 1) & 3], P.qy[(a + 1) & 3], bad);
  poly_refresh_max(P);
}

// clip the cell by the bisector of site (mx, my); returns false on overflow
template <int CAP>
__device__ __forceinline__ bool poly_clip(Poly<CAP>& P, int32_t mx, int32_t my, int32_t mid, int32_t mslot,
                                          float Dm, bool* bad, bool* touch) {
  const int m = P.m;
  // the vertices strictly beyond the bisector form one cyclic run [s, s+c)
  int c = 0, s = -1;
  bool first_cut = false, prev_cut = false;
  *touch = false;
  for (int a = 0; a < m; ++a) {
    bool cut = false;
    if (!(Dm > 4.0f * P.vr2[a])) {  // a vertex closer than |m|/2 cannot be cut
      const int b = (a + 1 == m) ? 0 : a + 1;
      const int sg = vertex_cut_sign(P.qx[a], P.qy[a], P.qx[b], P.qy[b], mx, my);
      cut = sg > 0;
      *touch = *touch || sg == 0;
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
      }
    } else if (delta > 0) {
      for (int a = m - 1; a >= t + 1; --a) {
        P.qx[a + delta] = P.qx[a]; P.qy[a + delta] = P.qy[a]; P.id[a + delta] = P.id[a];
        P.slot[a + delta] = P.slot[a]; P.vr2[a + delta] = P.vr2[a];
      }
    }
    mpos = s + 1;
  } else {
    // the run wraps: keep e_{t+1}..e_s (contiguous), then m
    const int sh = t + 1;
    for (int a = sh; a <= s; ++a) {
      P.qx[a - sh] = P.qx[a]; P.qy[a - sh] = P.qy[a]; P.id[a - sh] = P.id[a];
      P.slot[a - sh] = P.slot[a]; P.vr2[a - sh] = P.vr2[a];
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
  P.vr2[before] = vertex_r2_upper(P.qx[before], P.qy[before], mx, my, bad);
  P.vr2[mpos] = vertex_r2_upper(mx, my, P.qx[after], P.qy[after], bad);
  poly_refresh_max(P);
  return true;
}

// Voronoi cell of the particle at slot `self`.  Status codes are latched on
// internal inconsistencies (kStRange); capacity overflow is returned.
// Returns false (and leaves the cell unusable) if the polygon or the twin list
// outgrew its capacity.
template <int CAP>
__device__ bool voronoi_cell(const Rep& R, int64_t self, const int32_t* pi, int32_t self_id,
                             const int2* __restrict__ pos, const int32_t* __restrict__ ids,
                             const GridView& G, Poly<CAP>& P, int32_t* status, uint32_t* n_cand = nullptr,
                             uint32_t* n_runs = nullptr) {
  bool bad = false, overflow = false;
  poly_init(P, self_id, R.L[0], R.L[1], &bad);
  const int64_t Lx = R.L[0], Ly = R.L[1];
  auto add_twin = [&](int32_t slot, int32_t jid, int32_t of) {
    if (P.nt == Poly<CAP>::TW) {
      overflow = true;
      return;
    }
    P.tw_slot[P.nt] = slot;
    P.tw_id[P.nt] = jid;
    P.tw_of[P.nt] = of;
    ++P.nt;
  };
  auto visit = [&](int32_t qx, int32_t qy, int32_t jid, int32_t slot) {
    if (overflow) return;
    const uint64_t D = (uint64_t)((int64_t)qx * qx) + (uint64_t)((int64_t)qy * qy);
    if (D == 0) {
      add_twin(slot, jid, -2);  // coincident with the particle itself
      return;
    }
    const float Df = (float)D * (1.0f - 2.384185791015625e-07f);  // rounded down
    if (Df > 4.0f * P.max_r2) return;
    bool touch = false;
    if (!poly_clip(P, qx, qy, jid, slot, Df, &bad, &touch)) {
      overflow = true;
      return;
    }
    if (touch) {
      // no vertex cut but some vertex on the bisector: a twin of an edge site?
      for (int a = 0; a < P.m; ++a)
        if (P.qx[a] == qx && P.qy[a] == qy && P.slot[a] >= 0) {
          add_twin(slot, jid, P.slot[a]);
          break;
        }
    }
  };
  auto run = [&](uint32_t qb, uint32_t qe) {
    if (n_cand) {
      *n_cand += qe - qb;
      *n_runs += 1;
    }
    for (uint32_t q = qb; q < qe; ++q) {
      if ((int64_t)q == self) continue;
      const int2 pj = pos[q];
      const int32_t qx = (int32_t)min_image((int64_t)pj.x - pi[0], Lx);
      const int32_t qy = (int32_t)min_image((int64_t)pj.y - pi[1], Ly);
      visit(qx, qy, ids[q], (int32_t)q);
    }
  };
  auto stop = [&](uint64_t B2) {
    const float b2 = (float)B2 * (1.0f - 2.384185791015625e-07f);
    return b2 > 4.0f * P.max_r2;
  };
  // sites farther than twice the largest vertex distance cannot clip
  auto radius2 = [&]() -> uint64_t {
    const float r = 4.0f * P.max_r2 * 1.0000005f;
    return r >= 1.8e19f ? ~0ull : (uint64_t)r + 1ull;
  };
  const bool all = grid_walk<2>(R, pi, G, run, radius2, stop);
  if (all) {
    // tiny boxes: other periodic images than the minimum one can still shape
    // the cell when the security radius exceeds half the box
    const float half = 0.5f * (float)min(Lx, Ly);
    if (4.0f * P.max_r2 > half * half) {
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
  }
  if (bad) set_status(status, kStRange);
  return !overflow;
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

// the Vicsek update of one particle from its finished cell
template <int CAP>
__device__ __forceinline__ void voronoi_update(const Rep& R, const StepParams& Pm, int64_t step, int64_t s,
                                               const Poly<CAP>& P, const int32_t* pi, const float* ni,
                                               int32_t id, const float2* __restrict__ S_dir,
                                               int2* __restrict__ U_pos, float2* __restrict__ U_dir,
                                               int32_t* __restrict__ U_id, uint32_t* __restrict__ counts,
                                               float* nnew) {
  int32_t nid[CAP + Poly<CAP>::TW], nslot[CAP + Poly<CAP>::TW];
  const int cnt = voronoi_neighbors(P, id, nid, nslot);
  HeadSum<2> H;
  H.init();
  if (Pm.include_self) H.add(ni, Pm.sum_mode);
  for (int j = 0; j < cnt; ++j) {
    const float2 d = S_dir[nslot[j]];
    const float v[2] = {d.x, d.y};
    H.add(v, Pm.sum_mode);
  }
  int32_t pout[3] = {0, 0, 0};
  align_advect<2>(R, Pm, (uint32_t)step, id, ni, H, cnt + (Pm.include_self ? 1 : 0), pi, pout, nnew);
  U_pos[s] = make_int2(pout[0], pout[1]);
  U_dir[s] = make_float2(nnew[0], nnew[1]);
  U_id[s] = id;
  atomicAdd(counts + linear_cell<2>(R, pout), 1u);
}

// Main kernel: cells of up to kFastCap edges.  Particles whose cell outgrows
// it are appended to the overflow list and finished by the overflow kernel.
__global__ void __launch_bounds__(kBlock) voronoi_step_kernel(
    const Rep* __restrict__ reps, const BlockTask* __restrict__ tasks, const int2* __restrict__ S_pos,
    const float2* __restrict__ S_dir, const int32_t* __restrict__ S_id, GridView G,
    int2* __restrict__ U_pos, float2* __restrict__ U_dir, int32_t* __restrict__ U_id,
    uint32_t* __restrict__ counts, double* __restrict__ phi_acc, const int64_t* __restrict__ d_step, StepParams Pm,
    int2* __restrict__ ovf_list, int32_t* __restrict__ ovf_count, int32_t* status) {
  const BlockTask t = tasks[blockIdx.x];
  const Rep R = reps[t.rep];
  const int li = t.first + (int)threadIdx.x;
  const int64_t step = *d_step;
  float nnew[3] = {0.f, 0.f, 0.f};
  uint32_t n_cand = 0, n_runs = 0;
  if (li < R.n) {
    const int64_t s = R.p0 + li;
    const int2 p = S_pos[s];
    const float2 nv = S_dir[s];
    const int32_t pi[3] = {p.x, p.y, 0};
    const float ni[3] = {nv.x, nv.y, 0.f};
    const int32_t id = S_id[s];
    Poly<kFastCap> P;
    const bool ok = Pm.stats ? voronoi_cell(R, s, pi, id, S_pos, S_id, G, P, status, &n_cand, &n_runs)
                             : voronoi_cell(R, s, pi, id, S_pos, S_id, G, P, status);
    if (ok) {
      voronoi_update(R, Pm, step, s, P, pi, ni, id, S_dir, U_pos, U_dir, U_id, counts, nnew);
    } else {
      const int q = atomicAdd(ovf_count, 1);
      ovf_list[q] = make_int2((int)s, t.rep);
    }
  }
  record_search_stats(Pm.stats, li < R.n, n_cand, n_runs);
  block_phi_accumulate<2>(nnew, phi_acc + ((size_t)(step % Pm.phi_cap) * (size_t)Pm.n_rep + (size_t)t.rep) * 3);
}

// Overflow kernel: the few particles with very large cells (a particle
// bordering a void can have dozens of Voronoi neighbors).
__global__ void __launch_bounds__(64) voronoi_overflow_kernel(
    const Rep* __restrict__ reps, const int2* __restrict__ S_pos, const float2* __restrict__ S_dir,
    const int32_t* __restrict__ S_id, GridView G, int2* __restrict__ U_pos,
    float2* __restrict__ U_dir, int32_t* __restrict__ U_id,
    uint32_t* __restrict__ counts, double* __restrict__ phi_acc, const int64_t* __restrict__ d_step, StepParams Pm,
    const int2* __restrict__ ovf_list, const int32_t* __restrict__ ovf_count, int32_t* status) {
  const int total = *ovf_count;
  const int64_t step = *d_step;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < total; q += gridDim.x * blockDim.x) {
    const int2 e = ovf_list[q];
    const Rep R = reps[e.y];
    const int64_t s = e.x;
    const int2 p = S_pos[s];
    const float2 nv = S_dir[s];
    const int32_t pi[3] = {p.x, p.y, 0};
    const float ni[3] = {nv.x, nv.y, 0.f};
    const int32_t id = S_id[s];
    Poly<kSlowCap> P;
    if (!voronoi_cell(R, s, pi, id, S_pos, S_id, G, P, status)) {
      set_status(status, kStCapacity);
      continue;
    }
    float nnew[3] = {0.f, 0.f, 0.f};
    voronoi_update(R, Pm, step, s, P, pi, ni, id, S_dir, U_pos, U_dir, U_id, counts, nnew);
    double* acc = phi_acc + ((size_t)(step % Pm.phi_cap) * (size_t)Pm.n_rep + (size_t)e.y) * 3;
    atomicAdd(acc + 0, (double)nnew[0]);
    atomicAdd(acc + 1, (double)nnew[1]);
  }
}

// Export (not on the hot path): pass 0 writes the degree of every particle
// (by id), pass 1 writes the sorted ids at out_off[id].
__global__ void __launch_bounds__(64) voronoi_export_kernel(const Rep* __restrict__ reps, int rep,
                                                            const int2* __restrict__ S_pos,
                                                            const int32_t* __restrict__ S_id,
                                                            GridView G, int pass,
                                                            int32_t* __restrict__ deg,
                                                            const int64_t* __restrict__ out_off,
                                                            int32_t* __restrict__ out_ids, int32_t* status) {
  const Rep R = reps[rep];
  for (int li = blockIdx.x * blockDim.x + threadIdx.x; li < R.n; li += gridDim.x * blockDim.x) {
    const int64_t s = R.p0 + li;
    const int2 p = S_pos[s];
    const int32_t pi[3] = {p.x, p.y, 0};
    const int32_t id = S_id[s];
    Poly<kSlowCap> P;
    if (!voronoi_cell(R, s, pi, id, S_pos, S_id, G, P, status)) {
      set_status(status, kStCapacity);
      if (pass == 0) deg[id] = 0;
      continue;
    }
    int32_t nid[kSlowCap + Poly<kSlowCap>::TW], nslot[kSlowCap + Poly<kSlowCap>::TW];
    const int cnt = voronoi_neighbors(P, id, nid, nslot);
    if (pass == 0) {
      deg[id] = cnt;
    } else {
      const int64_t o = out_off[id];
      for (int j = 0; j < cnt; ++j) out_ids[o + j] = nid[j];
    }
  }
}

}  // namespace

static GridView grid_view(const Buffers& b) {
  GridView G;
  G.off = b.offsets;
  G.sub_s = b.sub_s;
  G.sub_base = b.sub_base;
  G.sub_off = b.sub_off;
  return G;
}

cudaError_t launch_voronoi_step(const Geometry& g, const Buffers& b, const StepParams& P, cudaStream_t st) {
  const GridView G = grid_view(b);
  voronoi_step_kernel<<<g.n_tasks, kBlock, 0, st>>>(g.reps, g.tasks, (const int2*)b.S_pos, (const float2*)b.S_dir,
                                                    b.S_id, G, (int2*)b.U_pos, (float2*)b.U_dir, b.U_id,
                                                    b.counts, b.phi_acc, b.d_step, P, b.ovf_list,
                                                    b.ovf_count, b.d_status);
  voronoi_overflow_kernel<<<152, 64, 0, st>>>(g.reps, (const int2*)b.S_pos, (const float2*)b.S_dir, b.S_id,
                                              G, (int2*)b.U_pos, (float2*)b.U_dir, b.U_id,
                                              b.counts, b.phi_acc, b.d_step, P, b.ovf_list, b.ovf_count,
                                              b.d_status);
  return cudaGetLastError();
}

cudaError_t launch_voronoi_export(const Geometry& g, const Buffers& b, int rep, int n, int pass, int32_t* deg,
                                  const int64_t* out_off, int32_t* out_ids, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  const int nb = std::min((n + 63) / 64, 152 * 8);
  voronoi_export_kernel<<<nb, 64, 0, st>>>(g.reps, rep, (const int2*)b.S_pos, b.S_id, grid_view(b), pass, deg,
                                           out_off, out_ids, b.d_status);
  return cudaGetLastError();
}

}  // namespace vk
