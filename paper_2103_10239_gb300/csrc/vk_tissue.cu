// vk_tissue.cu -- the Voronoi tissue model (Sec. "Geometric models of dense
// tissue": each particle generates its Voronoi cell, of area A_i and
// perimeter P_i, with the energy of Eq. (vmEnergy)
//   E = sum_i KA (A_i - A0)^2 + KP (P_i - P0)^2;
// Sec. "Voronoi model forces": F_i = -dE/dr_i by the chain rule through the
// Voronoi vertices h, the circumcenters of the Delaunay triangles).
//
// Three kernels over one replica, FP64 geometry from exact integer offsets:
//   1. cells: every particle builds its cell with the Voronoi rule's clipper
//      (vk_voronoi.cuh) and stores its edge sites in counter-clockwise order
//      (sorted slot and exact offset), its area and its perimeter;
//   2. forces: for every vertex h of cell i (edge sites a, b) the three cells
//      i, a, b that share h contribute dE_c/dh; the vertex's neighbors in
//      cells a and b come from their stored edge lists (found by slot and
//      offset, so periodic images of the same particle stay apart), and
//      dh/dr_i is the Jacobian of the circumcenter in the paper's notation
//      (c, d, beta d, gamma d, z);
//   3. energy: one block sums the cells' terms in a fixed order.
#include "vk_voronoi.cuh"

namespace vk {

namespace {

struct TissueParams {
  double KA, KP, A0, P0;
  double unit;  // length of one grid unit, 2^-F
};

// circumcenter of (0, a, b), FP64
__device__ __forceinline__ double2 circum64(double ax, double ay, double bx, double by) {
  const double D = 2.0 * (ax * by - ay * bx);
  const double a2 = ax * ax + ay * ay, b2 = bx * bx + by * by;
  return make_double2((by * a2 - ay * b2) / D, (ax * b2 - bx * a2) / D);
}

__device__ __forceinline__ double2 circum_off(int2 a, int2 b, double u) {
  return circum64((double)a.x * u, (double)a.y * u, (double)b.x * u, (double)b.y * u);
}

// Pass 1: the cell of every particle of the replica
__global__ void __launch_bounds__(64) tissue_cells_kernel(const Rep* __restrict__ reps, int rep,
                                                          const int2* __restrict__ S_pos,
                                                          const int32_t* __restrict__ S_id, GridView G,
                                                          TissueParams T, int32_t* __restrict__ nb_n,
                                                          int32_t* __restrict__ nb_slot, int2* __restrict__ nb_off,
                                                          double* __restrict__ area, double* __restrict__ perim,
                                                          int32_t* status, const int32_t* __restrict__ vor_seed,
                                                          const int32_t* __restrict__ vor_seed_n,
                                                          const int32_t* __restrict__ slot_of) {
  const Rep R = reps[rep];
  for (int li = blockIdx.x * blockDim.x + threadIdx.x; li < R.n; li += gridDim.x * blockDim.x) {
    const int64_t s = R.p0 + li;
    const int2 p = S_pos[s];
    const int32_t pi[3] = {p.x, p.y, 0};
    const int32_t id = S_id[s];
    // a Voronoi-rule sim's last neighbors seed the cell (any seeds give the same cell)
    const int64_t gi = R.p0 + id;
    const Seeds sd{vor_seed ? vor_seed + gi * kVorSeed : nullptr, vor_seed ? vor_seed_n[gi] & kSeedCount : 0,
                   slot_of};
    Poly<kFastCap> P;
    int m = 0;
    area[s] = 0.0;
    perim[s] = 0.0;
    if (!voronoi_cell(R, s, pi, id, S_pos, S_id, G, P, status, 0u, sd, nullptr) || P.m > kTissueCap) {
      set_status(status, kStCapacity);
    } else if (P.nt > 0) {
      set_status(status, kStDegenerate);  // coincident particles: one site, no cell each
    } else {
      m = P.m;
      for (int a = 0; a < m; ++a) {
        const int pa = a == 0 ? m - 1 : a - 1, na = a + 1 == m ? 0 : a + 1;
        // an edge of zero length (four cocircular particles): no derivative
        if (vertex_cut_sign(P.qx[pa], P.qy[pa], P.qx[a], P.qy[a], P.qx[na], P.qy[na]) == 0)
          set_status(status, kStDegenerate);
        // an edge to an image of the particle itself (tiny boxes) is kept
        // with the particle's own slot and the image's offset
        nb_slot[s * kTissueCap + a] = P.slot[a] >= 0 ? P.slot[a] : (int32_t)s;
        nb_off[s * kTissueCap + a] = make_int2(P.qx[a], P.qy[a]);
      }
      double A = 0.0, Pm = 0.0;
      double2 h0 = circum_off(make_int2(P.qx[m - 1], P.qy[m - 1]), make_int2(P.qx[0], P.qy[0]), T.unit);
      for (int a = 0; a < m; ++a) {
        const int na = a + 1 == m ? 0 : a + 1;
        const double2 h1 = circum_off(make_int2(P.qx[a], P.qy[a]), make_int2(P.qx[na], P.qy[na]), T.unit);
        A += 0.5 * (h0.x * h1.y - h1.x * h0.y);
        Pm += hypot(h1.x - h0.x, h1.y - h0.y);
        h0 = h1;
      }
      area[s] = A;
      perim[s] = Pm;
    }
    nb_n[s] = m;
  }
}

// dE_c/dh for a vertex h of cell c with polygon neighbors prev, next
// (counter-clockwise, one frame): from the shoelace area, dA/dh =
// (1/2)(y_next - y_prev, x_prev - x_next); from the perimeter, dP/dh =
// (h - prev)/|h - prev| + (h - next)/|h - next|.
__device__ __forceinline__ double2 cell_grad(double2 h, double2 pv, double2 nx, double gA, double gP) {
  const double l1 = hypot(h.x - pv.x, h.y - pv.y), l2 = hypot(h.x - nx.x, h.y - nx.y);
  return make_double2(gA * 0.5 * (nx.y - pv.y) + gP * ((h.x - pv.x) / l1 + (h.x - nx.x) / l2),
                      gA * 0.5 * (pv.x - nx.x) + gP * ((h.y - pv.y) / l1 + (h.y - nx.y) / l2));
}

// position of the entry (slot, offset) in a stored edge list, or -1
__device__ __forceinline__ int find_entry(const int32_t* __restrict__ sl, const int2* __restrict__ off, int m,
                                          int32_t slot, int2 o) {
  for (int t = 0; t < m; ++t) {
    const int2 e = off[t];
    if (sl[t] == slot && e.x == o.x && e.y == o.y) return t;
  }
  return -1;
}

// Pass 2: F_i = -sum over the vertices h of cell i of (dh/dr_i)^T (dE_i/dh +
// dE_a/dh + dE_b/dh)
__global__ void __launch_bounds__(128) tissue_force_kernel(const Rep* __restrict__ reps, int rep,
                                                           const int32_t* __restrict__ S_id, TissueParams T,
                                                           const int32_t* __restrict__ nb_n,
                                                           const int32_t* __restrict__ nb_slot,
                                                           const int2* __restrict__ nb_off,
                                                           const double* __restrict__ area,
                                                           const double* __restrict__ perim,
                                                           double* __restrict__ force_out,
                                                           double* __restrict__ area_out,
                                                           double* __restrict__ perim_out, int32_t* status) {
  const Rep R = reps[rep];
  const double u = T.unit;
  for (int li = blockIdx.x * blockDim.x + threadIdx.x; li < R.n; li += gridDim.x * blockDim.x) {
    const int64_t s = R.p0 + li;
    const int32_t id = S_id[s];
    const int m = nb_n[s];
    if (area_out) area_out[id] = area[s];
    if (perim_out) perim_out[id] = perim[s];
    if (!force_out) continue;
    if (m < 3) {  // the cell pass failed (its status is latched)
      force_out[2 * (int64_t)id] = 0.0;
      force_out[2 * (int64_t)id + 1] = 0.0;
      continue;
    }
    double Fx = 0.0, Fy = 0.0;
    const int32_t* sl = nb_slot + s * kTissueCap;
    const int2* of = nb_off + s * kTissueCap;
    const double gAi = 2.0 * T.KA * (area[s] - T.A0), gPi = 2.0 * T.KP * (perim[s] - T.P0);
    bool ok = true;
    for (int k = 0; k < m && ok; ++k) {
      const int kp = k == 0 ? m - 1 : k - 1, kn = k + 1 == m ? 0 : k + 1, kn2 = kn + 1 == m ? 0 : kn + 1;
      const int32_t sa = sl[k], sb = sl[kn];
      const int2 da = of[k], db = of[kn];
      // cell i: h between sites a and b, neighbors between (prev, a) and (b, next)
      const double2 h = circum_off(da, db, u);
      double2 g = cell_grad(h, circum_off(of[kp], da, u), circum_off(db, of[kn2], u), gAi, gPi);
      // cell a: around a the sites run ... b, i ...; h lies between b and i
      {
        const int ma = nb_n[sa];
        const int32_t* sla = nb_slot + (int64_t)sa * kTissueCap;
        const int2* ofa = nb_off + (int64_t)sa * kTissueCap;
        const int t = find_entry(sla, ofa, ma, (int32_t)s, make_int2(-da.x, -da.y));
        const int tp = t <= 0 ? ma - 1 : t - 1;
        const int2 bexp = make_int2(db.x - da.x, db.y - da.y);
        if (t < 0 || sla[tp] != sb || ofa[tp].x != bexp.x || ofa[tp].y != bexp.y) {
          ok = false;
          break;
        }
        const int tpp = tp == 0 ? ma - 1 : tp - 1, tn = t + 1 == ma ? 0 : t + 1;
        const double2 ha = circum_off(ofa[tp], ofa[t], u);
        const double2 c = cell_grad(ha, circum_off(ofa[tpp], ofa[tp], u), circum_off(ofa[t], ofa[tn], u),
                                    2.0 * T.KA * (area[sa] - T.A0), 2.0 * T.KP * (perim[sa] - T.P0));
        g.x += c.x;
        g.y += c.y;
      }
      // cell b: around b the sites run ... i, a ...; h lies between i and a
      {
        const int mb = nb_n[sb];
        const int32_t* slb = nb_slot + (int64_t)sb * kTissueCap;
        const int2* ofb = nb_off + (int64_t)sb * kTissueCap;
        const int t = find_entry(slb, ofb, mb, (int32_t)s, make_int2(-db.x, -db.y));
        const int tn = t < 0 || t + 1 == mb ? 0 : t + 1;
        const int2 aexp = make_int2(da.x - db.x, da.y - db.y);
        if (t < 0 || slb[tn] != sa || ofb[tn].x != aexp.x || ofb[tn].y != aexp.y) {
          ok = false;
          break;
        }
        const int tp = t == 0 ? mb - 1 : t - 1, tnn = tn + 1 == mb ? 0 : tn + 1;
        const double2 hb = circum_off(ofb[t], ofb[tn], u);
        const double2 c = cell_grad(hb, circum_off(ofb[tp], ofb[t], u), circum_off(ofb[tn], ofb[tnn], u),
                                    2.0 * T.KA * (area[sb] - T.A0), 2.0 * T.KP * (perim[sb] - T.P0));
        g.x += c.x;
        g.y += c.y;
      }
      // dh/dr_i (Sec. "Voronoi model forces"; j = a, k = b): r_ij, r_ik from
      // i, r_jk = r_k - r_j; c, d = 2 c^2, beta d, gamma d, z = beta d r_ij +
      // gamma d r_ik (so h - r_i = z / d), and
      //   dh/dr_i = I + [r_ij (x) d(beta d)/dr_i + r_ik (x) d(gamma d)/dr_i
      //                  - (beta d + gamma d) I - z (x) (1/d) dd/dr_i] / d
      // with the derivatives of beta d, gamma d and d as they follow from
      // their definitions
      const double ijx = da.x * u, ijy = da.y * u, ikx = db.x * u, iky = db.y * u;
      const double jkx = ikx - ijx, jky = iky - ijy;
      const double c = ijx * (-jky) - ijy * (-jkx);  // r_ij x r_kj
      const double d = 2.0 * c * c;
      const double ij_jk = ijx * jkx + ijy * jky, ik_jk = ikx * jkx + iky * jky;
      const double ij2 = ijx * ijx + ijy * ijy, ik2 = ikx * ikx + iky * iky;
      const double bd = -ik2 * ij_jk, gd = ij2 * ik_jk;
      const double zx = bd * ijx + gd * ikx, zy = bd * ijy + gd * iky;
      const double dbx = 2.0 * ij_jk * ikx + ik2 * jkx, dby = 2.0 * ij_jk * iky + ik2 * jky;
      const double dgx = -2.0 * ik_jk * ijx - ij2 * jkx, dgy = -2.0 * ik_jk * ijy - ij2 * jky;
      const double ddx = 2.0 / c * jky, ddy = -2.0 / c * jkx;
      const double J00 = 1.0 + (ijx * dbx + ikx * dgx - (bd + gd) - zx * ddx) / d;
      const double J01 = (ijx * dby + ikx * dgy - zx * ddy) / d;
      const double J10 = (ijy * dbx + iky * dgx - zy * ddx) / d;
      const double J11 = 1.0 + (ijy * dby + iky * dgy - (bd + gd) - zy * ddy) / d;
      Fx -= g.x * J00 + g.y * J10;
      Fy -= g.x * J01 + g.y * J11;
    }
    // the cells around a vertex do not fit together as three: with exact
    // predicates only where four or more particles are cocircular (a vertex
    // shared by more than three cells), where the energy has no derivative
    if (!ok) set_status(status, kStDegenerate);
    force_out[2 * (int64_t)id] = ok ? Fx : 0.0;
    force_out[2 * (int64_t)id + 1] = ok ? Fy : 0.0;
  }
}

// Pass 3: the energy, summed by one block in a fixed order
__global__ void __launch_bounds__(256) tissue_energy_kernel(const Rep* __restrict__ reps, int rep, TissueParams T,
                                                            const double* __restrict__ area,
                                                            const double* __restrict__ perim,
                                                            double* __restrict__ energy) {
  __shared__ double part[256];
  const Rep R = reps[rep];
  double e = 0.0;
  for (int li = threadIdx.x; li < R.n; li += blockDim.x) {
    const double dA = area[R.p0 + li] - T.A0, dP = perim[R.p0 + li] - T.P0;
    e += T.KA * dA * dA + T.KP * dP * dP;
  }
  part[threadIdx.x] = e;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *energy = part[0];
}

GridView tissue_view(const Buffers& b) {
  GridView G;
  G.off = b.offsets;
  G.sub_s = b.sub_s;
  G.sub_base = b.sub_base;
  G.sub_off = b.sub_off;
  return G;
}

}  // namespace

cudaError_t launch_tissue(const Geometry& g, const Buffers& b, int rep, int n, double KA, double KP, double A0,
                          double P0, double unit, TissueScratch w, double* area_out, double* perim_out,
                          double* force_out, double* energy_out, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  const TissueParams T{KA, KP, A0, P0, unit};
  const int nb = std::min((n + 63) / 64, device_sm_count() * 16);
  tissue_cells_kernel<<<nb, 64, 0, st>>>(g.reps, rep, (const int2*)b.S_pos, b.S_id, tissue_view(b), T, w.nb_n,
                                         w.nb_slot, w.nb_off, w.area, w.perim, b.d_status, b.vor_seed, b.vor_seed_n,
                                         b.slot_of);
  const int nf = std::min((n + 127) / 128, device_sm_count() * 16);
  tissue_force_kernel<<<nf, 128, 0, st>>>(g.reps, rep, b.S_id, T, w.nb_n, w.nb_slot, w.nb_off, w.area, w.perim,
                                          force_out, area_out, perim_out, b.d_status);
  if (energy_out) tissue_energy_kernel<<<1, 256, 0, st>>>(g.reps, rep, T, w.area, w.perim, energy_out);
  return cudaGetLastError();
}

}  // namespace vk
