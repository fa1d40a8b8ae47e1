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
#include <climits>

#include "vk_internal.cuh"

namespace vk {

namespace {

template <int KC>
struct Top {
  uint64_t d[KC];
  int32_t id[KC];
  int32_t slot[KC];
};

template <int KC>
__device__ __forceinline__ void top_init(Top<KC>& T, int k) {
#pragma unroll
  for (int s = 0; s < KC; ++s) {
    const bool sentinel = s < KC - k;  // orders before every real candidate
    T.d[s] = sentinel ? 0ull : ~0ull;
    T.id[s] = sentinel ? INT_MIN : INT_MAX;
    T.slot[s] = -1;
  }
}

template <int KC>
__device__ __forceinline__ void top_insert(Top<KC>& T, uint64_t D, int32_t idj, int32_t q) {
  bool placed = false;
#pragma unroll
  for (int s = KC - 1; s > 0; --s) {
    const bool before = (D < T.d[s - 1]) || (D == T.d[s - 1] && idj < T.id[s - 1]);
    if (!placed) {
      if (before) {
        T.d[s] = T.d[s - 1];
        T.id[s] = T.id[s - 1];
        T.slot[s] = T.slot[s - 1];
      } else {
        T.d[s] = D;
        T.id[s] = idj;
        T.slot[s] = q;
        placed = true;
      }
    }
  }
  if (!placed) {
    T.d[0] = D;
    T.id[0] = idj;
    T.slot[0] = q;
  }
}

struct Ctx {
  int64_t self;
  uint32_t px, py;
  uint32_t Lx, Ly;
  int32_t hix, lox, hiy, loy;  // minimum image: d > hi -> d - L, d <= lo -> d + L
  uint32_t n_cand, n_runs;
};

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
    if (D <= T.d[KC - 1] && (int64_t)q != C.self) {
      const int32_t idj = __ldg(ids + q);
      if (D < T.d[KC - 1] || idj < T.id[KC - 1]) top_insert<KC>(T, D, idj, (int32_t)q);
    }
  }
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

// first offset of sub-cell b: ceil(b*w/s)
__device__ __forceinline__ int64_t sub_lo(int b, int64_t w, int s) {
  const int64_t bw = (int64_t)b * w;
  int64_t q = (int64_t)((float)bw / (float)s);
  while (q * s < bw) ++q;
  while (q > 0 && (q - 1) * s >= bw) --q;
  return q;
}

struct Walk {
  const Rep* R;
  const uint32_t* __restrict__ bx;
  const uint32_t* __restrict__ by;
  GridView G;
  int64_t own;
  bool own_done;
};

// coarse cells x0..x1 (actual indices, contiguous) of one row; ux0 is the
// unwrapped x index of cell x0 and ucy the unwrapped y index of the row
template <int KC>
__device__ __forceinline__ void visit_cells(Ctx& C, const Walk& W, const int2* __restrict__ pos,
                                            const int32_t* __restrict__ ids, int x0, int x1, int ux0, int ucy,
                                            int64_t rowbase, Top<KC>& T) {
  const GridView& G = W.G;
  const uint32_t sb0 = __ldg(G.sub_base + rowbase + x0), sb1 = __ldg(G.sub_base + rowbase + x1 + 1);
  if (sb1 - sb0 == (uint32_t)(x1 - x0 + 1)) {  // no sub-grid in the segment: one run
    scan_run<KC>(C, pos, ids, __ldg(G.off + rowbase + x0), __ldg(G.off + rowbase + x1 + 1), T);
    return;
  }
  const Rep& R = *W.R;
  uint32_t pb = 0, pe = 0;
  bool pend = false;
  for (int x = x0; x <= x1; ++x) {
    const int64_t g = rowbase + x;
    const uint32_t b0 = __ldg(G.sub_base + g), b1 = __ldg(G.sub_base + g + 1);
    if (b1 - b0 == 1) {
      const uint32_t qb = __ldg(G.off + g), qe = __ldg(G.off + g + 1);
      if (pend && qb == pe) {
        pe = qe;
      } else {
        if (pend) scan_run<KC>(C, pos, ids, pb, pe, T);
        pend = true;
        pb = qb;
        pe = qe;
      }
      continue;
    }
    if (pend) scan_run<KC>(C, pos, ids, pb, pe, T);
    pend = false;
    if (g == W.own && W.own_done) continue;
    const uint64_t r2 = T.d[KC - 1];
    if (r2 == ~0ull) {
      scan_run<KC>(C, pos, ids, __ldg(G.off + g), __ldg(G.off + g + 1), T);
      continue;
    }
    // only the sub-cells meeting the box [p - rad, p + rad]
    const int64_t rad = radius_upper(r2);
    const int ucx = ux0 + (x - x0);
    const int64_t cx0 = cell_lo_tab(ucx, R.nc[0], W.bx, R.L[0]);
    const int64_t wx = cell_lo_tab(ucx + 1, R.nc[0], W.bx, R.L[0]) - cx0;
    const int64_t cy0 = cell_lo_tab(ucy, R.nc[1], W.by, R.L[1]);
    const int64_t wy = cell_lo_tab(ucy + 1, R.nc[1], W.by, R.L[1]) - cy0;
    const int64_t lx = (int64_t)C.px - rad - cx0, hx = (int64_t)C.px + rad - cx0;
    const int64_t ly = (int64_t)C.py - rad - cy0, hy = (int64_t)C.py + rad - cy0;
    if (hx < 0 || lx >= wx || hy < 0 || ly >= wy) continue;
    const int s = __ldg(G.sub_s + g);
    const int sx0 = lx <= 0 ? 0 : sub_idx(lx, wx, s), sx1 = hx >= wx ? s - 1 : sub_idx(hx, wx, s);
    const int sy0 = ly <= 0 ? 0 : sub_idx(ly, wy, s), sy1 = hy >= wy ? s - 1 : sub_idx(hy, wy, s);
    for (int yy = sy0; yy <= sy1; ++yy) {
      const uint32_t rb = b0 + (uint32_t)yy * s;
      scan_run<KC>(C, pos, ids, __ldg(G.sub_off + rb + sx0), __ldg(G.sub_off + rb + sx1 + 1), T);
    }
  }
  if (pend) scan_run<KC>(C, pos, ids, pb, pe, T);
}

// row segment of x offsets [a, b] around the particle's cell cx
template <int KC>
__device__ __forceinline__ void visit_segment(Ctx& C, const Walk& W, const int2* __restrict__ pos,
                                              const int32_t* __restrict__ ids, int cx, int a, int b, int ucy,
                                              int64_t rowbase, Top<KC>& T) {
  if (a > b) return;
  const int nx = W.R->nc[0];
  const int ua = cx + a;
  const int start = ua < 0 ? ua + nx : (ua >= nx ? ua - nx : ua);
  const int len = b - a + 1;
  if (start + len <= nx) {
    visit_cells<KC>(C, W, pos, ids, start, start + len - 1, ua, ucy, rowbase, T);
  } else {
    visit_cells<KC>(C, W, pos, ids, start, nx - 1, ua, ucy, rowbase, T);
    visit_cells<KC>(C, W, pos, ids, 0, start + len - nx - 1, ua + (nx - start), ucy, rowbase, T);
  }
}

template <int KC>
__device__ __forceinline__ void knn2_search(Ctx& C, const Rep& R, const uint32_t* __restrict__ bounds,
                                            const GridView& G, const int2* __restrict__ pos,
                                            const int32_t* __restrict__ ids, Top<KC>& T) {
  Walk W;
  W.R = &R;
  W.bx = bounds + R.bnd[0];
  W.by = bounds + R.bnd[1];
  W.G = G;
  const int nx = R.nc[0], ny = R.nc[1];
  const int cx = cell_of_tab(C.px, nx, W.bx, R.inv_w[0]);
  const int cy = cell_of_tab(C.py, ny, W.by, R.inv_w[1]);
  W.own = R.c0 + (int64_t)cy * nx + cx;
  W.own_done = false;
  const uint32_t ob0 = __ldg(G.sub_base + W.own), ob1 = __ldg(G.sub_base + W.own + 1);
  if (ob1 - ob0 > 1) {
    // phase 1: rings of sub-cells in the own coarse cell
    const int s = __ldg(G.sub_s + W.own);
    const int64_t cx0 = __ldg(W.bx + cx), wx = (int64_t)__ldg(W.bx + cx + 1) - cx0;
    const int64_t cy0 = __ldg(W.by + cy), wy = (int64_t)__ldg(W.by + cy + 1) - cy0;
    const int sx = sub_idx((int64_t)C.px - cx0, wx, s), sy = sub_idx((int64_t)C.py - cy0, wy, s);
    for (int r = 0;; ++r) {
      const int bx0 = max(sx - r, 0), bx1 = min(sx + r, s - 1), by0 = max(sy - r, 0), by1 = min(sy + r, s - 1);
      const int px0 = r ? max(sx - r + 1, 0) : 1, px1 = r ? min(sx + r - 1, s - 1) : 0;
      const int py0 = r ? max(sy - r + 1, 0) : 1, py1 = r ? min(sy + r - 1, s - 1) : 0;
      for (int yy = by0; yy <= by1; ++yy) {
        const uint32_t rb = ob0 + (uint32_t)yy * s;
        if (yy < py0 || yy > py1 || px0 > px1) {
          scan_run<KC>(C, pos, ids, __ldg(G.sub_off + rb + bx0), __ldg(G.sub_off + rb + bx1 + 1), T);
        } else {
          if (bx0 < px0) scan_run<KC>(C, pos, ids, __ldg(G.sub_off + rb + bx0), __ldg(G.sub_off + rb + px0), T);
          if (bx1 > px1)
            scan_run<KC>(C, pos, ids, __ldg(G.sub_off + rb + px1 + 1), __ldg(G.sub_off + rb + bx1 + 1), T);
        }
      }
      if (bx0 == 0 && by0 == 0 && bx1 == s - 1 && by1 == s - 1) break;
      int64_t B = INT64_MAX;
      if (bx0 > 0) B = min(B, (int64_t)C.px - (cx0 + sub_lo(bx0, wx, s)) + 1);
      if (bx1 < s - 1) B = min(B, cx0 + sub_lo(bx1 + 1, wx, s) - (int64_t)C.px);
      if (by0 > 0) B = min(B, (int64_t)C.py - (cy0 + sub_lo(by0, wy, s)) + 1);
      if (by1 < s - 1) B = min(B, cy0 + sub_lo(by1 + 1, wy, s) - (int64_t)C.py);
      if (T.d[KC - 1] < (uint64_t)B * (uint64_t)B) break;
    }
    W.own_done = true;
  }
  // phase 2: rings of coarse cells
  for (int r = 0;; ++r) {
    const int lox = -min(r, (nx - 1) / 2), hix = min(r, nx / 2);
    const int loy = -min(r, (ny - 1) / 2), hiy = min(r, ny / 2);
    const int plox = r ? -min(r - 1, (nx - 1) / 2) : 1, phix = r ? min(r - 1, nx / 2) : 0;
    const int ploy = r ? -min(r - 1, (ny - 1) / 2) : 1, phiy = r ? min(r - 1, ny / 2) : 0;
    const bool fullx = hix - lox + 1 == nx, fully = hiy - loy + 1 == ny;
    if (r > 0 && lox == plox && hix == phix && loy == ploy && hiy == phiy) break;  // nothing new
    for (int oy = loy; oy <= hiy; ++oy) {
      const int ucy = cy + oy;
      const int ay = ucy < 0 ? ucy + ny : (ucy >= ny ? ucy - ny : ucy);
      const int64_t rowbase = R.c0 + (int64_t)ay * nx;
      if (oy < ploy || oy > phiy) {
        visit_segment<KC>(C, W, pos, ids, cx, lox, hix, ucy, rowbase, T);
      } else {
        visit_segment<KC>(C, W, pos, ids, cx, lox, plox - 1, ucy, rowbase, T);
        visit_segment<KC>(C, W, pos, ids, cx, phix + 1, hix, ucy, rowbase, T);
      }
    }
    if (fullx && fully) break;
    int64_t B = INT64_MAX;
    if (!fullx) {
      B = min(B, (int64_t)C.px - cell_lo_tab(cx - r, nx, W.bx, R.L[0]) + 1);
      B = min(B, cell_lo_tab(cx + r + 1, nx, W.bx, R.L[0]) - (int64_t)C.px);
    }
    if (!fully) {
      B = min(B, (int64_t)C.py - cell_lo_tab(cy - r, ny, W.by, R.L[1]) + 1);
      B = min(B, cell_lo_tab(cy + r + 1, ny, W.by, R.L[1]) - (int64_t)C.py);
    }
    // every unscanned particle is at squared distance >= B^2; an equal
    // distance could still win on id, hence the strict test
    if (T.d[KC - 1] < (uint64_t)B * (uint64_t)B) break;
  }
}

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
}

// the general update (vectorial noise, FP64 sums), kept out of line
__device__ __noinline__ void align_advect_general(const Rep& R, const StepParams& P, uint32_t step, int32_t id,
                                                  const float* ni, const HeadSum<2>& H, int m, const int32_t* pi,
                                                  int32_t* pout, float* nout) {
  align_advect<2>(R, P, step, id, ni, H, m, pi, pout, nout);
}

template <int KC>
__global__ void __launch_bounds__(kBlock, 2) knn2_step_kernel(
    const Rep* __restrict__ reps, const BlockTask* __restrict__ tasks, const uint32_t* __restrict__ bounds,
    const int2* __restrict__ S_pos, const float2* __restrict__ S_dir, const int32_t* __restrict__ S_id, GridView G,
    int2* __restrict__ U_pos, float2* __restrict__ U_dir, int32_t* __restrict__ U_id, uint32_t* __restrict__ counts,
    double* __restrict__ phi_acc, const int64_t* __restrict__ d_step, StepParams P) {
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
  if (li < R.n) {
    const int64_t s = R.p0 + li;
    const int2 p = S_pos[s];
    const float2 nv = S_dir[s];
    const int32_t id = S_id[s];
    init_ctx(C, R, s, p);
    Top<KC> T;
    top_init<KC>(T, P.k);
    knn2_search<KC>(C, R, bounds, G, S_pos, S_id, T);
    // Eq. (2): neighbor headings in (D, id) order
    HeadSum<2> H;
    H.init();
    const float ni[3] = {nv.x, nv.y, 0.f};
    if (P.include_self) H.add(ni, P.sum_mode);
#pragma unroll
    for (int j = 0; j < KC; ++j) {
      if (j >= KC - P.k) {
        const float2 d = __ldg(S_dir + T.slot[j]);
        const float v[2] = {d.x, d.y};
        H.add(v, P.sum_mode);
      }
    }
    const int32_t pi[3] = {p.x, p.y, 0};
    int32_t pout[3] = {0, 0, 0};
    const int m = P.k + (P.include_self ? 1 : 0);
    if (P.noise == 0 && P.sum_mode != 2) {
      // angular noise, FP32 sums (the default) inline
      const uint4 w = philox4x32_10(make_uint4((uint32_t)id, (uint32_t)step, R.replica, 0u),
                                    make_uint2(P.seed_lo, P.seed_hi));
      const float u = unit24(w.x);
      const float Sx = P.sum_mode == 1 ? __fadd_rn(H.s[0], H.c[0]) : H.s[0];
      const float Sy = P.sum_mode == 1 ? __fadd_rn(H.s[1], H.c[1]) : H.s[1];
      float th = (Sx == 0.f && Sy == 0.f) ? atan2f(nv.y, nv.x) : atan2f(Sy, Sx);
      th = th + R.eta * (u - 0.5f);
      sincosf(th, &nnew[1], &nnew[0]);
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
  record_search_stats(P.stats, li < R.n, C.n_cand, C.n_runs);
  phi_block_end<2>(phs, nnew, phi_acc + ((size_t)(step % P.phi_cap) * (size_t)P.n_rep + (size_t)t.rep) * 3);
}

template <int KC>
__global__ void __launch_bounds__(kBlock, 2) knn2_export_kernel(const Rep* __restrict__ reps, int rep,
                                                                const uint32_t* __restrict__ bounds,
                                                                const int2* __restrict__ S_pos,
                                                                const int32_t* __restrict__ S_id, GridView G, int k,
                                                                int32_t* __restrict__ out) {
  const Rep R = reps[rep];
  const int li = blockIdx.x * kBlock + (int)threadIdx.x;
  if (li >= R.n) return;
  const int64_t s = R.p0 + li;
  Ctx C;
  init_ctx(C, R, s, S_pos[s]);
  Top<KC> T;
  top_init<KC>(T, k);
  knn2_search<KC>(C, R, bounds, G, S_pos, S_id, T);
  const int32_t id = S_id[s];
#pragma unroll
  for (int j = 0; j < KC; ++j)
    if (j >= KC - k) out[(int64_t)id * k + (j - (KC - k))] = T.id[j];
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
cudaError_t step2(const Geometry& g, const Buffers& b, const StepParams& P, cudaStream_t st) {
  knn2_step_kernel<KC><<<g.n_tasks, kBlock, 0, st>>>(g.reps, g.tasks, b.bounds, (const int2*)b.S_pos,
                                                     (const float2*)b.S_dir, b.S_id, view_of(b), (int2*)b.U_pos,
                                                     (float2*)b.U_dir, b.U_id, b.counts, b.phi_acc, b.d_step, P);
  return cudaGetLastError();
}

template <int KC>
cudaError_t export2(const Geometry& g, const Buffers& b, int k, int rep, int n, int32_t* out, cudaStream_t st) {
  const int nb = (n + kBlock - 1) / kBlock;
  if (nb == 0) return cudaSuccess;
  knn2_export_kernel<KC><<<nb, kBlock, 0, st>>>(g.reps, rep, b.bounds, (const int2*)b.S_pos, b.S_id, view_of(b), k,
                                                out);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_knn2_step(const Geometry& g, const Buffers& b, const StepParams& P, cudaStream_t st) {
  if (P.k <= 8) return step2<8>(g, b, P, st);
  if (P.k <= 16) return step2<16>(g, b, P, st);
  return step2<32>(g, b, P, st);
}

cudaError_t launch_knn2_export(const Geometry& g, const Buffers& b, int k, int rep, int n, int32_t* out,
                               cudaStream_t st) {
  if (k <= 8) return export2<8>(g, b, k, rep, n, out, st);
  if (k <= 16) return export2<16>(g, b, k, rep, n, out, st);
  return export2<32>(g, b, k, rep, n, out, st);
}

}  // namespace vk
