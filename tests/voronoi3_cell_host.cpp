// Host build of the 3D Voronoi cell builder of the CUDA path
// (paper_2103_10239_gb300/csrc/vk_voronoi3.cuh is plain C++ for the host and
// the device), driven by a brute-force candidate enumeration in a chosen
// order, for the CPU tests that compare it with the oracle.  Test code only.
#include "../paper_2103_10239_gb300/csrc/vk_voronoi3.cuh"

#include <algorithm>
#include <cmath>
#include <vector>

using namespace vk::v3;

namespace {

int64_t min_image(int64_t d, int64_t L) {
  if (2 * d > L) d -= L;
  if (2 * d <= -L) d += L;
  return d;
}

// the cell of particle i, candidates in the given order: 0 index order,
// 1 by distance, 2 pseudo-random; then every image within 2R when the cell
// reaches a quarter of the box (as the kernel does)
template <class Cell>
int build(Cell& C, int8_t* sg, int64_t n, const int32_t* pos, const int64_t* box, int order, int64_t i,
          std::vector<int32_t>& row) {
  const uint32_t L[3] = {(uint32_t)box[0], (uint32_t)box[1], (uint32_t)box[2]};
  const int64_t Lmin = std::min(box[0], std::min(box[1], box[2]));
  auto off = [&](int64_t j, int k) { return min_image((int64_t)pos[3 * j + k] - pos[3 * i + k], box[k]); };
  std::vector<int64_t> ord(n);
  for (int64_t j = 0; j < n; ++j) ord[j] = j;
  if (order == 1) {
    auto w = [&](int64_t j) { return off(j, 0) * off(j, 0) + off(j, 1) * off(j, 1) + off(j, 2) * off(j, 2); };
    std::stable_sort(ord.begin(), ord.end(), [&](int64_t a, int64_t b) { return w(a) < w(b); });
  } else if (order == 2) {
    uint64_t s = 88172645463325252ull ^ (uint64_t)i;
    for (int64_t j = n - 1; j > 0; --j) {
      s ^= s << 13;
      s ^= s >> 7;
      s ^= s << 17;
      std::swap(ord[j], ord[s % (uint64_t)(j + 1)]);
    }
  }
  cell_init(C, L, sg);
  for (int64_t j : ord) {
    if (j == i) continue;
    const int32_t d[3] = {(int32_t)off(j, 0), (int32_t)off(j, 1), (int32_t)off(j, 2)};
    if (!d[0] && !d[1] && !d[2]) return kCoincident;
    if (cell_clip(C, d, (int32_t)j, sg) < 0) return C.status;
  }
  if (16.0 * C.r2 > (double)Lmin * (double)Lmin) {
    const double R = std::sqrt((double)C.r2);
    int64_t K[3];
    for (int a = 0; a < 3; ++a) K[a] = (int64_t)std::floor((2.0 * R + 0.5 * box[a]) / box[a]) + 1;
    for (int64_t j = 0; j < n; ++j) {
      if (j == i) continue;
      for (int64_t kx = -K[0]; kx <= K[0]; ++kx)
        for (int64_t ky = -K[1]; ky <= K[1]; ++ky)
          for (int64_t kz = -K[2]; kz <= K[2]; ++kz) {
            const int32_t d[3] = {(int32_t)(off(j, 0) + kx * box[0]), (int32_t)(off(j, 1) + ky * box[1]),
                                  (int32_t)(off(j, 2) + kz * box[2])};
            if (cell_clip(C, d, (int32_t)j, sg) < 0) return C.status;
          }
    }
  }
  row.clear();
  for (int p = 0; p < C.np; ++p)
    if (C.pref[p] > 0 && C.pslot[p] >= 0 && face_positive(C, p)) row.push_back(C.pslot[p]);
  std::sort(row.begin(), row.end());
  row.erase(std::unique(row.begin(), row.end()), row.end());
  return kOk;
}

}  // namespace

// Neighbor rows of every particle (ids sorted; deg[i] < 0: -status).  The
// kernel's cell (64 planes, 128 vertices) first, the overflow kernel's
// (128, 256) when it runs out of room.  Returns how many cells needed the
// larger one.
extern "C" int64_t v3_host_neighbors(int64_t n, const int32_t* pos, const int64_t* box, int32_t order,
                                     int32_t maxdeg, int32_t* deg, int32_t* ids) {
  static Cell<64, 128> small;
  static Cell<128, 256> large;
  static int8_t sg[256];
  std::vector<int32_t> row;
  int64_t n_large = 0;
  for (int64_t i = 0; i < n; ++i) {
    int st = build(small, sg, n, pos, box, order, i, row);
    if (st == kCapacity) {
      ++n_large;
      st = build(large, sg, n, pos, box, order, i, row);
    }
    if (st != kOk || (int32_t)row.size() > maxdeg) {
      deg[i] = st != kOk ? -st : -100;
      continue;
    }
    deg[i] = (int32_t)row.size();
    for (size_t t = 0; t < row.size(); ++t) ids[i * maxdeg + (int64_t)t] = row[t];
  }
  return n_large;
}

// The exact side test and the FP32 vertex estimate of the builder, on
// explicit plane offsets (for the predicate tests).
extern "C" int v3_host_side(const int32_t* da, const int32_t* db, const int32_t* dc, const int32_t* de) {
  return side_exact(da, db, dc, de);
}

extern "C" void v3_host_vertex(const int32_t* da, const int32_t* db, const int32_t* dc, float* y) {
  vertex_y(da, db, dc, y);
}
