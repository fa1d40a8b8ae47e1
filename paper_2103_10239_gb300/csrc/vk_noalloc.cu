// vk_noalloc.cu -- k-nearest-neighbor lists without any device allocation.
//
// Who needs this: callers that must not allocate GPU memory at the point of
// the call.  Examples: code that records its work into a CUDA graph (plain
// cudaMalloc/cudaFree are not allowed while a stream is being captured);
// real-time or tightly scheduled loops, where cudaMalloc/cudaFree can block on
// or synchronise the device and add unpredictable latency; and hosts that own
// the device memory budget themselves (a fixed pool, a framework allocator)
// and forbid a library from taking memory behind their back.  For them this
// entry point works entirely inside one fixed scratch array that is part of
// the library image and sized for at most kNoAllocMaxN particles.
//
// It runs the same kernels as vk_init + vk_get_neighbors (cell histogram,
// two-level grid build, scatter, 2D kNN search) on the caller's stream, with
// every intermediate array carved out of that static array.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "../../include/vk.h"
#include "vk_internal.cuh"

namespace vk {

namespace {

constexpr int64_t kNoAllocMaxN = VK_NOALLOC_MAX_N;
constexpr float kNoAllocOccupancy = 2.0f;
// generous bound of the scratch the layout below needs for kNoAllocMaxN
constexpr size_t kScratchBytes = (size_t)6 << 20;

// The scratch array: every GPU that loads the library keeps these bytes
// until the process exits.  Host code must not use the symbol as a pointer;
// its device address comes from cudaGetSymbolAddress (see scratch_ptr).
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_mu;
void* g_ptr[256] = {nullptr};

// Device address of the scratch on the current device, looked up once per
// device (the first call on a device does it; that call must not be made
// while the stream is being captured).
cudaError_t scratch_ptr(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 256) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_ptr[dev] = p;
  }
  *out = g_ptr[dev];
  return cudaSuccess;
}

// lays out the intermediate arrays as 256-byte aligned offsets into the scratch
struct Carver {
  size_t used;
  template <class T>
  size_t take(size_t count) {
    used = (used + 255) & ~(size_t)255;
    const size_t off = used;
    used += sizeof(T) * (count ? count : 1);
    return off;
  }
};

// tables, grid bounds and cleared counters for one call
__global__ void noalloc_setup_kernel(Rep R, BlockTask* tasks, int n_tasks, Rep* rep_out, uint32_t* bounds,
                                     uint32_t* counts, int64_t n_cells, uint32_t* sub_count, int64_t n_sub,
                                     int32_t* status) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  if (tid == 0) {
    *rep_out = R;
    *status = 0;
  }
  for (int64_t i = tid; i < n_tasks; i += stride) tasks[i] = BlockTask{0, (int32_t)(i * kBlock)};
  for (int a = 0; a < 3; ++a)
    for (int64_t b = tid; b <= R.nc[a]; b += stride)
      bounds[R.bnd[a] + b] = (uint32_t)((b * (int64_t)R.L[a] + R.nc[a] - 1) / R.nc[a]);
  for (int64_t i = tid; i < n_cells; i += stride) counts[i] = 0u;
  for (int64_t i = tid; i < n_sub; i += stride) sub_count[i] = 0u;
}

// caller positions -> U; positions outside the box are wrapped into it so
// that every later index stays in bounds, and the status records it
__global__ void noalloc_load_kernel(const int32_t* __restrict__ pos, int32_t n, uint32_t Lx, uint32_t Ly,
                                    int2* __restrict__ U_pos, float2* __restrict__ U_dir, int32_t* __restrict__ U_id,
                                    int32_t* status) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int64_t x = pos[2 * (int64_t)i], y = pos[2 * (int64_t)i + 1];
  if (x < 0 || x >= (int64_t)Lx || y < 0 || y >= (int64_t)Ly) {
    atomicCAS(status, 0, (int32_t)VK_ERR_RANGE);
    x %= (int64_t)Lx;
    if (x < 0) x += Lx;
    y %= (int64_t)Ly;
    if (y < 0) y += Ly;
  }
  U_pos[i] = make_int2((int32_t)x, (int32_t)y);
  U_dir[i] = make_float2(0.f, 0.f);
  U_id[i] = i;
}

}  // namespace

}  // namespace vk

using namespace vk;

extern "C" vk_status vk_knn_lists_noalloc(const int32_t* pos_q, int64_t n, const vk_box* box, int32_t k,
                                          int32_t* out_ids, int32_t* dev_status, void* cuda_stream) {
  if (!pos_q || !box || !out_ids) return VK_ERR_ARG;
  if (n < 2 || n > kNoAllocMaxN) return VK_ERR_ARG;  // beyond the fixed scratch: see VK_NOALLOC_MAX_N
  if (k < 1 || k > kMaxK || k > n - 1) return VK_ERR_ARG;
  if (box->dim != 2) return VK_ERR_ARG;
  for (int a = 0; a < 2; ++a)
    if (box->box_q[a] < 1 || box->box_q[a] > (1u << 31)) return VK_ERR_RANGE;
  cudaStream_t st = (cudaStream_t)cuda_stream;

  // grid plan (host arithmetic only)
  Rep R;
  std::memset(&R, 0, sizeof(R));
  R.p0 = 0;
  R.c0 = 0;
  R.n = (int32_t)n;
  R.L[0] = box->box_q[0];
  R.L[1] = box->box_q[1];
  R.L[2] = 1;
  const double side = std::sqrt((double)kNoAllocOccupancy * (double)R.L[0] * (double)R.L[1] / (double)n);
  int64_t n_cells = 1;
  for (int a = 0; a < 3; ++a) {
    double ncd = a < 2 ? std::floor((double)R.L[a] / side) : 1.0;
    ncd = std::max(1.0, std::min(ncd, std::min((double)R.L[a], 65536.0)));
    R.nc[a] = (int32_t)ncd;
    n_cells *= R.nc[a];
    R.inv_w[a] = (float)R.nc[a] / (float)R.L[a];
  }
  R.bnd[0] = 0;
  R.bnd[1] = R.nc[0] + 1;
  R.bnd[2] = R.bnd[1] + R.nc[1] + 1;
  const int64_t n_bounds = (int64_t)R.nc[0] + R.nc[1] + R.nc[2] + 3;
  const int64_t n_sub = n_cells + n / kSubTarget + 1;
  const int n_tasks = (int)((n + kBlock - 1) / kBlock);

  // carve the scratch: offsets first (host arithmetic, checked against the
  // array's size before any device work), then the device address
  Carver cv{0};
  const size_t o_upos = cv.take<int2>(n), o_udir = cv.take<float2>(n), o_uid = cv.take<int32_t>(n);
  const size_t o_urank = cv.take<uint32_t>(n);
  const size_t o_spos = cv.take<int2>(n), o_sdir = cv.take<float2>(n), o_sid = cv.take<int32_t>(n);
  const size_t o_counts = cv.take<uint32_t>(n_cells), o_offsets = cv.take<uint32_t>(n_cells + 1);
  const size_t o_bsum = cv.take<uint32_t>(2 * ((n_cells + 2047) / 2048 + 1));
  const size_t o_subs = cv.take<uint8_t>(n_cells), o_subbase = cv.take<uint32_t>(n_cells + 1);
  const size_t o_subcount = cv.take<uint32_t>(n_sub), o_suboff = cv.take<uint32_t>(n_sub + 1);
  const size_t o_bsum2 = cv.take<uint32_t>((n_sub + 2047) / 2048 + 1);
  const size_t o_bounds = cv.take<uint32_t>(n_bounds);
  const size_t o_rep = cv.take<Rep>(1), o_tasks = cv.take<BlockTask>(n_tasks), o_status = cv.take<int32_t>(1);
  if (cv.used > kScratchBytes) return VK_ERR_CAPACITY;  // cannot happen for n <= kNoAllocMaxN
  // an error left pending by the caller's earlier work is reported, not
  // cleared (this call's status then says nothing about its own work)
  if (cudaPeekAtLastError() != cudaSuccess) return VK_ERR_CUDA;
  void* base_v = nullptr;
  if (scratch_ptr(&base_v) != cudaSuccess) {
    cudaGetLastError();  // the failed lookup's own error
    return VK_ERR_CUDA;
  }
  unsigned char* base = reinterpret_cast<unsigned char*>(base_v);
  Buffers b;
  std::memset(&b, 0, sizeof(b));
  b.U_pos = base + o_upos;
  b.U_dir = base + o_udir;
  b.U_id = reinterpret_cast<int32_t*>(base + o_uid);
  b.U_rank = reinterpret_cast<uint32_t*>(base + o_urank);
  b.S_pos = base + o_spos;
  b.S_dir = base + o_sdir;
  b.S_id = reinterpret_cast<int32_t*>(base + o_sid);
  b.counts = reinterpret_cast<uint32_t*>(base + o_counts);
  b.offsets = reinterpret_cast<uint32_t*>(base + o_offsets);
  b.bsum = reinterpret_cast<uint32_t*>(base + o_bsum);
  b.sub_s = base + o_subs;
  b.sub_base = reinterpret_cast<uint32_t*>(base + o_subbase);
  b.sub_count = reinterpret_cast<uint32_t*>(base + o_subcount);
  b.sub_off = reinterpret_cast<uint32_t*>(base + o_suboff);
  b.bsum2 = reinterpret_cast<uint32_t*>(base + o_bsum2);
  b.bounds = reinterpret_cast<uint32_t*>(base + o_bounds);
  Rep* rep_d = reinterpret_cast<Rep*>(base + o_rep);
  BlockTask* tasks_d = reinterpret_cast<BlockTask*>(base + o_tasks);
  int32_t* status_d = reinterpret_cast<int32_t*>(base + o_status);

  Geometry g;
  g.dim = 2;
  g.rule = VK_RULE_KNN;
  g.n_rep = 1;
  g.n_total = n;
  g.n_cells = n_cells;
  g.n_sub_max = n_sub;
  g.n_tasks = n_tasks;
  g.reps = rep_d;
  g.tasks = tasks_d;
  StepParams P;
  std::memset(&P, 0, sizeof(P));
  P.k = k;
  P.n_rep = 1;
  P.phi_cap = 2;
  P.knn_search = 1;  // the per-particle walk: no hint buffers, no shared-memory attribute to set
  P.fov_cq = kViewAll;

  noalloc_setup_kernel<<<64, 256, 0, st>>>(R, tasks_d, n_tasks, rep_d, b.bounds, b.counts, n_cells, b.sub_count,
                                           n_sub, status_d);
  noalloc_load_kernel<<<(int)((n + 255) / 256), 256, 0, st>>>(pos_q, (int32_t)n, R.L[0], R.L[1], (int2*)b.U_pos,
                                                              (float2*)b.U_dir, b.U_id, status_d);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = launch_count(g, b, st);
  if (e == cudaSuccess) e = launch_build(g, b, st);
  if (e == cudaSuccess) e = launch_scatter(g, b, P, 0, st);
  if (e == cudaSuccess) e = launch_knn2_export(g, b, k, 0, (int)n, out_ids, st, P);
  if (e == cudaSuccess && dev_status)
    e = cudaMemcpyAsync(dev_status, status_d, sizeof(int32_t), cudaMemcpyDefault, st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return VK_ERR_CUDA;
  }
  return VK_OK;
}
