// Run-time dispatch of the σ-Laplace launchers on the GLL order, the element-to-global map,
// the apply's edge pass, and the allocation-free apply (arXiv 1512.02548, §3.1.2).  The
// order-templated kernels live in laplace_device.cuh and are compiled once per order.
#include <dlfcn.h>

#include <array>
#include <atomic>
#include <functional>
#include <map>
#include <mutex>

#include "mesh_index.cuh"

namespace semgb {


__global__ void k_apply_fix(DevGeom g, const double* __restrict__ q, const double* __restrict__ edge,
                            double* __restrict__ y) {
  const long long n = (long long)g.ncol * g.nrow;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int col = (int)(t / g.nrow), iz = (int)(t - (long long)col * g.nrow);
  double v = q[t];
  if (has_left_edge(g, col)) v += edge[(size_t)left_element(g, col) * g.nrow + iz];
  y[t] = -v;   // 𝓛 = −A
}

__global__ void k_l2g(DevGeom g, int32_t* __restrict__ l2g) {
  const int Q = g.P + 1;
  const long long total = (long long)g.Nx * g.Nz * Q * Q;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= total) return;
  const int b = (int)(t % Q);
  const int a = (int)((t / Q) % Q);
  const int l = (int)((t / (Q * Q)) % g.Nz);
  const int ex = (int)(t / ((long long)Q * Q * g.Nz));
  l2g[t] = col_of(g, ex, a) * g.nrow + l * g.P + b;
}

// ------------------------------------------------------------------------------------
// Launchers: dispatch on the GLL order to the per-order entry points (kernels_order.cu).
// ------------------------------------------------------------------------------------
#define SEM_DISPATCH_P(P_, ...) \
  switch (P_) {                  \
    case 2: { constexpr int PP = 2; __VA_ARGS__; } break;   \
    case 3: { constexpr int PP = 3; __VA_ARGS__; } break;   \
    case 4: { constexpr int PP = 4; __VA_ARGS__; } break;   \
    case 5: { constexpr int PP = 5; __VA_ARGS__; } break;   \
    case 6: { constexpr int PP = 6; __VA_ARGS__; } break;   \
    case 7: { constexpr int PP = 7; __VA_ARGS__; } break;   \
    case 8: { constexpr int PP = 8; __VA_ARGS__; } break;   \
    case 9: { constexpr int PP = 9; __VA_ARGS__; } break;   \
    case 10: { constexpr int PP = 10; __VA_ARGS__; } break; \
    case 11: { constexpr int PP = 11; __VA_ARGS__; } break; \
    case 12: { constexpr int PP = 12; __VA_ARGS__; } break; \
    default: return cudaErrorInvalidValue;           \
  }

cudaError_t upload_line_tables(const double* D64, const double* w64) {
  for (int P = 2; P <= kMaxP; ++P) {
    cudaError_t e = cudaSuccess;
    SEM_DISPATCH_P(P, (e = upload_tables_impl<PP>(D64, w64)));
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_geometry(const DevGeom& g, const double* eta, bool with_diag, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  SEM_DISPATCH_P(g.P, (e = launch_geometry_impl<PP>(g, eta, with_diag, s)));
  return e;
}

cudaError_t launch_apply(const DevGeom& g, const double* x, double* y, double* qtmp, double* edge,
                         cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  SEM_DISPATCH_P(g.P, (e = launch_apply_elem_impl<PP>(g, x, qtmp, edge, s)));
  if (e != cudaSuccess) return e;
  const long long n = (long long)g.ncol * g.nrow;
  k_apply_fix<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(g, qtmp, edge, y);
  count_launch();
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------
// Allocation-free variant of the stand-alone apply.  The only scratch the apply needs
// beyond its input and output is the per-element-column copy of the shared x-interface
// column; here it lives in one file-scope device array instead of the mesh workspace, and
// the output array doubles as the owned-column buffer.  The array is shared by every call
// on a device: calls that overlap on the GPU race on it.  Every entry that a call reads
// is written earlier in the same call, so nothing has to be cleared between calls.
// ------------------------------------------------------------------------------------
static __device__ __align__(256) double g_noalloc_edge[kNoAllocEdgeMax];

// Device address of g_noalloc_edge, looked up with cudaGetSymbolAddress at the first call on a
// device (with that device current) and kept for later calls.  The address belongs to the CUDA
// context that loaded this module, so the cache is keyed on that context as well: after
// cudaDeviceReset a new primary context may load the module at another address, and the next
// call looks it up again.  The context handle comes from the driver's cuCtxGetCurrent, found
// in the already loaded driver library; without it the key is the device alone.
static std::mutex g_noalloc_mu;
struct NoallocSlot { void* ctx; double* ptr; };
static NoallocSlot g_noalloc_slot[64] = {};

static void* current_context() {
  using GetCurrent = int (*)(void**);
  static GetCurrent fn = []() -> GetCurrent {
    void* h = dlopen("libcuda.so.1", RTLD_NOW | RTLD_NOLOAD);
    return h ? reinterpret_cast<GetCurrent>(dlsym(h, "cuCtxGetCurrent")) : nullptr;
  }();
  void* ctx = nullptr;
  if (fn && fn(&ctx) != 0) ctx = nullptr;
  return ctx;
}

static cudaError_t noalloc_edge_address(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  void* ctx = current_context();   // null on a thread the runtime has not bound yet
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  NoallocSlot& sl = g_noalloc_slot[dev];
  if (!sl.ptr || sl.ctx != ctx) {
    double* p = nullptr;
    e = cudaGetSymbolAddress(reinterpret_cast<void**>(&p), g_noalloc_edge);
    if (e != cudaSuccess) return e;
    sl.ptr = p;
    sl.ctx = current_context();      // the lookup has bound the device's context to this thread
  }
  *out = sl.ptr;
  return cudaSuccess;
}

// y ← −(y + edge of the left neighbour) in place: y holds the owned columns' A x.
__global__ void k_apply_fix_inplace(DevGeom g, const double* __restrict__ edge, double* y) {
  const long long n = (long long)g.ncol * g.nrow;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int col = (int)(t / g.nrow), iz = (int)(t - (long long)col * g.nrow);
  double v = y[t];
  if (has_left_edge(g, col)) v += edge[(size_t)left_element(g, col) * g.nrow + iz];
  y[t] = -v;
}

cudaError_t launch_apply_noalloc(const DevGeom& g, const double* x, double* y, cudaStream_t s) {
  if ((size_t)g.Nx * (size_t)g.nrow > kNoAllocEdgeMax) return cudaErrorInvalidValue;
  double* edge = nullptr;
  cudaError_t e = noalloc_edge_address(&edge);
  if (e != cudaSuccess) return e;
  SEM_DISPATCH_P(g.P, (e = launch_apply_elem_impl<PP>(g, x, y, edge, s)));
  if (e != cudaSuccess) return e;
  const long long n = (long long)g.ncol * g.nrow;
  k_apply_fix_inplace<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(g, edge, y);
  count_launch();
  return cudaGetLastError();
}

static std::atomic<int> g_tile_width[kMaxP + 1][kMaxNz + 1];

void set_apply_tile_width(int P, int Nz, int E) { g_tile_width[P][Nz].store(E, std::memory_order_relaxed); }
int apply_tile_width(int P, int Nz) {
  return (P >= 0 && P <= kMaxP && Nz >= 0 && Nz <= kMaxNz) ? g_tile_width[P][Nz].load(std::memory_order_relaxed) : 0;
}

cudaError_t launch_apply_tile(int fp32, const DevGeom& g, const void* x, void* y, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  SEM_DISPATCH_P(g.P, (e = launch_apply_tile_impl<PP>(fp32, g, x, y, s)));
  return e;
}

cudaError_t launch_l2g(const DevGeom& g, int32_t* l2g, cudaStream_t s) {
  const long long total = (long long)g.Nx * g.Nz * (g.P + 1) * (g.P + 1);
  k_l2g<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(g, l2g);
  count_launch();
  return cudaGetLastError();
}

cudaError_t pcg_grid_size(int P, int Nz, int nrow, int Nx, int chunk, int mixed, int* grid, size_t* smem) {
  *smem = apply_smem_bytes(P, nrow, Nz, chunk, sizeof(double));
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  SEM_DISPATCH_P(P, (e = pcg_occupancy_impl<PP>(mixed, *smem, &per_sm)));
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const long long cap = (long long)per_sm * sms, want = (Nx + chunk - 1) / chunk;
  *grid = (int)(want < cap ? want : cap);
  return cudaSuccess;
}

size_t stage_smem_bytes(int P, int nrow, int Nz, int chunk) {
  return apply_smem_bytes(P, nrow, Nz, chunk, sizeof(double));
}

// Occupancy queries are answered once per (device, kernel variant, shared memory) and kept: the
// serving loop creates batches every tick.
static std::mutex g_occ_mu;
static std::map<std::array<long long, 6>, int> g_occ;

static cudaError_t cached_query(std::array<long long, 6> key, int* out, const std::function<cudaError_t(int*)>& q) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  key[0] = dev;
  {
    std::lock_guard<std::mutex> lk(g_occ_mu);
    auto it = g_occ.find(key);
    if (it != g_occ.end()) { *out = it->second; return cudaSuccess; }
  }
  if ((e = q(out)) != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(g_occ_mu);
  g_occ[key] = *out;
  return cudaSuccess;
}

cudaError_t stage_occupancy(int P, int mixed, int wide, size_t smem, int* per_sm) {
  return cached_query({0, P, mixed, wide, 0, (long long)smem}, per_sm, [&](int* o) {
    cudaError_t e = cudaSuccess;
    SEM_DISPATCH_P(P, (e = stage_occupancy_impl<PP>(mixed, wide, smem, o)));
    return e;
  });
}

cudaError_t launch_stage(int P, int mixed, int wide, const StageArgs& a, int grid, size_t smem, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  SEM_DISPATCH_P(P, (e = launch_stage_impl<PP>(mixed, wide, a, grid, smem, s)));
  count_launch();
  return e;
}

cudaError_t cluster_fit(int P, int mixed, int wide, int csize, size_t smem, int* active_clusters) {
  return cached_query({0, P, mixed, wide, csize, (long long)smem}, active_clusters, [&](int* o) {
    cudaError_t e = cudaSuccess;
    SEM_DISPATCH_P(P, (e = cluster_fit_impl<PP>(mixed, wide, csize, smem, o)));
    return e;
  });
}

cudaError_t launch_stage_cluster(int P, int mixed, int wide, const StageArgs& a, int grid, int csize, size_t smem,
                                 cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  SEM_DISPATCH_P(P, (e = launch_stage_cluster_impl<PP>(mixed, wide, a, grid, csize, smem, s)));
  count_launch();
  return e;
}

__global__ void k_gather_status(const Instance* __restrict__ inst, int n, int* __restrict__ out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  int* p = inst[k].g.status;
  const int v = *p;
  out[k] = v;
  if (v) *p = 0;
}

cudaError_t launch_gather_status(const Instance* inst, int n, int* out, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_gather_status<<<(n + 127) / 128, 128, 0, s>>>(inst, n, out);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_prec_setup(const DevGeom& g, const PrecSetup& ps, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  SEM_DISPATCH_P(g.P, (e = launch_prec_setup_impl<PP>(g, ps, s)));
  return e;
}

cudaError_t launch_pcg(const DevGeom& g, const PcgArgs& a, int grid, size_t smem, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(a.bar, 0, 2 * sizeof(unsigned int), s);
  if (e != cudaSuccess) return e;
  SEM_DISPATCH_P(g.P, (e = launch_pcg_impl<PP>(a.mixed, g, a, grid, smem, s)));
  count_launch();
  return e;
}

}  // namespace semgb
