// Device code of the σ-Laplace path (§2 and §3.1.2 of arXiv 1512.02548), templated on the GLL
// order P: geometry, the matrix-free operator, the persistent Krylov solver with the σ-separable
// preconditioner, and the fused RK stage.  Included by kernels_order.cu, which is compiled once
// per order (-DSEM_ORDER=P) and instantiates the host entry points at the end of this file;
// everything else here has internal linkage, including each order's copy of the constant tables.
//
// Operator.  For element (ex,l) with local nodal values u_ab, a along x and b along
// σ, GLL collocation gives the gradients u_r = (D⊗I)u, u_t = (I⊗D)u; with weights
// W_ab = w_a w_b |J^k| and K = JJᵀ/det J (eq. symTransformedLaplace2) the element
// contribution to A = −𝓛 is
//     (A_e u) = (Dᵀ⊗I) F1 + (I⊗Dᵀ) F2,
//     F1 = w_a w_b (Δσ/Δx · K11 u_r + K12 u_t),  F2 = w_a w_b (K12 u_r + Δx/Δσ · K22 u_t),
// with K11 = d, K12 = ∂xh − σ ∂xd, K22 = (1 + K12²)/d evaluated on the fly from four
// numbers per element-local column.  Nothing is stored per node except the vectors.
//
// Work decomposition.  A team of CTAs (the whole grid for one mesh, or the CTAs given to one
// instance of a batch) splits the x-elements into contiguous ranges; a CTA processes its
// element columns (all Nz layers of an x-element) in chunks of consecutive columns staged in
// shared memory.  Columns a = 0..P−1 of an element are written straight to the output and
// column a = P (shared with the next x-element) to an edge buffer that the owner of that
// column adds after a team barrier.  All sums are in a fixed order, so results are bitwise
// reproducible for a given team size.
//
// Krylov.  Preconditioned conjugate gradients (Chronopoulos–Gear form: one reduction per
// iteration) on the Dirichlet-eliminated SPD system, inside one cooperative persistent kernel:
// team barriers with acquire/release atomics and a wall-clock limit, deterministic reductions,
// a halo column per CTA so the preconditioned residual needs no extra barrier, and a
// device-side convergence test (no host round trip).  The σ-separable preconditioner applies
// the exact inverse of the operator without its slope coupling (σ-eigenbasis, per-mode 1D
// condensation and a warp-parallel interface solve).  In mixed precision the inner iterations
// run in FP32 and the kernel refines the FP64 residual.
#pragma once
#include <cooperative_groups.h>
#include <mutex>

#include "mesh_index.cuh"
#include "surface_device.cuh"

namespace semgb {

static __constant__ double c_D64[kDTotal];
static __constant__ float c_D32[kDTotal];
static __constant__ double c_w64[kWTotal];
static __constant__ float c_w32[kWTotal];

template <class T> struct CT;
template <> struct CT<double> {
  static __device__ __forceinline__ const double* D() { return c_D64; }
  static __device__ __forceinline__ const double* w() { return c_w64; }
};
template <> struct CT<float> {
  static __device__ __forceinline__ const float* D() { return c_D32; }
  static __device__ __forceinline__ const float* w() { return c_w32; }
};


// L2-coherent load for data another CTA wrote before the last grid barrier.


// ------------------------------------------------------------------------------------
// Geometry: per element-local column (ex, a) store d, 1/d, ∂x h, ∂x d (element-local
// collocation derivative of d = η + h, the exact Jacobian of the interpolated σ-map).
// ------------------------------------------------------------------------------------
template <int P>
__device__ __forceinline__ void geometry_item(const DevGeom& g, const double* __restrict__ eta, int t) {
  constexpr int Q = P + 1;
  const int ex = t / Q, a = t - ex * Q;
  const double* D = c_D64 + d_off(P) + a * Q;
  double etax = 0.0;
#pragma unroll
  for (int c = 0; c < Q; ++c) etax = fma(D[c], __ldcg(eta + col_of(g, ex, c)), etax);
  etax *= g.r2dx[ex];
  const int col = col_of(g, ex, a);
  const double d = __ldcg(eta + col) + g.h[col];
  const double hx = g.hx_loc[t];
  const double dxd = etax + hx;
  if (!(d > 0.0) || !isfinite(d) || !isfinite(dxd)) atomicOr(g.status, ST_BAD_DEPTH);
  const double invd = 1.0 / d;
  double* o = g.geo64 + (size_t)t * 4;
  o[0] = d; o[1] = invd; o[2] = hx; o[3] = dxd;
  float* o32 = g.geo32 + (size_t)t * 4;
  o32[0] = (float)d; o32[1] = (float)invd; o32[2] = (float)hx; o32[3] = (float)dxd;
}

template <int P>
__global__ void k_geometry(DevGeom g, const double* __restrict__ eta) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= g.Nx * (P + 1)) return;
  geometry_item<P>(g, eta, t);
}

// Jacobi diagonal of A = −𝓛: for element-local node (i,j),
//   A_e[(i,j),(i,j)] = Σ_a D_ai² G11_aj + 2 D_ii D_jj G12_ij + Σ_b D_bj² G22_ib,
// summed over the (up to four) elements sharing the node (gather, no atomics).
template <int P>
__global__ void k_diag(DevGeom g) {
  constexpr int Q = P + 1;
  const long long n = (long long)g.ncol * g.nrow;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int col = (int)(t / g.nrow), iz = (int)(t - (long long)col * g.nrow);
  if (iz == g.nrow - 1) { g.invdiag64[t] = 0.0; g.invdiag32[t] = 0.0f; return; }
  const double* D = c_D64 + d_off(P);
  const double* w = c_w64 + w_off(P);
  int exs[2], as[2], ne = 0;
  if (col % P != 0) { exs[0] = col / P; as[0] = col % P; ne = 1; }
  else {
    const int exr = col / P;
    if (exr < g.Nx) { exs[ne] = exr; as[ne] = 0; ++ne; }
    if (g.periodic) { exs[ne] = (exr == 0 ? g.Nx - 1 : exr - 1); as[ne] = P; ++ne; }
    else if (exr >= 1) { exs[ne] = exr - 1; as[ne] = P; ++ne; }
  }
  int ls[2], bs[2], nl = 0;
  { const int l = iz / P, b = iz - l * P;
    if (l < g.Nz) { ls[nl] = l; bs[nl] = b; ++nl; }
    if (b == 0 && l > 0) { ls[nl] = l - 1; bs[nl] = P; ++nl; } }
  double diag = 0.0;
  for (int ie = 0; ie < ne; ++ie) {
    const int ex = exs[ie], i = as[ie];
    const double* geo = g.geo64 + (size_t)ex * Q * 4;
    const double dxe = g.dxe[ex];
    for (int il = 0; il < nl; ++il) {
      const int l = ls[il], j = bs[il];
      const double dsl = g.dsl[l], cx = dsl / dxe, cz = dxe / dsl;
      const double sj = g.sig[l * P + j];
      double s = 0.0;
      for (int a = 0; a < Q; ++a) {                       // Σ_a D_ai² G11_aj
        const double Dai = D[a * Q + i];
        s += Dai * Dai * w[a] * w[j] * cx * geo[a * 4 + 0];
      }
      {                                                    // 2 D_ii D_jj G12_ij
        const double K12 = geo[i * 4 + 2] - sj * geo[i * 4 + 3];
        s += 2.0 * D[i * Q + i] * D[j * Q + j] * w[i] * w[j] * K12;
      }
      for (int b = 0; b < Q; ++b) {                       // Σ_b D_bj² G22_ib
        const double sb = g.sig[l * P + b];
        const double K12 = geo[i * 4 + 2] - sb * geo[i * 4 + 3];
        const double K22 = (1.0 + K12 * K12) * geo[i * 4 + 1];
        const double Dbj = D[b * Q + j];
        s += Dbj * Dbj * w[i] * w[b] * cz * K22;
      }
      diag += s;
    }
  }
  const double inv = 1.0 / diag;
  g.invdiag64[t] = inv;
  g.invdiag32[t] = (float)inv;
}

// ------------------------------------------------------------------------------------
// Shared-memory layout of one CTA and the element-column apply.
// ------------------------------------------------------------------------------------
template <int P, class T>
struct Smem {
  static constexpr int Q = P + 1;
  T* D;     // Q*Q
  T* w;     // Q
  T* sig;   // nrow
  T* cxz;   // E*2*Nz: Δσ_l/Δx_e, Δx_e/Δσ_l of the chunk's element columns
  T* geo;   // E*4*Q
  T* X;     // E*Q*nrow
  T* F1;    // E*Nz*Q*Q
  T* F2;    // E*Nz*Q*Q
  __device__ void carve(unsigned char* base, int nrow, int Nz, int E) {
    T* p = reinterpret_cast<T*>(base);
    D = p; p += Q * Q;
    w = p; p += Q;
    sig = p; p += nrow;
    cxz = p; p += 2 * Nz * E;
    geo = p; p += 4 * Q * E;
    X = p; p += Q * nrow * E;
    F1 = p; p += Nz * Q * Q * E;
    F2 = p;
  }
  __device__ void load_tables(const DevGeom& g) {
    const T* cD = CT<T>::D() + d_off(P);
    const T* cw = CT<T>::w() + w_off(P);
    for (int t = threadIdx.x; t < Q * Q; t += blockDim.x) D[t] = cD[t];
    for (int t = threadIdx.x; t < Q; t += blockDim.x) w[t] = cw[t];
    for (int t = threadIdx.x; t < g.nrow; t += blockDim.x) sig[t] = (T)g.sig[t];
  }
};

template <class T> __device__ __forceinline__ const T* geo_ptr(const DevGeom& g);
template <> __device__ __forceinline__ const double* geo_ptr<double>(const DevGeom& g) { return g.geo64; }
template <> __device__ __forceinline__ const float* geo_ptr<float>(const DevGeom& g) { return g.geo32; }

// Apply A = −𝓛 on the ne consecutive element columns ex0..ex0+ne−1 (a chunk, processed
// together so that small element columns still occupy the CTA).  `loadx(ex,a,iz)` gives the
// input value of local column a, row iz of element column ex; `store(ex,a,iz,y)` receives the
// element column's contribution.  Returns this thread's share of Σ x·(A_e x) over the chunk
// (accumulated in T).
// Geometric factors of the σ-transformed operator at element-local node (a, b) of layer l:
// G11 = w_a w_b (Δσ/Δx) d, G12 = w_a w_b K12, G22 = w_a w_b (Δx/Δσ) (1 + K12²)/d, K12 = ∂xh − σ ∂xd.
template <class T>
__device__ __forceinline__ void geo_factors(T d, T invd, T hx, T dxd, T cz0, T cz1, T wa, T wb, T sig, T& G11,
                                            T& G12, T& G22) {
  const T wab = wa * wb;
  const T K12 = hx - sig * dxd;
  const T K22 = fmx(K12, K12, (T)1) * invd;
  G11 = wab * cz0 * d;
  G12 = wab * K12;
  G22 = wab * cz1 * K22;
}

// The factors of every element-local node of the CTA's element columns R.e0..R.e1−1, three per
// node in the order of the apply's work items; FP64, computed as in apply_element_chunk.
template <int P>
__device__ void fill_gcache(const DevGeom& g, int e0, int e1, double* gc) {
  constexpr int Q = P + 1;
  const int elsz = g.Nz * Q * Q;
  const double* w = c_w64 + w_off(P);
  for (int t = threadIdx.x; t < (e1 - e0) * elsz; t += blockDim.x) {
    const int e = g.dv_elsz.div(t), rem0 = t - e * elsz;
    const int l = rem0 / (Q * Q), rem = rem0 - l * (Q * Q), a = rem / Q, b = rem - a * Q;
    const int ge = e0 + e;
    const double* geo = g.geo64 + (size_t)ge * Q * 4 + a * 4;
    const double* cz = g.cxz + ((size_t)ge * g.Nz + l) * 2;   // the layer's ratios, not a division per node
    double G11, G12, G22;
    geo_factors<double>(geo[0], geo[1], geo[2], geo[3], cz[0], cz[1], w[a], w[b], g.sig[l * P + b], G11, G12, G22);
    gc[3 * t] = G11;
    gc[3 * t + 1] = G12;
    gc[3 * t + 2] = G22;
  }
}

// gc (FP64 only, optional): the chunk's geometric factors from fill_gcache, used instead of
// staging the geometry and recomputing them.
// TOP: only the top element layer (an input that is zero below the surface row, whose image is zero
// below the top layer's lowest row): rows under that row get no store.
template <int P, class T, bool TOP = false, class LoadX, class Store>
__device__ __forceinline__ T apply_element_chunk(const DevGeom& g, Smem<P, T>& s, int ex0, int ne,
                                                 LoadX loadx, Store store, const double* gc = nullptr) {
  constexpr int Q = P + 1;
  const int nrow = g.nrow, Nz = g.Nz;
  const int colsz = Q * nrow, elsz = Nz * Q * Q;
  const int l_first = TOP ? Nz - 1 : 0;   // first layer computed
  const int nl = Nz - l_first;
  if (gc == nullptr) {
    const T* geo = geo_ptr<T>(g) + (size_t)ex0 * Q * 4;
    for (int t = threadIdx.x; t < ne * 4 * Q; t += blockDim.x) s.geo[t] = geo[t];
    const double* cz = g.cxz + (size_t)ex0 * Nz * 2;
    for (int t = threadIdx.x; t < ne * Nz * 2; t += blockDim.x) s.cxz[t] = (T)cz[t];
  }
  for (int t = threadIdx.x; t < ne * colsz; t += blockDim.x) {
    const int e = g.dv_colsz.div(t), rem = t - e * colsz;
    const int a = g.dv_nrow.div(rem), iz = rem - a * nrow;
    s.X[t] = loadx(ex0 + e, a, iz);
  }
  __syncthreads();
  for (int tt = threadIdx.x; tt < ne * nl * Q * Q; tt += blockDim.x) {
    int t = tt;
    if constexpr (TOP) {   // layer l_first of element e: its items in the full numbering
      const int e = tt / (Q * Q);
      t = e * elsz + l_first * Q * Q + (tt - e * Q * Q);
    }
    const int e = g.dv_elsz.div(t), rem0 = t - e * elsz;
    const int l = rem0 / (Q * Q), rem = rem0 - l * (Q * Q), a = rem / Q, b = rem - a * Q;
    const T* Xe = s.X + e * colsz;
    const T* Xrow = Xe + l * P + b;              // Xrow[c*nrow]: row l·P+b, column c
    const T* Xcol = Xe + a * nrow + l * P;       // Xcol[c]: column a, row l·P+c
    const T* Da = s.D + a * Q;
    const T* Db = s.D + b * Q;
    T ur = 0, ut = 0;
#pragma unroll
    for (int c = 0; c < Q; ++c) {
      ur = fmx(Da[c], Xrow[c * nrow], ur);
      ut = fmx(Db[c], Xcol[c], ut);
    }
    T G11, G12, G22;
    if (gc != nullptr) {
      G11 = (T)gc[3 * t];
      G12 = (T)gc[3 * t + 1];
      G22 = (T)gc[3 * t + 2];
    } else {
      const T* ge = s.geo + e * 4 * Q + a * 4;
      const T* cz = s.cxz + 2 * (e * Nz + l);
      geo_factors<T>(ge[0], ge[1], ge[2], ge[3], cz[0], cz[1], s.w[a], s.w[b], s.sig[l * P + b], G11, G12, G22);
    }
    s.F1[t] = fmx(G11, ur, G12 * ut);
    s.F2[t] = fmx(G12, ur, G22 * ut);
  }
  __syncthreads();
  T part = 0;
  for (int t = threadIdx.x; t < ne * colsz; t += blockDim.x) {
    const int e = g.dv_colsz.div(t), rem = t - e * colsz;
    const int a = g.dv_nrow.div(rem), iz = rem - a * nrow;
    const int l = iz / P, b = iz - l * P;
    if (TOP && l < l_first) continue;
    const T* F1e = s.F1 + e * elsz;
    const T* F2e = s.F2 + e * elsz;
    T y = 0;
    if (l < Nz) {
      const T* F1 = F1e + (l * Q) * Q + b;       // F1[(l*Q+a')*Q+b] = F1[a'*Q]
      const T* F2 = F2e + (l * Q + a) * Q;       // F2[(l*Q+a)*Q+b']
#pragma unroll
      for (int c = 0; c < Q; ++c) {
        y = fmx(s.D[c * Q + a], F1[c * Q], y);
        y = fmx(s.D[c * Q + b], F2[c], y);
      }
    }
    if (b == 0 && l > l_first) {
      const int lm = l - 1;
      const T* F1 = F1e + (lm * Q) * Q + P;
      const T* F2 = F2e + (lm * Q + a) * Q;
#pragma unroll
      for (int c = 0; c < Q; ++c) {
        y = fmx(s.D[c * Q + a], F1[c * Q], y);
        y = fmx(s.D[c * Q + P], F2[c], y);
      }
    }
    store(ex0 + e, a, iz, y);
    part = fmx(s.X[t], y, part);
  }
  __syncthreads();
  return part;
}

// ------------------------------------------------------------------------------------
// Stand-alone apply: y = 𝓛x (two kernels: element columns, then the edge columns).
// ------------------------------------------------------------------------------------
template <int P>
__global__ void __launch_bounds__(kThreads) k_apply(DevGeom g, const double* __restrict__ x,
                                                    double* __restrict__ q, double* __restrict__ edge) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem<P, double> s;
  s.carve(smem_raw, g.nrow, g.Nz, g.chunk);
  s.load_tables(g);
  __syncthreads();
  const int nrow = g.nrow, E = g.chunk;
  for (int ex0 = blockIdx.x * E; ex0 < g.Nx; ex0 += gridDim.x * E) {
    apply_element_chunk<P, double>(
        g, s, ex0, min(E, g.Nx - ex0),
        [&](int e, int a, int iz) { return x[(size_t)col_of(g, e, a) * nrow + iz]; },
        [&](int e, int a, int iz, double y) {
          if (a < P || (!g.periodic && e == g.Nx - 1)) q[(size_t)col_of(g, e, a) * nrow + iz] = y;
          else edge[(size_t)e * nrow + iz] = y;
        });
  }
}




}  // namespace semgb

#include "apply_tile.cuh"
#include "apply_tc.cuh"

namespace semgb {

// ------------------------------------------------------------------------------------
// Grid barrier for the cooperative kernel, with a wall-clock limit.
// ------------------------------------------------------------------------------------

// A team of CTAs that synchronise among themselves: the whole grid for one mesh, or the CTAs
// assigned to one instance of a batch.
struct Team {
  int rank, size;        // this CTA's index in the team, number of CTAs
  unsigned int* bar;     // arrival counter (and one spare word), zero at launch
  int* status;           // device status word of the instance
  double* part;          // reduction partials [4 slots][4 values][stride]
  int stride;
  unsigned long long timeout_ns;   // limit of each barrier wait (2 s unless a test sets it)
  int cluster;           // 1: the team is one thread-block cluster (hardware cluster barrier)
};

// Barrier of every thread of a thread-block cluster, with release/acquire at cluster scope: the
// writes of every CTA of the cluster before it (global and shared memory) are visible to every
// CTA after it.  Executed by all threads of every CTA of the cluster.
static __device__ __forceinline__ void cluster_barrier() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Returns false (and sets ST_TIMEOUT) if the other CTAs of the team did not arrive in time;
// the caller must then return without touching another barrier.
// The arrival counter only grows during a launch: the n-th barrier of the launch is passed once
// it reaches n·size, so the last arrival's own increment releases the waiters (one round trip
// to L2 fewer than a separate generation word).  Arrivals are acquire-release RMWs, waiters poll
// with acquire loads; successive RMWs extend each arrival's release sequence, so a waiter that
// reads n·size has acquired every CTA's writes before its arrival.  The CTA's own writes are
// ordered before thread 0's arrival by the __syncthreads that precedes it; after the wait, the
// closing __syncthreads orders the other CTAs' writes before every thread of this CTA.
static __device__ __forceinline__ unsigned bar_arrive(unsigned* p) {
  unsigned old;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;" : "=r"(old) : "l"(p) : "memory");
  return old;
}
static __device__ __forceinline__ unsigned bar_load(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

#ifdef SEM_TRACE
static __device__ __forceinline__ void trace_mark(const DevGeom& g, const Team& tm, int tag) {
  if (threadIdx.x == 0 && tm.rank == 0 && g.trace) {
    const unsigned long long n = g.trace[0];
    if (n < (unsigned long long)kTraceMax) {
      g.trace[1 + 2 * n] = (unsigned long long)tag;
      g.trace[2 + 2 * n] = global_ns();
      g.trace[0] = n + 1;
    }
  }
}
#define SEM_MARK(g, tm, tag) trace_mark(g, tm, tag)
#else
#define SEM_MARK(g, tm, tag) ((void)0)
#endif

static __device__ __forceinline__ bool grid_barrier(const Team& tm, int* s_flag) {
  if (tm.cluster && tm.size > 1) {
    cluster_barrier();
    return true;
  }
  __syncthreads();
  if (tm.size == 1) return true;
  if (threadIdx.x == 0) {
    const unsigned size = (unsigned)tm.size;
    const unsigned prev = bar_arrive(tm.bar);
    const unsigned target = prev - prev % size + size;   // arrivals that complete this barrier
    int ok = 1;
    if (prev + 1 != target) {
      const unsigned long long t0 = global_ns();
      unsigned int spins = 0;
      while (bar_load(tm.bar) < target) {
        if ((++spins & 63u) == 0 && global_ns() - t0 > tm.timeout_ns) {
          atomicOr(tm.status, ST_TIMEOUT);
          ok = 0;
          break;
        }
        __nanosleep(20);
      }
    }
    *s_flag = ok;
  }
  __syncthreads();
  return *s_flag != 0;
}

// Shared reduction buffer of the persistent kernels: K·blockDim partials of block_sum, then the
// block sums and the grid sums.
constexpr int kRedOut = 4 * kThreads, kRedGrid = kRedOut + 8, kRedSize = kRedGrid + 8;

// Deterministic block sum of K ≤ 4 values of type A (all threads get the result).  The values go
// to shared memory and warp k adds up value k (lane j: threads j, j + 32, …, then a shuffle
// tree), so the K sums run on different SM sub-partitions.  FP64 adds issue slowly on this
// GPU; a shuffle tree in every warp would issue about eight times as many.
template <int K, class A>
__device__ __forceinline__ void block_sum(A (&v)[K], double* red) {
  A* rr = reinterpret_cast<A*>(red);
  const int nt = blockDim.x, tid = threadIdx.x, wid = tid >> 5, lane = tid & 31;
  __syncthreads();                               // earlier readers of the buffer are done
#pragma unroll
  for (int k = 0; k < K; ++k) rr[k * nt + tid] = v[k];
  __syncthreads();
  if (wid < K) {
    const A* row = rr + wid * nt;
    A s = A(0);
    for (int j = lane; j < nt; j += 32) s += row[j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) red[kRedOut + wid] = (double)s;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < K; ++k) v[k] = (A)red[kRedOut + k];
}

// Sum of K per-CTA partials part[slot][k][cta] over all CTAs, same order in every CTA; warp k
// sums value k.
template <int K>
__device__ __forceinline__ void grid_sum(const Team& tm, int slot, double (&v)[K], double* red) {
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (wid < K) {
    const double* p = tm.part + ((size_t)slot * 4 + wid) * tm.stride;
    double s = 0.0;
    for (int c = lane; c < tm.size; c += 32) s += __ldcg(p + c);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) red[kRedGrid + wid] = s;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < K; ++k) v[k] = red[kRedGrid + k];
  __syncthreads();
}

template <int K, class A>
__device__ __forceinline__ void put_partials(const Team& tm, int slot, const A (&v)[K]) {
  if (threadIdx.x == 0)
#pragma unroll
    for (int k = 0; k < K; ++k) tm.part[((size_t)slot * 4 + k) * tm.stride + tm.rank] = (double)v[k];
}

// ------------------------------------------------------------------------------------
// Persistent preconditioned CG.  One level (FP64) or two levels (FP32 inner, FP64
// residual refinement).
// ------------------------------------------------------------------------------------
struct Range { int e0, e1, c0, c1; };   // owned element columns and global columns

static __device__ __forceinline__ Range my_range(const DevGeom& g, const Team& tm) {
  Range r;
  r.e0 = (int)(((long long)tm.rank * g.Nx) / tm.size);
  r.e1 = (int)(((long long)(tm.rank + 1) * g.Nx) / tm.size);
  r.c0 = r.e0 * g.P;
  r.c1 = r.e1 * g.P + ((!g.periodic && r.e1 == g.Nx) ? 1 : 0);
  return r;
}

static __device__ __forceinline__ bool owns_local_col(const DevGeom& g, int ex, int a) {
  return a < g.P || (!g.periodic && ex == g.Nx - 1);
}

// ---- σ-separable preconditioner ----------------------------------------------------
// M⁻¹ = (I⊗S) [Kx(d) ⊗ I + Mx(1/d) ⊗ Λ]⁻¹ (I⊗Sᵀ), the exact inverse of the Kronecker-sum
// operator obtained from A by dropping the K12 (slope) coupling and the K12² part of K22.
// Kx(d) = Σ_e (2/Δx) Dᵀ diag(w d) D and Mx(1/d) = Σ_e (Δx/2) diag(w/d) are 1D operators in x
// (periodic or walls); Kσ S = Mσ S Λ is the generalized eigenproblem of the 1D σ stiffness
// (Dirichlet at the surface) against the GLL-lumped σ mass.  Each σ-mode is a 1D SEM problem
// in x, solved by static condensation of the element interiors and a tridiagonal (cyclic)
// interface system.

// Vectors of one Krylov level (type T).  Owned-column values live in the global arrays; `uh`
// holds M⁻¹r on this CTA's halo column (the first column of the next CTA), which each CTA
// rebuilds itself so that no barrier separates the preconditioner from the next apply.
template <class T>
struct CgVecs {
  T* x;              // solution (FP64 level) or correction (FP32 level)
  T* r[2];           // residual, double-buffered
  T* s[2];           // s = A p, double-buffered
  T* p;              // search direction (owned columns only)
  T* u;              // u = M⁻¹ r (owned columns)
  T* uh;             // u on the CTA's halo column, [grid][nrow]
  T* w;              // w = A u (owned columns)
  T* edge;           // A u contribution to the next element column's first column
  const T* invdiag;  // Jacobi preconditioner
};

static __device__ __forceinline__ bool is_halo_col(const DevGeom& g, const Range& R, int ex, int a) {
  return a == g.P && ex == R.e1 - 1 && !owns_local_col(g, ex, g.P);
}

// o[q] = Σ_j M[j·nr + c0 + q] x[j], j < nr, for four consecutive columns c0..c0+3 of the nr×nr
// matrix M: each x[j] is loaded once for the four, and when nr is a multiple of 4 the four M
// values are one 16-byte load (the rows are then 16-byte aligned).  Columns past nr are read at
// nr − 1 and their sums are meaningless (the caller drops them).  One chain per column, j in order.
template <class TP>
__device__ __forceinline__ void dot_cols4(const TP* M, int nr, int c0, const TP* x, TP (&o)[4]) {
  o[0] = o[1] = o[2] = o[3] = TP(0);
  if constexpr (sizeof(TP) == 4) {
    if ((nr & 3) == 0) {
      const float4* M4 = reinterpret_cast<const float4*>(M + c0);
      const int s4 = nr >> 2;
      for (int j = 0; j < nr; ++j) {
        const float4 m = M4[j * s4];
        const float xj = x[j];
        o[0] = fmaf(m.x, xj, o[0]);
        o[1] = fmaf(m.y, xj, o[1]);
        o[2] = fmaf(m.z, xj, o[2]);
        o[3] = fmaf(m.w, xj, o[3]);
      }
      return;
    }
  }
  const int c1 = min(c0 + 1, nr - 1), c2 = min(c0 + 2, nr - 1), c3 = min(c0 + 3, nr - 1);
  for (int j = 0; j < nr; ++j) {
    const TP* Mj = M + j * nr;
    const TP xj = x[j];
    o[0] = fmx(Mj[c0], xj, o[0]);
    o[1] = fmx(Mj[c1], xj, o[1]);
    o[2] = fmx(Mj[c2], xj, o[2]);
    o[3] = fmx(Mj[c3], xj, o[3]);
  }
}

// Update of the Chronopoulos–Gear recurrences on owned nodes (and, for r, on the halo column),
// then the first part of u = M⁻¹ r:
//   s ← w + β s,  r ← r − α s,  p ← u + β p,  x ← x + α p      (first iteration: s ← w, p ← u).
// With update == false only the preconditioner part runs on r[cur].  Jacobi completes u here;
// the separable preconditioner transforms the residual to the σ-eigenbasis and condenses.
// ILP (compile time, the one-CTA-per-SM build, which has the registers): two items per thread
// and pass with their loads issued together.
template <int P, class T, class TP, bool ILP = false>
__device__ void cg_update(const DevGeom& g, Smem<P, T>& s, const Range& R, const Team& tm,
                          const PrecView<TP>& pv, int precond, const CgVecs<T>& V, int cur, bool update,
                          bool first, T alpha, T beta) {
  constexpr int Q = P + 1, Pm = P - 1;
  const int nrow = g.nrow, nr = nrow - 1;
  const T* r_old = V.r[cur];
  T* r_new = V.r[cur ^ 1];
  const T* s_old = V.s[cur];
  T* s_new = V.s[cur ^ 1];
  // the preconditioner works in TP (FP32 also under FP64 vectors); its staging buffers reuse
  // the apply's shared memory, which holds at least as many values of type T
  TP* X = reinterpret_cast<TP*>(s.X);     // [E][Q][nr] residual of the chunk's element columns
  TP* RH = reinterpret_cast<TP*>(s.F1);   // [E][Q][nr] σ-transformed residual
  const int E = g.chunk, qn = Q * nr;
  // U items per thread and pass: all their loads are issued before any of their stores, so that
  // the L2 round trips of consecutive items overlap (a store to the vectors could alias the next
  // item's loads, which the compiler would otherwise leave behind it)
  constexpr int U = ILP ? 2 : 1;
  for (int ex0 = R.e0; ex0 < R.e1; ex0 += E) {
    const int ne = min(E, R.e1 - ex0), nt = ne * qn;
    for (int t0 = threadIdx.x; t0 < nt; t0 += U * blockDim.x) {
      T wv[U], so[U], ro[U], uo[U], po[U], xo[U];
      int ia[U];                                   // the item's (e, a, j), packed
      bool own[U];
#pragma unroll
      for (int q = 0; q < U; ++q) {
        const int t = t0 + q * blockDim.x;
        if (t >= nt) continue;
        const int e = g.dv_qn.div(t), rem = t - e * qn;
        const int a = g.dv_nr.div(rem), j = rem - a * nr, ex = ex0 + e;
        const int col = col_of(g, ex, a);
        const size_t i = (size_t)col * nrow + j;
        ia[q] = rem;
        own[q] = owns_local_col(g, ex, a);
        ro[q] = ldcg(r_old + i);
        if (update) {
          wv[q] = ldcg(V.w + i);
          if (has_left_edge_p<P>(g, col)) wv[q] += ldcg(V.edge + (size_t)left_element_p<P>(g, col) * nrow + j);
          so[q] = first ? T(0) : ldcg(s_old + i);
          if (own[q]) {
            uo[q] = V.u[i];
            po[q] = first ? T(0) : V.p[i];
            xo[q] = V.x[i];
          }
        }
      }
#pragma unroll
      for (int q = 0; q < U; ++q) {
        const int t = t0 + q * blockDim.x;
        if (t >= nt) continue;
        const int e = g.dv_qn.div(t), a = g.dv_nr.div(ia[q]), j = ia[q] - a * nr, ex = ex0 + e;
        const size_t i = (size_t)col_of(g, ex, a) * nrow + j;
        T rv = ro[q];
        if (update) {
          const T sv = first ? wv[q] : fmx(beta, so[q], wv[q]);
          rv = fmx(-alpha, sv, ro[q]);
          if (own[q]) {
            s_new[i] = sv;
            r_new[i] = rv;
            const T pn = first ? uo[q] : fmx(beta, po[q], uo[q]);
            V.p[i] = pn;
            V.x[i] = fmx(alpha, pn, xo[q]);
          }
        }
        if (precond == PREC_JACOBI) {
          const T uv = rv * V.invdiag[i];
          if (own[q]) V.u[i] = uv;
          else if (is_halo_col(g, R, ex, a)) V.uh[(size_t)tm.rank * nrow + j] = uv;
        } else {
          X[t] = (TP)rv;
        }
      }
    }
    if (precond == PREC_JACOBI) continue;
    __syncthreads();
    SEM_MARK(g, tm, TR_UPD_VEC);
    // r̂ = Sᵀ r per element-local column, four modes per thread
    const int nq = (nr + 3) >> 2;
    for (int t = threadIdx.x; t < ne * Q * nq; t += blockDim.x) {
      const int ea = t / nq, k0 = (t - ea * nq) * 4;
      const int e = ea / Q, a = ea - e * Q, ex = ex0 + e;
      TP v[4];
      dot_cols4<TP>(pv.S, nr, k0, X + e * qn + a * nr, v);
      const bool own = owns_local_col(g, ex, a);
      TP* rh = pv.rhat + (size_t)col_of(g, ex, a) * nr;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int k = k0 + q;
        if (k >= nr) break;
        RH[e * qn + a * nr + k] = v[q];
        if (own) rh[k] = v[q];
      }
    }
    __syncthreads();
    SEM_MARK(g, tm, TR_UPD_SIGMA);
    for (int t = threadIdx.x; t < ne * nr; t += blockDim.x) {
      const int e = g.dv_nr.div(t), k = t - e * nr, ex = ex0 + e;
      const TP* RHe = RH + e * qn;
      const TP* Zl = pv.Z + (size_t)ex * 2 * Pm * nr + k;   // Zl[m·nr]: left row, Zl[(Pm + m)·nr]: right
      // the assembled residual at an interface node enters once: with the element that owns
      // that column (its left end), plus the walls' last column with the last element
      TP l = RHe[k], r = owns_local_col(g, ex, P) ? RHe[P * nr + k] : TP(0);
#pragma unroll
      for (int m = 0; m < Pm; ++m) {
        const TP f = RHe[(1 + m) * nr + k];
        l = fmx(-Zl[m * nr], f, l);
        r = fmx(-Zl[(Pm + m) * nr], f, r);
      }
      pv.gL[(size_t)k * g.Nx + ex] = l;
      pv.gR[(size_t)k * g.Nx + ex] = r;
    }
    __syncthreads();
    SEM_MARK(g, tm, TR_UPD_COND);
  }
}

// Interface solve per σ-mode: one warp (warp 0 of a CTA) per mode, or the whole CTA for long
// systems, modes spread over CTAs;
// g_j = gL_j + gR_{j−1} assembled on the fly, then the warp-parallel tridiagonal solve.
template <class T, bool CACHE = false>
__device__ void phase_interface(const DevGeom& g, const PrecView<T>& pv, const Team& tm) {
  const int N = pv.nif, Nx = g.Nx;
  const bool whole_cta = N > 32 * kTridiagRegs;   // long systems: all warps of the CTA per mode
  // short systems: one warp per mode, the modes spread over the team's CTAs and their warps
  const int w = whole_cta ? 0 : (int)(threadIdx.x >> 5), nw = whole_cta ? 1 : (int)(blockDim.x >> 5);
  for (int k = tm.rank + tm.size * w; k < pv.nr; k += tm.size * nw) {
    const T* gl = pv.gL + (size_t)k * Nx;
    const T* gr = pv.gR + (size_t)k * Nx;
    auto gfun = [&](int j) -> T {
      if (g.periodic) return ldcg(gl + j) + ldcg(gr + (j == 0 ? Nx - 1 : j - 1));
      return (j < Nx ? ldcg(gl + j) : T(0)) + (j > 0 ? ldcg(gr + j - 1) : T(0));
    };
    if (whole_cta)
      cta_tridiag<T, decltype(gfun), CACHE>(N, gfun, pv.te + (size_t)k * N, pv.tm + (size_t)k * N, pv.tcp + (size_t)k * N,
                     g.periodic != 0, pv.tz + (size_t)k * N, g.periodic ? pv.tvl[k] : T(0),
                     g.periodic ? pv.tfac[k] : T(0), pv.zb + (size_t)k * N);
    else
      warp_tridiag<T>(N, gfun, pv.te + (size_t)k * N, pv.tm + (size_t)k * N, pv.tcp + (size_t)k * N,
                      g.periodic != 0, pv.tz + (size_t)k * N, g.periodic ? pv.tvl[k] : T(0),
                      g.periodic ? pv.tfac[k] : T(0), pv.zb + (size_t)k * N);
  }
}

// Back-substitution of the element interiors, then u = S ẑ on owned columns and on the halo
// column (whose modal values are interface unknowns, known to every CTA after the solve).
template <int P, class T, class TP>
__device__ void phase_backsub(const DevGeom& g, Smem<P, T>& s, const Range& R, const Team& tm,
                              const PrecView<TP>& pv, const CgVecs<T>& V) {
  constexpr int Q = P + 1, Pm = P - 1;
  const int nrow = g.nrow, nr = pv.nr, N = pv.nif;
  TP* ZH = reinterpret_cast<TP*>(s.F1);   // [E][Q][nr]
  const int E = g.chunk, qn = Q * nr;
  for (int ex0 = R.e0; ex0 < R.e1; ex0 += E) {
    const int ne = min(E, R.e1 - ex0);
    // chunks with few (element, mode) pairs (under a quarter of the threads; a one-element chunk of a
    // C2-like column): one (element, column, mode) per thread
    const bool by_row = ne * nr * 4 < (int)blockDim.x;
    if (by_row) {
      for (int t = threadIdx.x; t < ne * qn; t += blockDim.x) {
        const int e = g.dv_qn.div(t), rem = t - e * qn;
        const int a = g.dv_nr.div(rem), k = rem - a * nr, ex = ex0 + e;
        TP v;
        if (a == 0) v = ldcg(pv.zb + (size_t)k * N + ex);
        else if (a == P) v = ldcg(pv.zb + (size_t)k * N + ((ex + 1 == N) ? 0 : ex + 1));
        else {
          const int i = a - 1;
          const TP zl = ldcg(pv.zb + (size_t)k * N + ex);
          const TP zr = ldcg(pv.zb + (size_t)k * N + ((ex + 1 == N) ? 0 : ex + 1));
          const TP* Ai = pv.Aii + ((size_t)ex * Pm + i) * Pm * nr + k;   // Ai[m·nr]
          const TP* Zl = pv.Z + (size_t)ex * 2 * Pm * nr + k;
          v = 0;
#pragma unroll
          for (int m = 0; m < Pm; ++m) v = fmx(Ai[m * nr], pv.rhat[(size_t)(ex * P + 1 + m) * nr + k], v);
          v = fmx(-Zl[i * nr], zl, v);
          v = fmx(-Zl[(Pm + i) * nr], zr, v);
        }
        ZH[t] = v;
      }
    }
    // otherwise one (element, mode) per thread: the element's interior values of the mode from
    // the condensed residual and the two interface values, each loaded once for all P−1 rows
    // (the same sums in the same order either way)
    for (int t = threadIdx.x; !by_row && t < ne * nr; t += blockDim.x) {
      const int e = g.dv_nr.div(t), k = t - e * nr, ex = ex0 + e;
      const int jr = (ex + 1 == N) ? 0 : ex + 1;
      const TP zl = ldcg(pv.zb + (size_t)k * N + ex);
      const TP zr = ldcg(pv.zb + (size_t)k * N + jr);
      TP rh[Pm];
#pragma unroll
      for (int m = 0; m < Pm; ++m) rh[m] = pv.rhat[(size_t)(ex * P + 1 + m) * nr + k];
      TP* zh = ZH + e * qn + k;
      zh[0] = zl;
      zh[P * nr] = zr;
      const TP* Zl = pv.Z + (size_t)ex * 2 * Pm * nr + k;
#pragma unroll
      for (int i = 0; i < Pm; ++i) {
        const TP* Ai = pv.Aii + ((size_t)ex * Pm + i) * Pm * nr + k;   // Ai[m·nr]
        TP v = 0;
#pragma unroll
        for (int m = 0; m < Pm; ++m) v = fmx(Ai[m * nr], rh[m], v);
        v = fmx(-Zl[i * nr], zl, v);
        v = fmx(-Zl[(Pm + i) * nr], zr, v);
        zh[(1 + i) * nr] = v;
      }
    }
    __syncthreads();
    SEM_MARK(g, tm, TR_BS_INTERIOR);
    // u = S ẑ per element-local column, four rows per thread (threads of consecutive row quads
    // read consecutive words of Sᵀ)
    const int nq = (nr + 3) >> 2;
    for (int t = threadIdx.x; t < ne * Q * nq; t += blockDim.x) {
      const int ea = t / nq, j0 = (t - ea * nq) * 4;
      const int e = ea / Q, a = ea - e * Q, ex = ex0 + e;
      const bool own = owns_local_col(g, ex, a);
      const bool halo = is_halo_col(g, R, ex, a);
      if (!own && !halo) continue;
      TP v[4];
      dot_cols4<TP>(pv.ST, nr, j0, ZH + e * qn + a * nr, v);
      T* dst = own ? V.u + (size_t)col_of(g, ex, a) * nrow : V.uh + (size_t)tm.rank * nrow;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int j = j0 + q;
        if (j >= nr) break;
        dst[j] = (T)v[q];
      }
    }
    __syncthreads();
    SEM_MARK(g, tm, TR_BS_SIGMA);
  }
}

// Remaining grid phases of u = M⁻¹ r after cg_update (separable: interface solve and
// back-substitution; Jacobi: nothing but a barrier that protects w and edge).
template <int P, class T, class TP, bool CACHE = false>
__device__ bool finish_precondition(const DevGeom& g, Smem<P, T>& s, const Range& R, const Team& tm,
                                    const PcgArgs& PA, const PrecView<TP>& pv, const CgVecs<T>& V, int* s_flag) {
  if (PA.precond == PREC_JACOBI) return grid_barrier(tm, s_flag);
  if (!grid_barrier(tm, s_flag)) return false;
  SEM_MARK(g, tm, TR_IT_BAR2);
  phase_interface<TP, CACHE>(g, pv, tm);
  SEM_MARK(g, tm, TR_IT_INTERFACE);
  if (!grid_barrier(tm, s_flag)) return false;
  SEM_MARK(g, tm, TR_IT_BAR3);
  phase_backsub<P, T, TP>(g, s, R, tm, pv, V);
  return true;
}

// Preconditioned conjugate gradients in the Chronopoulos–Gear form: one grid reduction per
// iteration, (γ, δ, ‖r‖²) = ((r,u), (u,Au), (r,r)) taken together with the apply w = A u.
//   β = γ/γ_prev, α = γ/(δ − βγ/α_prev)  (first: β = 0, α = γ/δ).
// Starts from V.x with its residual in V.r[0].  Stops when ‖r‖² ≤ target or after max_it
// iterations.  Returns the iterations, or −1 on a barrier timeout; ‖r‖² of the final residual
// (on thread 0) in *rr_out.
template <int P, class T, class A, class TP, bool CACHE = false>
__device__ int cg_solve(const DevGeom& g, Smem<P, T>& s, const Range& R, const Team& tm, const PcgArgs& PA,
                        const PrecView<TP>& pv, const CgVecs<T>& V, double target, int max_it, double* red,
                        int* s_flag, double* rr_out, const double* gc = nullptr) {
  const int nrow = g.nrow;
  __shared__ T s_scal[2];
  __shared__ int s_stop;
  int cur = 0;
  SEM_MARK(g, tm, TR_CG_START);
  cg_update<P, T, TP, CACHE>(g, s, R, tm, pv, PA.precond, V, cur, false, true, T(0), T(0));
  if (!finish_precondition<P, T, TP, CACHE>(g, s, R, tm, PA, pv, V, s_flag)) return -1;
  SEM_MARK(g, tm, TR_IT_BACKSUB);
  int k = 0;
  double rr = 0.0;
  // 1/γ and 1/α of the last iteration, double-buffered by iteration parity: thread 32 (another SM
  // sub-partition, so another FP64 pipe) divides for the next iteration while thread 0 divides for α
  __shared__ double s_inv[2][2];
  while (true) {
    // w = A u and the three inner products (u on owned columns and the halo column)
    const T* rc = V.r[cur];
    A acc[3] = {A(0), A(0), A(0)};   // γ = (r,u), δ = (u,Au), (r,r)
    for (int ex0 = R.e0; ex0 < R.e1; ex0 += g.chunk) {
      const double* gce = gc ? gc + (size_t)(ex0 - R.e0) * 3 * g.Nz * (P + 1) * (P + 1) : nullptr;
      acc[1] += (A)apply_element_chunk<P, T>(
          g, s, ex0, min(g.chunk, R.e1 - ex0),
          [&](int e, int a, int iz) -> T {
            if (iz == nrow - 1) return T(0);
            if (is_halo_col(g, R, e, a)) return V.uh[(size_t)tm.rank * nrow + iz];
            const size_t i = (size_t)col_of(g, e, a) * nrow + iz;
            const T uv = V.u[i];
            if (owns_local_col(g, e, a)) {
              const T rv = rc[i];
              acc[0] += (A)rv * (A)uv;
              acc[2] += (A)rv * (A)rv;
            }
            return uv;
          },
          [&](int e, int a, int iz, T y) {
            if (owns_local_col(g, e, a)) V.w[(size_t)col_of(g, e, a) * nrow + iz] = y;
            else V.edge[(size_t)e * nrow + iz] = y;
          },
          gce);
    }
    block_sum<3, A>(acc, red);
    put_partials<3, A>(tm, 2, acc);
    SEM_MARK(g, tm, TR_IT_APPLY);
    if (!grid_barrier(tm, s_flag)) return -1;
    SEM_MARK(g, tm, TR_IT_BAR1);
    double sums[3];
    grid_sum<3>(tm, 2, sums, red);
    if (threadIdx.x == 32) {
      const double gam = sums[0], del = sums[1];
      const double* ip = s_inv[(k + 1) & 1];
      const double beta = k == 0 ? 0.0 : gam * ip[0];
      const double den = k == 0 ? del : del - beta * gam * ip[1];
      const double ig = 1.0 / gam;
      s_inv[k & 1][0] = ig;
      s_inv[k & 1][1] = den * ig;
    }
    if (threadIdx.x == 0) {
      rr = sums[2];
      int stop = 0;
      if (!(rr == rr) || isinf(rr) || !(sums[1] == sums[1])) { atomicOr(g.status, ST_NONFINITE); stop = 1; }
      else if (rr <= target || k >= max_it) stop = 1;
      if (!stop) {
        // α = γ/(δ − βγ/α_prev); thread 32 takes the next iteration's 1/γ and 1/α = den/γ
        const double gam = sums[0], del = sums[1];
        const double* ip = s_inv[(k + 1) & 1];
        const double beta = k == 0 ? 0.0 : gam * ip[0];
        const double den = k == 0 ? del : del - beta * gam * ip[1];
        const double alpha = gam / den;
        s_scal[0] = (T)alpha;
        s_scal[1] = (T)beta;
      }
      s_stop = stop;
    }
    __syncthreads();
    SEM_MARK(g, tm, TR_IT_SCALARS);
    if (s_stop) break;
    const T alpha = s_scal[0], beta = s_scal[1];
    cg_update<P, T, TP, CACHE>(g, s, R, tm, pv, PA.precond, V, cur, true, k == 0, alpha, beta);
    cur ^= 1;
    SEM_MARK(g, tm, TR_IT_UPDATE);
    if (!finish_precondition<P, T, TP, CACHE>(g, s, R, tm, PA, pv, V, s_flag)) return -1;
    SEM_MARK(g, tm, TR_IT_BACKSUB);
    ++k;
  }
  SEM_MARK(g, tm, TR_CG_END);
  *rr_out = rr;
  return k;
}

// FP64 residual r = b − A_II x = −(A [x; φ̃])_I on owned nodes, with ‖b‖² when asked
// (b = −(A [0; φ̃])_I).  Returns false on a barrier timeout; rr (and bb) summed on return.
template <int P>
__device__ bool fp64_residual(const DevGeom& g, Smem<P, double>& s, const Range& R, const Team& tm,
                              const PcgArgs& A, bool want_b, double* red, int* s_flag, double& rr, double& bb,
                              double* dx = nullptr, const double* gc = nullptr, float* d32 = nullptr,
                              float* r32 = nullptr) {
  // dx (optional): on exit dx[0] = ‖δ‖² of the correction d32 and dx[1] = ‖x‖² over the whole team
  // (interior nodes).
  // d32 (optional, mixed precision): the FP32 correction of the last inner solve, not yet added:
  // the apply takes x + δ, then x ← x + δ on owned nodes and δ ← 0 (the next inner solve's start).
  // r32 (optional): receives the FP32 copy of the residual (0 on the surface row), the next inner
  // solve's right-hand side.
  const int nrow = g.nrow;
  const double* x = A.x;
  const double* phis = A.phis;
  const size_t gstride = (size_t)3 * g.Nz * (g.P + 1) * (g.P + 1);   // cached factors per element
  for (int ex0 = R.e0; ex0 < R.e1; ex0 += g.chunk) {
    const int ne = min(g.chunk, R.e1 - ex0);
    const double* gce = gc ? gc + (size_t)(ex0 - R.e0) * gstride : nullptr;
    apply_element_chunk<P, double>(
        g, s, ex0, ne,
        [&](int e, int a, int iz) -> double {
          const int col = col_of(g, e, a);
          if (iz == nrow - 1) return phis[col];
          const size_t i = (size_t)col * nrow + iz;
          return d32 ? ldcg(x + i) + (double)ldcg(d32 + i) : ldcg(x + i);
        },
        [&](int e, int a, int iz, double y) {
          if (owns_local_col(g, e, a)) A.q64[(size_t)col_of(g, e, a) * nrow + iz] = y;
          else A.edge64[(size_t)e * nrow + iz] = y;
        },
        gce);
  }
  if (want_b) {
    // b = −(A[0; φ̃])_I enters only through ‖b‖, the scale of the stopping test, which FP32 gives to
    // far better than the tolerance needs: an FP32 apply on the same shared memory (the FP64
    // tables are reloaded after it)
    Smem<P, float> s32;
    s32.carve(reinterpret_cast<unsigned char*>(s.D), nrow, g.Nz, g.chunk);
    s32.load_tables(g);
    // only the top element layer: [0; φ̃] is zero below the surface row, and the rows below the top
    // layer keep the zeros they were created with
    for (int ex0 = R.e0; ex0 < R.e1; ex0 += g.chunk)
      apply_element_chunk<P, float, true>(
          g, s32, ex0, min(g.chunk, R.e1 - ex0),
          [&](int e, int a, int iz) -> float { return iz == nrow - 1 ? (float)phis[col_of(g, e, a)] : 0.f; },
          [&](int e, int a, int iz, float y) {
            if (owns_local_col(g, e, a)) A.q64b[(size_t)col_of(g, e, a) * nrow + iz] = (double)y;
            else A.edge64b[(size_t)e * nrow + iz] = (double)y;
          });
    s.load_tables(g);
  }
  if (!grid_barrier(tm, s_flag)) return false;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  const int ncols = R.c1 - R.c0;
  for (int t = threadIdx.x; t < ncols * nrow; t += blockDim.x) {
    const int cq = g.dv_nrow.div(t), col = R.c0 + cq, iz = t - cq * nrow;
    const size_t i = (size_t)col * nrow + iz;
    if (iz == nrow - 1) {
      A.x[i] = phis[col];
      if (d32) d32[i] = 0.f;
      if (r32) r32[i] = 0.f;
      continue;
    }
    if (d32) {
      const double d = (double)d32[i];
      const double xn = A.x[i] + d;
      A.x[i] = xn;
      d32[i] = 0.f;
      acc[2] += d * d;
      acc[3] += xn * xn;
    } else if (dx) {
      acc[3] += A.x[i] * A.x[i];
    }
    const bool le = has_left_edge_p<P>(g, col);
    const size_t ie = le ? (size_t)left_element_p<P>(g, col) * nrow + iz : 0;
    double qv = A.q64[i];
    if (le) qv += ldcg(A.edge64 + ie);
    const double rv = -qv;
    A.r64[i] = rv;
    if (r32) r32[i] = (float)rv;
    acc[0] += rv * rv;
    if (want_b) {
      double bv = A.q64b[i];
      if (le) bv += ldcg(A.edge64b + ie);
      acc[1] += bv * bv;
    }
  }
  block_sum<4, double>(acc, red);
  put_partials<4, double>(tm, 0, acc);
  if (!grid_barrier(tm, s_flag)) return false;
  grid_sum<4>(tm, 0, acc, red);
  rr = acc[0];
  if (want_b) bb = acc[1];
  if (dx) { dx[0] = acc[2]; dx[1] = acc[3]; }
  return true;
}

// One Laplace solve by a team of CTAs: FP64 residual of the lifted system, then PCG in FP64, or
// FP32 inner PCG with FP64 residual refinement (MIXED).  Returns false after a barrier timeout.
template <int P, bool MIXED, bool CACHE = false>
__device__ bool solve_body(const DevGeom& g, const PcgArgs& A, const Team& tm, unsigned char* smem_raw,
                           double* red, int* s_flag_p) {
  int& s_flag = *s_flag_p;
  const Range R = my_range(g, tm);
  const int nrow = g.nrow;
  Smem<P, double> s64;
  s64.carve(smem_raw, nrow, g.Nz, g.chunk);
  s64.load_tables(g);
  // the geometric factors of the FP64 applies, once per solve, where the launch reserved room
  // for them after the apply's buffers
  // (in shared memory where the launch reserved room, else in the mesh's global array)
  const double* gc = nullptr;
  const size_t per_e = (size_t)3 * g.Nz * (P + 1) * (P + 1);
  if (g.gcache > 0 && per_e * (R.e1 - R.e0) <= (size_t)g.gcache) {
    double* c = s64.F2 + (size_t)g.Nz * (P + 1) * (P + 1) * g.chunk;
    fill_gcache<P>(g, R.e0, R.e1, c);
    __syncthreads();
    gc = c;
  } else if (g.gglob != nullptr) {
    double* c = g.gglob + (size_t)R.e0 * per_e;
    fill_gcache<P>(g, R.e0, R.e1, c);
    __syncthreads();
    gc = c;
  }
  SEM_MARK(g, tm, TR_GCACHE);
  double rr = 0.0, bb = 0.0;
  // mixed precision: the residual loop also starts the first inner solve (δ = 0, FP32 residual)
  if (!fp64_residual<P>(g, s64, R, tm, A, true, red, &s_flag, rr, bb, nullptr, gc, nullptr,
                        MIXED ? A.r32 : nullptr))
    return false;
  if (MIXED) {
    const int ncols = R.c1 - R.c0;
    for (int t = threadIdx.x; t < ncols * nrow; t += blockDim.x) {
      const int cq = g.dv_nrow.div(t);
      A.d32[(size_t)(R.c0 + cq) * nrow + (t - cq * nrow)] = 0.f;
    }
    __syncthreads();
  }
  SEM_MARK(g, tm, TR_RESIDUAL);
  const double target = A.tol * A.tol * bb;
  int iters = 0, refinements = 0;
  bool rr_floor_ok = false;   // stopped at the FP64 residual floor with converged corrections
  if (bb == 0.0) {
    // φ̃ ≡ 0 on the surface: Φ = 0 is the solution.
    const int ncols = R.c1 - R.c0;
    for (int t = threadIdx.x; t < ncols * nrow; t += blockDim.x) {
      const int cq = g.dv_nrow.div(t), col = R.c0 + cq, iz = t - cq * nrow;
      if (iz != nrow - 1) A.x[(size_t)col * nrow + iz] = 0.0;
    }
    rr = 0.0;
  } else if (!MIXED) {
    const CgVecs<double> V{A.x, {A.r64, A.r64b}, {A.p64b, A.s64b}, A.p64a, A.z64, A.uh64, A.q64, A.edge64,
                           g.invdiag64};
    double rr_out = rr;
    // FP64 vectors, FP32 preconditioner: u = M⁻¹r only steers the search directions, and the
    // FP32 pipe is 64 times the FP64 pipe on this part
    iters = cg_solve<P, double, double, float, CACHE>(g, s64, R, tm, A, A.pv32, V, target, A.max_iter, red, &s_flag,
                                               &rr_out, gc);
    if (iters < 0) return false;
    rr = rr_out;
  } else {
    Smem<P, float> s32;
    s32.carve(smem_raw, nrow, g.Nz, g.chunk);
    const CgVecs<float> V{A.d32, {A.r32, A.r32b}, {A.p32b, A.s32b}, A.p32a, A.z32, A.uh32, A.q32, A.edge32,
                          g.invdiag32};
    // Refinement stops at the target residual, or once the corrections stop shrinking
    // (‖δ_i‖ > ½‖δ_{i−1}‖): the true residual has then reached the rounding floor of its
    // FP64 evaluation, which can lie above tol·‖b‖ when ‖A‖‖x‖ ≫ ‖b‖.  A stalled solve
    // counts as converged only if its last correction is below tol·‖x‖.
    __shared__ int s_go;
    double dd_prev = INFINITY, dx[2] = {0.0, 0.0};
    bool stalled = false;
    while (true) {
      if (threadIdx.x == 0) {
        int go = rr > target && iters < A.max_iter && !stalled;
        if (!(rr == rr) || isinf(rr)) { atomicOr(g.status, ST_NONFINITE); go = 0; }
        s_go = go;
      }
      __syncthreads();
      if (!s_go) break;
      s32.load_tables(g);
      // inner: A δ = r in FP32 from δ = 0 (δ and the FP32 residual were set by the last FP64
      // residual, whose closing barrier orders them before every CTA's reads), to a relative
      // residual inner_rtol (or the outer target)
      const double tgt_in = fmax(A.inner_rtol * A.inner_rtol * rr, 0.25 * target);
      double rr_in = rr;
      const int it = cg_solve<P, float, float, float, CACHE>(g, s32, R, tm, A, A.pv32, V, tgt_in, A.max_iter - iters, red,
                                               &s_flag, &rr_in);
      if (it < 0) return false;
      iters += it;
      ++refinements;
      // the true FP64 residual of x + δ; x ← x + δ, δ ← 0 and the FP32 residual on the way
      __syncthreads();
      s64.load_tables(g);
      double dummy_b = 0.0;
      if (!fp64_residual<P>(g, s64, R, tm, A, false, red, &s_flag, rr, dummy_b, dx, gc, A.d32, A.r32))
        return false;
      SEM_MARK(g, tm, TR_REFINE);
      stalled = dx[0] > 0.25 * dd_prev;
      dd_prev = dx[0];
      if (it == 0) break;   // no progress possible
    }
    if (rr > target && stalled && dx[0] <= A.tol * A.tol * dx[1]) rr_floor_ok = true;
  }
  if (tm.rank == 0 && threadIdx.x == 0) {
    const double rel = bb > 0.0 ? sqrt(rr / bb) : 0.0;
    SolveRecord* rec = A.rec;
    rec->iterations = iters;
    rec->refinements = refinements;
    rec->rel_residual = rel;
    rec->solves += 1;
    rec->total_iterations += iters;
    rec->total_refinements += refinements;
    if (rel > rec->max_rel_residual) rec->max_rel_residual = rel;
    if (rr > target && !rr_floor_ok) atomicOr(g.status, ST_NOT_CONVERGED);
  }
  return true;
}

template <int P, bool MIXED>
__global__ void __launch_bounds__(kThreads) k_pcg(DevGeom g, PcgArgs A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[kRedSize];
  __shared__ int s_flag;
  const Team tm{(int)blockIdx.x, (int)gridDim.x, A.bar, g.status, A.part, A.part_stride, g.bar_timeout_ns, 0};
  if (tm.rank == g.drop_rank) return;   // testing hook: see sem_set_barrier_test
  solve_body<P, MIXED>(g, A, tm, smem_raw, red, &s_flag);
}

// ------------------------------------------------------------------------------------
// Set-up of the separable preconditioner for the current geometry.
// ------------------------------------------------------------------------------------
// Block per element, one thread per mode: the mode-independent x-stiffness Kx = (2/Δx) Dᵀ
// diag(w d) D is formed once in shared memory (FP64); each mode adds λ_k (Δx/2) diag(w/d) and
// inverts the interior block in FP32 (a sequential FP64 Gauss–Jordan costs ~64 cycles per
// instruction on this part).  The inverse is symmetrised, so the condensed solve is the exact
// inverse of a symmetric operator within FP32 of E; Z = E_bi Ã_ii and the 2×2 Schur block are
// then formed in FP64 from that same Ã_ii, which keeps the FP64 preconditioner symmetric.
constexpr int kPrecModesPerBlock = 32;
constexpr size_t kTriStageMax = 160 * 1024;

// Mode-independent part of element ex: entry t (row-major) of Kx and entry i of the lumped mass
// weights (Δx/2) w/d; prec_elem_kx fills both with all threads of the block (sync after).
template <int P>
__device__ __forceinline__ double prec_kx_entry(const DevGeom& g, int ex, int t) {
  constexpr int Q = P + 1;
  const double* D = c_D64 + d_off(P);
  const double* w = c_w64 + w_off(P);
  const double* geo = g.geo64 + (size_t)ex * Q * 4;
  const int i = t / Q, j = t - i * Q;
  double s = 0.0;
#pragma unroll
  for (int a = 0; a < Q; ++a) s = fma(D[a * Q + i] * w[a] * geo[a * 4 + 0], D[a * Q + j], s);
  return g.r2dx[ex] * s;
}
template <int P>
__device__ __forceinline__ double prec_mw_entry(const DevGeom& g, int ex, int i) {
  constexpr int Q = P + 1;
  const double* w = c_w64 + w_off(P);
  return 0.5 * g.dxe[ex] * w[i] * g.geo64[(size_t)ex * Q * 4 + i * 4 + 1];
}
template <int P>
__device__ __forceinline__ void prec_elem_kx(const DevGeom& g, int ex, double* Kx, double* mw) {
  constexpr int Q = P + 1;
  for (int t = threadIdx.x; t < Q * Q; t += blockDim.x) Kx[t] = prec_kx_entry<P>(g, ex, t);
  for (int i = threadIdx.x; i < Q; i += blockDim.x) mw[i] = prec_mw_entry<P>(g, ex, i);
}

// Mode k of element ex (one thread).
template <int P>
__device__ __forceinline__ void prec_elem_mode(const DevGeom& g, const PrecSetup& ps, int ex, int k,
                                               const double* Kx, const double* mw) {
  constexpr int Q = P + 1, Pm = P - 1;
  const double lam = ps.lam[k];
  float Ai[Pm][Pm], Bm[Pm][Pm];
#pragma unroll
  for (int i = 0; i < Pm; ++i)
#pragma unroll
    for (int j = 0; j < Pm; ++j) {
      Bm[i][j] = (float)(Kx[(1 + i) * Q + 1 + j] + (i == j ? lam * mw[1 + i] : 0.0));
      Ai[i][j] = (i == j) ? 1.f : 0.f;
    }
#pragma unroll
  for (int c = 0; c < Pm; ++c) {
    const float inv = 1.f / Bm[c][c];
#pragma unroll
    for (int j = 0; j < Pm; ++j) { Bm[c][j] *= inv; Ai[c][j] *= inv; }
#pragma unroll
    for (int r = 0; r < Pm; ++r) {
      if (r == c) continue;
      const float f = Bm[r][c];
#pragma unroll
      for (int j = 0; j < Pm; ++j) { Bm[r][j] = fmaf(-f, Bm[c][j], Bm[r][j]); Ai[r][j] = fmaf(-f, Ai[c][j], Ai[r][j]); }
    }
  }
  const size_t base = (size_t)k * g.Nx + ex;
  const int nr = ps.nr;
  float* A32 = ps.Aii32 + (size_t)ex * Pm * Pm * nr + k;   // mode-fastest: A32[(i·Pm + j)·nr]
#pragma unroll
  for (int i = 0; i < Pm; ++i)
#pragma unroll
    for (int j = 0; j < Pm; ++j) A32[(i * Pm + j) * nr] = 0.5f * (Ai[i][j] + Ai[j][i]);
  // Z = E_bi E_ii⁻¹ from the FP32 inverse, accumulated in FP32: the inverse carries FP32 error
  // already, and the FP64 pipe is the scarce one (the Schur complements below stay FP64)
  float kb0[Pm], kb1[Pm];
#pragma unroll
  for (int m = 0; m < Pm; ++m) { kb0[m] = (float)Kx[1 + m]; kb1[m] = (float)Kx[P * Q + 1 + m]; }
  double Z0[Pm], Z1[Pm];
#pragma unroll
  for (int i = 0; i < Pm; ++i) {
    float a0 = 0.f, a1 = 0.f;
#pragma unroll
    for (int m = 0; m < Pm; ++m) {
      const float am = 0.5f * (Ai[m][i] + Ai[i][m]);
      a0 = fmaf(kb0[m], am, a0);
      a1 = fmaf(kb1[m], am, a1);
    }
    Z0[i] = a0; Z1[i] = a1;
  }
  double S00 = Kx[0] + lam * mw[0], S01 = Kx[P], S11 = Kx[P * Q + P] + lam * mw[P];
#pragma unroll
  for (int i = 0; i < Pm; ++i) {
    S00 -= Z0[i] * Kx[(1 + i) * Q];
    S01 -= Z0[i] * Kx[(1 + i) * Q + P];
    S11 -= Z1[i] * Kx[(1 + i) * Q + P];
  }
  float* Z32 = ps.Z32 + (size_t)ex * 2 * Pm * nr + k;      // mode-fastest: Z32[(s·Pm + i)·nr]
#pragma unroll
  for (int i = 0; i < Pm; ++i) {
    Z32[i * nr] = (float)Z0[i];
    Z32[(Pm + i) * nr] = (float)Z1[i];
  }
  ps.schur[base * 3 + 0] = S00;
  ps.schur[base * 3 + 1] = S01;
  ps.schur[base * 3 + 2] = S11;
}

template <int P>
__global__ void __launch_bounds__(kPrecModesPerBlock) k_prec_elem(DevGeom g, PrecSetup ps) {
  constexpr int Q = P + 1;
  __shared__ double Kx[Q * Q];
  __shared__ double mw[Q];
  prec_elem_kx<P>(g, blockIdx.x, Kx, mw);
  __syncthreads();
  const int k = blockIdx.y * blockDim.x + threadIdx.x;
  if (k < ps.nr) prec_elem_mode<P>(g, ps, blockIdx.x, k, Kx, mw);
}

// One warp per mode: interface tridiagonal d_j = S00(j) + S11(j−1), e_j = S01(j) and its Thomas
// pivots.  The pivot recurrence m_j = 1/(d_j − e_{j−1}² m_{j−1}) runs on lane 0 in FP32 from
// shared memory (a sequential FP64 chain costs ~64 cycles per instruction on this part); the
// FP64 factors are taken from those pivots, m⁶⁴ = m³², c' = e m, which makes them the exact
// LDLᵀ factors of a symmetric tridiagonal within FP32 of the true one.  The Sherman–Morrison
// vector T'⁻¹u of the periodic closure (γ = −d_0, u = (γ,0,…,0,e_{N−1}), v = (1,0,…,0,
// e_{N−1}/γ)) is then solved with the warp-parallel tridiagonal solver and the same factors,
// once in FP64 and once in FP32.  Staged in shared memory when 3·nif values fit, otherwise the
// recurrence reads and writes the destination arrays directly.
// `stage_sm`: 2·nif floats of shared memory, or nullptr to run the recurrence on the
// destination arrays.  Called by one full warp.
static __device__ void prec_tri_mode(const DevGeom& g, const PrecSetup& ps, int k, float* stage_sm) {
  const bool staged = stage_sm != nullptr;
  const int N = ps.nif, Nx = g.Nx;
  const double* sc = ps.schur + (size_t)k * Nx * 3;
  float* te32 = ps.te32 + (size_t)k * N;
  float* tm32 = ps.tm32 + (size_t)k * N;
  float* tcp32 = ps.tcp32 + (size_t)k * N;
  float* tz32 = ps.tz32 + (size_t)k * N;
  const double corner = g.periodic ? sc[(Nx - 1) * 3 + 1] : 0.0;
  float* dd = staged ? stage_sm : tm32;     // modified diagonal
  float* ee = staged ? dd + N : te32;
  for (int j = (threadIdx.x & 31); j < N; j += 32) {
    double d;
    if (g.periodic) d = sc[j * 3 + 0] + sc[(j == 0 ? Nx - 1 : j - 1) * 3 + 2];
    else d = (j < Nx ? sc[j * 3 + 0] : 0.0) + (j > 0 ? sc[(j - 1) * 3 + 2] : 0.0);
    dd[j] = (float)d;
    ee[j] = (float)((j < N - 1) ? sc[j * 3 + 1] : 0.0);
  }
  __syncwarp();
  const double gamma = g.periodic ? -(double)(sc[0] + sc[(Nx - 1) * 3 + 2]) : 0.0;
  if ((threadIdx.x & 31) == 0) {
    if (g.periodic) {
      dd[0] = (float)(2.0 * (sc[0] + sc[(Nx - 1) * 3 + 2]));
      dd[N - 1] = (float)((double)dd[N - 1] - corner * corner / gamma);
    }
    float cp_prev = 0.f, e_prev = 0.f;
    for (int j = 0; j < N; ++j) {
      const float m = 1.f / (j == 0 ? dd[0] : fmaf(-e_prev, cp_prev, dd[j]));
      const float e = ee[j];
      dd[j] = m;                 // pivots overwrite the diagonal
      cp_prev = e * m;
      e_prev = e;
    }
  }
  __syncwarp();
  for (int j = (threadIdx.x & 31); j < N; j += 32) {
    const float m = dd[j], e32 = ee[j];
    tm32[j] = m;
    te32[j] = e32;
    tcp32[j] = e32 * m;
  }
  __syncwarp();
  if (g.periodic) {
    auto u32 = [&](int j) -> float { return j == 0 ? (float)gamma : (j == N - 1 ? (float)corner : 0.f); };
    warp_tridiag<float>(N, u32, te32, tm32, tcp32, false, (const float*)nullptr, 0.f, 0.f, tz32);
    if ((threadIdx.x & 31) == 0) {
      const double vl = corner / gamma;
      ps.tvl32[k] = (float)vl;
      ps.tfac32[k] = 1.f / (1.f + tz32[0] + (float)vl * tz32[N - 1]);
    }
  } else {
    for (int j = (threadIdx.x & 31); j < N; j += 32) tz32[j] = 0.f;
  }
}

// 2×2 matrix product A·B scaled by a power of two (exact) so that its largest entry lies in
// [½, 1): the pivot scan below needs only ratios of the entries.
static __device__ __forceinline__ void mat2_mul_norm(const float (&A)[4], const float (&B)[4], float (&C)[4]) {
  float c0 = fmaf(A[0], B[0], A[1] * B[2]), c1 = fmaf(A[0], B[1], A[1] * B[3]);
  float c2 = fmaf(A[2], B[0], A[3] * B[2]), c3 = fmaf(A[2], B[1], A[3] * B[3]);
  const float mx = fmaxf(fmaxf(fabsf(c0), fabsf(c1)), fmaxf(fabsf(c2), fabsf(c3)));
  if (mx > 0.f && mx < INFINITY) {
    int ex;
    frexpf(mx, &ex);
    c0 = ldexpf(c0, -ex); c1 = ldexpf(c1, -ex); c2 = ldexpf(c2, -ex); c3 = ldexpf(c3, -ex);
  }
  C[0] = c0; C[1] = c1; C[2] = c2; C[3] = c3;
}

// prec_tri_mode by every thread of the CTA, for long interface systems between walls
// (N > 32·kTridiagRegs).  The
// pivots p_j = d_j − e_{j−1}²/p_{j−1} are the ratios of the continuants [u_j; v_j] = M_j [u_{j−1};
// v_{j−1}], M_j = [[d_j, −e_{j−1}²], [1, 0]], [u_{−1}; v_{−1}] = [1; 0].  Each thread multiplies
// the M_j of its chunk, a CTA-wide scan of these products gives the continuant before every
// chunk, and each thread then runs the scalar recurrence of prec_tri_mode from that pivot.
static __device__ void prec_tri_mode_cta(const DevGeom& g, const PrecSetup& ps, int k) {
  __shared__ float sM[32][4];
  const int N = ps.nif, Nx = g.Nx;
  const int nt = blockDim.x, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
  const unsigned full = 0xffffffffu;
  const double* sc = ps.schur + (size_t)k * Nx * 3;
  float* te32 = ps.te32 + (size_t)k * N;
  float* tm32 = ps.tm32 + (size_t)k * N;
  float* tcp32 = ps.tcp32 + (size_t)k * N;
  float* tz32 = ps.tz32 + (size_t)k * N;
  const double corner = g.periodic ? sc[(Nx - 1) * 3 + 1] : 0.0;
  const double gamma = g.periodic ? -(double)(sc[0] + sc[(Nx - 1) * 3 + 2]) : 0.0;
  // diagonal (staged in tm32, replaced by the pivots) and off-diagonal
  for (int j = tid; j < N; j += nt) {
    double d;
    if (g.periodic) d = sc[j * 3 + 0] + sc[(j == 0 ? Nx - 1 : j - 1) * 3 + 2];
    else d = (j < Nx ? sc[j * 3 + 0] : 0.0) + (j > 0 ? sc[(j - 1) * 3 + 2] : 0.0);
    if (g.periodic && j == 0) d = 2.0 * (sc[0] + sc[(Nx - 1) * 3 + 2]);
    tm32[j] = (float)d;
    te32[j] = (float)((j < N - 1) ? sc[j * 3 + 1] : 0.0);
  }
  __syncthreads();
  if (g.periodic && tid == 0) tm32[N - 1] = (float)((double)tm32[N - 1] - corner * corner / gamma);
  __syncthreads();
  const int c = (N + nt - 1) / nt;
  const int j0 = min(N, tid * c), j1 = min(N, j0 + c);
  float M[4] = {1.f, 0.f, 0.f, 1.f};
  for (int j = j0; j < j1; ++j) {
    const float ej = j > 0 ? te32[j - 1] : 0.f;
    const float Mj[4] = {tm32[j], -ej * ej, 1.f, 0.f};
    mat2_mul_norm(Mj, M, M);
  }
  for (int o = 1; o < 32; o <<= 1) {               // inclusive scan over the lanes (later on the left)
    float Mp[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) Mp[q] = __shfl_up_sync(full, M[q], o);
    if (lane >= o) mat2_mul_norm(M, Mp, M);
  }
  if (lane == 31)
#pragma unroll
    for (int q = 0; q < 4; ++q) sM[wid][q] = M[q];
  __syncthreads();
  if (wid == 0) {                                   // exclusive scan over the warps
    float W[4] = {1.f, 0.f, 0.f, 1.f};
    if (lane < nw)
#pragma unroll
      for (int q = 0; q < 4; ++q) W[q] = sM[lane][q];
    for (int o = 1; o < 32; o <<= 1) {
      float Wp[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) Wp[q] = __shfl_up_sync(full, W[q], o);
      if (lane >= o) mat2_mul_norm(W, Wp, W);
    }
    float E[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) E[q] = __shfl_up_sync(full, W[q], 1);
    if (lane == 0) { E[0] = 1.f; E[1] = 0.f; E[2] = 0.f; E[3] = 1.f; }
    __syncwarp();
    if (lane < nw)
#pragma unroll
      for (int q = 0; q < 4; ++q) sM[lane][q] = E[q];
  }
  __syncthreads();
  float Lx[4];                                      // lanes before this one in the warp
#pragma unroll
  for (int q = 0; q < 4; ++q) Lx[q] = __shfl_up_sync(full, M[q], 1);
  if (lane == 0) { Lx[0] = 1.f; Lx[1] = 0.f; Lx[2] = 0.f; Lx[3] = 1.f; }
  float Ew[4], Pf[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) Ew[q] = sM[wid][q];
  mat2_mul_norm(Lx, Ew, Pf);                        // continuant map up to the end of the last chunk
  // the scalar recurrence of prec_tri_mode from the pivot before the chunk
  float e_prev = 0.f, cp_prev = 0.f;
  if (j0 > 0 && j0 < j1) {
    e_prev = te32[j0 - 1];
    cp_prev = e_prev * (Pf[2] / Pf[0]);             // e_{j0−1} / p_{j0−1}
  }
  __syncthreads();                                  // every chunk has read its diagonal
  for (int j = j0; j < j1; ++j) {
    const float m = 1.f / (j == 0 ? tm32[0] : fmaf(-e_prev, cp_prev, tm32[j]));
    const float e = te32[j];
    tm32[j] = m;
    tcp32[j] = e * m;
    cp_prev = e * m;
    e_prev = e;
  }
  __syncthreads();
  if (g.periodic) {
    auto u32 = [&](int j) -> float { return j == 0 ? (float)gamma : (j == N - 1 ? (float)corner : 0.f); };
    cta_tridiag<float>(N, u32, te32, tm32, tcp32, false, (const float*)nullptr, 0.f, 0.f, tz32);
    if (tid == 0) {
      const double vl = corner / gamma;
      ps.tvl32[k] = (float)vl;
      ps.tfac32[k] = 1.f / (1.f + tz32[0] + (float)vl * tz32[N - 1]);
    }
  } else {
    for (int j = tid; j < N; j += nt) tz32[j] = 0.f;
  }
}

static __global__ void __launch_bounds__(32) k_prec_tri(DevGeom g, PrecSetup ps, int staged) {
  extern __shared__ __align__(16) double tri_sm[];
  prec_tri_mode(g, ps, blockIdx.x, staged ? reinterpret_cast<float*>(tri_sm) : nullptr);
}

// ------------------------------------------------------------------------------------
// Fused RK stage: one cooperative launch runs a whole RK4 stage for one or many instances of
// order P.  Each instance is served by a team of CTAs (barriers and reductions are per team):
//   σ-geometry → preconditioner set-up → Laplace solve → w̃ and M'-projected ∂x of η, φ̃ →
//   over-integrated Zakharov right-hand side and its M' solve → relaxation source → RK4 update
//   (→ modal filter after stage 4).
// ------------------------------------------------------------------------------------
constexpr int kStageWarps = kThreads / 32;

// The interface systems of the two right-hand sides (η, φ̃) of an M' solve: short systems on one
// warp each (warps 0 and 1 of a one-CTA team, warp 0 of ranks 0 and 1 otherwise), long ones on a
// whole CTA each.  Every thread of the CTA calls it.
template <bool CACHE>
__device__ __forceinline__ void mass1d_interfaces(const SurfTables& t, const Team& tm, double* scr) {
  if (t.nif <= 32 * kTridiagRegs) {
    const int warp = threadIdx.x >> 5;
    if (tm.size == 1) {
      if (warp < 2) mass1d_interface(t, 2, scr, warp);
    } else if (tm.rank < 2 && warp == 0) {
      mass1d_interface(t, 2, scr, tm.rank);
    }
    return;
  }
  for (int rh = tm.rank; rh < 2; rh += tm.size) mass1d_interface_cta<CACHE>(t, 2, scr, rh);
}

template <int P, bool MIXED, bool CACHE = false>
__device__ void stage_body(Instance& I, const Team& tm, int stage, int step, unsigned char* smem_raw,
                           double* red, int* s_flag, double (*sh)[kSurfWarpScratch]) {
  constexpr int Q = P + 1;
  const DevGeom& g = I.g;
  const SurfTables& t = I.st;
  const Range R = my_range(g, tm);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  // stage 0: Laplace solve only (geometry, preconditioner and solve from the state itself)
  const double* ein = stage <= 1 ? I.eta : (stage == 3 ? I.s1e : I.s0e);
  const double* pin = stage <= 1 ? I.phis : (stage == 3 ? I.s1p : I.s0p);
  double* eout = stage == 2 ? I.s1e : I.s0e;   // stage inputs of the next stage (not used at stage 4)
  double* pout = stage == 2 ? I.s1p : I.s0p;
  const double t0 = I.tstart + step * I.dt;
  const double time = t0 + (stage == 1 ? 0.0 : (stage == 4 ? I.dt : 0.5 * I.dt));
  const int ne = R.e1 - R.e0, nc = R.c1 - R.c0;
  SEM_MARK(g, tm, TR_START);

  // σ-geometry of the owned element columns
  for (int q = threadIdx.x; q < ne * Q; q += blockDim.x) geometry_item<P>(g, ein, R.e0 * Q + q);
  // Initial guess of the stage's Laplace solve.  x holds the previous stage's potential; the
  // stage states of RK4 lie on lines from y_n, so linear extrapolation in the stage time turns the
  // first-order starts of stages 2 and 4 into second-order ones: stage 2 (y_n + ½dt k₁) from
  // 2Φ₁ − Φ₃ of the last step, stage 4 (y_n + dt k₃) from 2Φ₃ − Φ₁.  Stage 3 (y_n + ½dt k₂)
  // differs from stage 2 by ¼dt²k₁' + …, which changes little from step to step: Φ₂ + (Φ₃ − Φ₂)
  // of the last step.  Owned nodes only; the barriers below order these writes before any
  // neighbour reads them.
  // generated signal of the left relaxation zone at this stage's time: component angles now
  // (all CTAs of the team), the zone columns after the next barrier, read by the relaxation term
  const bool wave_tab = I.relax && t.wkx != nullptr && t.ncomp > 0 && t.nzl > 0 && stage >= 1;
  if (wave_tab) wave_angles(t, time, tm.rank * blockDim.x + threadIdx.x, tm.size * blockDim.x);
  const bool cont = step > 0 || I.hist;        // the last step belongs to this trajectory
  if (stage == 4 || (stage == 2 && cont)) {
    const double* Pold = stage == 2 ? I.P3 : I.P1;
    double* x = I.pa.x;
    for (int i = R.c0 * g.nrow + threadIdx.x; i < R.c1 * g.nrow; i += blockDim.x) x[i] = fma(2.0, x[i], -Pold[i]);
  } else if (stage == 3 && cont) {
    double* x = I.pa.x;
    for (int i = R.c0 * g.nrow + threadIdx.x; i < R.c1 * g.nrow; i += blockDim.x) x[i] += I.D32[i];
  }
  __syncthreads();
  // preconditioner: condensation of the owned elements for every mode, then interface pivots.
  // The apply's shared memory is free until the solve: it holds Kx and mw of a batch of elements,
  // so that all (element, mode) pairs of the batch run at once.
  {
    double* kxs = reinterpret_cast<double*>(smem_raw);
    constexpr int per = Q * Q + Q;
    const int avail = Q * Q + Q + g.nrow + g.chunk * (2 * g.Nz + 4 * Q + Q * g.nrow + 2 * g.Nz * Q * Q);
    const int nb_max = max(1, min(ne, avail / per));
    const int nr = I.ps.nr;
    for (int e0 = R.e0; e0 < R.e1; e0 += nb_max) {
      const int nb = min(nb_max, R.e1 - e0);
      for (int t = threadIdx.x; t < nb * Q * Q; t += blockDim.x) {
        const int b = t / (Q * Q);
        kxs[b * per + (t - b * Q * Q)] = prec_kx_entry<P>(g, e0 + b, t - b * Q * Q);
      }
      for (int t = threadIdx.x; t < nb * Q; t += blockDim.x) {
        const int b = t / Q;
        kxs[b * per + Q * Q + (t - b * Q)] = prec_mw_entry<P>(g, e0 + b, t - b * Q);
      }
      __syncthreads();
      for (int t = threadIdx.x; t < nb * nr; t += blockDim.x) {
        const int b = g.dv_nr.div(t), k = t - b * nr;
        prec_elem_mode<P>(g, I.ps, e0 + b, k, kxs + b * per, kxs + b * per + Q * Q);
      }
      __syncthreads();
    }
  }
  SEM_MARK(g, tm, TR_SETUP);
  if (!grid_barrier(tm, s_flag)) return;
  SEM_MARK(g, tm, TR_BAR_SETUP);
  if (wave_tab)
    for (int col = tm.rank * nw + warp; col < t.nzl; col += tm.size * nw) wave_zone_column(t, col, lane);
  // long systems between walls: the whole CTA per mode.  Periodic systems keep the serial
  // recurrence: their Sherman–Morrison closure divides by 1 + vᵀT'⁻¹u, which for a nearly
  // singular lowest mode magnifies any difference in the pivots (a 192 k-node periodic tank
  // stopped converging with the scanned pivots).
  if (I.ps.nif > 32 * kTridiagRegs && !g.periodic) {
    for (int k = tm.rank; k < I.ps.nr; k += tm.size) prec_tri_mode_cta(g, I.ps, k);
  } else {
    // one warp per mode, the modes spread over the team's CTAs and their warps
    float* stg = 2 * I.ps.nif <= 2 * kSurfWarpScratch ? reinterpret_cast<float*>(sh[warp]) : nullptr;
    for (int k = tm.rank + tm.size * warp; k < I.ps.nr; k += tm.size * nw) prec_tri_mode(g, I.ps, k, stg);
  }
  if (!grid_barrier(tm, s_flag)) return;
  SEM_MARK(g, tm, TR_PIVOTS);
  // Laplace solve, warm-started from the previous stage's potential
  if (threadIdx.x == 0) I.pa.phis = pin;
  __syncthreads();
  if (!solve_body<P, MIXED, CACHE>(g, I.pa, tm, smem_raw, red, s_flag)) return;
  SEM_MARK(g, tm, TR_SOLVED);
  if (stage == 0) return;
  // kept for the initial guesses of the next stages
  if (stage == 3) {
    for (int i = R.c0 * g.nrow + threadIdx.x; i < R.c1 * g.nrow; i += blockDim.x) {
      const double v = I.pa.x[i];
      I.D32[i] = v - I.P2[i];
      I.P3[i] = v;
    }
  } else {
    double* Pk = stage == 1 ? I.P1 : (stage == 2 ? I.P2 : nullptr);
    if (Pk)
      for (int i = R.c0 * g.nrow + threadIdx.x; i < R.c1 * g.nrow; i += blockDim.x) Pk[i] = I.pa.x[i];
  }
  // w̃ on owned columns; element S_x of η and φ̃; condensation of M'
  for (int c0 = R.c0 + 4 * warp; c0 < R.c1; c0 += 4 * nw) {
    const int col = c0 + (lane >> 3);
    wsurf_column8(t, I.pa.x, ein, I.wt, col < R.c1 ? col : -1, lane & 7);
  }
  for (int q = threadIdx.x; q < 2 * ne * Q; q += blockDim.x) {
    const int fld = q / (ne * Q), r = q - fld * ne * Q;
    sx_item(t, ein, pin, I.R, fld * t.Nx * Q + R.e0 * Q + r);
  }
  __syncthreads();
  for (int q = threadIdx.x; q < 2 * ne; q += blockDim.x) {
    const int rh = q / ne, ex = R.e0 + (q - rh * ne);
    mass1d_condense(t, I.R, 2, I.scr, rh * t.Nx + ex);
  }
  SEM_MARK(g, tm, TR_WSX);
  if (!grid_barrier(tm, s_flag)) return;
  mass1d_interfaces<CACHE>(t, tm, I.scr);
  if (!grid_barrier(tm, s_flag)) return;
  SEM_MARK(g, tm, TR_MINT1);
  for (int q = threadIdx.x; q < 2 * nc; q += blockDim.x) {
    const int rh = q / nc, col = R.c0 + (q - rh * nc);
    mass1d_backsub(t, I.R, 2, rh == 0 ? I.etax : I.phisx, I.scr, rh, col);
  }
  if (!grid_barrier(tm, s_flag)) return;
  SEM_MARK(g, tm, TR_MBACK1);
  // over-integrated Zakharov right-hand side of the owned elements and its M' solve
  for (int ex = R.e0 + warp; ex < R.e1; ex += nw) zak_element(t, ein, I.etax, I.phisx, I.wt, I.R, ex, lane, sh[warp]);
  __syncthreads();
  for (int q = threadIdx.x; q < 2 * ne; q += blockDim.x) {
    const int rh = q / ne, ex = R.e0 + (q - rh * ne);
    mass1d_condense(t, I.R, 2, I.scr, rh * t.Nx + ex);
  }
  SEM_MARK(g, tm, TR_ZAK);
  if (!grid_barrier(tm, s_flag)) return;
  mass1d_interfaces<CACHE>(t, tm, I.scr);
  if (!grid_barrier(tm, s_flag)) return;
  SEM_MARK(g, tm, TR_MINT2);
  for (int q = threadIdx.x; q < 2 * nc; q += blockDim.x) {
    const int rh = q / nc, col = R.c0 + (q - rh * nc);
    mass1d_backsub(t, I.R, 2, rh == 0 ? I.ke : I.kp, I.scr, rh, col);
  }
  __syncthreads();
  // relaxation source and the RK4 bookkeeping on owned columns
  for (int col = R.c0 + threadIdx.x; col < R.c1; col += blockDim.x) {
    if (I.relax) relax_column(t, ein, pin, time, 1.0 / I.tau, I.ke, I.kp, col, wave_tab ? t.wEP : nullptr);
    rk4_item(stage, I.dt, I.eta, I.phis, I.ke, I.kp, I.ae, I.ap, eout, pout, col);
  }
  SEM_MARK(g, tm, TR_RK4);
  if (stage == 4 && t.filter_on) {
    if (!grid_barrier(tm, s_flag)) return;
    for (int ex = R.e0 + warp; ex < R.e1; ex += nw) filter_element(t, I.eta, I.phis, ex, lane, sh[warp]);
    SEM_MARK(g, tm, TR_FILTER);
  }
}

// WIDE = false: one CTA per SM and the full register file, so the stage keeps its values in
// registers (single meshes: one team, latency bound).  WIDE = true: two CTAs per SM at 128
// registers, more co-resident teams for batches of many small instances.
// Two launch forms.  Cooperative (B.cluster = 0): the grid is co-resident and a team's barrier is
// the bounded global one.  Cluster teams (B.cluster = 1): every instance's CTAs are one thread-block
// cluster (team0 a multiple of the cluster size) and the team barrier is the hardware cluster
// barrier; no CTA waits on a CTA of another cluster, so the launch needs no co-residency and the
// launches of other groups may run at the same time.  Every CTA of a cluster takes the same
// sequence of barriers: no control path leaves the kernel early in one CTA only.
template <int P, bool MIXED, bool WIDE>
__global__ void __launch_bounds__(kThreads, WIDE ? 2 : 1) k_stage(StageArgs B) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[kRedSize];
  __shared__ int s_flag;
  __shared__ __align__(16) double sh[kStageWarps][kSurfWarpScratch];
  __shared__ __align__(16) Instance I;
  const int ii = B.cta_inst[blockIdx.x];
  {
    const unsigned int* src = reinterpret_cast<const unsigned int*>(B.inst + ii);
    unsigned int* dst = reinterpret_cast<unsigned int*>(&I);
    for (int q = threadIdx.x; q < (int)(sizeof(Instance) / 4); q += blockDim.x) dst[q] = src[q];
  }
  __syncthreads();
  const Team tm{(int)blockIdx.x - I.team0, I.nteam, B.bars + 2 * ii, I.g.status, I.pa.part, I.pa.part_stride,
                I.g.bar_timeout_ns, B.cluster};
  // testing hook (see sem_set_barrier_test); the cluster plan never serves a mesh that carries it
  if (!B.cluster && tm.rank == I.g.drop_rank) return;
  stage_body<P, MIXED, !WIDE>(I, tm, B.stage, B.step, smem_raw, red, &s_flag, sh);
}

// ------------------------------------------------------------------------------------
// Host entry points for one order P (explicitly instantiated per order in kernels_order.cu).
// ------------------------------------------------------------------------------------
template <int P>
cudaError_t upload_tables_impl(const double* D64, const double* w64) {
  float D32[kDTotal], w32[kWTotal];
  for (int i = 0; i < kDTotal; ++i) D32[i] = static_cast<float>(D64[i]);
  for (int i = 0; i < kWTotal; ++i) w32[i] = static_cast<float>(w64[i]);
  cudaError_t e;
  if ((e = cudaMemcpyToSymbol(c_D64, D64, sizeof(double) * kDTotal)) != cudaSuccess) return e;
  if ((e = cudaMemcpyToSymbol(c_D32, D32, sizeof(float) * kDTotal)) != cudaSuccess) return e;
  if ((e = cudaMemcpyToSymbol(c_w64, w64, sizeof(double) * kWTotal)) != cudaSuccess) return e;
  return cudaMemcpyToSymbol(c_w32, w32, sizeof(float) * kWTotal);
}

template <int P>
cudaError_t launch_geometry_impl(const DevGeom& g, const double* eta, bool with_diag, cudaStream_t s) {
  const int n1 = g.Nx * (P + 1);
  k_geometry<P><<<(n1 + 127) / 128, 128, 0, s>>>(g, eta);
  count_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || !with_diag) return e;
  const long long n = (long long)g.ncol * g.nrow;
  k_diag<P><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(g);
  count_launch();
  return cudaGetLastError();
}

template <int P>
cudaError_t launch_apply_elem_impl(const DevGeom& g, const double* x, double* q, double* edge, cudaStream_t s) {
  const size_t smem = apply_smem_bytes(P, g.nrow, g.Nz, g.chunk, sizeof(double));
  const int nch = (g.Nx + g.chunk - 1) / g.chunk;
  const int grid = nch < 4096 ? nch : 4096;
  cudaError_t e = cudaFuncSetAttribute(k_apply<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDynSmem);
  if (e != cudaSuccess) return e;
  k_apply<P><<<grid, kThreads, smem, s>>>(g, x, q, edge);
  count_launch();
  return cudaGetLastError();
}

template <int P>
cudaError_t pcg_occupancy_impl(int mixed, size_t smem, int* per_sm) {
  const void* fn = mixed ? (const void*)k_pcg<P, true> : (const void*)k_pcg<P, false>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDynSmem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, fn, kThreads, smem);
}

template <int P>
cudaError_t launch_pcg_impl(int mixed, const DevGeom& g, const PcgArgs& a, int grid, size_t smem, cudaStream_t s) {
  DevGeom gg = g;
  PcgArgs aa = a;
  void* args[] = {&gg, &aa};
  const void* fn = mixed ? (const void*)k_pcg<P, true> : (const void*)k_pcg<P, false>;
  return cudaLaunchCooperativeKernel(fn, grid, kThreads, args, smem, s);
}

template <int P>
cudaError_t launch_prec_setup_impl(const DevGeom& g, const PrecSetup& ps, cudaStream_t s) {
  const dim3 grid_e(g.Nx, (ps.nr + kPrecModesPerBlock - 1) / kPrecModesPerBlock);
  k_prec_elem<P><<<grid_e, kPrecModesPerBlock, 0, s>>>(g, ps);
  count_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const size_t bytes = (size_t)2 * ps.nif * sizeof(float);
  const int staged = bytes <= kTriStageMax ? 1 : 0;
  if (staged) {
    e = cudaFuncSetAttribute(k_prec_tri, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTriStageMax);
    if (e != cudaSuccess) return e;
  }
  k_prec_tri<<<ps.nr, 32, staged ? bytes : 0, s>>>(g, ps, staged);
  count_launch();
  return cudaGetLastError();
}

template <int P>
static const void* stage_fn(int mixed, int wide) {
  if (wide) return mixed ? (const void*)k_stage<P, true, true> : (const void*)k_stage<P, false, true>;
  return mixed ? (const void*)k_stage<P, true, false> : (const void*)k_stage<P, false, false>;
}

template <int P>
cudaError_t stage_occupancy_impl(int mixed, int wide, size_t smem, int* per_sm) {
  const void* fn = stage_fn<P>(mixed, wide);
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDynSmem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, fn, kThreads, smem);
}

template <int P>
cudaError_t launch_stage_impl(int mixed, int wide, const StageArgs& a, int grid, size_t smem, cudaStream_t s) {
  StageArgs aa = a;
  void* args[] = {&aa};
  const void* fn = stage_fn<P>(mixed, wide);
  return cudaLaunchCooperativeKernel(fn, grid, kThreads, args, smem, s);
}


template <int P>
static cudaLaunchConfig_t cluster_config(int grid, int csize, size_t smem, cudaStream_t s, cudaLaunchAttribute* attr) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)csize;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cfg;
}

template <int P>
cudaError_t cluster_fit_impl(int mixed, int wide, int csize, size_t smem, int* active_clusters) {
  const void* fn = stage_fn<P>(mixed, wide);
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDynSmem);
  if (e != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1)) != cudaSuccess) return e;
  cudaLaunchAttribute attr[1];
  const cudaLaunchConfig_t cfg = cluster_config<P>(csize, csize, smem, nullptr, attr);
  return cudaOccupancyMaxActiveClusters(active_clusters, fn, &cfg);
}

template <int P>
cudaError_t launch_stage_cluster_impl(int mixed, int wide, const StageArgs& a, int grid, int csize, size_t smem,
                                      cudaStream_t s) {
  cudaLaunchAttribute attr[1];
  const cudaLaunchConfig_t cfg = cluster_config<P>(grid, csize, smem, s, attr);
  StageArgs aa = a;
  void* args[] = {&aa};
  return cudaLaunchKernelExC(&cfg, stage_fn<P>(mixed, wide), args);
}

// Tiled apply (apply_tile.cuh): widest tile of at most 16 elements whose shared memory keeps
// three CTAs per SM (FP32; the measured width where one is set) or fits at all (FP64, one CTA per
// SM); persistent CTAs (at most the co-resident count) stride over the tiles.
// The tensor-core FP32 kernel (apply_tc.cuh, fp32 = 3, orders 4..7) takes tiles of 64/Nz − 1
// elements: with the recomputed left neighbour, 64 element blocks, four block pairs per warp.
constexpr size_t kTileSmemTarget = 76 * 1024;

template <int P>
static int tile_grid(const void* fn, size_t smem, int E, int Nx, int slot, cudaError_t* err) {
  // the attribute, the SM count and the occupancy for the last (device, smem) of each kernel
  // variant are kept, so that a repeated apply costs one launch on the host
  static std::mutex mu;
  static int last_dev[9] = {-1, -1, -1, -1, -1, -1, -1, -1, -1}, last_sms[9] = {0}, last_per_sm[9] = {0};
  static size_t last_smem[9] = {0};
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) { *err = e; return 0; }
  {
    std::lock_guard<std::mutex> lk(mu);
    if (last_dev[slot] != dev || last_smem[slot] != smem) {
      if ((e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDynSmem)) != cudaSuccess ||
          (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess ||
          (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kThreads, smem)) != cudaSuccess) {
        *err = e;
        return 0;
      }
      last_dev[slot] = dev; last_smem[slot] = smem; last_sms[slot] = sms; last_per_sm[slot] = per_sm;
    }
    sms = last_sms[slot];
    per_sm = last_per_sm[slot];
  }
  if (per_sm < 1) { *err = cudaErrorInvalidConfiguration; return 0; }
  const long long ntiles = (Nx + E - 1) / E;
  *err = cudaSuccess;
  return (int)(ntiles < (long long)per_sm * sms ? ntiles : (long long)per_sm * sms);
}

template <int P>
cudaError_t launch_apply_tile_impl(int fp32, const DevGeom& g, const void* x, void* y, cudaStream_t s) {
  const int bulk_ok = (reinterpret_cast<uintptr_t>(x) % 16) == 0 ? 1 : 0;   // bulk copies need 16-B alignment
  const float* xf = static_cast<const float*>(x);
  float* yf = static_cast<float*>(y);
  cudaError_t e = cudaSuccess;
  if constexpr (P >= 4 && P <= 7) {
    if (fp32 == 3) {   // tensor-core kernel
      int E = g.Nz < 64 ? 64 / g.Nz - 1 : 1;
      while (E > 1 && apply_tile_tc_smem<P>(E, g.nrow, g.Nz) > kTileSmemTarget) E = (E + 1) / 2 - 1;
      const size_t smem = apply_tile_tc_smem<P>(E, g.nrow, g.Nz);
      if (smem > (size_t)kMaxDynSmem) return cudaErrorInvalidValue;
      const int nzc = (g.Nz == 1 || g.Nz == 2 || g.Nz == 4) ? g.Nz : 0;
      const int k = 5 + (nzc == 4 ? 3 : nzc);
      const void* fns[4] = {(const void*)k_apply_tile_tc<P, 0>, (const void*)k_apply_tile_tc<P, 1>,
                            (const void*)k_apply_tile_tc<P, 2>, (const void*)k_apply_tile_tc<P, 4>};
      const int grid = tile_grid<P>(fns[k - 5], smem, E, g.Nx, k, &e);
      if (e != cudaSuccess) return e;
      switch (k) {
        case 5: k_apply_tile_tc<P, 0><<<grid, kThreads, smem, s>>>(g, xf, yf, E, bulk_ok); break;
        case 6: k_apply_tile_tc<P, 1><<<grid, kThreads, smem, s>>>(g, xf, yf, E, bulk_ok); break;
        case 7: k_apply_tile_tc<P, 2><<<grid, kThreads, smem, s>>>(g, xf, yf, E, bulk_ok); break;
        default: k_apply_tile_tc<P, 4><<<grid, kThreads, smem, s>>>(g, xf, yf, E, bulk_ok); break;
      }
      count_launch();
      return cudaGetLastError();
    }
  }
  const size_t elem = fp32 ? sizeof(float) : sizeof(double);
  // the FP64 kernel holds one CTA per SM (its registers), so only the shared-memory maximum caps it
  const size_t cap = fp32 ? kTileSmemTarget : (size_t)kMaxDynSmem;
  int E = 16;
  while (E > 1 && apply_tile_smem<P>(E, g.nrow, g.Nz, elem) > cap) E >>= 1;
  const int Et = fp32 ? apply_tile_width(P, g.Nz) : 0;   // a measured FP32 width (autotuner), if set
  if (Et > 0 && apply_tile_smem<P>(Et, g.nrow, g.Nz, elem) <= (size_t)kMaxDynSmem) E = Et;
  const size_t smem = apply_tile_smem<P>(E, g.nrow, g.Nz, elem);
  if (smem > (size_t)kMaxDynSmem) return cudaErrorInvalidValue;
  // FP32 kernels specialised on the common layer counts 1, 2 and 4 (constant row arithmetic)
  const int nzc = fp32 && (g.Nz == 1 || g.Nz == 2 || g.Nz == 4) ? g.Nz : 0;
  const int k = fp32 ? 1 + (nzc == 4 ? 3 : nzc) : 0;   // kernel variant 0..4
  const void* fns[5] = {(const void*)k_apply_tile<P, double, 0>, (const void*)k_apply_tile<P, float, 0>,
                        (const void*)k_apply_tile<P, float, 1>, (const void*)k_apply_tile<P, float, 2>,
                        (const void*)k_apply_tile<P, float, 4>};
  const int grid = tile_grid<P>(fns[k], smem, E, g.Nx, k, &e);
  if (e != cudaSuccess) return e;
  switch (k) {
    case 0: k_apply_tile<P, double, 0><<<grid, kThreads, smem, s>>>(g, static_cast<const double*>(x),
                                                                   static_cast<double*>(y), E, bulk_ok); break;
    case 1: k_apply_tile<P, float, 0><<<grid, kThreads, smem, s>>>(g, xf, yf, E, bulk_ok); break;
    case 2: k_apply_tile<P, float, 1><<<grid, kThreads, smem, s>>>(g, xf, yf, E, bulk_ok); break;
    case 3: k_apply_tile<P, float, 2><<<grid, kThreads, smem, s>>>(g, xf, yf, E, bulk_ok); break;
    default: k_apply_tile<P, float, 4><<<grid, kThreads, smem, s>>>(g, xf, yf, E, bulk_ok); break;
  }
  count_launch();
  return cudaGetLastError();
}

}  // namespace semgb
