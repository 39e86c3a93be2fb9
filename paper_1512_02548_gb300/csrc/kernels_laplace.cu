// σ-geometry, the matrix-free Laplace operator and the persistent Krylov solver
// (§2 and §3.1.2 of arXiv 1512.02548), for sm_103a.
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
// Work decomposition.  One CTA processes an "element column" (all Nz layers of
// x-element ex) at a time: its (P+1)·Nrow nodes are staged in shared memory, the
// layers are summed in shared memory, columns a = 0..P−1 are written straight to
// the output and column a = P (shared with the next x-element) to an edge buffer
// that the owner of that column adds after a grid barrier.  All sums are in a fixed
// order, so results are bitwise reproducible.
//
// Krylov.  Conjugate gradients on the Dirichlet-eliminated SPD system with the
// Jacobi preconditioner run inside ONE cooperative persistent kernel: two grid
// barriers per iteration, deterministic reductions, a double-buffered search
// direction so each CTA can rebuild its halo column without a third barrier, and a
// device-side convergence test (no host round trip).  In mixed precision the inner
// iterations run in FP32 and the kernel refines the FP64 residual.
#include <cooperative_groups.h>

#include "sem_internal.cuh"

namespace semgb {

__constant__ double c_D64[kDTotal];
__constant__ float c_D32[kDTotal];
__constant__ double c_w64[kWTotal];
__constant__ float c_w32[kWTotal];

template <class T> struct CT;
template <> struct CT<double> {
  static __device__ __forceinline__ const double* D() { return c_D64; }
  static __device__ __forceinline__ const double* w() { return c_w64; }
};
template <> struct CT<float> {
  static __device__ __forceinline__ const float* D() { return c_D32; }
  static __device__ __forceinline__ const float* w() { return c_w32; }
};

cudaError_t upload_line_tables(const double* D64, const double* w64) {
  float D32[kDTotal], w32[kWTotal];
  for (int i = 0; i < kDTotal; ++i) D32[i] = static_cast<float>(D64[i]);
  for (int i = 0; i < kWTotal; ++i) w32[i] = static_cast<float>(w64[i]);
  cudaError_t e;
  if ((e = cudaMemcpyToSymbol(c_D64, D64, sizeof(double) * kDTotal)) != cudaSuccess) return e;
  if ((e = cudaMemcpyToSymbol(c_D32, D32, sizeof(float) * kDTotal)) != cudaSuccess) return e;
  if ((e = cudaMemcpyToSymbol(c_w64, w64, sizeof(double) * kWTotal)) != cudaSuccess) return e;
  return cudaMemcpyToSymbol(c_w32, w32, sizeof(float) * kWTotal);
}

__device__ __forceinline__ double fmx(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fmx(float a, float b, float c) { return fmaf(a, b, c); }
// L2-coherent load for data another CTA wrote before the last grid barrier.
__device__ __forceinline__ double ldcg(const double* p) { return __ldcg(p); }
__device__ __forceinline__ float ldcg(const float* p) { return __ldcg(p); }

__device__ __forceinline__ int col_of(const DevGeom& g, int ex, int a) {
  int c = ex * g.P + a;
  return c >= g.ncol ? c - g.ncol : c;
}

// ------------------------------------------------------------------------------------
// Geometry: per element-local column (ex, a) store d, 1/d, ∂x h, ∂x d (element-local
// collocation derivative of d = η + h, the exact Jacobian of the interpolated σ-map).
// ------------------------------------------------------------------------------------
template <int P>
__global__ void k_geometry(DevGeom g, const double* __restrict__ eta) {
  constexpr int Q = P + 1;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= g.Nx * Q) return;
  const int ex = t / Q, a = t - ex * Q;
  const double* D = c_D64 + d_off(P) + a * Q;
  double etax = 0.0;
#pragma unroll
  for (int c = 0; c < Q; ++c) etax = fma(D[c], eta[col_of(g, ex, c)], etax);
  etax *= 2.0 / g.dxe[ex];
  const int col = col_of(g, ex, a);
  const double d = eta[col] + g.h[col];
  const double hx = g.hx_loc[t];
  const double dxd = etax + hx;
  if (!(d > 0.0) || !isfinite(d) || !isfinite(dxd)) atomicOr(g.status, ST_BAD_DEPTH);
  const double invd = 1.0 / d;
  double* o = g.geo64 + (size_t)t * 4;
  o[0] = d; o[1] = invd; o[2] = hx; o[3] = dxd;
  float* o32 = g.geo32 + (size_t)t * 4;
  o32[0] = (float)d; o32[1] = (float)invd; o32[2] = (float)hx; o32[3] = (float)dxd;
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
  T* cxz;   // 2*Nz: Δσ_l/Δx_e, Δx_e/Δσ_l for the current element column
  T* geo;   // 4*Q
  T* X;     // Q*nrow
  T* F1;    // Nz*Q*Q
  T* F2;    // Nz*Q*Q
  __device__ static size_t bytes(int nrow, int Nz) {
    return sizeof(T) * (size_t)(Q * Q + Q + nrow + 2 * Nz + 4 * Q + Q * nrow + 2 * Nz * Q * Q);
  }
  __device__ void carve(unsigned char* base, int nrow, int Nz) {
    T* p = reinterpret_cast<T*>(base);
    D = p; p += Q * Q;
    w = p; p += Q;
    sig = p; p += nrow;
    cxz = p; p += 2 * Nz;
    geo = p; p += 4 * Q;
    X = p; p += Q * nrow;
    F1 = p; p += Nz * Q * Q;
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

// Apply A = −𝓛 on element column ex.  `loadx(ex,a,iz)` gives the input value of local
// column a, row iz; `store(ex,a,iz,y)` receives the element column's contribution.
// Returns this thread's share of Σ x·(A_e x) over the element column.
template <int P, class T, class LoadX, class Store>
__device__ __forceinline__ double apply_element_column(const DevGeom& g, Smem<P, T>& s, int ex,
                                                       LoadX loadx, Store store) {
  constexpr int Q = P + 1;
  const int nrow = g.nrow, Nz = g.Nz;
  const T* geo = geo_ptr<T>(g) + (size_t)ex * Q * 4;
  for (int t = threadIdx.x; t < 4 * Q; t += blockDim.x) s.geo[t] = geo[t];
  for (int t = threadIdx.x; t < Nz; t += blockDim.x) {
    const double dxe = g.dxe[ex], dsl = g.dsl[t];
    s.cxz[2 * t] = (T)(dsl / dxe);
    s.cxz[2 * t + 1] = (T)(dxe / dsl);
  }
  for (int t = threadIdx.x; t < Q * nrow; t += blockDim.x) {
    const int a = t / nrow, iz = t - a * nrow;
    s.X[t] = loadx(ex, a, iz);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < Nz * Q * Q; t += blockDim.x) {
    const int l = t / (Q * Q), rem = t - l * (Q * Q), a = rem / Q, b = rem - a * Q;
    const T* Xrow = s.X + l * P + b;             // Xrow[c*nrow]: row l·P+b, column c
    const T* Xcol = s.X + a * nrow + l * P;      // Xcol[c]: column a, row l·P+c
    const T* Da = s.D + a * Q;
    const T* Db = s.D + b * Q;
    T ur = 0, ut = 0;
#pragma unroll
    for (int c = 0; c < Q; ++c) {
      ur = fmx(Da[c], Xrow[c * nrow], ur);
      ut = fmx(Db[c], Xcol[c], ut);
    }
    const T d = s.geo[a * 4 + 0], invd = s.geo[a * 4 + 1], hx = s.geo[a * 4 + 2], dxd = s.geo[a * 4 + 3];
    const T wab = s.w[a] * s.w[b];
    const T K12 = hx - s.sig[l * P + b] * dxd;
    const T K22 = fmx(K12, K12, (T)1) * invd;
    const T G11 = wab * s.cxz[2 * l] * d;
    const T G12 = wab * K12;
    const T G22 = wab * s.cxz[2 * l + 1] * K22;
    s.F1[t] = fmx(G11, ur, G12 * ut);
    s.F2[t] = fmx(G12, ur, G22 * ut);
  }
  __syncthreads();
  double part = 0.0;
  for (int t = threadIdx.x; t < Q * nrow; t += blockDim.x) {
    const int a = t / nrow, iz = t - a * nrow;
    const int l = iz / P, b = iz - l * P;
    T y = 0;
    if (l < Nz) {
      const T* F1 = s.F1 + (l * Q) * Q + b;      // F1[(l*Q+a')*Q+b] = F1[a'*Q]
      const T* F2 = s.F2 + (l * Q + a) * Q;      // F2[(l*Q+a)*Q+b']
#pragma unroll
      for (int c = 0; c < Q; ++c) {
        y = fmx(s.D[c * Q + a], F1[c * Q], y);
        y = fmx(s.D[c * Q + b], F2[c], y);
      }
    }
    if (b == 0 && l > 0) {
      const int lm = l - 1;
      const T* F1 = s.F1 + (lm * Q) * Q + P;
      const T* F2 = s.F2 + (lm * Q + a) * Q;
#pragma unroll
      for (int c = 0; c < Q; ++c) {
        y = fmx(s.D[c * Q + a], F1[c * Q], y);
        y = fmx(s.D[c * Q + P], F2[c], y);
      }
    }
    store(ex, a, iz, y);
    part += (double)s.X[t] * (double)y;
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
  s.carve(smem_raw, g.nrow, g.Nz);
  s.load_tables(g);
  __syncthreads();
  const int nrow = g.nrow;
  for (int ex = blockIdx.x; ex < g.Nx; ex += gridDim.x) {
    apply_element_column<P, double>(
        g, s, ex,
        [&](int e, int a, int iz) { return x[(size_t)col_of(g, e, a) * nrow + iz]; },
        [&](int e, int a, int iz, double y) {
          if (a < P || (!g.periodic && e == g.Nx - 1)) q[(size_t)col_of(g, e, a) * nrow + iz] = y;
          else edge[(size_t)e * nrow + iz] = y;
        });
  }
}

__device__ __forceinline__ bool has_left_edge(const DevGeom& g, int col) {
  if (col % g.P != 0) return false;
  if (g.periodic) return true;
  return col > 0 && col < g.Nx * g.P;
}
__device__ __forceinline__ int left_element(const DevGeom& g, int col) {
  const int ex = col / g.P;
  return ex == 0 ? g.Nx - 1 : ex - 1;
}

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
// Grid barrier for the cooperative kernel, with a wall-clock limit.
// ------------------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

constexpr unsigned long long kBarrierTimeoutNs = 2000000000ull;  // 2 s

// Returns false (and sets ST_TIMEOUT) if the other CTAs did not arrive in time; the
// caller must then return without touching another barrier.
__device__ __forceinline__ bool grid_barrier(unsigned int* bar, int* status, int* s_flag) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned int* vgen = bar + 1;
    const unsigned int gen = *vgen;
    __threadfence();
    const unsigned int prev = atomicAdd(bar, 1u);
    int ok = 1;
    if (prev == gridDim.x - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      const unsigned long long t0 = global_ns();
      unsigned int spins = 0;
      while (*vgen == gen) {
        if ((++spins & 63u) == 0 && global_ns() - t0 > kBarrierTimeoutNs) {
          atomicOr(status, ST_TIMEOUT);
          ok = 0;
          break;
        }
        __nanosleep(20);
      }
    }
    __threadfence();
    *s_flag = ok;
  }
  __syncthreads();
  return *s_flag != 0;
}

// Deterministic block sum of K values (all threads get the result).
template <int K>
__device__ __forceinline__ void block_sum(double (&v)[K], double* red) {
#pragma unroll
  for (int k = 0; k < K; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < K; ++k) red[k * 32 + wid] = v[k];
  __syncthreads();
#pragma unroll
  for (int k = 0; k < K; ++k) {
    double s = lane < nw ? red[k * 32 + lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    v[k] = s;
  }
  __syncthreads();
}

// Sum of K per-CTA partials part[slot][k][cta] over all CTAs, same order in every CTA.
template <int K>
__device__ __forceinline__ void grid_sum(const double* part, int stride, int slot, double (&v)[K],
                                         double* red) {
  const int lane = threadIdx.x & 31;
  if (threadIdx.x < 32) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const volatile double* p = part + ((size_t)slot * 4 + k) * stride;
      double s = 0.0;
      for (int c = lane; c < (int)gridDim.x; c += 32) s += p[c];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) red[128 + k] = s;
    }
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < K; ++k) v[k] = red[128 + k];
  __syncthreads();
}

template <int K>
__device__ __forceinline__ void put_partials(double* part, int stride, int slot, const double (&v)[K]) {
  if (threadIdx.x == 0)
#pragma unroll
    for (int k = 0; k < K; ++k) part[((size_t)slot * 4 + k) * stride + blockIdx.x] = v[k];
}

// ------------------------------------------------------------------------------------
// Persistent preconditioned CG.  One level (FP64) or two levels (FP32 inner, FP64
// residual refinement).
// ------------------------------------------------------------------------------------
struct Range { int e0, e1, c0, c1; };   // owned element columns and global columns

__device__ __forceinline__ Range my_range(const DevGeom& g) {
  Range r;
  r.e0 = (int)(((long long)blockIdx.x * g.Nx) / gridDim.x);
  r.e1 = (int)(((long long)(blockIdx.x + 1) * g.Nx) / gridDim.x);
  r.c0 = r.e0 * g.P;
  r.c1 = r.e1 * g.P + ((!g.periodic && r.e1 == g.Nx) ? 1 : 0);
  return r;
}

// Inner PCG on A x = r0 (vectors of type T), starting from x (given) and residual r.
// Expects r, z, rz, rr already computed for the start (slot `sl` holds rr, rz).
// Stops when rr ≤ target or after max_it iterations.  Returns iterations, or −1 on
// a barrier timeout.
template <int P, class T>
__device__ int inner_pcg(const DevGeom& g, Smem<P, T>& s, const Range& R, T* x, T* r, T* z, T* pa,
                         T* pb, T* q, T* edge, const T* invdiag, double* part, int stride,
                         unsigned int* bar, double* red, int* s_flag, double rr, double rz,
                         double target, int max_it, double* rr_out) {
  const int nrow = g.nrow;
  int k = 0;
  double rz_prev = 1.0;
  T* p_old = pa;
  T* p_new = pb;
  while (true) {
    if (!(rr == rr) || isinf(rr)) { if (threadIdx.x == 0) atomicOr(g.status, ST_NONFINITE); break; }
    if (rr <= target || k >= max_it) break;
    const T beta = (T)(k == 0 ? 0.0 : rz / rz_prev);
    const bool first = (k == 0);
    // Phase A: p_new = z + β p_old (own columns written, halo column rebuilt), q = A p_new
    double pap[1] = {0.0};
    for (int ex = R.e0; ex < R.e1; ++ex) {
      pap[0] += apply_element_column<P, T>(
          g, s, ex,
          [&](int e, int a, int iz) -> T {
            if (iz == nrow - 1) return (T)0;
            const size_t i = (size_t)col_of(g, e, a) * nrow + iz;
            const T zi = ldcg(z + i);
            const T pn = first ? zi : fmx(beta, ldcg(p_old + i), zi);
            if (a < P || (!g.periodic && e == g.Nx - 1)) p_new[i] = pn;
            return pn;
          },
          [&](int e, int a, int iz, T y) {
            if (a < P || (!g.periodic && e == g.Nx - 1)) q[(size_t)col_of(g, e, a) * nrow + iz] = y;
            else edge[(size_t)e * nrow + iz] = y;
          });
    }
    block_sum<1>(pap, red);
    put_partials<1>(part, stride, 2, pap);
    if (!grid_barrier(bar, g.status, s_flag)) return -1;
    grid_sum<1>(part, stride, 2, pap, red);
    const T alpha = (T)(rz / pap[0]);
    // Phase B: x += α p, r −= α q, z = M⁻¹ r on owned nodes
    double acc[2] = {0.0, 0.0};
    const int ncols = R.c1 - R.c0;
    for (int t = threadIdx.x; t < ncols * nrow; t += blockDim.x) {
      const int col = R.c0 + t / nrow, iz = t - (t / nrow) * nrow;
      if (iz == nrow - 1) continue;
      const size_t i = (size_t)col * nrow + iz;
      T qv = q[i];
      if (has_left_edge(g, col)) qv += ldcg(edge + (size_t)left_element(g, col) * nrow + iz);
      x[i] = fmx(alpha, p_new[i], x[i]);
      const T rv = fmx(-alpha, qv, r[i]);
      r[i] = rv;
      const T zv = rv * invdiag[i];
      z[i] = zv;
      acc[0] += (double)rv * (double)rv;
      acc[1] += (double)rv * (double)zv;
    }
    block_sum<2>(acc, red);
    put_partials<2>(part, stride, 3, acc);
    if (!grid_barrier(bar, g.status, s_flag)) return -1;
    grid_sum<2>(part, stride, 3, acc, red);
    rr = acc[0];
    rz_prev = rz;
    rz = acc[1];
    T* tmp = p_old; p_old = p_new; p_new = tmp;
    ++k;
  }
  *rr_out = rr;
  return k;
}

// FP64 residual r = b − A_II x = −(A [x; φ̃])_I on owned nodes, with ‖b‖² when asked
// (b = −(A [0; φ̃])_I).  Two passes: element columns, then edge fix.  Returns false on
// a barrier timeout.  On return rr/bb (and rz for z = M⁻¹r when want_z) are summed.
template <int P>
__device__ bool fp64_residual(const DevGeom& g, Smem<P, double>& s, const Range& R, const PcgArgs& A,
                              bool want_b, bool want_z, double* red, int* s_flag, double& rr,
                              double& bb, double& rz) {
  const int nrow = g.nrow;
  const double* x = A.x;
  const double* phis = A.phis;
  for (int ex = R.e0; ex < R.e1; ++ex) {
    apply_element_column<P, double>(
        g, s, ex,
        [&](int e, int a, int iz) -> double {
          const int col = col_of(g, e, a);
          return iz == nrow - 1 ? phis[col] : ldcg(x + (size_t)col * nrow + iz);
        },
        [&](int e, int a, int iz, double y) {
          if (a < P || (!g.periodic && e == g.Nx - 1)) A.q64[(size_t)col_of(g, e, a) * nrow + iz] = y;
          else A.edge64[(size_t)e * nrow + iz] = y;
        });
    if (want_b)
      apply_element_column<P, double>(
          g, s, ex,
          [&](int e, int a, int iz) -> double { return iz == nrow - 1 ? phis[col_of(g, e, a)] : 0.0; },
          [&](int e, int a, int iz, double y) {
            if (a < P || (!g.periodic && e == g.Nx - 1)) A.q64b[(size_t)col_of(g, e, a) * nrow + iz] = y;
            else A.edge64b[(size_t)e * nrow + iz] = y;
          });
  }
  if (!grid_barrier(A.bar, g.status, s_flag)) return false;
  double acc[3] = {0.0, 0.0, 0.0};
  const int ncols = R.c1 - R.c0;
  for (int t = threadIdx.x; t < ncols * nrow; t += blockDim.x) {
    const int col = R.c0 + t / nrow, iz = t - (t / nrow) * nrow;
    const size_t i = (size_t)col * nrow + iz;
    if (iz == nrow - 1) { A.x[i] = phis[col]; continue; }
    const bool le = has_left_edge(g, col);
    const size_t ie = le ? (size_t)left_element(g, col) * nrow + iz : 0;
    double qv = A.q64[i];
    if (le) qv += ldcg(A.edge64 + ie);
    const double rv = -qv;
    A.r64[i] = rv;
    acc[0] += rv * rv;
    if (want_b) {
      double bv = A.q64b[i];
      if (le) bv += ldcg(A.edge64b + ie);
      acc[1] += bv * bv;
    }
    if (want_z) {
      const double zv = rv * g.invdiag64[i];
      A.z64[i] = zv;
      acc[2] += rv * zv;
    }
  }
  block_sum<3>(acc, red);
  put_partials<3>(A.part, A.part_stride, 0, acc);
  if (!grid_barrier(A.bar, g.status, s_flag)) return false;
  grid_sum<3>(A.part, A.part_stride, 0, acc, red);
  rr = acc[0];
  if (want_b) bb = acc[1];
  rz = acc[2];
  return true;
}

template <int P, bool MIXED>
__global__ void __launch_bounds__(kThreads) k_pcg(DevGeom g, PcgArgs A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[160];
  __shared__ int s_flag;
  const Range R = my_range(g);
  const int nrow = g.nrow;
  Smem<P, double> s64;
  s64.carve(smem_raw, nrow, g.Nz);
  s64.load_tables(g);
  double rr = 0.0, bb = 0.0, rz = 0.0;
  // r = b − A x0 and ‖b‖ (FP64)
  if (!fp64_residual<P>(g, s64, R, A, true, !MIXED, red, &s_flag, rr, bb, rz)) return;
  const double target = A.tol * A.tol * bb;
  int iters = 0, refinements = 0;
  if (bb == 0.0) {
    // φ̃ ≡ 0 on the surface: Φ = 0 is the solution.
    const int ncols = R.c1 - R.c0;
    for (int t = threadIdx.x; t < ncols * nrow; t += blockDim.x) {
      const int col = R.c0 + t / nrow, iz = t - (t / nrow) * nrow;
      if (iz != nrow - 1) A.x[(size_t)col * nrow + iz] = 0.0;
    }
    rr = 0.0;
  } else if (!MIXED) {
    double rr_out = rr;
    iters = inner_pcg<P, double>(g, s64, R, A.x, A.r64, A.z64, A.p64a, A.p64b, A.q64, A.edge64,
                                 g.invdiag64, A.part, A.part_stride, A.bar, red, &s_flag, rr, rz,
                                 target, A.max_iter, &rr_out);
    if (iters < 0) return;
    rr = rr_out;
  } else {
    Smem<P, float> s32;
    s32.carve(smem_raw, nrow, g.Nz);
    while (rr > target && iters < A.max_iter) {
      if (!(rr == rr) || isinf(rr)) { if (threadIdx.x == 0) atomicOr(g.status, ST_NONFINITE); break; }
      // inner: A δ = r in FP32 from δ = 0
      __syncthreads();
      s32.load_tables(g);
      __syncthreads();
      double acc[2] = {0.0, 0.0};
      const int ncols = R.c1 - R.c0;
      for (int t = threadIdx.x; t < ncols * nrow; t += blockDim.x) {
        const int col = R.c0 + t / nrow, iz = t - (t / nrow) * nrow;
        const size_t i = (size_t)col * nrow + iz;
        if (iz == nrow - 1) { A.d32[i] = 0.f; A.r32[i] = 0.f; A.z32[i] = 0.f; continue; }
        const float rv = (float)A.r64[i];
        const float zv = rv * g.invdiag32[i];
        A.d32[i] = 0.f;
        A.r32[i] = rv;
        A.z32[i] = zv;
        acc[0] += (double)rv * rv;
        acc[1] += (double)rv * zv;
      }
      block_sum<2>(acc, red);
      put_partials<2>(A.part, A.part_stride, 1, acc);
      if (!grid_barrier(A.bar, g.status, &s_flag)) return;
      grid_sum<2>(A.part, A.part_stride, 1, acc, red);
      double rr_in = acc[0];
      const double tgt_in = fmax(A.inner_rtol * A.inner_rtol * acc[0], 0.25 * target);
      const int it = inner_pcg<P, float>(g, s32, R, A.d32, A.r32, A.z32, A.p32a, A.p32b, A.q32,
                                         A.edge32, g.invdiag32, A.part, A.part_stride, A.bar, red,
                                         &s_flag, acc[0], acc[1], tgt_in, A.max_iter - iters, &rr_in);
      if (it < 0) return;
      iters += it;
      ++refinements;
      // x += δ (FP64), then the true FP64 residual
      for (int t = threadIdx.x; t < ncols * nrow; t += blockDim.x) {
        const int col = R.c0 + t / nrow, iz = t - (t / nrow) * nrow;
        if (iz == nrow - 1) continue;
        const size_t i = (size_t)col * nrow + iz;
        A.x[i] += (double)A.d32[i];
      }
      __syncthreads();
      s64.load_tables(g);
      if (!grid_barrier(A.bar, g.status, &s_flag)) return;
      double dummy_b = 0.0, dummy_z = 0.0;
      if (!fp64_residual<P>(g, s64, R, A, false, false, red, &s_flag, rr, dummy_b, dummy_z)) return;
      if (it == 0) break;   // no progress possible
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const double rel = bb > 0.0 ? sqrt(rr / bb) : 0.0;
    SolveRecord* rec = A.rec;
    rec->iterations = iters;
    rec->refinements = refinements;
    rec->rel_residual = rel;
    rec->solves += 1;
    rec->total_iterations += iters;
    rec->total_refinements += refinements;
    if (rel > rec->max_rel_residual) rec->max_rel_residual = rel;
    if (rr > target) atomicOr(g.status, ST_NOT_CONVERGED);
  }
}

// ------------------------------------------------------------------------------------
// Launchers (dispatch on P).
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

static size_t apply_smem_bytes(int P, int nrow, int Nz, size_t elem) {
  const int Q = P + 1;
  return elem * (size_t)(Q * Q + Q + nrow + 2 * Nz + 4 * Q + Q * nrow + 2 * Nz * Q * Q) + 16;
}

cudaError_t launch_geometry(const DevGeom& g, const double* eta, cudaStream_t s) {
  const int n1 = g.Nx * (g.P + 1);
  SEM_DISPATCH_P(g.P, (k_geometry<PP><<<(n1 + 127) / 128, 128, 0, s>>>(g, eta)));
  count_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const long long n = (long long)g.ncol * g.nrow;
  SEM_DISPATCH_P(g.P, (k_diag<PP><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(g)));
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_apply(const DevGeom& g, const double* x, double* y, double* qtmp, double* edge,
                         cudaStream_t s) {
  const size_t smem = apply_smem_bytes(g.P, g.nrow, g.Nz, sizeof(double));
  const int grid = g.Nx < 4096 ? g.Nx : 4096;
  cudaError_t e = cudaSuccess;
  SEM_DISPATCH_P(g.P, {
    e = cudaFuncSetAttribute(k_apply<PP>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e == cudaSuccess) k_apply<PP><<<grid, kThreads, smem, s>>>(g, x, qtmp, edge);
  });
  if (e != cudaSuccess) return e;
  count_launch();
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const long long n = (long long)g.ncol * g.nrow;
  k_apply_fix<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(g, qtmp, edge, y);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_l2g(const DevGeom& g, int32_t* l2g, cudaStream_t s) {
  const long long total = (long long)g.Nx * g.Nz * (g.P + 1) * (g.P + 1);
  k_l2g<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(g, l2g);
  count_launch();
  return cudaGetLastError();
}

constexpr int kMaxDynSmem = 200 * 1024;   // opt-in ceiling; each launch passes its own size

template <int P, bool MIXED>
static cudaError_t pcg_occupancy(size_t smem, int* per_sm) {
  cudaError_t e = cudaFuncSetAttribute(k_pcg<P, MIXED>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       kMaxDynSmem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_pcg<P, MIXED>, kThreads, smem);
}

cudaError_t pcg_grid_size(int P, int Nz, int nrow, int Nx, int mixed, int* grid, size_t* smem) {
  *smem = apply_smem_bytes(P, nrow, Nz, sizeof(double));
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if (mixed) { SEM_DISPATCH_P(P, (e = pcg_occupancy<PP, true>(*smem, &per_sm))); }
  else { SEM_DISPATCH_P(P, (e = pcg_occupancy<PP, false>(*smem, &per_sm))); }
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  long long cap = (long long)per_sm * sms;
  *grid = (int)(Nx < cap ? Nx : cap);
  return cudaSuccess;
}

cudaError_t launch_pcg(const DevGeom& g, const PcgArgs& a, int grid, size_t smem, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(a.bar, 0, 2 * sizeof(unsigned int), s);
  if (e != cudaSuccess) return e;
  DevGeom gg = g;
  PcgArgs aa = a;
  void* args[] = {&gg, &aa};
  if (a.mixed) {
    SEM_DISPATCH_P(g.P, (e = cudaLaunchCooperativeKernel((const void*)k_pcg<PP, true>, grid, kThreads,
                                                         args, smem, s)));
  } else {
    SEM_DISPATCH_P(g.P, (e = cudaLaunchCooperativeKernel((const void*)k_pcg<PP, false>, grid, kThreads,
                                                         args, smem, s)));
  }
  count_launch();
  return e;
}

}  // namespace semgb
