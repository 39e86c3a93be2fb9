// Internal declarations shared by the library's translation units (not installed).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace semgb {

constexpr int kMaxP = 12;
constexpr int kMaxNz = 16;
constexpr int kThreads = 256;

// Offsets of the order-P tables inside the packed constant arrays (orders 1..kMaxP).
__host__ __device__ constexpr int d_off(int P) { return P * (P + 1) * (2 * P + 1) / 6 - 1; }
__host__ __device__ constexpr int w_off(int P) { return P * (P + 1) / 2 - 1; }
constexpr int kDTotal = d_off(kMaxP + 1);
constexpr int kWTotal = w_off(kMaxP + 1);

// Wall-clock limit of a team barrier wait (sem_set_barrier_test can shorten it).
constexpr unsigned long long kBarrierTimeoutNs = 2000000000ull;   // 2 s

// Device status bits (OR-ed into the mesh's status word).
enum : int { ST_NOT_CONVERGED = 1, ST_NONFINITE = 2, ST_TIMEOUT = 4, ST_BAD_DEPTH = 8 };

// Division by a divisor fixed per mesh, for the work-item decompositions of the kernels (an
// integer division by a run-time value costs tens of instructions): ⌊n/d⌋ = umulhi(n, ⌈2³²/d⌉),
// exact for 0 ≤ n < 2³²/d (d ≥ 2).
struct FastDiv {
  unsigned m;
  int d;
  static FastDiv make(int dd) { return FastDiv{(unsigned)((0x100000000ull + (unsigned)dd - 1) / (unsigned)dd), dd}; }
  __device__ __forceinline__ int div(int n) const { return (int)__umulhi((unsigned)n, m); }
};

// Read-only view of a mesh for the volume kernels.
struct DevGeom {
  int P, Nx, Nz, ncol, nrow, periodic;
  int chunk;             // element columns a CTA processes together in one pass (≥ 1)
  const double* h;       // [ncol] still-water depth at the columns
  const double* hx_loc;  // [Nx*(P+1)] element-local ∂x h
  const double* dxe;     // [Nx] element widths Δx_e
  const double* dsl;     // [Nz] layer heights Δσ_l
  const double* sig;     // [nrow] σ of each row
  const double* cxz;     // [Nx][Nz][2] Δσ_l/Δx_e, Δx_e/Δσ_l (constant per mesh)
  const double* r2dx;    // [Nx] 2/Δx_e
  double* geo64;         // [Nx*(P+1)*4] per element-local column: d, 1/d, ∂x h, ∂x d
  float* geo32;          // same in FP32 (inner solves of the mixed path)
  double* invdiag64;     // [n] 1 / diag(−𝓛) at interior nodes, 0 at the surface
  float* invdiag32;      // same in FP32
  int* status;           // device status word
  int gcache;            // doubles of dynamic shared memory after the FP64 apply's buffers that
                         // hold a solve's geometric factors (single-mesh fused stage; 0 = none)
  double* gglob;         // [Nx][Nz][(P+1)²][3] geometric factors of the FP64 applies of a solve,
                         // when they do not fit in shared memory (each CTA fills its own elements)
  unsigned long long bar_timeout_ns;   // wall-clock limit of every team barrier wait
  int drop_rank;         // testing: this team rank leaves the next launch before its first
                         // barrier, so the others' bounded waits run out (−1: none)
  FastDiv dv_nrow, dv_nr, dv_colsz, dv_elsz, dv_qn;   // Nrow, Nrow−1, (P+1)Nrow, Nz(P+1)², (P+1)(Nrow−1)
  unsigned long long* trace;   // phase trace of builds compiled with -DSEM_TRACE (else unused):
                               // [0] = marks so far, then (tag, %globaltimer) pairs
};

// Phase trace (diagnostic builds only, compiled with -DSEM_TRACE): thread 0 of team rank 0
// stamps %globaltimer with a tag at the phase boundaries of the Krylov and fused stage kernels.
constexpr int kTraceMax = 4096;
enum : int {
  TR_START = 1, TR_SETUP = 2, TR_BAR_SETUP = 3, TR_PIVOTS = 4, TR_RESIDUAL = 5, TR_GCACHE = 6,
  TR_IT_APPLY = 10, TR_IT_BAR1 = 11, TR_IT_SCALARS = 12, TR_IT_UPDATE = 13, TR_IT_BAR2 = 14,
  TR_IT_INTERFACE = 15, TR_IT_BAR3 = 16, TR_IT_BACKSUB = 17, TR_CG_START = 18, TR_CG_END = 19,
  TR_REFINE = 20, TR_SOLVED = 30, TR_WSX = 31, TR_MINT1 = 32, TR_MBACK1 = 33, TR_ZAK = 34, TR_MINT2 = 35,
  TR_RK4 = 36, TR_FILTER = 37, TR_END = 38,
  TR_UPD_VEC = 40, TR_UPD_SIGMA = 41, TR_UPD_COND = 42, TR_BS_INTERIOR = 43, TR_BS_SIGMA = 44,
  TR_AP_LOAD = 45, TR_AP_F = 46, TR_AP_Y = 47
};

// Element columns processed together per CTA pass: enough that a pass has ~256–512 work
// items when the element columns are small (few layers, low order), at most 16.
inline int chunk_width(int P, int Nz) {
  const int per = Nz * (P + 1) * (P + 1);
  const int E = 384 / per;
  return E < 1 ? 1 : (E > 16 ? 16 : E);
}

// Per-solve record written by the Krylov kernel and accumulated counters.
struct SolveRecord {
  int iterations;
  int refinements;
  double rel_residual;
  long long solves;
  long long total_iterations;
  long long total_refinements;
  double max_rel_residual;
};

enum : int { PREC_SEPARABLE = 0, PREC_JACOBI = 1 };

// σ-separable preconditioner (exact inverse of Kx(d)⊗Mσ + Mx(1/d)⊗Kσ, see kernels_laplace.cu).
// All per-mode arrays are mode-major.
template <class T>
struct PrecView {
  int nr;                  // σ modes = interior rows (Nrow − 1)
  int nif;                 // interface unknowns per mode (Nx periodic, Nx+1 walls)
  const T* S;              // [nr*nr]   S[j*nr + k]: σ-eigenvectors, Sᵀ Mσ S = I
  const T* ST;             // [nr*nr]   ST[k*nr + j] = S[j*nr + k] (the backward transform reads it)
  // the element blocks are stored mode-fastest, so that threads of consecutive modes read
  // consecutive words
  const T* Aii;            // [Nx][P−1][P−1][nr] inverse interior block of the mode-k element matrix
  const T* Z;              // [Nx][2][P−1][nr]  E_bi E_ii⁻¹ (left, right boundary rows)
  const T* te;             // [nr][nif] interface tridiagonal off-diagonals
  const T* tm;             // [nr][nif] Thomas pivots 1/(d_j − e_{j−1} c'_{j−1})
  const T* tcp;            // [nr][nif] Thomas c'_j
  const T* tz;             // [nr][nif] periodic: T'⁻¹u of the Sherman–Morrison closure
  const T* tvl;            // [nr] periodic: v_{N−1}
  const T* tfac;           // [nr] periodic: 1/(1 + vᵀT'⁻¹u)
  T* gL;                   // [nr][Nx] condensed right-hand side, left interface of element
  T* gR;                   // [nr][Nx] condensed right-hand side, right interface of element
  T* zb;                   // [nr][nif] interface solution
  T* rhat;                 // [ncol][nr] σ-transformed residual
};

// Set-up data written per stage by the preconditioner set-up kernels.  The preconditioner is
// applied in FP32 by both precisions' solves, so its factors are FP32 (the element Schur
// complements are formed in FP64 before they are rounded).
struct PrecSetup {
  int nr, nif;
  const double* lam;       // [nr] σ eigenvalues
  double* schur;           // [nr][Nx][3]  S00, S01, S11 of the condensed element matrix
  PrecView<float> v32;
  // writable aliases of the factor arrays
  float *Aii32, *Z32, *te32, *tm32, *tcp32, *tz32, *tvl32, *tfac32;
};

struct PcgArgs {
  double* x;              // Φ [n]
  const double* phis;     // φ̃ [ncol]
  // FP64 level: residual, CG vectors and apply outputs
  double *r64, *z64, *p64a, *p64b, *q64, *q64b, *edge64, *edge64b;
  // FP32 level (mixed precision inner solve)
  float *d32, *r32, *z32, *p32a, *p32b, *q32, *edge32;
  double* part;           // reduction partials [4 slots][4 values][max grid]
  int part_stride;        // max grid
  unsigned int* bar;      // grid barrier: arrival counter (two words), zero at launch
  SolveRecord* rec;
  double* r64b;           // second residual buffer (double-buffered update)
  float* r32b;
  double* s64b;           // second buffer of s = A p
  float* s32b;
  double* uh64;           // preconditioned residual on each CTA's halo column, [grid][nrow]
  float* uh32;
  PrecView<float> pv32;    // the preconditioner of both precisions' solves
  int precond;            // PREC_SEPARABLE or PREC_JACOBI
  double tol;
  double inner_rtol;
  int max_iter;
  int mixed;
};

// Tables for the surface kernels (per mesh, device memory), offsets into one buffer.
struct SurfTables {
  int P, Pf, Nx, Nz, ncol, nrow, periodic;
  double g;
  const double* D;        // (P+1)²  differentiation on the GLL nodes
  const double* MD;       // (P+1)²  M·D (element S_x without scale)
  const double* B;        // (P+1)×(Pf+1)  Iᵀ M_f (over-integration projection)
  const double* I;        // (Pf+1)×(P+1)  interpolation to the fine nodes
  const double* F;        // (P+1)²  modal filter
  const double* wrow;     // [nrow] row weights of the w̃ projection: w̃ d = Σ_iz wrow_iz Φ_iz
  const double* Aii;      // (P−1)²  inverse interior block of M
  const double* Z;        // 2×(P−1) M_bi M_ii⁻¹
  const double* se;       // [Nx] Δx_e / 2
  const double* dsl;      // [Nz]
  const double* h;        // [ncol]
  const double* th_e;     // interface tridiagonal: off-diagonals  [N]
  const double* th_m;     // Thomas pivots                           [N]
  const double* th_cp;    // Thomas c'                               [N]
  const double* th_z;     // periodic: T'⁻¹u                         [N]
  double th_vlast;        // periodic: v_{N−1}
  double th_fac;          // periodic: 1/(1 + vᵀ T'⁻¹u)
  int nif;                // interface unknowns N
  int filter_on;
  // relaxation zones (§2.2)
  const double* xcol;     // [ncol] column positions
  double x0, x1;          // tank ends
  double relax_left, relax_right;
  int ncomp;              // components of the generated signal
  const double* wave;     // [4][ncomp]: a, ω, k, θ
  // the generated signal by angle addition (fused stage): cos(ωt + θ − kx) from cos, sin of
  // ωt + θ (per stage) and of kx (per column, fixed); nzl = columns of the left zone, which are
  // the first columns; wkx = nullptr: evaluated directly
  int nzl;
  const double* wkx;      // [nzl][ncomp][2]: cos k_i x, sin k_i x
  double* wA;             // [4][ncomp] per stage: a cos A, a sin A, c sin A, c cos A (A = ωt + θ, c = −g a/ω)
  double* wEP;            // [nzl][2] per stage: generated η and φ̃ at the left-zone columns
};

// One instance (mesh + state) of a fused RK stage launch.
struct Instance {
  DevGeom g;
  SurfTables st;
  PcgArgs pa;            // pa.x = the mesh's potential (warm start), pa.phis set per stage
  PrecSetup ps;
  double *eta, *phis;    // state, updated at stage 4
  double *s0e, *s0p;     // stage inputs (double-buffered: stages 2 and 4 read s0, stage 3 reads s1)
  double *s1e, *s1p;
  double *ke, *kp, *ae, *ap;
  double *wt, *etax, *phisx, *R, *scr;
  double *P1, *P2, *P3;  // stage potentials: P1, P2 of this step, P3 of the last stage 3
  double *D32;           // Φ₃ − Φ₂ of the last step
  double tstart, dt, tau;
  int team0, nteam;      // first CTA and number of CTAs of this instance's team
  int relax;
  int hist;              // P3 belongs to the step before this call's first step (same trajectory)
};

struct StageArgs {
  const Instance* inst;  // device array
  const int* cta_inst;   // CTA → instance
  unsigned int* bars;    // 2 per instance, zero at launch (cooperative launches)
  int stage;             // 1..4; 0 = Laplace solve only
  int step;              // steps since tstart
  int cluster;           // 1: cluster-team launch (each instance's CTAs are one cluster)
};

// ---- per-order entry points (laplace_device.cuh, instantiated in kernels_order.cu) ----
template <int P> cudaError_t upload_tables_impl(const double* D64, const double* w64);
template <int P> cudaError_t launch_geometry_impl(const DevGeom& g, const double* eta, bool with_diag,
                                                  cudaStream_t s);
template <int P> cudaError_t launch_apply_elem_impl(const DevGeom& g, const double* x, double* q, double* edge,
                                                    cudaStream_t s);
template <int P> cudaError_t pcg_occupancy_impl(int mixed, size_t smem, int* per_sm);
template <int P> cudaError_t launch_pcg_impl(int mixed, const DevGeom& g, const PcgArgs& a, int grid, size_t smem,
                                             cudaStream_t s);
template <int P> cudaError_t launch_prec_setup_impl(const DevGeom& g, const PrecSetup& ps, cudaStream_t s);
template <int P> cudaError_t launch_apply_tile_impl(int fp32, const DevGeom& g, const void* x, void* y,
                                                    cudaStream_t s);
template <int P> cudaError_t stage_occupancy_impl(int mixed, int wide, size_t smem, int* per_sm);
template <int P> cudaError_t launch_stage_impl(int mixed, int wide, const StageArgs& a, int grid, size_t smem,
                                               cudaStream_t s);
template <int P> cudaError_t cluster_fit_impl(int mixed, int wide, int csize, size_t smem, int* active_clusters);
template <int P> cudaError_t launch_stage_cluster_impl(int mixed, int wide, const StageArgs& a, int grid, int csize,
                                                       size_t smem, cudaStream_t s);

// ---- launchers (kernels_laplace.cu) ----
// Fused RK stage for instances of order P: capacity (CTAs per SM) at a given dynamic smem,
// and the cooperative launch.  wide = 0: the one-CTA-per-SM variant (single meshes);
// wide = 1: the two-CTAs-per-SM variant (batches).
cudaError_t stage_occupancy(int P, int mixed, int wide, size_t smem, int* per_sm);
size_t stage_smem_bytes(int P, int nrow, int Nz, int chunk);
cudaError_t launch_stage(int P, int mixed, int wide, const StageArgs& a, int grid, size_t smem, cudaStream_t s);
// Cluster teams (every instance's CTAs form one thread-block cluster of csize CTAs, grid = members ×
// csize): no cooperative launch, so launches of different groups may run at once.  cluster_fit
// gives how many such clusters can be resident at once (0: the cluster size does not fit).
cudaError_t cluster_fit(int P, int mixed, int wide, int csize, size_t smem, int* active_clusters);
cudaError_t launch_stage_cluster(int P, int mixed, int wide, const StageArgs& a, int grid, int csize, size_t smem,
                                 cudaStream_t s);
// out[k] = status word of inst[k]; a nonzero word is cleared after it is read.
cudaError_t launch_gather_status(const Instance* inst, int n, int* out, cudaStream_t s);
cudaError_t upload_line_tables(const double* D64, const double* w64);  // packed, all orders
// σ-geometry per element-local column; with_diag also builds the Jacobi diagonal.
cudaError_t launch_geometry(const DevGeom& g, const double* eta, bool with_diag, cudaStream_t s);
cudaError_t launch_apply(const DevGeom& g, const double* x, double* y, double* qtmp, double* edge,
                         cudaStream_t s);
cudaError_t launch_l2g(const DevGeom& g, int32_t* l2g, cudaStream_t s);
// Tiled apply y = 𝓛x at every node in FP32 (fp32 = 1: CUDA-core kernel; fp32 = 3: tensor-core
// kernel for orders 4..7, else the CUDA-core one; x, y float) or FP64 (fp32 = 0, x, y double), from
// the geometry of the last launch_geometry; x and y must not overlap.  No workspace.
cudaError_t launch_apply_tile(int fp32, const DevGeom& g, const void* x, void* y, cudaStream_t s);
// Tile width of the tiled apply for (P, Nz): 0 = the widest that keeps three CTAs per SM.
void set_apply_tile_width(int P, int Nz, int E);
int apply_tile_width(int P, int Nz);
// Allocation-free apply (scratch in a static device array of kNoAllocEdgeMax doubles).
constexpr size_t kNoAllocEdgeMax = size_t(1) << 20;
cudaError_t launch_apply_noalloc(const DevGeom& g, const double* x, double* y, cudaStream_t s);
cudaError_t pcg_grid_size(int P, int Nz, int nrow, int Nx, int chunk, int mixed, int* grid, size_t* smem);
cudaError_t launch_prec_setup(const DevGeom& g, const PrecSetup& ps, cudaStream_t s);
cudaError_t launch_pcg(const DevGeom& g, const PcgArgs& a, int grid, size_t smem, cudaStream_t s);

// ---- launchers (kernels_surface.cu) ----
cudaError_t launch_wsurf(const SurfTables& t, const double* Phi, const double* eta, double* w,
                         cudaStream_t s);
cudaError_t launch_sx(const SurfTables& t, const double* f0, const double* f1, double* R,
                      cudaStream_t s);
cudaError_t launch_mass1d(const SurfTables& t, const double* R, int nrhs, double* u0, double* u1,
                          double* scratch, cudaStream_t s);
cudaError_t launch_zakharov(const SurfTables& t, const double* eta, const double* etax,
                            const double* phisx, const double* w, double* R, cudaStream_t s);
cudaError_t launch_filter(const SurfTables& t, double* q0, double* q1, cudaStream_t s);
// Adds the relaxation source (1 − γ)(q_a − q)/τ to (de, dp) in the zones.
cudaError_t launch_relax(const SurfTables& t, const double* eta, const double* phis, double time,
                         double inv_tau, double* de, double* dp, cudaStream_t s);
// RK4 stage update on (η, φ̃): see kernels_surface.cu for the stage semantics.
cudaError_t launch_rk4_stage(int stage, int n, double dt, double* eta, double* phis,
                             const double* keta, const double* kphis, double* acc_eta,
                             double* acc_phis, double* st_eta, double* st_phis, cudaStream_t s);

// ---- device helpers shared by the translation units ----
__device__ __forceinline__ double fmx(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fmx(float a, float b, float c) { return fmaf(a, b, c); }

// One warp solves a tridiagonal system with precomputed Thomas factors (pivots m_j, c'_j,
// off-diagonals e_j), closed by Sherman–Morrison when `periodic` (T'⁻¹u = tz, v_{N−1} =
// tvl, factor tfac).  The two first-order recurrences
//     y_j = g_j m_j − (e_{j−1} m_j) y_{j−1},        x_j = y_j − c'_j x_{j+1},
// are evaluated as a parallel prefix over affine maps: each lane composes a contiguous
// chunk, the lanes scan the composed maps with shuffles, then each lane replays its chunk.
// `gfun(j)` returns the right-hand side; `out` (N values, global or shared) receives x.
// Must be called by all 32 lanes of a warp.
// Chunks of at most kTridiagRegs values per lane (N ≤ 32·kTridiagRegs) are kept in registers
// between the passes: the right-hand side and the factors are read once, y never leaves the lane.
constexpr int kTridiagRegs = 4;

template <class T, class GFun>
__device__ __forceinline__ void warp_tridiag(int N, GFun gfun, const T* te, const T* tm, const T* tcp,
                                             bool periodic, const T* tz, T tvl, T tfac, T* out) {
  const int lane = threadIdx.x & 31;
  const int c = (N + 31) / 32;
  const int j0 = min(N, lane * c), j1 = min(N, j0 + c);
  const unsigned full = 0xffffffffu;
  if (c <= kTridiagRegs) {
    // the same operations in the same order as below, on register copies of the chunk
    T al[kTridiagRegs], gm[kTridiagRegs], cp[kTridiagRegs], v[kTridiagRegs];
#pragma unroll
    for (int q = 0; q < kTridiagRegs; ++q) {
      const int j = j0 + q;
      if (j < j1) {
        const T m = tm[j];
        al[q] = j > 0 ? -te[j - 1] * m : T(0);
        gm[q] = gfun(j) * m;
        cp[q] = tcp[j];
      }
    }
    T A = T(1), B = T(0);
#pragma unroll
    for (int q = 0; q < kTridiagRegs; ++q)
      if (j0 + q < j1) { B = fmx(al[q], B, gm[q]); A = al[q] * A; }
    for (int o = 1; o < 32; o <<= 1) {
      const T Ap = __shfl_up_sync(full, A, o), Bp = __shfl_up_sync(full, B, o);
      if (lane >= o) { B = fmx(A, Bp, B); A = A * Ap; }
    }
    T y = __shfl_up_sync(full, B, 1);
    if (lane == 0) y = T(0);
#pragma unroll
    for (int q = 0; q < kTridiagRegs; ++q)
      if (j0 + q < j1) { y = fmx(al[q], y, gm[q]); v[q] = y; }
    A = T(1); B = T(0);
#pragma unroll
    for (int q = kTridiagRegs - 1; q >= 0; --q)
      if (j0 + q < j1) { const T ga = -cp[q]; B = fmx(ga, B, v[q]); A = ga * A; }
    for (int o = 1; o < 32; o <<= 1) {
      const T An = __shfl_down_sync(full, A, o), Bn = __shfl_down_sync(full, B, o);
      if (lane + o < 32) { B = fmx(A, Bn, B); A = A * An; }
    }
    T x = __shfl_down_sync(full, B, 1);
    if (lane == 31) x = T(0);
#pragma unroll
    for (int q = kTridiagRegs - 1; q >= 0; --q)
      if (j0 + q < j1) { x = fmx(-cp[q], x, v[q]); v[q] = x; }
    if (periodic) {
      // x_0 is on lane 0, x_{N−1} on the lane whose chunk ends at N
      const T x0 = __shfl_sync(full, v[0], 0);
      const int ln = (N - 1) / c;
      T xl = v[0];
#pragma unroll
      for (int q = 1; q < kTridiagRegs; ++q)
        if (j0 + q == N - 1) xl = v[q];
      const T xN = __shfl_sync(full, xl, ln);
      const T cc = (x0 + tvl * xN) * tfac;
#pragma unroll
      for (int q = 0; q < kTridiagRegs; ++q)
        if (j0 + q < j1) v[q] = fmx(-cc, tz[j0 + q], v[q]);
    }
#pragma unroll
    for (int q = 0; q < kTridiagRegs; ++q)
      if (j0 + q < j1) out[j0 + q] = v[q];
    __syncwarp();
    return;
  }
  // forward: y_j = α_j y_{j−1} + β_j, α_j = −e_{j−1} m_j, β_j = g_j m_j
  T A = T(1), B = T(0);
  for (int j = j0; j < j1; ++j) {
    const T m = tm[j];
    const T al = j > 0 ? -te[j - 1] * m : T(0);
    B = fmx(al, B, gfun(j) * m);
    A = al * A;
  }
  for (int o = 1; o < 32; o <<= 1) {
    const T Ap = __shfl_up_sync(full, A, o), Bp = __shfl_up_sync(full, B, o);
    if (lane >= o) { B = fmx(A, Bp, B); A = A * Ap; }
  }
  T y = __shfl_up_sync(full, B, 1);
  if (lane == 0) y = T(0);
  for (int j = j0; j < j1; ++j) {
    const T m = tm[j];
    const T al = j > 0 ? -te[j - 1] * m : T(0);
    y = fmx(al, y, gfun(j) * m);
    out[j] = y;
  }
  __syncwarp();
  // backward: x_j = γ_j x_{j+1} + y_j, γ_j = −c'_j (c'_{N−1} = 0)
  A = T(1); B = T(0);
  for (int j = j1 - 1; j >= j0; --j) {
    const T ga = -tcp[j];
    B = fmx(ga, B, out[j]);
    A = ga * A;
  }
  for (int o = 1; o < 32; o <<= 1) {
    const T An = __shfl_down_sync(full, A, o), Bn = __shfl_down_sync(full, B, o);
    if (lane + o < 32) { B = fmx(A, Bn, B); A = A * An; }
  }
  T x = __shfl_down_sync(full, B, 1);
  if (lane == 31) x = T(0);
  for (int j = j1 - 1; j >= j0; --j) {
    x = fmx(-tcp[j], x, out[j]);
    out[j] = x;
  }
  __syncwarp();
  if (periodic) {
    const T cc = (out[0] + tvl * out[N - 1]) * tfac;
    __syncwarp();
    for (int j = lane; j < N; j += 32) out[j] = fmx(-cc, tz[j], out[j]);
    __syncwarp();
  }
}

// All threads of the CTA solve one tridiagonal system: the factors and recurrences of
// warp_tridiag, with chunks of ⌈N/blockDim⌉ values per thread and the scan of the composed affine
// maps across the CTA (shuffles within each warp, the warps' totals scanned by warp 0 through
// shared memory).  For long systems (N > 32·kTridiagRegs), where a warp alone would walk chunks of
// N/32 values.  Must be called by every thread of the CTA (it synchronises the CTA).
// Chunks of at most kCtaRegs values per thread keep the right-hand side and y in registers
// between the passes of cta_tridiag (N ≤ kCtaRegs·blockDim).
constexpr int kCtaRegs = 12;

// CACHE (compile time): keep the chunk in registers (the one-CTA-per-SM build, which has the registers).
template <class T, class GFun, bool CACHE = false>
__device__ void cta_tridiag(int N, GFun gfun, const T* te, const T* tm, const T* tcp, bool periodic,
                            const T* tz, T tvl, T tfac, T* out) {
  __shared__ T sA[32], sB[32];
  const int nt = blockDim.x, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
  const int c = (N + nt - 1) / nt;
  const int j0 = min(N, tid * c), j1 = min(N, j0 + c);
  const unsigned full = 0xffffffffu;
  const bool regs = CACHE && c <= kCtaRegs;
  T gr[kCtaRegs], vr[kCtaRegs];                   // g_j m_j, then y_j and x_j, of this chunk
  // forward: y_j = α_j y_{j−1} + β_j over this thread's chunk
  T A = T(1), B = T(0);
  if (regs) {
#pragma unroll
    for (int q = 0; q < kCtaRegs; ++q) {
      const int j = j0 + q;
      if (j < j1) {
        const T m = tm[j];
        const T al = j > 0 ? -te[j - 1] * m : T(0);
        gr[q] = gfun(j) * m;
        B = fmx(al, B, gr[q]);
        A = al * A;
      }
    }
  } else {
    for (int j = j0; j < j1; ++j) {
      const T m = tm[j];
      const T al = j > 0 ? -te[j - 1] * m : T(0);
      B = fmx(al, B, gfun(j) * m);
      A = al * A;
    }
  }
  for (int o = 1; o < 32; o <<= 1) {             // inclusive scan over the lanes
    const T Ap = __shfl_up_sync(full, A, o), Bp = __shfl_up_sync(full, B, o);
    if (lane >= o) { B = fmx(A, Bp, B); A = A * Ap; }
  }
  __syncthreads();                                // earlier users of sA, sB are done
  if (lane == 31) { sA[wid] = A; sB[wid] = B; }
  __syncthreads();
  if (wid == 0) {                                 // exclusive scan over the warps
    T a = lane < nw ? sA[lane] : T(1), b = lane < nw ? sB[lane] : T(0);
    for (int o = 1; o < 32; o <<= 1) {
      const T ap = __shfl_up_sync(full, a, o), bp = __shfl_up_sync(full, b, o);
      if (lane >= o) { b = fmx(a, bp, b); a = a * ap; }
    }
    T eb = __shfl_up_sync(full, b, 1);
    if (lane == 0) eb = T(0);
    if (lane < nw) sB[lane] = eb;                 // y at the end of the warps before
  }
  __syncthreads();
  {
    T Al = __shfl_up_sync(full, A, 1), Bl = __shfl_up_sync(full, B, 1);
    if (lane == 0) { Al = T(1); Bl = T(0); }
    T y = fmx(Al, sB[wid], Bl);                   // y_{j0−1}
    if (regs) {
#pragma unroll
      for (int q = 0; q < kCtaRegs; ++q) {
        const int j = j0 + q;
        if (j < j1) {
          const T al = j > 0 ? -te[j - 1] * tm[j] : T(0);
          y = fmx(al, y, gr[q]);
          vr[q] = y;
        }
      }
    } else {
      for (int j = j0; j < j1; ++j) {
        const T m = tm[j];
        const T al = j > 0 ? -te[j - 1] * m : T(0);
        y = fmx(al, y, gfun(j) * m);
        out[j] = y;
      }
    }
  }
  // backward: x_j = γ_j x_{j+1} + y_j, γ_j = −c'_j (c'_{N−1} = 0), chunks from the top
  A = T(1); B = T(0);
  if (regs) {
#pragma unroll
    for (int q = kCtaRegs - 1; q >= 0; --q) {
      const int j = j0 + q;
      if (j < j1) {
        const T ga = -tcp[j];
        B = fmx(ga, B, vr[q]);
        A = ga * A;
      }
    }
  } else {
    for (int j = j1 - 1; j >= j0; --j) {
      const T ga = -tcp[j];
      B = fmx(ga, B, out[j]);
      A = ga * A;
    }
  }
  for (int o = 1; o < 32; o <<= 1) {
    const T An = __shfl_down_sync(full, A, o), Bn = __shfl_down_sync(full, B, o);
    if (lane + o < 32) { B = fmx(A, Bn, B); A = A * An; }
  }
  __syncthreads();
  if (lane == 0) { sA[wid] = A; sB[wid] = B; }
  __syncthreads();
  if (wid == 0) {
    T a = lane < nw ? sA[lane] : T(1), b = lane < nw ? sB[lane] : T(0);
    for (int o = 1; o < 32; o <<= 1) {
      const T an = __shfl_down_sync(full, a, o), bn = __shfl_down_sync(full, b, o);
      if (lane + o < 32) { b = fmx(a, bn, b); a = a * an; }
    }
    T eb = __shfl_down_sync(full, b, 1);
    if (lane == 31) eb = T(0);
    if (lane < nw) sB[lane] = eb;                 // x at the start of the warps after
  }
  __syncthreads();
  {
    T An = __shfl_down_sync(full, A, 1), Bn = __shfl_down_sync(full, B, 1);
    if (lane == 31) { An = T(1); Bn = T(0); }
    T x = fmx(An, sB[wid], Bn);                   // x_{j1}
    if (regs) {
#pragma unroll
      for (int q = kCtaRegs - 1; q >= 0; --q) {
        const int j = j0 + q;
        if (j < j1) {
          x = fmx(-tcp[j], x, vr[q]);
          vr[q] = x;
          out[j] = x;
        }
      }
    } else {
      for (int j = j1 - 1; j >= j0; --j) {
        x = fmx(-tcp[j], x, out[j]);
        out[j] = x;
      }
    }
  }
  __syncthreads();
  if (periodic) {
    const T cc = (out[0] + tvl * out[N - 1]) * tfac;
    __syncthreads();
    for (int j = j0; j < j1; ++j) out[j] = fmx(-cc, tz[j], out[j]);
    __syncthreads();
  }
}

// Launch counter (all kernels of this library).
void count_launch(int k = 1);

}  // namespace semgb
