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

// Device status bits (OR-ed into the mesh's status word).
enum : int { ST_NOT_CONVERGED = 1, ST_NONFINITE = 2, ST_TIMEOUT = 4, ST_BAD_DEPTH = 8 };

// Read-only view of a mesh for the volume kernels.
struct DevGeom {
  int P, Nx, Nz, ncol, nrow, periodic;
  const double* h;       // [ncol] still-water depth at the columns
  const double* hx_loc;  // [Nx*(P+1)] element-local ∂x h
  const double* dxe;     // [Nx] element widths Δx_e
  const double* dsl;     // [Nz] layer heights Δσ_l
  const double* sig;     // [nrow] σ of each row
  double* geo64;         // [Nx*(P+1)*4] per element-local column: d, 1/d, ∂x h, ∂x d
  float* geo32;          // same in FP32 (inner solves of the mixed path)
  double* invdiag64;     // [n] 1 / diag(−𝓛) at interior nodes, 0 at the surface
  float* invdiag32;      // same in FP32
  int* status;           // device status word
};

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

struct PcgArgs {
  double* x;              // Φ [n]
  const double* phis;     // φ̃ [ncol]
  // FP64 level: residual, CG vectors and apply outputs
  double *r64, *z64, *p64a, *p64b, *q64, *q64b, *edge64, *edge64b;
  // FP32 level (mixed precision inner solve)
  float *d32, *r32, *z32, *p32a, *p32b, *q32, *edge32;
  double* part;           // reduction partials [4 slots][4 values][max grid]
  int part_stride;        // max grid
  unsigned int* bar;      // grid barrier {arrive, generation}
  SolveRecord* rec;
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
  const double* cw;       // Nz×(P+1) σ-contraction weights of the w̃ projection
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
};

// ---- launchers (kernels_laplace.cu) ----
cudaError_t upload_line_tables(const double* D64, const double* w64);  // packed, all orders
cudaError_t launch_geometry(const DevGeom& g, const double* eta, cudaStream_t s);
cudaError_t launch_apply(const DevGeom& g, const double* x, double* y, double* qtmp, double* edge,
                         cudaStream_t s);
cudaError_t launch_l2g(const DevGeom& g, int32_t* l2g, cudaStream_t s);
cudaError_t pcg_grid_size(int P, int Nz, int nrow, int Nx, int mixed, int* grid, size_t* smem);
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
// RK4 stage update on (η, φ̃): see kernels_surface.cu for the stage semantics.
cudaError_t launch_rk4_stage(int stage, int n, double dt, double* eta, double* phis,
                             const double* keta, const double* kphis, double* acc_eta,
                             double* acc_phis, double* st_eta, double* st_phis, cudaStream_t s);

// Launch counter (all kernels of this library).
void count_launch(int k = 1);

}  // namespace semgb
