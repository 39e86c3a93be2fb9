// Free-surface kernels (§3.1.1, §3.1.3, §3.3, §3.4 of arXiv 1512.02548), FP64, sm_103a.
//
//  * w̃ (eq. velocpot2).  On the tensor-product mesh the 2D mass is M = M_x ⊗ M_σ and
//    the σ-derivative (1/d)∂σΦ is continuous across x-element edges, so the surface row
//    of M⁻¹ S_z Φ reduces exactly to a per-column contraction
//        w̃(x_i) = Σ_l Σ_b c_{l,b} · (1/d_i) (2/Δσ_l) (D Φ_{i,l})_b,
//    with c_l = (Δσ_l/2) M · (M_σ⁻¹ e_top)|_layer l precomputed on the host.  No 2D mass
//    solve is needed; the result equals the global projection up to rounding.
//  * S_x f and the over-integrated Zakharov integrals are formed per element
//    (unassembled), and one kernel solves M' u = Σ_e Q_eᵀ R_e by static condensation:
//    element-interior unknowns are eliminated with the precomputed M_ii⁻¹, the interface
//    unknowns form a tridiagonal system (cyclic when periodic, closed by
//    Sherman–Morrison) solved with precomputed Thomas factors, then the interiors are
//    recovered.  M' is constant in time, so only the right-hand sides change.
//  * The modal filter F = V̂SV̂⁻¹ acts per element on interior nodes only: the hat
//    modes are untouched, so shared end values are unchanged by construction.
#include "surface_device.cuh"

namespace semgb {

__global__ void k_wsurf(SurfTables t, const double* __restrict__ Phi, const double* __restrict__ eta,
                        double* __restrict__ w) {
  const int col = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (col >= t.ncol) return;
  wsurf_column(t, Phi, eta, w, col, threadIdx.x & 31);
}

__global__ void k_sx(SurfTables t, const double* __restrict__ f0, const double* __restrict__ f1,
                     double* __restrict__ R) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= 2 * t.Nx * (t.P + 1)) return;
  sx_item(t, f0, f1, R, k);
}

// One CTA: condensation, the interface solves (one warp per right-hand side), back-substitution.
__global__ void k_mass1d(SurfTables t, const double* __restrict__ R, int nrhs, double* __restrict__ u0,
                         double* __restrict__ u1, double* __restrict__ scr) {
  for (int k = threadIdx.x; k < nrhs * t.Nx; k += blockDim.x) mass1d_condense(t, R, nrhs, scr, k);
  __syncthreads();
  if ((threadIdx.x >> 5) < nrhs) mass1d_interface(t, nrhs, scr, threadIdx.x >> 5);
  __syncthreads();
  const int ncols = t.Nx * t.P + (t.periodic ? 0 : 1);
  for (int k = threadIdx.x; k < nrhs * ncols; k += blockDim.x) {
    const int rh = k / ncols, col = k - rh * ncols;
    mass1d_backsub(t, R, nrhs, rh == 0 ? u0 : u1, scr, rh, col);
  }
}

constexpr int kZakWarps = 4;

__global__ void __launch_bounds__(32 * kZakWarps) k_zak(SurfTables t, const double* __restrict__ eta,
                                                        const double* __restrict__ etax,
                                                        const double* __restrict__ phisx,
                                                        const double* __restrict__ w,
                                                        double* __restrict__ R) {
  __shared__ double sh[kZakWarps][kSurfWarpScratch];
  const int wid = threadIdx.x >> 5;
  const int ex = blockIdx.x * kZakWarps + wid;
  if (ex >= t.Nx) return;
  zak_element(t, eta, etax, phisx, w, R, ex, threadIdx.x & 31, sh[wid]);
}

__global__ void k_filter(SurfTables t, double* __restrict__ q0, double* __restrict__ q1) {
  __shared__ double sh[kZakWarps][kSurfWarpScratch];
  const int wid = threadIdx.x >> 5;
  const int ex = blockIdx.x * kZakWarps + wid;
  if (ex >= t.Nx) return;
  filter_element(t, q0, q1, ex, threadIdx.x & 31, sh[wid]);
}

__global__ void k_relax(SurfTables t, const double* __restrict__ eta, const double* __restrict__ phis,
                        double time, double inv_tau, double* __restrict__ de, double* __restrict__ dp) {
  const int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= t.ncol) return;
  relax_column(t, eta, phis, time, inv_tau, de, dp, col);
}

__global__ void k_rk4(int stage, int n, double dt, double* __restrict__ eta, double* __restrict__ phis,
                      const double* __restrict__ ke, const double* __restrict__ kp,
                      double* __restrict__ ae, double* __restrict__ ap, double* __restrict__ se,
                      double* __restrict__ sp) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  rk4_item(stage, dt, eta, phis, ke, kp, ae, ap, se, sp, i);
}

cudaError_t launch_wsurf(const SurfTables& t, const double* Phi, const double* eta, double* w,
                         cudaStream_t s) {
  k_wsurf<<<(t.ncol + 3) / 4, 128, 0, s>>>(t, Phi, eta, w);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_sx(const SurfTables& t, const double* f0, const double* f1, double* R,
                      cudaStream_t s) {
  const int n = 2 * t.Nx * (t.P + 1);
  k_sx<<<(n + 255) / 256, 256, 0, s>>>(t, f0, f1, R);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_mass1d(const SurfTables& t, const double* R, int nrhs, double* u0, double* u1,
                          double* scratch, cudaStream_t s) {
  k_mass1d<<<1, 256, 0, s>>>(t, R, nrhs, u0, u1, scratch);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_zakharov(const SurfTables& t, const double* eta, const double* etax,
                            const double* phisx, const double* w, double* R, cudaStream_t s) {
  k_zak<<<(t.Nx + kZakWarps - 1) / kZakWarps, 32 * kZakWarps, 0, s>>>(t, eta, etax, phisx, w, R);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_filter(const SurfTables& t, double* q0, double* q1, cudaStream_t s) {
  if (!t.filter_on) return cudaSuccess;
  k_filter<<<(t.Nx + kZakWarps - 1) / kZakWarps, 32 * kZakWarps, 0, s>>>(t, q0, q1);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_relax(const SurfTables& t, const double* eta, const double* phis, double time,
                         double inv_tau, double* de, double* dp, cudaStream_t s) {
  if (!(t.relax_left > 0.0) && !(t.relax_right > 0.0)) return cudaSuccess;
  k_relax<<<(t.ncol + 127) / 128, 128, 0, s>>>(t, eta, phis, time, inv_tau, de, dp);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_rk4_stage(int stage, int n, double dt, double* eta, double* phis,
                             const double* keta, const double* kphis, double* acc_eta,
                             double* acc_phis, double* st_eta, double* st_phis, cudaStream_t s) {
  k_rk4<<<(n + 255) / 256, 256, 0, s>>>(stage, n, dt, eta, phis, keta, kphis, acc_eta, acc_phis,
                                        st_eta, st_phis);
  count_launch();
  return cudaGetLastError();
}

}  // namespace semgb
