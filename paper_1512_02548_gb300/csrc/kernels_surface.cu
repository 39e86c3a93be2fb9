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
#include "sem_internal.cuh"

namespace semgb {

__device__ __forceinline__ int scol(const SurfTables& t, int ex, int a) {
  int c = ex * t.P + a;
  return c >= t.ncol ? c - t.ncol : c;
}

// One warp per column: lanes take (layer, row) pairs, each forms the σ-derivative at its
// row from the layer's P+1 values and weights it by c_{l,b}; the warp sums the terms.
__global__ void k_wsurf(SurfTables t, const double* __restrict__ Phi, const double* __restrict__ eta,
                        double* __restrict__ w) {
  const int col = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (col >= t.ncol) return;
  const int P = t.P, Q = P + 1;
  const double* phi = Phi + (size_t)col * t.nrow;
  double acc = 0.0;
  for (int lb = lane; lb < t.Nz * Q; lb += 32) {
    const int l = lb / Q, b = lb - l * Q;
    const double* pl = phi + l * P;
    const double* Db = t.D + b * Q;
    double d = 0.0;
    for (int c = 0; c < Q; ++c) d = fma(Db[c], pl[c], d);
    acc = fma(t.cw[lb] * (2.0 / t.dsl[l]), d, acc);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) w[col] = acc / (eta[col] + t.h[col]);
}

// Element-local S_x f = M·D f_e (the Δx/2 and 2/Δx scales cancel), two fields.
__global__ void k_sx(SurfTables t, const double* __restrict__ f0, const double* __restrict__ f1,
                     double* __restrict__ R) {
  const int Q = t.P + 1;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= 2 * t.Nx * Q) return;
  const int fld = k / (t.Nx * Q), rem = k - fld * t.Nx * Q, ex = rem / Q, a = rem - ex * Q;
  const double* f = fld == 0 ? f0 : f1;
  double s = 0.0;
  for (int c = 0; c < Q; ++c) s = fma(t.MD[a * Q + c], f[scol(t, ex, c)], s);
  R[k] = s;
}

// M' u = Σ_e Q_eᵀ R_e for nrhs element-local right-hand sides R[rhs][ex][a].
__global__ void k_mass1d(SurfTables t, const double* __restrict__ R, int nrhs, double* __restrict__ u0,
                         double* __restrict__ u1, double* __restrict__ scr) {
  const int P = t.P, Q = P + 1, Pm = P - 1, Nx = t.Nx, N = t.nif;
  double* gL = scr;
  double* gR = scr + nrhs * Nx;
  double* ub = scr + 2 * nrhs * Nx;
  for (int k = threadIdx.x; k < nrhs * Nx; k += blockDim.x) {
    const double* Re = R + (size_t)k * Q;
    double l = Re[0], r = Re[P];
    for (int i = 0; i < Pm; ++i) {
      l = fma(-t.Z[i], Re[1 + i], l);
      r = fma(-t.Z[Pm + i], Re[1 + i], r);
    }
    gL[k] = l;
    gR[k] = r;
  }
  __syncthreads();
  if ((threadIdx.x >> 5) < nrhs) {
    const int rh = threadIdx.x >> 5;
    const double* gl = gL + rh * Nx;
    const double* gr = gR + rh * Nx;
    auto gfun = [&](int j) -> double {
      if (t.periodic) return gl[j] + gr[j == 0 ? Nx - 1 : j - 1];
      return (j < Nx ? gl[j] : 0.0) + (j > 0 ? gr[j - 1] : 0.0);
    };
    warp_tridiag<double>(N, gfun, t.th_e, t.th_m, t.th_cp, t.periodic != 0, t.th_z, t.th_vlast, t.th_fac,
                         ub + rh * N);
  }
  __syncthreads();
  const int extra = t.periodic ? 0 : 1;
  for (int k = threadIdx.x; k < nrhs * (Nx * P + extra); k += blockDim.x) {
    const int rh = k / (Nx * P + extra), col = k - rh * (Nx * P + extra);
    double* u = rh == 0 ? u0 : u1;
    const double* y = ub + rh * N;
    const int ex = col / P, a = col - ex * P;
    double v;
    if (a == 0) v = y[ex];                       // interface node (incl. the walls' last column)
    else {
      const double* Re = R + ((size_t)rh * Nx + ex) * Q;
      const int i = a - 1;
      double s = 0.0;
      for (int m = 0; m < Pm; ++m) s = fma(t.Aii[i * Pm + m], Re[1 + m], s);
      const int jr = (ex + 1 == N) ? 0 : ex + 1;
      v = s / t.se[ex] - (t.Z[i] * y[ex] + t.Z[Pm + i] * y[jr]);
    }
    u[col] = v;
  }
}

// Over-integrated Zakharov integrals per surface element (§3.1.1, §3.3): one warp per
// element; fields are interpolated to the Pf+1 fine GLL nodes, the PDE integrands of
// eq. (FSeqs) evaluated pointwise and projected with Iᵀ M_f (Δx/2).
constexpr int kZakWarps = 4;
constexpr int kMaxQf = 3 * kMaxP + 1;

__global__ void __launch_bounds__(32 * kZakWarps) k_zak(SurfTables t, const double* __restrict__ eta,
                                                        const double* __restrict__ etax,
                                                        const double* __restrict__ phisx,
                                                        const double* __restrict__ w,
                                                        double* __restrict__ R) {
  __shared__ double sh[kZakWarps][2 * kMaxQf + 4 * (kMaxP + 1)];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ex = blockIdx.x * kZakWarps + wid;
  if (ex >= t.Nx) return;
  const int Q = t.P + 1, Qf = t.Pf + 1;
  double* Fe = sh[wid];
  double* Fp = Fe + kMaxQf;
  double* cv = Fp + kMaxQf;   // 4*Q coarse values: η, ηx, φ̃x, w̃
  if (lane < Q) {
    const int c = scol(t, ex, lane);
    cv[lane] = eta[c];
    cv[Q + lane] = etax[c];
    cv[2 * Q + lane] = phisx[c];
    cv[3 * Q + lane] = w[c];
  }
  __syncwarp();
  for (int q = lane; q < Qf; q += 32) {
    const double* Iq = t.I + q * Q;
    double e = 0, ex_ = 0, px = 0, wv = 0;
    for (int c = 0; c < Q; ++c) {
      e = fma(Iq[c], cv[c], e);
      ex_ = fma(Iq[c], cv[Q + c], ex_);
      px = fma(Iq[c], cv[2 * Q + c], px);
      wv = fma(Iq[c], cv[3 * Q + c], wv);
    }
    const double s2 = fma(ex_, ex_, 1.0);
    Fe[q] = fma(wv, s2, -ex_ * px);
    Fp[q] = -t.g * e - 0.5 * fma(px, px, -wv * wv * s2);
  }
  __syncwarp();
  const double se = t.se[ex];
  for (int a = lane; a < Q; a += 32) {
    const double* Ba = t.B + a * Qf;
    double se0 = 0, se1 = 0;
    for (int q = 0; q < Qf; ++q) {
      se0 = fma(Ba[q], Fe[q], se0);
      se1 = fma(Ba[q], Fp[q], se1);
    }
    R[(size_t)ex * Q + a] = se * se0;
    R[((size_t)t.Nx + ex) * Q + a] = se * se1;
  }
}

// Modal filter on element interiors, two fields; one warp per element.
__global__ void k_filter(SurfTables t, double* __restrict__ q0, double* __restrict__ q1) {
  __shared__ double sh[kZakWarps][2 * (kMaxP + 1)];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ex = blockIdx.x * kZakWarps + wid;
  if (ex >= t.Nx) return;
  const int P = t.P, Q = P + 1;
  double* v0 = sh[wid];
  double* v1 = v0 + Q;
  if (lane < Q) {
    const int c = scol(t, ex, lane);
    v0[lane] = q0[c];
    v1[lane] = q1 ? q1[c] : 0.0;
  }
  __syncwarp();
  if (lane >= 1 && lane < P) {
    const double* Fa = t.F + lane * Q;
    double s0 = 0, s1 = 0;
    for (int c = 0; c < Q; ++c) {
      s0 = fma(Fa[c], v0[c], s0);
      s1 = fma(Fa[c], v1[c], s1);
    }
    const int c = scol(t, ex, lane);
    q0[c] = s0;
    if (q1) q1[c] = s1;
  }
}

// Embedded penalty forcing of §2.2 at the surface nodes: q̇ += (1 − γ(x))(q_a(x,t) − q)/τ with
// γ = ξ²(3 − 2ξ) across each zone (1 outside); q_a is the linear superposition of the wave
// input in the left zone, rest in the right zone.
__global__ void k_relax(SurfTables t, const double* __restrict__ eta, const double* __restrict__ phis,
                        double time, double inv_tau, double* __restrict__ de, double* __restrict__ dp) {
  const int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= t.ncol) return;
  const double x = t.xcol[col];
  double gam = 1.0;
  const bool left = t.relax_left > 0.0 && x < t.x0 + t.relax_left;
  if (left) {
    const double xi = fmin(fmax((x - t.x0) / t.relax_left, 0.0), 1.0);
    gam = xi * xi * (3.0 - 2.0 * xi);
  }
  if (t.relax_right > 0.0 && x > t.x1 - t.relax_right) {
    const double xi = fmin(fmax((t.x1 - x) / t.relax_right, 0.0), 1.0);
    gam = fmin(gam, xi * xi * (3.0 - 2.0 * xi));
  }
  if (gam >= 1.0) return;
  double ea = 0.0, pa = 0.0;
  if (left) {
    const double* a = t.wave;
    const double* om = a + t.ncomp;
    const double* k = om + t.ncomp;
    const double* th = k + t.ncomp;
    for (int i = 0; i < t.ncomp; ++i) {
      double sn, cs;
      sincos(om[i] * time - k[i] * x + th[i], &sn, &cs);
      ea = fma(a[i], cs, ea);
      pa = fma(-t.g * a[i] / om[i], sn, pa);
    }
  }
  const double c = (1.0 - gam) * inv_tau;
  de[col] = fma(c, ea - eta[col], de[col]);
  dp[col] = fma(c, pa - phis[col], dp[col]);
}

// Classical RK4 stage bookkeeping on (η, φ̃) with k = right-hand side of this stage:
//   stage 1: acc = k,   st = q + dt/2 k
//   stage 2: acc += 2k, st = q + dt/2 k
//   stage 3: acc += 2k, st = q + dt k
//   stage 4: q += dt/6 (acc + k)
__global__ void k_rk4(int stage, int n, double dt, double* __restrict__ eta, double* __restrict__ phis,
                      const double* __restrict__ ke, const double* __restrict__ kp,
                      double* __restrict__ ae, double* __restrict__ ap, double* __restrict__ se,
                      double* __restrict__ sp) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double a = ke[i], b = kp[i];
  if (stage == 1) {
    ae[i] = a; ap[i] = b;
    se[i] = fma(0.5 * dt, a, eta[i]); sp[i] = fma(0.5 * dt, b, phis[i]);
  } else if (stage == 2 || stage == 3) {
    ae[i] = fma(2.0, a, ae[i]); ap[i] = fma(2.0, b, ap[i]);
    const double c = stage == 2 ? 0.5 * dt : dt;
    se[i] = fma(c, a, eta[i]); sp[i] = fma(c, b, phis[i]);
  } else {
    eta[i] = fma(dt / 6.0, ae[i] + a, eta[i]);
    phis[i] = fma(dt / 6.0, ap[i] + b, phis[i]);
  }
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
