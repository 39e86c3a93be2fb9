// Device bodies of the free-surface operations (§3.1.1, §3.1.3, §3.3, §3.4, §2.2), shared by
// the stand-alone kernels (kernels_surface.cu) and the fused per-stage kernel
// (kernels_laplace.cu).  Each body computes one work item (a column, an element, a
// right-hand side); the callers decide which items a thread, warp or CTA takes.
#pragma once
#include "sem_internal.cuh"

namespace semgb {

constexpr int kMaxQf = 3 * kMaxP + 1;
// shared scratch of one warp in the element bodies (zak, filter)
constexpr int kSurfWarpScratch = 2 * kMaxQf + 4 * (kMaxP + 1);

__device__ __forceinline__ int scol(const SurfTables& t, int ex, int a) {
  int c = ex * t.P + a;
  return c >= t.ncol ? c - t.ncol : c;
}

// w̃ at column `col` (one warp).  On the tensor-product mesh the 2D mass is M_x ⊗ M_σ and the
// σ-derivative (1/d)∂σΦ is continuous across x-element edges, so the surface row of
// M⁻¹S_zΦ (eq. velocpot2) is the per-column contraction
//     w̃ = (1/d) Σ_l Σ_b c_{l,b} (2/Δσ_l) (D Φ_l)_b,  c_l = (Δσ_l/2) M (M_σ⁻¹ e_top)|_l,
// whose weights are folded on the host into one weight per row, w̃ = (1/d) Σ_iz wrow_iz Φ_iz.
// Lanes take rows; the warp sums.
__device__ __forceinline__ void wsurf_column(const SurfTables& t, const double* __restrict__ Phi,
                                             const double* __restrict__ eta, double* __restrict__ w,
                                             int col, int lane) {
  const double* phi = Phi + (size_t)col * t.nrow;
  double acc = 0.0;
  for (int iz = lane; iz < t.nrow; iz += 32) acc = fma(t.wrow[iz], phi[iz], acc);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) w[col] = acc / (eta[col] + t.h[col]);
}

// The same for four columns per warp, eight lanes per column (col < 0: no column; every lane of
// the warp must call it).
__device__ __forceinline__ void wsurf_column8(const SurfTables& t, const double* __restrict__ Phi,
                                              const double* __restrict__ eta, double* __restrict__ w,
                                              int col, int sub) {
  double acc = 0.0;
  if (col >= 0) {
    const double* phi = Phi + (size_t)col * t.nrow;
    for (int iz = sub; iz < t.nrow; iz += 8) acc = fma(t.wrow[iz], phi[iz], acc);
  }
#pragma unroll
  for (int o = 4; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (col >= 0 && sub == 0) w[col] = acc / (eta[col] + t.h[col]);
}

// Element-local S_x f = M·D f_e (the Δx/2 and 2/Δx scales cancel); item k over
// [field][ex][a], two fields.
__device__ __forceinline__ void sx_item(const SurfTables& t, const double* __restrict__ f0,
                                        const double* __restrict__ f1, double* __restrict__ R, int k) {
  const int Q = t.P + 1;
  const int fld = k / (t.Nx * Q), rem = k - fld * t.Nx * Q, ex = rem / Q, a = rem - ex * Q;
  const double* f = fld == 0 ? f0 : f1;
  double s = 0.0;
  for (int c = 0; c < Q; ++c) s = fma(t.MD[a * Q + c], f[scol(t, ex, c)], s);
  R[k] = s;
}

// M'u = Σ_e Q_eᵀ R_e by static condensation (M' is constant in time).  Scratch layout:
// gL[nrhs][Nx], gR[nrhs][Nx], ub[nrhs][nif].
// Phase 1, item k over [rhs][ex]: condensed boundary right-hand sides of element ex.
__device__ __forceinline__ void mass1d_condense(const SurfTables& t, const double* __restrict__ R, int nrhs,
                                                double* __restrict__ scr, int k) {
  const int P = t.P, Q = P + 1, Pm = P - 1, Nx = t.Nx;
  const double* Re = R + (size_t)k * Q;
  double l = Re[0], r = Re[P];
  for (int i = 0; i < Pm; ++i) {
    l = fma(-t.Z[i], Re[1 + i], l);
    r = fma(-t.Z[Pm + i], Re[1 + i], r);
  }
  scr[k] = l;
  scr[nrhs * Nx + k] = r;
}

// Phase 2, one warp per right-hand side: the interface tridiagonal (cyclic when periodic).
__device__ __forceinline__ void mass1d_interface(const SurfTables& t, int nrhs, double* __restrict__ scr,
                                                 int rh) {
  const int Nx = t.Nx, N = t.nif;
  const double* gl = scr + rh * Nx;
  const double* gr = scr + nrhs * Nx + rh * Nx;
  double* ub = scr + 2 * nrhs * Nx + rh * N;
  auto gfun = [&](int j) -> double {
    if (t.periodic) return __ldcg(gl + j) + __ldcg(gr + (j == 0 ? Nx - 1 : j - 1));
    return (j < Nx ? __ldcg(gl + j) : 0.0) + (j > 0 ? __ldcg(gr + j - 1) : 0.0);
  };
  warp_tridiag<double>(N, gfun, t.th_e, t.th_m, t.th_cp, t.periodic != 0, t.th_z, t.th_vlast, t.th_fac, ub);
}

// The same solve by a whole CTA (every thread must call it): long systems (N > 32·kTridiagRegs)
// use the CTA-wide scan (CACHE: with register-held chunks), short ones warp 0 alone.
template <bool CACHE = false>
__device__ __forceinline__ void mass1d_interface_cta(const SurfTables& t, int nrhs, double* __restrict__ scr,
                                                     int rh) {
  const int Nx = t.Nx, N = t.nif;
  if (N <= 32 * kTridiagRegs) {
    if (threadIdx.x < 32) mass1d_interface(t, nrhs, scr, rh);
    return;
  }
  const double* gl = scr + rh * Nx;
  const double* gr = scr + nrhs * Nx + rh * Nx;
  double* ub = scr + 2 * nrhs * Nx + rh * N;
  auto gfun = [&](int j) -> double {
    if (t.periodic) return __ldcg(gl + j) + __ldcg(gr + (j == 0 ? Nx - 1 : j - 1));
    return (j < Nx ? __ldcg(gl + j) : 0.0) + (j > 0 ? __ldcg(gr + j - 1) : 0.0);
  };
  cta_tridiag<double, decltype(gfun), CACHE>(N, gfun, t.th_e, t.th_m, t.th_cp, t.periodic != 0, t.th_z, t.th_vlast,
                                             t.th_fac, ub);
}

// Phase 3, column `col` of right-hand side `rh`: interface value or back-substituted interior.
__device__ __forceinline__ void mass1d_backsub(const SurfTables& t, const double* __restrict__ R, int nrhs,
                                               double* __restrict__ u, const double* __restrict__ scr,
                                               int rh, int col) {
  const int P = t.P, Q = P + 1, Pm = P - 1, Nx = t.Nx, N = t.nif;
  const double* y = scr + 2 * nrhs * Nx + rh * N;
  const int ex = col / P, a = col - ex * P;
  double v;
  if (a == 0) v = __ldcg(y + ex);   // interface node (incl. the walls' last column)
  else {
    const double* Re = R + ((size_t)rh * Nx + ex) * Q;
    const int i = a - 1;
    double s = 0.0;
    for (int m = 0; m < Pm; ++m) s = fma(t.Aii[i * Pm + m], Re[1 + m], s);
    const int jr = (ex + 1 == N) ? 0 : ex + 1;
    v = s / t.se[ex] - (t.Z[i] * __ldcg(y + ex) + t.Z[Pm + i] * __ldcg(y + jr));
  }
  u[col] = v;
}

// Over-integrated Zakharov integrals of element ex (one warp, `sh` = kSurfWarpScratch doubles):
// η, ηx, φ̃x, w̃ are interpolated to the Pf+1 fine GLL nodes, the PDE integrands of eq. FSeqs
// evaluated pointwise and projected with Iᵀ M_f (Δx/2) (§3.1.1, §3.3).  R[0][ex][·] and
// R[1][ex][·] receive the element right-hand sides of ∂tη and ∂tφ̃.
__device__ __forceinline__ void zak_element(const SurfTables& t, const double* __restrict__ eta,
                                            const double* __restrict__ etax, const double* __restrict__ phisx,
                                            const double* __restrict__ w, double* __restrict__ R, int ex,
                                            int lane, double* sh) {
  const int Q = t.P + 1, Qf = t.Pf + 1;
  double* Fe = sh;
  double* Fp = Fe + kMaxQf;
  double* cv = Fp + kMaxQf;   // 4*Q coarse values: η, ηx, φ̃x, w̃
  if (lane < Q) {
    const int c = scol(t, ex, lane);
    cv[lane] = __ldcg(eta + c);
    cv[Q + lane] = __ldcg(etax + c);
    cv[2 * Q + lane] = __ldcg(phisx + c);
    cv[3 * Q + lane] = __ldcg(w + c);
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
  __syncwarp();
}

// Modal filter of element ex on its interior nodes, two fields (one warp, `sh` scratch).  The
// hat modes are untouched, so the shared end values keep their value by construction.
__device__ __forceinline__ void filter_element(const SurfTables& t, double* q0, double* q1, int ex, int lane,
                                               double* sh) {
  const int P = t.P, Q = P + 1;
  double* v0 = sh;
  double* v1 = v0 + Q;
  if (lane < Q) {
    const int c = scol(t, ex, lane);
    v0[lane] = __ldcg(q0 + c);
    v1[lane] = q1 ? __ldcg(q1 + c) : 0.0;
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
  __syncwarp();
}

// Embedded penalty forcing of §2.2 at column `col`: q̇ += (1 − γ(x))(q_a(x,t) − q)/τ with
// γ = ξ²(3 − 2ξ) across each zone (1 outside); q_a is the linear superposition of the wave
// input in the left zone, rest in the right zone.
// Per time level, the component factors of the generated signal (§2.2): with A = ωt + θ and
// c = −g a/ω, wA = (a cos A, a sin A, c sin A, c cos A).  Items i = first, first + stride, ….
__device__ __forceinline__ void wave_angles(const SurfTables& t, double time, int first, int stride) {
  const int n = t.ncomp;
  const double* a = t.wave;
  const double* om = a + n;
  const double* th = om + 2 * n;
  for (int i = first; i < n; i += stride) {
    double sn, cs;
    sincos(fma(om[i], time, th[i]), &sn, &cs);
    const double c = -t.g * a[i] / om[i];
    t.wA[i] = a[i] * cs;
    t.wA[n + i] = a[i] * sn;
    t.wA[2 * n + i] = c * sn;
    t.wA[3 * n + i] = c * cs;
  }
}

// The generated η = Σ a cos(A − kx) and φ̃ = Σ c sin(A − kx) at left-zone column `col`, by one
// warp (lanes over the components, then a shuffle tree): cos(A − kx) = cos A cos kx + sin A sin kx,
// sin(A − kx) = sin A cos kx − cos A sin kx.  Written to wEP by lane 0.
__device__ __forceinline__ void wave_zone_column(const SurfTables& t, int col, int lane) {
  const int n = t.ncomp;
  const double* ck = t.wkx + (size_t)col * n * 2;
  double ea = 0.0, pa = 0.0;
  for (int i = lane; i < n; i += 32) {
    const double cb = ck[2 * i], sb = ck[2 * i + 1];
    ea = fma(t.wA[i], cb, fma(t.wA[n + i], sb, ea));
    pa = fma(t.wA[2 * n + i], cb, fma(-t.wA[3 * n + i], sb, pa));
  }
  for (int o = 16; o > 0; o >>= 1) {
    ea += __shfl_xor_sync(0xffffffffu, ea, o);
    pa += __shfl_xor_sync(0xffffffffu, pa, o);
  }
  if (lane == 0) {
    t.wEP[2 * col] = ea;
    t.wEP[2 * col + 1] = pa;
  }
}

// ep: the generated (η, φ̃) of the left-zone columns for this time (wave_zone_columns), or
// nullptr to sum the components here.
__device__ __forceinline__ void relax_column(const SurfTables& t, const double* __restrict__ eta,
                                             const double* __restrict__ phis, double time, double inv_tau,
                                             double* de, double* dp, int col, const double* ep = nullptr) {
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
  if (left && ep != nullptr && col < t.nzl) {
    ea = ep[2 * col];
    pa = ep[2 * col + 1];
  } else if (left) {
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

// Classical RK4 stage bookkeeping at index i, with k = right-hand side of this stage:
//   stage 1: acc = k,   st = q + dt/2 k
//   stage 2: acc += 2k, st = q + dt/2 k
//   stage 3: acc += 2k, st = q + dt k
//   stage 4: q += dt/6 (acc + k)
__device__ __forceinline__ void rk4_item(int stage, double dt, double* eta, double* phis, const double* ke,
                                         const double* kp, double* ae, double* ap, double* se, double* sp,
                                         int i) {
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

}  // namespace semgb
