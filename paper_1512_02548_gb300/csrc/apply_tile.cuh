// Tiled matrix-free σ-Laplace apply, y = 𝓛x at every node (§3.1.2, element change of
// variables), for long meshes where the apply streams x and y through HBM.  Included by
// laplace_device.cuh (order-templated, internal linkage).
//
// A CTA takes a tile of E consecutive x-elements (all Nz layers) plus the element to the
// left of the tile, whose contribution completes the tile's first column; every output
// column of the tile is then complete inside the CTA, so y is written once, with no edge
// buffer, no second kernel and no atomics.  The left element is recomputed by both
// neighbouring tiles (1/E extra arithmetic, its x values come from L2).
//
// Per tile, with the tile's nodal values staged in shared memory:
//   1. x-lines (element e, layer l, row b): u_r(a) = Σ_c D_ac u(c,b) for all a, in registers;
//   2. σ-lines (e, l, column a): u_t(b) = Σ_c D_bc u(a,c); the geometric factors of column a
//      (d, 1/d, ∂xh, ∂xd) and the layer ratios give
//        F1 = w_a w_b (Δσ/Δx · d · u_r + K12 u_t),  F2 = w_a w_b (K12 u_r + Δx/Δσ · K22 u_t),
//      K12 = ∂xh − σ ∂xd, K22 = (1 + K12²)/d, and the σ part of the transpose,
//      y_σ(b) = Σ_c D_cb F2(c), in registers;
//   3. x-lines: y_e(a) = Σ_c D_ca F1(c) + y_σ(a) — the element's contribution to A = −𝓛;
//   4. every tile node sums the contributions of the ≤ 4 elements that share it (left/right
//      element, lower/upper layer) in a fixed order and writes −sum.
// All sums have a fixed order: results are bitwise reproducible.
#pragma once

namespace semgb {

template <int P>
struct TileLayout {
  static constexpr int Q = P + 1;
  static constexpr int QP = (Q % 2 == 0) ? Q + 1 : Q;   // odd stride of the line buffers
  int E, en_max, XS, tcols, nline;
  __host__ __device__ TileLayout(int E_, int nrow, int Nz) {
    E = E_;
    en_max = E + 1;
    XS = nrow | 1;
    tcols = en_max * P + 1;
    nline = en_max * Nz * Q * QP;
  }
  // elements of the dynamic shared memory (of type T)
  __host__ __device__ size_t count(int nrow, int Nz) const {
    return (size_t)tcols * XS + 3 * (size_t)nline + (size_t)en_max * Q * 4 + (size_t)en_max * Nz * 2 + nrow + Q;
  }
};

template <int P, class T>
__global__ void __launch_bounds__(kThreads) k_apply_tile(DevGeom g, const T* __restrict__ x, T* __restrict__ y,
                                                         int E) {
  constexpr int Q = P + 1;
  constexpr int QP = TileLayout<P>::QP;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nrow = g.nrow, Nz = g.Nz, Nx = g.Nx, ncol = g.ncol;
  const TileLayout<P> L(E, nrow, Nz);
  const int XS = L.XS;
  T* Xs = reinterpret_cast<T*>(smem_raw);   // [tcols][XS] nodal values of the tile
  T* Ur = Xs + (size_t)L.tcols * XS;        // [en][Nz][Q b][QP a] u_r, then the element contributions
  T* Fs = Ur + L.nline;                     // [en][Nz][Q b][QP a] F1
  T* Ys = Fs + L.nline;                     // [en][Nz][Q b][QP a] σ part of the transpose
  T* Gs = Ys + L.nline;                     // [en][Q][4] d, 1/d, ∂xh, ∂xd
  T* Cs = Gs + (size_t)L.en_max * Q * 4;    // [en][Nz][2] Δσ/Δx, Δx/Δσ
  T* Ss = Cs + (size_t)L.en_max * Nz * 2;   // [nrow] σ
  T* Ws = Ss + nrow;                        // [Q] GLL weights (indexed per thread)
  const T* D = CT<T>::D() + d_off(P);       // compile-time indices only: constant operands
  const T* w = CT<T>::w() + w_off(P);
  const T* geo = geo_ptr<T>(g);
  for (int t = threadIdx.x; t < nrow; t += blockDim.x) Ss[t] = (T)g.sig[t];
  for (int t = threadIdx.x; t < Q; t += blockDim.x) Ws[t] = w[t];
  const int ntiles = (Nx + E - 1) / E;
  const int lpe = Nz * Q;                                   // lines per element (x- or σ-lines)
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  // line index li = threadIdx.x + k·blockDim.x as (element, line in element), stepped without
  // dividing: line 0 of the loop and the step of blockDim.x lines
  const int le0 = threadIdx.x / lpe, lr0 = threadIdx.x - le0 * lpe;
  const int lde = blockDim.x / lpe, ldr = blockDim.x - lde * lpe;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int ex0 = tile * E;
    const int ne = min(E, Nx - ex0);
    const int en = ne + 1;                       // local element 0 is the left neighbour
    const bool has_left = g.periodic || ex0 > 0;
    const int nc = en * P + 1;
    __syncthreads();                             // the previous tile's readers are done
    // ---- stage the tile: nodal values (a warp per column), geometry, layer ratios ----
    for (int j = warp; j < nc; j += nwarps) {
      int gc = (ex0 - 1) * P + j;
      if (gc < 0) gc = g.periodic ? gc + ncol : -1;
      else if (gc >= ncol) gc -= ncol;           // periodic: column Nx·P is column 0
      const T* xc = x + (size_t)(gc < 0 ? 0 : gc) * nrow;
      for (int r = lane; r < nrow; r += 32) Xs[j * XS + r] = gc >= 0 ? __ldg(xc + r) : T(0);
    }
    for (int t = threadIdx.x; t < en * Q * 4; t += blockDim.x) {
      const int e = t / (Q * 4);
      int ge = ex0 - 1 + e;
      if (ge < 0) ge = g.periodic ? ge + Nx : 0;
      Gs[t] = geo[(size_t)ge * Q * 4 + (t - e * Q * 4)];
    }
    for (int t = threadIdx.x; t < en * Nz; t += blockDim.x) {
      const int e = t / Nz, l = t - e * Nz;
      int ge = ex0 - 1 + e;
      if (ge < 0) ge = g.periodic ? ge + Nx : 0;
      const T dxe = (T)g.dxe[ge], dsl = (T)g.dsl[l];   // ratios in the kernel's own precision
      Cs[2 * t] = dsl / dxe;
      Cs[2 * t + 1] = dxe / dsl;
    }
    __syncthreads();
    const int e_first = has_left ? 0 : 1;        // walls: no element left of x = 0
    // ---- 1. x-lines: u_r ----
    for (int e = e_first + le0, rem = lr0; e < en; e += lde, rem += ldr) {
      if (rem >= lpe) { rem -= lpe; ++e; if (e >= en) break; }
      const int l = rem / Q, b = rem - l * Q;
      const T* X = Xs + (e * P) * XS + l * P + b;
      T u[Q];
#pragma unroll
      for (int c = 0; c < Q; ++c) u[c] = X[c * XS];
      T* out = Ur + ((e * Nz + l) * Q + b) * QP;
#pragma unroll
      for (int a = 0; a < Q; ++a) {
        T s = T(0);
#pragma unroll
        for (int c = 0; c < Q; ++c) s = fmx(D[a * Q + c], u[c], s);
        out[a] = s;
      }
    }
    __syncthreads();
    // ---- 2. σ-lines: u_t, F1, F2 and the σ part of the transpose ----
    for (int e = e_first + le0, rem = lr0; e < en; e += lde, rem += ldr) {
      if (rem >= lpe) { rem -= lpe; ++e; if (e >= en) break; }
      const int l = rem / Q, a = rem - l * Q;
      const T* X = Xs + (e * P + a) * XS + l * P;
      T u[Q];
#pragma unroll
      for (int c = 0; c < Q; ++c) u[c] = X[c];
      const T* gq = Gs + (e * Q + a) * 4;
      const T c0 = Cs[2 * (e * Nz + l)], c1 = Cs[2 * (e * Nz + l) + 1];
      const T wa = Ws[a], hx = gq[2], dxd = gq[3];
      const T g11 = wa * c0 * gq[0];             // w_a Δσ/Δx d
      const T g22 = wa * c1 * gq[1];             // w_a Δx/Δσ /d
      const T* sg = Ss + l * P;
      const int base = (e * Nz + l) * Q;
      T f2[Q];
#pragma unroll
      for (int b = 0; b < Q; ++b) {
        T ut = T(0);
#pragma unroll
        for (int c = 0; c < Q; ++c) ut = fmx(D[b * Q + c], u[c], ut);
        const T ur = Ur[(base + b) * QP + a];
        const T K12 = fmx(-sg[b], dxd, hx);
        const T wb = w[b];
        const T G12 = wa * wb * K12;
        Fs[(base + b) * QP + a] = fmx(g11 * wb, ur, G12 * ut);
        f2[b] = fmx(G12, ur, g22 * wb * fmx(K12, K12, T(1)) * ut);
      }
#pragma unroll
      for (int b = 0; b < Q; ++b) {
        T s = T(0);
#pragma unroll
        for (int c = 0; c < Q; ++c) s = fmx(D[c * Q + b], f2[c], s);
        Ys[(base + b) * QP + a] = s;
      }
    }
    __syncthreads();
    // ---- 3. x-lines: the element contribution (into the u_r buffer) ----
    for (int e = e_first + le0, rem = lr0; e < en; e += lde, rem += ldr) {
      if (rem >= lpe) { rem -= lpe; ++e; if (e >= en) break; }
      const int l = rem / Q, b = rem - l * Q;
      const int row = ((e * Nz + l) * Q + b) * QP;
      T f1[Q];
#pragma unroll
      for (int c = 0; c < Q; ++c) f1[c] = Fs[row + c];
#pragma unroll
      for (int a = 0; a < Q; ++a) {
        T s = Ys[row + a];
#pragma unroll
        for (int c = 0; c < Q; ++c) s = fmx(D[c * Q + a], f1[c], s);
        Ur[row + a] = s;
      }
    }
    __syncthreads();
    // ---- 4. gather: own columns [P, P + ne·P) (plus the last column between walls) ----
    const bool last_wall = !g.periodic && ex0 + ne == Nx;
    const int nout = ne * P + (last_wall ? 1 : 0);   // output columns
    T* yt = y + (size_t)ex0 * P * nrow;
    for (int jj = warp; jj < nout; jj += nwarps) {   // a warp per output column
      const int j = P + jj;
      int e = j / P, a = j - e * P;
      if (e == en) { e = en - 1; a = P; }       // right wall column
      const bool left = a == 0 && (e > 1 || has_left);   // the element left of column j exists
      T* yc = yt + (size_t)jj * nrow;
      for (int r = lane; r < nrow; r += 32) {
        int l = r / P, b = r - l * P;
        if (l == Nz) { l = Nz - 1; b = P; }     // surface row
        T s = Ur[((e * Nz + l) * Q + b) * QP + a];
        if (left) s += Ur[(((e - 1) * Nz + l) * Q + b) * QP + P];
        if (b == 0 && l > 0) {
          s += Ur[((e * Nz + l - 1) * Q + P) * QP + a];
          if (left) s += Ur[(((e - 1) * Nz + l - 1) * Q + P) * QP + P];
        }
        yc[r] = -s;
      }
    }
  }
}

// Dynamic shared memory of the tiled apply for tile width E.
template <int P>
size_t apply_tile_smem(int E, int nrow, int Nz, size_t elem) {
  return TileLayout<P>(E, nrow, Nz).count(nrow, Nz) * elem;
}

}  // namespace semgb
