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
// The CTAs are persistent and stage their tiles' nodal values with bulk copies (TMA,
// cp.async.bulk) into two shared-memory buffers: the copy of the next tile is in flight
// while the current one is computed.  A tile's values are one contiguous range of x
// (columns are stored back to back); the copy starts at the 16-byte boundary below the
// range and the tile is read at the resulting offset.  Tiles whose range wraps around the
// periodic end, or whose rounded range would pass the end of x, are staged with plain loads.
//
// Per tile, with the tile's nodal values staged in shared memory:
//   1. x-lines (element e, layer l, row b): u_r(a) = Σ_c D_ac u(c,b) for all a, in registers;
//   2. σ-lines (e, l, column a): u_t(b) = Σ_c D_bc u(a,c); the geometric factors of column a
//      (d, 1/d, ∂xh, ∂xd) and the layer ratios give
//        F1 = w_a w_b (Δσ/Δx · d · u_r + K12 u_t),  F2 = w_a w_b (K12 u_r + Δx/Δσ · K22 u_t),
//      K12 = ∂xh − σ ∂xd, K22 = (1 + K12²)/d, and the σ part of the transpose,
//      y_σ(b) = Σ_c D_cb F2(c), in registers;
//   3. x-lines: y_e(a) = Σ_c D_ca F1(c) + y_σ(a) — the element's contribution to A = −𝓛;
//   4. the contributions are stored into the tile's nodes; the nodes shared between layers
//      and between elements are completed by two small fix-up sweeps in a fixed order (no
//      atomics), and the tile's own columns are written as −sum with contiguous stores.
// All sums have a fixed order: results are bitwise reproducible.
#pragma once

namespace semgb {

// ---- bulk copies with mbarrier completion (sm_90+ PTX) ----
static __device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
static __device__ __forceinline__ void mbar_init(unsigned long long* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(bar)) : "memory");
}
static __device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// Generic-proxy accesses of shared memory before this point are ordered before later
// async-proxy (bulk copy) accesses.
static __device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
static __device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
  asm volatile(
      "{\n\t.reg .b64 st;\n\t"
      "mbarrier.arrive.expect_tx.shared::cta.b64 st, [%3], %2;\n\t"
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n\t}"
      :: "r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}
static __device__ __forceinline__ bool mbar_test(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity) : "memory");
  return ok != 0;
}
// Wait for a phase of the mbarrier, at most `limit_ns` of wall-clock time.
static __device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity,
                                                 unsigned long long limit_ns) {
  if (mbar_test(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (unsigned spins = 1;; ++spins) {
    if (mbar_test(bar, parity)) return true;
    if ((spins & 255u) == 0 && global_ns() - t0 > limit_ns) return false;
  }
}

constexpr unsigned long long kCopyTimeoutNs = 2000000000ull;   // 2 s

template <int P>
struct TileLayout {
  static constexpr int Q = P + 1;
  static constexpr int QP = (Q % 2 == 0) ? Q + 1 : Q;   // odd stride of the line buffers
  // stride of one (element, layer) block of a line buffer: at least Q·QP and ≡ 8 (mod 16), so
  // that the σ-lines of consecutive layers (one warp) fall in different shared-memory banks
  static constexpr int BS = Q * QP + ((8 - (Q * QP) % 16) + 16) % 16;
  int E, en_max, tcols, xbuf, nline, ybuf;
  __host__ __device__ TileLayout(int E_, int nrow, int Nz, int elem) {
    E = E_;
    en_max = E + 1;
    tcols = en_max * P + 1;
    // one staging buffer: the tile's columns back to back; the 16-byte-aligned copy adds less
    // than 16 bytes on each side; rounded up to 16 bytes
    const int per16 = 16 / elem;
    xbuf = ((tcols * nrow + 2 * per16 + per16 - 1) / per16) * per16;
    nline = en_max * Nz * BS;
    ybuf = ((tcols * nrow + 3) / 4) * 4;   // the tile's nodes (tensor-core kernel), 16-byte multiple
  }
  // bytes of dynamic shared memory for element size `elem`: two mbarriers (16 B), two staging
  // buffers, the line buffers and the tile's geometry
  __host__ __device__ size_t bytes(int nrow, int Nz, int elem) const {
    return 16 + (size_t)elem * (2 * (size_t)xbuf + 3 * (size_t)nline + (size_t)en_max * Q * 4 +
                                (size_t)en_max * Nz * 2 + nrow + Q + 2 * (size_t)en_max * Nz * Q);
  }
  // the same for the tensor-core kernel (FP32): the tile's node buffer and `scratch` floats per
  // warp in place of the three line buffers
  __host__ __device__ size_t bytes_tc(int nrow, int Nz, int scratch) const {
    return 16 + 4 * (2 * (size_t)xbuf + (size_t)ybuf + (size_t)(kThreads / 32) * scratch +
                     (size_t)en_max * Q * 4 + (size_t)en_max * Nz * 2 + nrow + Q + 2 * (size_t)en_max * Nz * Q);
  }
};

// Range of x (in elements of T) that a tile reads: columns (ex0−1)·P … (ex0+ne)·P.
// Returns true when it can be bulk-copied: no periodic wrap, and the 16-byte-aligned
// superset [*lo, *lo + *count) stays inside x; *shift is the tile's offset in the copy.
template <int P, class T>
static __device__ __forceinline__ bool tile_range(const DevGeom& g, int ex0, int ne, long long* lo, int* count,
                                                  int* shift) {
  constexpr int per16 = 16 / (int)sizeof(T);
  const long long c_lo = (long long)(ex0 - 1) * P, c_hi = (long long)(ex0 + ne) * P;
  if (c_lo < 0 || c_hi >= g.ncol) return false;
  const long long first = c_lo * g.nrow, last = (c_hi + 1) * g.nrow;   // [first, last)
  const long long a = first - first % per16;
  const long long b = ((last + per16 - 1) / per16) * per16;
  if (b > (long long)g.ncol * g.nrow) return false;
  *lo = a;
  *count = (int)(b - a);
  *shift = (int)(first - a);
  return true;
}

// bulk_ok != 0: x is 16-byte aligned and interior tiles are staged by bulk copies.
// NZC > 0: the layer count is the compile-time constant NZC (= g.Nz), which turns the row
// arithmetic into constants; NZC = 0 reads it from g.
// Minimum of 3 CTAs per SM (at most 85 registers) only for FP32, P = 8, four layers, which the
// compiler otherwise builds with 96 registers (two CTAs per SM); 0 leaves the choice to it.
template <int P, class T, int NZC>
__global__ void __launch_bounds__(kThreads, (sizeof(T) == 4 && P == 8 && NZC == 4) ? 3 : 0)
    k_apply_tile(DevGeom g, const T* __restrict__ x, T* __restrict__ y,
                                                         int E, int bulk_ok) {
  constexpr int Q = P + 1;
  constexpr int QP = TileLayout<P>::QP;
  constexpr int BS = TileLayout<P>::BS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nrow = NZC ? NZC * P + 1 : g.nrow, Nz = NZC ? NZC : g.Nz, Nx = g.Nx, ncol = g.ncol;
  const TileLayout<P> L(E, nrow, Nz, (int)sizeof(T));
  unsigned long long* mbar = reinterpret_cast<unsigned long long*>(smem_raw);   // [2]
  T* const Xb0 = reinterpret_cast<T*>(smem_raw + 16);   // staging buffers b = 0, 1 at Xb0 + b·xbuf
  T* Ur = Xb0 + 2 * L.xbuf;                 // [en][Nz][Q b][QP a] u_r, then the element contributions
  T* Fs = Ur + L.nline;                     // [en][Nz][Q b][QP a] F1
  T* Ys = Fs + L.nline;                     // [en][Nz][Q b][QP a] σ part of the transpose
  T* Gs = Ys + L.nline;                     // [en][Q][4] d, 1/d, ∂xh, ∂xd
  T* Cs = Gs + (size_t)L.en_max * Q * 4;    // [en][Nz][2] Δσ/Δx, Δx/Δσ
  T* Ss = Cs + (size_t)L.en_max * Nz * 2;   // [nrow] σ
  T* Ws = Ss + nrow;                        // [Q] GLL weights (indexed per thread)
  T* Rrow = Ws + Q;                         // [en][Nz][Q] top-row (b = P) contributions, a < P
  T* Ccol = Rrow + (size_t)L.en_max * Nz * Q;   // [en][Nz][Q] right-column (a = P) contributions
  __shared__ int s_ok;
  const T* D = CT<T>::D() + d_off(P);       // compile-time indices only: constant operands
  const T* w = CT<T>::w() + w_off(P);
  const T* geo = geo_ptr<T>(g);
  for (int t = threadIdx.x; t < nrow; t += blockDim.x) Ss[t] = (T)g.sig[t];
  for (int t = threadIdx.x; t < Q; t += blockDim.x) Ws[t] = w[t];
  if (threadIdx.x == 0) {
    mbar_init(&mbar[0]);
    mbar_init(&mbar[1]);
    mbar_init_fence();
    s_ok = 1;
  }
  __syncthreads();
  const int ntiles = (Nx + E - 1) / E;
  const int lpe = Nz * Q;                                   // lines per element (x- or σ-lines)
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  // line index li = threadIdx.x + k·blockDim.x as (element, line in element), stepped without
  // dividing: line 0 of the loop and the step of blockDim.x lines
  const int le0 = threadIdx.x / lpe, lr0 = threadIdx.x - le0 * lpe;
  const int lde = blockDim.x / lpe, ldr = blockDim.x - lde * lpe;
  unsigned parity0 = 0u, parity1 = 0u;   // next phase to wait for, per staging buffer (thread 0)
  int pending0 = 0, pending1 = 0;        // a bulk copy is in flight into the buffer (thread 0)

  // thread 0: issue the copy of `tile` into buffer `bf` if it can be bulk-copied
  auto issue = [&](int tile, int bf) {
    const int ex0 = tile * E, ne = min(E, Nx - ex0);
    long long lo;
    int count, shift;
    if (bulk_ok && tile_range<P, T>(g, ex0, ne, &lo, &count, &shift)) {
      fence_proxy_async_smem();
      bulk_load(Xb0 + bf * L.xbuf, x + lo, (unsigned)(count * sizeof(T)), &mbar[bf]);
      if (bf) pending1 = 1;
      else pending0 = 1;
    }
  };
  if (threadIdx.x == 0 && (int)blockIdx.x < ntiles) issue(blockIdx.x, 0);

  int k = 0;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++k) {
    const int b = k & 1;
    const int ex0 = tile * E;
    const int ne = min(E, Nx - ex0);
    const int en = ne + 1;                       // local element 0 is the left neighbour
    const bool has_left = g.periodic || ex0 > 0;
    const int nc = en * P + 1;
    long long lo;
    int count, shift;
    const bool bulk = bulk_ok && tile_range<P, T>(g, ex0, ne, &lo, &count, &shift);
    __syncthreads();                             // the previous tile's readers are done
    if (threadIdx.x == 0) {
      // prefetch the next tile into the other buffer, then wait for this one
      if (tile + (int)gridDim.x < ntiles) issue(tile + gridDim.x, b ^ 1);
      const int pend = b ? pending1 : pending0;
      if (pend) {
        const unsigned par = b ? parity1 : parity0;
        if (!mbar_wait(&mbar[b], par, kCopyTimeoutNs)) s_ok = 0;
        else if (b) { parity1 ^= 1u; pending1 = 0; }
        else { parity0 ^= 1u; pending0 = 0; }
      }
    }
    // ---- stage the tile: nodal values (a warp per column unless bulk-copied), geometry ----
    T* X = Xb0 + b * L.xbuf;
    if (bulk) {
      X += shift;
    } else {
      for (int j = warp; j < nc; j += nwarps) {
        int gc = (ex0 - 1) * P + j;
        if (gc < 0) gc = g.periodic ? gc + ncol : -1;
        else if (gc >= ncol) gc -= ncol;         // periodic: column Nx·P is column 0
        const T* xc = x + (size_t)(gc < 0 ? 0 : gc) * nrow;
        for (int r = lane; r < nrow; r += 32) X[j * nrow + r] = gc >= 0 ? __ldg(xc + r) : T(0);
      }
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
    if (!s_ok) break;                            // a copy did not complete: stop (status set below)
    const int e_first = has_left ? 0 : 1;        // walls: no element left of x = 0
    // ---- 1. x-lines: u_r ----
    for (int e = e_first + le0, rem = lr0; e < en; e += lde, rem += ldr) {
      if (rem >= lpe) { rem -= lpe; ++e; if (e >= en) break; }
      const int l = rem / Q, bb = rem - l * Q;
      const T* Xl = X + (e * P) * nrow + l * P + bb;
      T u[Q];
#pragma unroll
      for (int c = 0; c < Q; ++c) u[c] = Xl[c * nrow];
      T* out = Ur + (e * Nz + l) * BS + bb * QP;
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
      const T* Xl = X + (e * P + a) * nrow + l * P;
      T u[Q];
#pragma unroll
      for (int c = 0; c < Q; ++c) u[c] = Xl[c];
      const T* gq = Gs + (e * Q + a) * 4;
      const T c0 = Cs[2 * (e * Nz + l)], c1 = Cs[2 * (e * Nz + l) + 1];
      const T wa = Ws[a], hx = gq[2], dxd = gq[3];
      const T g11 = wa * c0 * gq[0];             // w_a Δσ/Δx d
      const T g22 = wa * c1 * gq[1];             // w_a Δx/Δσ /d
      const T* sg = Ss + l * P;
      const int base = (e * Nz + l) * BS;
      T f2[Q];
#pragma unroll
      for (int bb = 0; bb < Q; ++bb) {
        T ut = T(0);
#pragma unroll
        for (int c = 0; c < Q; ++c) ut = fmx(D[bb * Q + c], u[c], ut);
        const T ur = Ur[base + bb * QP + a];
        const T K12 = fmx(-sg[bb], dxd, hx);
        const T wb = w[bb];
        const T G12 = wa * wb * K12;
        Fs[base + bb * QP + a] = fmx(g11 * wb, ur, G12 * ut);
        f2[bb] = fmx(G12, ur, g22 * wb * fmx(K12, K12, T(1)) * ut);
      }
#pragma unroll
      for (int bb = 0; bb < Q; ++bb) {
        T s = T(0);
#pragma unroll
        for (int c = 0; c < Q; ++c) s = fmx(D[c * Q + bb], f2[c], s);
        Ys[base + bb * QP + a] = s;
      }
    }
    __syncthreads();
    // ---- 3. x-lines: element contributions into the tile's nodes ----
    // The u_r buffer is dead after step 2 and now holds the tile's nodes (column-major, like
    // x).  A node interior to its element's column range and layer is written by exactly one
    // x-line.  The shared nodes are completed in a fixed order: the value of the element to the
    // right (a = 0) and of the layer above (b = 0) is stored; the top row of a layer (b = P)
    // and the right column of an element (a = P) go to small buffers and are added afterwards,
    // rows first, then columns.
    T* Yt = Ur;
    for (int e = e_first + le0, rem = lr0; e < en; e += lde, rem += ldr) {
      if (rem >= lpe) { rem -= lpe; ++e; if (e >= en) break; }
      const int l = rem / Q, bb = rem - l * Q;
      const int row = (e * Nz + l) * BS + bb * QP;
      T f1[Q];
#pragma unroll
      for (int c = 0; c < Q; ++c) f1[c] = Fs[row + c];
      const bool top = bb == P && l < Nz - 1;   // row shared with the layer above
      T* yn = Yt + (e * P) * nrow + l * P + bb;
#pragma unroll
      for (int a = 0; a < Q; ++a) {
        T s = Ys[row + a];
#pragma unroll
        for (int c = 0; c < Q; ++c) s = fmx(D[c * Q + a], f1[c], s);
        if (a == P) Ccol[(e * Nz + l) * Q + bb] = s;
        else if (top) Rrow[(e * Nz + l) * Q + a] = s;
        else yn[a * nrow] = s;
      }
    }
    __syncthreads();
    // rows shared between layers: (e, l, a < P) adds to row (l+1)·P
    const int rpe = (Nz > 1 ? Nz - 1 : 1) * P;   // shared rows per element (the loop is empty for Nz = 1)
    for (int t = threadIdx.x; t < en * (Nz - 1) * P; t += blockDim.x) {
      const int e = t / rpe, rem = t - e * rpe;
      const int l = rem / P, a = rem - l * P;
      if (e < e_first) continue;
      Yt[(e * P + a) * nrow + (l + 1) * P] += Rrow[(e * Nz + l) * Q + a];
    }
    __syncthreads();
    // columns shared between elements: (e, l, b) adds to column (e+1)·P; the layers' top nodes
    // (b = P, below the top layer) meet the next layer's b = 0 and are added in a second sweep
    for (int sweep = 0; sweep < 2; ++sweep) {
      const int per = sweep == 0 ? P : 1;        // b = 0..P−1, then b = P
      for (int t = threadIdx.x; t < en * Nz * per; t += blockDim.x) {
        const int e = t / (Nz * per), rem = t - e * (Nz * per);
        const int l = rem / per, bb = sweep == 0 ? rem - l * per : P;
        if (e < e_first) continue;
        T* dst = Yt + ((e + 1) * P) * nrow + l * P + bb;
        const T v = Ccol[(e * Nz + l) * Q + bb];
        // the tile's last column has no element to its right: its first contribution is a store
        // (rows l·P+b, b < P, and the surface node), the layer-top nodes then add
        const bool first_here = e == en - 1 && (sweep == 0 || l == Nz - 1);
        if (first_here) *dst = v;
        else *dst += v;
      }
      __syncthreads();
    }
    // ---- 4. own columns [P, P + ne·P) (plus the last column between walls), contiguous ----
    const bool last_wall = !g.periodic && ex0 + ne == Nx;
    const int nout = (ne * P + (last_wall ? 1 : 0)) * nrow;   // output values
    T* yt = y + (size_t)ex0 * P * nrow;
    const T* ys = Yt + P * nrow;
    for (int t = threadIdx.x; t < nout; t += blockDim.x) yt[t] = -ys[t];
  }
  // a copy still in flight (after a timeout, or the prefetch of a tile this CTA stopped
  // before) must land before the CTA's shared memory is released
  __syncthreads();
  if (threadIdx.x == 0) {
    if (!s_ok) atomicOr(g.status, ST_TIMEOUT);
    if (pending0 && !mbar_wait(&mbar[0], parity0, kCopyTimeoutNs)) atomicOr(g.status, ST_TIMEOUT);
    if (pending1 && !mbar_wait(&mbar[1], parity1, kCopyTimeoutNs)) atomicOr(g.status, ST_TIMEOUT);
  }
}

// Dynamic shared memory of the tiled apply for tile width E.
template <int P>
size_t apply_tile_smem(int E, int nrow, int Nz, size_t elem) {
  return TileLayout<P>(E, nrow, Nz, (int)elem).bytes(nrow, Nz, (int)elem);
}

}  // namespace semgb
