// Tensor-core FP32 tiled apply, orders P = 4..7 (P+1 ≤ 8): the tiles, bulk-copy staging,
// shared-node fix-ups and contiguous output of the tiled apply (apply_tile.cuh), with the element
// contributions computed on the tensor cores.  Included by laplace_device.cuh after apply_tile.cuh.
// Selected with SEM_APPLY_F32=tc.  On GB300 it is slower than the CUDA-core kernel (82.6 against
// 70.3 µs on a 65536×4, P = 6 tank): the contractions' FMAs it moves to the tensor pipe are a
// third of that kernel's instructions, and the operand splits, the fragment-layout exchanges
// through shared memory and the padding of 49 nodes to 64 slots cost more issue slots than they
// free (96 M against 86 M warp instructions on a 131072×4 tank).
//
// The four sum-factorised contractions of an element block (x-element e, layer l; nodal values
// U[b][a], b along σ, a along x, (P+1)² of them) are small dense products with the GLL
// derivative matrix D (§3.1.2):
//     u_r = U Dᵀ,   u_tᵀ = Uᵀ Dᵀ,   y_σᵀ = F2ᵀ D,   y = F1 D + y_σ,
// and each is one warp-wide mma.sync m16n8k8 (TF32 inputs, FP32 accumulation) over a PAIR of
// blocks: M = 16 rows are the two blocks' 8 lines, N = K = 8 hold the P+1 nodes of a line
// padded with zero rows/columns of D.  TF32 keeps 10 mantissa bits, which would perturb the
// operator by ~1e-3 relative — far above FP32 — so every product is split in the 3×TF32 way:
// a = a_hi + a_lo with a_hi = a rounded to TF32 and a_lo = a − a_hi (exact in FP32), likewise D,
// and a·D ≈ a_lo·D_hi + a_hi·D_lo + a_hi·D_hi (the a_lo·D_lo term is below FP32 rounding).
//
// Fragment layouts of m16n8k8 .tf32 (PTX ISA), lane = 4·g + t:
//   A (16×8): a0 (g, t), a1 (g+8, t), a2 (g, t+4), a3 (g+8, t+4)
//   B (8×8):  b0 (k = t, n = g), b1 (k = t+4, n = g)
//   C (16×8): c0 (g, 2t), c1 (g, 2t+1), c2 (g+8, 2t), c3 (g+8, 2t+1)
// Row g of the tile is line g of block 0 and row g+8 line g of block 1.  u_r comes out with the
// lines along b and u_t with the lines along a, so u_r is passed through a per-warp shared-memory
// scratch to meet u_t at the same nodes (lane holds nodes a = g, b = 2t, 2t+1 of both blocks).
// F2 is then used as the A operand of y_σᵀ directly, with D's rows permuted to match (the
// C-layout columns 2t, 2t+1 taken as the A-layout columns t, t+4); F1 and y_σ go through the
// scratch once more, to the A layout and the C layout of the last product.  Padding rows and
// columns read clamped (finite) nodes, and their products are either discarded or multiplied
// by D's zero padding.  All sums have a fixed order: results are bitwise reproducible.
#pragma once

#include "apply_tile.cuh"

namespace semgb {

// floats of per-warp scratch: lines-by-σ buffer of two blocks (2·8·12) and the F1 buffer (2·8·24)
constexpr int kTcScratch = 2 * 8 * 12 + 2 * 8 * 24;

// v rounded to TF32 (10 mantissa bits), to nearest with ties away from zero, on the bit pattern:
// adding half a TF32 ulp to the magnitude bits carries into the kept bits exactly when the
// dropped 13 bits are at least half an ulp (finite v; a carry into the exponent is the correct
// rounding up to the next binade).  Two integer instructions.
static __device__ __forceinline__ unsigned tf32_rna(float v) {
  return (__float_as_uint(v) + 0x1000u) & 0xFFFFE000u;
}
static __device__ __forceinline__ void tf32_split(float v, unsigned& hi, unsigned& lo) {
  hi = tf32_rna(v);
  lo = __float_as_uint(v - __uint_as_float(hi));   // exact; its low bits are ignored by the MMA
}
static __device__ __forceinline__ void mma_tf32(float (&c)[4], const unsigned (&a)[4], unsigned b0, unsigned b1) {
  asm("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
// c += a·B with FP32-level accuracy (3×TF32); B given as its TF32 high and low parts
static __device__ __forceinline__ void mma3(float (&c)[4], const float (&a)[4], const unsigned (&bh)[2],
                                            const unsigned (&bl)[2]) {
  unsigned ah[4], al[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) tf32_split(a[i], ah[i], al[i]);
  mma_tf32(c, al, bh[0], bh[1]);
  mma_tf32(c, ah, bl[0], bl[1]);
  mma_tf32(c, ah, bh[0], bh[1]);
}

// Per-lane constants of the tensor-core kernel: B fragments of D (high/low parts) for the three
// operand forms, the lane's clamped node indices and the weights of its nodes.
struct TcLane {
  unsigned bd_h[2], bd_l[2];   // B[k][n] = D[n][k]          (u_r, u_t)
  unsigned bp_h[2], bp_l[2];   // B[k][n] = D[π(k)][n], π(t) = 2t, π(t+4) = 2t+1  (y_σᵀ)
  unsigned bt_h[2], bt_l[2];   // B[k][n] = D[k][n]          (F1 D)
  int g, t, gc, t4c, t2c, t21c;
  float wab0, wab1;            // w_g w_{2t}, w_g w_{2t+1}
};

template <int P>
static __device__ __forceinline__ TcLane tc_lane(const float* D, const float* w) {
  constexpr int Q = P + 1;
  TcLane c;
  const int lane = threadIdx.x & 31;
  c.g = lane >> 2;
  c.t = lane & 3;
  c.gc = min(c.g, P);
  c.t4c = min(c.t + 4, P);
  c.t2c = min(2 * c.t, P);
  c.t21c = min(2 * c.t + 1, P);
  auto dv = [&](int r, int k) { return (r < Q && k < Q) ? D[r * Q + k] : 0.f; };
  tf32_split(dv(c.g, c.t), c.bd_h[0], c.bd_l[0]);
  tf32_split(dv(c.g, c.t + 4), c.bd_h[1], c.bd_l[1]);
  tf32_split(dv(2 * c.t, c.g), c.bp_h[0], c.bp_l[0]);
  tf32_split(dv(2 * c.t + 1, c.g), c.bp_h[1], c.bp_l[1]);
  tf32_split(dv(c.t, c.g), c.bt_h[0], c.bt_l[0]);
  tf32_split(dv(c.t + 4, c.g), c.bt_h[1], c.bt_l[1]);
  c.wab0 = w[c.gc] * w[c.t2c];
  c.wab1 = w[c.gc] * w[c.t21c];
  return c;
}

// One tile's element contributions: the (element, layer) blocks e = e_first..en−1, l = 0..Nz−1
// in pairs over the CTA's warps.  X: the tile's nodal values (column-major, `nrow` per column);
// Gs [en][P+1] float4 (d, 1/d, ∂xh, ∂xd); Cs [en][Nz] float2 (Δσ/Δx, Δx/Δσ); Ss [nrow] σ.
// Contributions go to Yt (tile nodes), Rrow (top rows shared with the layer above) and Ccol
// (right columns shared with the next element), as in the CUDA-core kernel.
template <int P, int NZC>
static __device__ __forceinline__ void tc_tile(const TcLane& c, const float* X, float* Yt, float* scr,
                                               const float* Gs, const float* Cs, const float* Ss, float* Rrow,
                                               float* Ccol, int en, int e_first, int Nz_rt, int nrow_rt) {
  constexpr int Q = P + 1;
  const int Nz = NZC ? NZC : Nz_rt;
  const int nrow = NZC ? NZC * P + 1 : nrow_rt;
  const int warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int nb = (en - e_first) * Nz;
  const int npair = (nb + 1) >> 1;
  float* sA = scr;                 // [2][8 b][12]: u_r by lines along b, then y_σ
  float* sB = scr + 2 * 8 * 12;    // [2][8 a][24]: F1 by lines along a
  const int offr = c.t * nrow + c.gc, offr4 = c.t4c * nrow + c.gc;   // A of u_r: U[b = g][k]
  const int offs = c.gc * nrow + c.t, offs4 = c.gc * nrow + c.t4c;   // A of u_t: U[k][a = g]
  const int g = c.g, t = c.t;
  for (int p = warp; p < npair; p += nwarps) {
    const int i0 = 2 * p, i1 = min(2 * p + 1, nb - 1);
    const bool has1 = 2 * p + 1 < nb;
    const int e0 = e_first + i0 / Nz, l0 = i0 - (i0 / Nz) * Nz;
    const int e1 = e_first + i1 / Nz, l1 = i1 - (i1 / Nz) * Nz;
    const float* X0 = X + e0 * P * nrow + l0 * P;
    const float* X1 = X + e1 * P * nrow + l1 * P;
    // ---- u_r and u_t ----
    float ur[4] = {0.f, 0.f, 0.f, 0.f}, ut[4] = {0.f, 0.f, 0.f, 0.f};
    {
      const float a[4] = {X0[offr], X1[offr], X0[offr4], X1[offr4]};
      mma3(ur, a, c.bd_h, c.bd_l);
    }
    {
      const float a[4] = {X0[offs], X1[offs], X0[offs4], X1[offs4]};
      mma3(ut, a, c.bd_h, c.bd_l);
    }
    // u_r (b = g, a = 2t, 2t+1) → the lane's nodes (a = g, b = 2t, 2t+1)
    __syncwarp();
    *reinterpret_cast<float2*>(sA + g * 12 + 2 * t) = make_float2(ur[0], ur[1]);
    *reinterpret_cast<float2*>(sA + 96 + g * 12 + 2 * t) = make_float2(ur[2], ur[3]);
    __syncwarp();
    ur[0] = sA[(2 * t) * 12 + g];
    ur[1] = sA[(2 * t + 1) * 12 + g];
    ur[2] = sA[96 + (2 * t) * 12 + g];
    ur[3] = sA[96 + (2 * t + 1) * 12 + g];
    // ---- fluxes F1, F2 at the lane's nodes ----
    float f1[4], f2[4];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const int e = k ? e1 : e0, l = k ? l1 : l0;
      const float4 gq = *reinterpret_cast<const float4*>(Gs + (e * Q + c.gc) * 4);
      const float2 cc = *reinterpret_cast<const float2*>(Cs + 2 * (e * Nz + l));
      const float al = cc.x * gq.x;      // Δσ/Δx · d
      const float be = cc.y * gq.y;      // Δx/Δσ / d
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const float sg = Ss[l * P + (j ? c.t21c : c.t2c)];
        const float wab = j ? c.wab1 : c.wab0;
        const float K12 = fmaf(-sg, gq.w, gq.z);
        const float G12 = wab * K12;
        const float u1 = ur[2 * k + j], u2 = ut[2 * k + j];
        f1[2 * k + j] = fmaf(al * wab, u1, G12 * u2);
        f2[2 * k + j] = fmaf(G12, u1, be * wab * fmaf(K12, K12, 1.f) * u2);
      }
    }
    *reinterpret_cast<float2*>(sB + g * 24 + 2 * t) = make_float2(f1[0], f1[1]);
    *reinterpret_cast<float2*>(sB + 192 + g * 24 + 2 * t) = make_float2(f1[2], f1[3]);
    // ---- y_σᵀ = F2ᵀ D (F2 in the C layout serves as A with D's rows permuted) ----
    float ys[4] = {0.f, 0.f, 0.f, 0.f};
    {
      const float a[4] = {f2[0], f2[2], f2[1], f2[3]};
      mma3(ys, a, c.bp_h, c.bp_l);
    }
    __syncwarp();   // every lane has read u_r from sA and written F1 to sB
    sA[(2 * t) * 12 + g] = ys[0];
    sA[(2 * t + 1) * 12 + g] = ys[1];
    sA[96 + (2 * t) * 12 + g] = ys[2];
    sA[96 + (2 * t + 1) * 12 + g] = ys[3];
    __syncwarp();
    // ---- y = F1 D + y_σ, lines along b ----
    float y[4];
    {
      const float2 c0 = *reinterpret_cast<const float2*>(sA + g * 12 + 2 * t);
      const float2 c1 = *reinterpret_cast<const float2*>(sA + 96 + g * 12 + 2 * t);
      y[0] = c0.x; y[1] = c0.y; y[2] = c1.x; y[3] = c1.y;
      const float a[4] = {sB[t * 24 + g], sB[192 + t * 24 + g], sB[(t + 4) * 24 + g], sB[192 + (t + 4) * 24 + g]};
      mma3(y, a, c.bt_h, c.bt_l);
    }
    // ---- contributions of the lane's nodes (b = g, a = 2t, 2t+1) ----
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      if (k == 1 && !has1) break;
      const int e = k ? e1 : e0, l = k ? l1 : l0;
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const int a = 2 * t + j, b = g;
        if (a > P || b > P) continue;
        const float v = y[2 * k + j];
        if (a == P) Ccol[(e * Nz + l) * Q + b] = v;
        else if (b == P && l < Nz - 1) Rrow[(e * Nz + l) * Q + a] = v;
        else Yt[(e * P + a) * nrow + l * P + b] = v;
      }
    }
  }
}

// Tensor-core tiled apply (FP32).  Same tiles, staging, fix-ups and output as k_apply_tile;
// NZC > 0: the layer count is the compile-time constant NZC.
template <int P, int NZC>
__global__ void __launch_bounds__(kThreads, 3)
    k_apply_tile_tc(DevGeom g, const float* __restrict__ x, float* __restrict__ y, int E, int bulk_ok) {
  constexpr int Q = P + 1;
  static_assert(P >= 4 && P <= 7, "tensor-core apply: orders 4..7");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nrow = NZC ? NZC * P + 1 : g.nrow, Nz = NZC ? NZC : g.Nz, Nx = g.Nx, ncol = g.ncol;
  const TileLayout<P> L(E, nrow, Nz, (int)sizeof(float));
  unsigned long long* mbar = reinterpret_cast<unsigned long long*>(smem_raw);   // [2]
  float* const Xb0 = reinterpret_cast<float*>(smem_raw + 16);   // staging buffers at Xb0 + b·xbuf
  float* Yt = Xb0 + 2 * L.xbuf;                       // [tcols][nrow] the tile's nodes
  float* Scr = Yt + L.ybuf;                           // [warps][kTcScratch]
  float* Gs = Scr + (kThreads / 32) * kTcScratch;     // [en][Q][4] d, 1/d, ∂xh, ∂xd (16-B aligned)
  float* Cs = Gs + (size_t)L.en_max * Q * 4;          // [en][Nz][2] Δσ/Δx, Δx/Δσ
  float* Ss = Cs + (size_t)L.en_max * Nz * 2;         // [nrow] σ
  float* Rrow = Ss + nrow + Q;                        // [en][Nz][Q] top-row (b = P) contributions, a < P
  float* Ccol = Rrow + (size_t)L.en_max * Nz * Q;     // [en][Nz][Q] right-column (a = P) contributions
  __shared__ int s_ok;
  const float* D = CT<float>::D() + d_off(P);
  const float* w = CT<float>::w() + w_off(P);
  const float* geo = geo_ptr<float>(g);
  const TcLane lane_c = tc_lane<P>(D, w);
  for (int t = threadIdx.x; t < nrow; t += blockDim.x) Ss[t] = (float)g.sig[t];
  if (threadIdx.x == 0) {
    mbar_init(&mbar[0]);
    mbar_init(&mbar[1]);
    mbar_init_fence();
    s_ok = 1;
  }
  __syncthreads();
  const int ntiles = (Nx + E - 1) / E;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  unsigned parity0 = 0u, parity1 = 0u;   // next phase to wait for, per staging buffer (thread 0)
  int pending0 = 0, pending1 = 0;        // a bulk copy is in flight into the buffer (thread 0)
  auto issue = [&](int tile, int bf) {
    const int ex0 = tile * E, ne = min(E, Nx - ex0);
    long long lo;
    int count, shift;
    if (bulk_ok && tile_range<P, float>(g, ex0, ne, &lo, &count, &shift)) {
      fence_proxy_async_smem();
      bulk_load(Xb0 + bf * L.xbuf, x + lo, (unsigned)(count * sizeof(float)), &mbar[bf]);
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
    const bool bulk = bulk_ok && tile_range<P, float>(g, ex0, ne, &lo, &count, &shift);
    __syncthreads();                             // the previous tile's readers are done
    if (threadIdx.x == 0) {
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
    float* X = Xb0 + b * L.xbuf;
    if (bulk) {
      X += shift;
    } else {
      for (int j = warp; j < nc; j += nwarps) {
        int gc = (ex0 - 1) * P + j;
        if (gc < 0) gc = g.periodic ? gc + ncol : -1;
        else if (gc >= ncol) gc -= ncol;
        const float* xc = x + (size_t)(gc < 0 ? 0 : gc) * nrow;
        for (int r = lane; r < nrow; r += 32) X[j * nrow + r] = gc >= 0 ? __ldg(xc + r) : 0.f;
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
      const float dxe = (float)g.dxe[ge], dsl = (float)g.dsl[l];
      Cs[2 * t] = dsl / dxe;
      Cs[2 * t + 1] = dxe / dsl;
    }
    __syncthreads();
    if (!s_ok) break;                            // a copy did not complete: stop (status set below)
    const int e_first = has_left ? 0 : 1;        // walls: no element left of x = 0
    tc_tile<P, NZC>(lane_c, X, Yt, Scr + warp * kTcScratch, Gs, Cs, Ss, Rrow, Ccol, en, e_first, Nz, nrow);
    __syncthreads();
    // rows shared between layers: (e, l, a < P) adds to row (l+1)·P
    const int rpe = (Nz > 1 ? Nz - 1 : 1) * P;
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
      const int per = sweep == 0 ? P : 1;
      for (int t = threadIdx.x; t < en * Nz * per; t += blockDim.x) {
        const int e = t / (Nz * per), rem = t - e * (Nz * per);
        const int l = rem / per, bb = sweep == 0 ? rem - l * per : P;
        if (e < e_first) continue;
        float* dst = Yt + ((e + 1) * P) * nrow + l * P + bb;
        const float v = Ccol[(e * Nz + l) * Q + bb];
        const bool first_here = e == en - 1 && (sweep == 0 || l == Nz - 1);
        if (first_here) *dst = v;
        else *dst += v;
      }
      __syncthreads();
    }
    // ---- own columns [P, P + ne·P) (plus the last column between walls), contiguous ----
    const bool last_wall = !g.periodic && ex0 + ne == Nx;
    const int nout = (ne * P + (last_wall ? 1 : 0)) * nrow;
    float* yt = y + (size_t)ex0 * P * nrow;
    const float* ys = Yt + P * nrow;
    for (int t = threadIdx.x; t < nout; t += blockDim.x) yt[t] = -ys[t];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (!s_ok) atomicOr(g.status, ST_TIMEOUT);
    if (pending0 && !mbar_wait(&mbar[0], parity0, kCopyTimeoutNs)) atomicOr(g.status, ST_TIMEOUT);
    if (pending1 && !mbar_wait(&mbar[1], parity1, kCopyTimeoutNs)) atomicOr(g.status, ST_TIMEOUT);
  }
}

// Dynamic shared memory of the tensor-core apply for tile width E.
template <int P>
size_t apply_tile_tc_smem(int E, int nrow, int Nz) {
  return TileLayout<P>(E, nrow, Nz, (int)sizeof(float)).bytes_tc(nrow, Nz, kTcScratch);
}

}  // namespace semgb
