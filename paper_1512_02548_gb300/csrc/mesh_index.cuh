// Index helpers of the structured σ-mesh and small device utilities shared by the
// translation units (internal linkage).
#pragma once
#include <cstddef>

#include "sem_internal.cuh"

namespace semgb {

static __device__ __forceinline__ double ldcg(const double* p) { return __ldcg(p); }
static __device__ __forceinline__ float ldcg(const float* p) { return __ldcg(p); }

static __device__ __forceinline__ int col_of(const DevGeom& g, int ex, int a) {
  int c = ex * g.P + a;
  return c >= g.ncol ? c - g.ncol : c;
}

static __device__ __forceinline__ bool has_left_edge(const DevGeom& g, int col) {
  if (col % g.P != 0) return false;
  if (g.periodic) return true;
  return col > 0 && col < g.Nx * g.P;
}

static __device__ __forceinline__ int left_element(const DevGeom& g, int col) {
  const int ex = col / g.P;
  return ex == 0 ? g.Nx - 1 : ex - 1;
}

// The same with the order known at compile time (no run-time division).
template <int P>
static __device__ __forceinline__ bool has_left_edge_p(const DevGeom& g, int col) {
  if (col % P != 0) return false;
  if (g.periodic) return true;
  return col > 0 && col < g.Nx * P;
}
template <int P>
static __device__ __forceinline__ int left_element_p(const DevGeom& g, int col) {
  const int ex = col / P;
  return ex == 0 ? g.Nx - 1 : ex - 1;
}

static __device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

constexpr int kMaxDynSmem = 180 * 1024;   // opt-in ceiling; each launch passes its own size

// Dynamic shared memory of the element-column apply (tables, one element column, fluxes).
static inline size_t apply_smem_bytes(int P, int nrow, int Nz, int E, size_t elem) {
  const int Q = P + 1;
  return elem * (size_t)(Q * Q + Q + nrow + (size_t)E * (2 * Nz + 4 * Q + Q * nrow + 2 * Nz * Q * Q)) + 16;
}

}  // namespace semgb
