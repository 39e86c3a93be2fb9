// C ABI of the library (declared in include/sem.h): mesh set-up, host-side tables and
// the orchestration of the kernels for one Laplace solve, the recovery, the Zakharov
// right-hand side and RK4 (§2–§3 of arXiv 1512.02548).
#include <algorithm>
#include <array>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <queue>
#include <mutex>
#include <tuple>
#include <memory>
#include <string>
#include <utility>
#include <vector>

#include "sem.h"
#include "mesh_index.cuh"
#include "sem_internal.cuh"
#include "tables.h"

using namespace semgb;

namespace semgb {
static std::atomic<long long> g_launches{0};
void count_launch(int k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
}  // namespace semgb

namespace {

constexpr int kMaxWaveComp = 4096;
thread_local std::string t_err;

int fail(int code, const std::string& msg) {
  t_err = msg;
  return code;
}

#define CUDA_TRY(call)                                                                      \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess)                                                                  \
      return fail(SEM_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));        \
  } while (0)

std::mutex g_tables_mu;
bool g_tables_done[64] = {false};

int ensure_device_tables(int dev) {
  std::lock_guard<std::mutex> lk(g_tables_mu);
  if (dev < 0 || dev >= 64) return fail(SEM_ERR_INVALID_ARG, "device index out of range");
  if (g_tables_done[dev]) return SEM_OK;
  std::vector<double> D(kDTotal, 0.0), w(kWTotal, 0.0);
  for (int P = 1; P <= kMaxP; ++P) {
    Line L = make_line(P);
    std::memcpy(&D[d_off(P)], L.D.data(), sizeof(double) * (P + 1) * (P + 1));
    std::memcpy(&w[w_off(P)], L.w.data(), sizeof(double) * (P + 1));
  }
  CUDA_TRY(upload_line_tables(D.data(), w.data()));
  g_tables_done[dev] = true;
  return SEM_OK;
}

// Device memory of meshes and batches comes from a per-device cache of freed blocks, so that
// a serving loop that creates and destroys meshes per request does not pay cudaMalloc and
// cudaFree for each.  A freed block is kept (up to kCacheBytes per device) and handed to a
// later request of at most its size and at least half of it.  sem_trim_cache returns the
// cached blocks to CUDA.
constexpr size_t kCacheBytes = 8ull << 30;
struct BlockCache {
  std::multimap<size_t, void*> free;          // size → block
  std::map<void*, size_t> size_of;            // every block this cache handed out or holds
  size_t cached = 0;
};
std::mutex g_cache_mu;
BlockCache g_cache[64];

cudaError_t dev_alloc(int dev, size_t bytes, void** p) {
  {
    std::lock_guard<std::mutex> lk(g_cache_mu);
    BlockCache& c = g_cache[dev];
    auto it = c.free.lower_bound(bytes);
    if (it != c.free.end() && it->first <= 2 * bytes) {
      *p = it->second;
      c.cached -= it->first;
      c.free.erase(it);
      return cudaSuccess;
    }
  }
  cudaError_t e = cudaMalloc(p, bytes);
  if (e == cudaErrorMemoryAllocation) {        // give the cached blocks back and retry once
    sem_trim_cache();
    cudaGetLastError();
    e = cudaMalloc(p, bytes);
  }
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(g_cache_mu);
  g_cache[dev].size_of[*p] = bytes;
  return cudaSuccess;
}

// The block must have no work in flight; the callers synchronise the device first.
void dev_free(int dev, void* p) {
  if (!p) return;
  std::lock_guard<std::mutex> lk(g_cache_mu);
  BlockCache& c = g_cache[dev];
  auto it = c.size_of.find(p);
  const size_t sz = it == c.size_of.end() ? 0 : it->second;
  if (sz > 0 && c.cached + sz <= kCacheBytes) {
    c.free.emplace(sz, p);
    c.cached += sz;
  } else {
    if (it != c.size_of.end()) c.size_of.erase(it);
    cudaFree(p);
  }
}

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

// Bump allocator over one device allocation (256-byte aligned slices).
struct Carve {
  size_t off = 0;
  template <class T> size_t take(size_t count) {
    size_t o = (off + 255) & ~size_t(255);
    off = o + count * sizeof(T);
    return o;
  }
};

}  // namespace

struct sem_mesh {
  sem_params p{};
  int device = 0;
  int ncol = 0, nrow = 0, Pf = 0, nif = 0;
  long long n = 0;
  int grid = 0;
  size_t smem = 0;
  unsigned char* pool = nullptr;
  size_t pool_bytes = 0;
  DevGeom g{};
  SurfTables st{};
  PcgArgs pa{};
  PrecSetup ps{};
  SolveRecord* rec = nullptr;
  // workspace
  double *Phi = nullptr, *qtmp = nullptr, *edgetmp = nullptr;
  double *wt = nullptr, *etax = nullptr, *phisx = nullptr, *R = nullptr, *scr = nullptr;
  double *ke = nullptr, *kp = nullptr, *ae = nullptr, *ap = nullptr, *se = nullptr, *sp = nullptr;
  double *eta_dev = nullptr, *phis_dev = nullptr;
  double *s1e = nullptr, *s1p = nullptr;   // second stage-input pair of the fused RK stage
  // stage potentials kept for the next stages' initial guesses, and the trajectory they belong
  // to (the state buffers and dt of the last fused RK call; hist_dt = 0: none)
  double *Phi1 = nullptr, *Phi2 = nullptr, *Phi3 = nullptr, *D32 = nullptr;
  // column positions on the host, and the cos/sin(k x) table of the left-zone columns for the
  // generated signal (its own device block, rebuilt by sem_set_wave_input)
  std::vector<double> xcol_h;
  double* wkx = nullptr;
  double hist_dt = 0.0;
  const double *hist_eta = nullptr, *hist_phis = nullptr;
  // fused-stage launch of this mesh alone: device descriptor, CTA map, barrier pair
  Instance* inst_d = nullptr;
  int* cta_inst_d = nullptr;
  unsigned int* stage_bars = nullptr;
  Instance inst_h{};
  int stage_team = 0;
  size_t stage_smem = 0;         // the mesh's own fused stage launch (with the factor cache)
  size_t stage_smem_batch = 0;   // in a batch launch (no factor cache)
  int gcache = 0;                // doubles of the factor cache in the own launch (0 = none)
  int own_chunk = 0;             // element columns per pass in the own launch (g.chunk elsewhere)
  bool fused = true;
  // optional event timing of the Krylov kernel
  bool timing = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> events;
  std::vector<cudaEvent_t> spare;
};

// A batch: instances grouped by (order, precision) and, within a group, into launches of at
// most the co-resident capacity; each instance gets a team of CTAs sized to its work.
struct BatchLaunch {
  int P = 0, mixed = 0, wide = 1;
  int csize = 0;                     // cluster teams of csize CTAs each (0: one cooperative launch)
  std::vector<int> members;          // mesh indices
  std::vector<int> team0, nteam;
  std::vector<int> chunk;            // element columns per pass of each member
  int grid = 0;
  size_t smem = 0;
  Instance* inst_d = nullptr;
  int* cta_d = nullptr;
  unsigned int* bars_d = nullptr;
  int* status_d = nullptr;           // gathered status words of the members
  std::vector<Instance> inst_h;
  std::vector<int> status_h;
  cudaStream_t stream = nullptr;     // cluster launches: the launch's own stream
  cudaEvent_t done = nullptr;        // ... and the event that joins it back to the caller's stream
};

struct sem_batch {
  std::vector<sem_mesh*> meshes;
  std::vector<int> codes;            // per-instance error code of the last step or solve
  std::vector<BatchLaunch> launches;     // cooperative plan: one launch per RK stage and group
  std::vector<BatchLaunch> cl_launches;  // cluster plan: launches on streams of their own (empty: none)
  cudaEvent_t fork = nullptr;
  int device = 0;
  unsigned char* pool = nullptr;
  // packed device copy of every member's (η, φ̃) for sem_batch_rk4_step_host: η of member i at
  // state + off[i], φ̃ at state + ncol_total + off[i]
  double* state = nullptr;
  std::vector<size_t> off;
  size_t ncol_total = 0;
  // optional event timing of the stage launches
  bool timing = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> events;
  std::vector<cudaEvent_t> spare;
};

namespace {

// Error code of a device status word (no message).
int status_code(int st) {
  if (st == 0) return SEM_OK;
  if (st & ST_TIMEOUT) return SEM_ERR_TIMEOUT;
  if (st & (ST_BAD_DEPTH | ST_NONFINITE)) return SEM_ERR_NONFINITE;
  if (st & ST_NOT_CONVERGED) return SEM_ERR_NOT_CONVERGED;
  return SEM_ERR_CUDA;
}

int status_error(int st) {
  if (st == 0) return SEM_OK;
  if (st & ST_TIMEOUT) return fail(SEM_ERR_TIMEOUT, "a grid barrier of the Krylov kernel timed out");
  if (st & ST_BAD_DEPTH) return fail(SEM_ERR_NONFINITE, "water depth d = eta + h is not positive and finite");
  if (st & ST_NONFINITE) return fail(SEM_ERR_NONFINITE, "non-finite residual in the Laplace solve");
  if (st & ST_NOT_CONVERGED) return fail(SEM_ERR_NOT_CONVERGED, "Laplace solve reached max_iter above tol");
  return fail(SEM_ERR_CUDA, "unknown device status");
}

// After a failed step the mesh's warm-start potential may hold non-finite values; the next
// solve on this mesh starts from zero instead.
cudaError_t reset_warm_start(sem_mesh* m, cudaStream_t s) {
  m->hist_dt = 0.0;   // the stage potentials kept for initial guesses may be from a failed step
  return cudaMemsetAsync(m->Phi, 0, sizeof(double) * (size_t)m->n, s);
}

int read_status(sem_mesh* m, cudaStream_t s) {
  int st = 0;
  CUDA_TRY(cudaMemcpyAsync(&st, m->g.status, sizeof(int), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  if (st == 0) return SEM_OK;
  CUDA_TRY(reset_warm_start(m, s));
  CUDA_TRY(cudaMemsetAsync(m->g.status, 0, sizeof(int), s));
  CUDA_TRY(cudaStreamSynchronize(s));
  return status_error(st);
}

cudaError_t take_event(sem_mesh* m, cudaEvent_t* ev) {
  if (!m->spare.empty()) { *ev = m->spare.back(); m->spare.pop_back(); return cudaSuccess; }
  return cudaEventCreate(ev);
}

int do_solve(sem_mesh* m, const double* phis, double* Phi, cudaStream_t s) {
  PcgArgs a = m->pa;
  a.x = Phi;
  a.phis = phis;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (m->timing) {
    CUDA_TRY(take_event(m, &e0));
    CUDA_TRY(take_event(m, &e1));
    CUDA_TRY(cudaEventRecord(e0, s));
  }
  CUDA_TRY(launch_pcg(m->g, a, m->grid, m->smem, s));
  if (m->timing) {
    CUDA_TRY(cudaEventRecord(e1, s));
    m->events.emplace_back(e0, e1);
  }
  return SEM_OK;
}

int do_geometry(sem_mesh* m, const double* eta, cudaStream_t s) {
  const bool jacobi = m->p.precond == SEM_PRECOND_JACOBI;
  CUDA_TRY(launch_geometry(m->g, eta, jacobi, s));
  if (!jacobi) CUDA_TRY(launch_prec_setup(m->g, m->ps, s));
  return SEM_OK;
}

bool has_zones(const sem_mesh* m) { return m->p.relax_left > 0.0 || m->p.relax_right > 0.0; }

int do_rhs(sem_mesh* m, const double* eta, const double* phis, double time, double tau, double* de,
           double* dp, cudaStream_t s) {
  const int Q = m->p.P + 1;
  int rc0 = do_geometry(m, eta, s);
  if (rc0) return rc0;
  int rc = do_solve(m, phis, m->Phi, s);
  if (rc) return rc;
  CUDA_TRY(launch_wsurf(m->st, m->Phi, eta, m->wt, s));
  CUDA_TRY(launch_sx(m->st, eta, phis, m->R, s));
  CUDA_TRY(launch_mass1d(m->st, m->R, 2, m->etax, m->phisx, m->scr, s));
  CUDA_TRY(launch_zakharov(m->st, eta, m->etax, m->phisx, m->wt, m->R, s));
  CUDA_TRY(launch_mass1d(m->st, m->R, 2, de, dp, m->scr, s));
  if (has_zones(m)) CUDA_TRY(launch_relax(m->st, eta, phis, time, 1.0 / tau, de, dp, s));
  (void)Q;
  return SEM_OK;
}

// After a fused RK call: the next call continues the trajectory if it steps the same state
// buffers with the same dt (then its stages 2 and 3 may extrapolate from the last step's stage
// potentials).
void set_history(sem_mesh* m, const double* eta, const double* phis, double dt) {
  m->hist_dt = dt;
  m->hist_eta = eta;
  m->hist_phis = phis;
}

// own_launch: the mesh's own fused stage launch, whose shared memory holds the factor cache.
// chunk > 0: element columns per pass in a batch launch.
Instance make_instance(sem_mesh* m, double* eta, double* phis, double tstart, double dt, int team0,
                       int nteam, bool own_launch = false, int chunk = 0) {
  Instance I{};
  I.g = m->g;
  I.g.gcache = own_launch ? m->gcache : 0;
  if (own_launch) I.g.chunk = m->own_chunk;
  else if (chunk > 0) I.g.chunk = chunk;
  I.st = m->st;
  I.pa = m->pa;
  I.pa.x = m->Phi;
  I.ps = m->ps;
  I.eta = eta; I.phis = phis;
  I.s0e = m->se; I.s0p = m->sp; I.s1e = m->s1e; I.s1p = m->s1p;
  I.ke = m->ke; I.kp = m->kp; I.ae = m->ae; I.ap = m->ap;
  I.wt = m->wt; I.etax = m->etax; I.phisx = m->phisx; I.R = m->R; I.scr = m->scr;
  I.P1 = m->Phi1; I.P2 = m->Phi2; I.P3 = m->Phi3; I.D32 = m->D32;
  I.hist = (m->hist_dt == dt && m->hist_eta == eta && m->hist_phis == phis) ? 1 : 0;
  I.tstart = tstart; I.dt = dt;
  I.tau = m->p.relax_tau > 0.0 ? m->p.relax_tau : dt;
  I.team0 = team0; I.nteam = nteam;
  I.relax = has_zones(m) ? 1 : 0;
  return I;
}

// nsteps RK4 steps of one mesh with the fused stage kernel: one cooperative launch per stage.
int do_rk4_fused(sem_mesh* m, double* eta, double* phis, double t0, double dt, int nsteps, cudaStream_t s) {
  m->inst_h = make_instance(m, eta, phis, t0, dt, 0, m->stage_team, true);
  CUDA_TRY(cudaMemcpyAsync(m->inst_d, &m->inst_h, sizeof(Instance), cudaMemcpyHostToDevice, s));
  StageArgs a{m->inst_d, m->cta_inst_d, m->stage_bars, 1, 0, 0};
  const int mixed = m->p.precision == SEM_PREC_MIXED;
  for (int step = 0; step < nsteps; ++step)
    for (int stage = 1; stage <= 4; ++stage) {
      a.stage = stage;
      a.step = step;
      CUDA_TRY(cudaMemsetAsync(m->stage_bars, 0, 2 * sizeof(unsigned int), s));
      cudaEvent_t e0 = nullptr, e1 = nullptr;
      if (m->timing) {
        CUDA_TRY(take_event(m, &e0));
        CUDA_TRY(take_event(m, &e1));
        CUDA_TRY(cudaEventRecord(e0, s));
      }
      CUDA_TRY(launch_stage(m->p.P, mixed, 0, a, m->stage_team, m->stage_smem, s));
      if (m->timing) {
        CUDA_TRY(cudaEventRecord(e1, s));
        m->events.emplace_back(e0, e1);
      }
    }
  if (nsteps > 0) set_history(m, eta, phis, dt);
  return SEM_OK;
}

int do_rk4(sem_mesh* m, double* eta, double* phis, double t0, double dt, int nsteps, cudaStream_t s) {
  if (m->fused) return do_rk4_fused(m, eta, phis, t0, dt, nsteps, s);
  const int n = m->ncol;
  const double tau = m->p.relax_tau > 0.0 ? m->p.relax_tau : dt;
  for (int step = 0; step < nsteps; ++step) {
    const double ts = t0 + step * dt;
    for (int stage = 1; stage <= 4; ++stage) {
      const double* ei = stage == 1 ? eta : m->se;
      const double* pi = stage == 1 ? phis : m->sp;
      const double tstage = ts + (stage == 1 ? 0.0 : (stage == 4 ? dt : 0.5 * dt));
      int rc = do_rhs(m, ei, pi, tstage, tau, m->ke, m->kp, s);
      if (rc) return rc;
      CUDA_TRY(launch_rk4_stage(stage, n, dt, eta, phis, m->ke, m->kp, m->ae, m->ap, m->se, m->sp, s));
    }
    CUDA_TRY(launch_filter(m->st, eta, phis, s));
  }
  return SEM_OK;
}

std::vector<double> matmul(const std::vector<double>& A, const std::vector<double>& B, int n, int k, int mcols) {
  std::vector<double> C((size_t)n * mcols, 0.0);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < mcols; ++j) {
      long double s = 0.0L;
      for (int q = 0; q < k; ++q) s += (long double)A[(size_t)i * k + q] * B[(size_t)q * mcols + j];
      C[(size_t)i * mcols + j] = (double)s;
    }
  return C;
}

}  // namespace

extern "C" {

const char* sem_last_error(void) { return t_err.c_str(); }

int64_t sem_launch_count(void) { return g_launches.load(); }

// Host tables of one (P, Nz, Pf, filter) combination, shared by every mesh that has it.
struct ColumnTables {
  Line L;
  std::vector<double> MD, I, B, F, wrow, Aii, Z, Sg, lam, dsl, sig;
  long double S00 = 0, S01 = 0, S11 = 0;
};

static std::mutex g_ct_mu;
static std::map<std::tuple<int, int, int, double, double, int>, std::shared_ptr<const ColumnTables>> g_ct;

static int column_tables(const sem_params& p, std::shared_ptr<const ColumnTables>* out) {
  const auto key = std::make_tuple(p.P, p.Nz, p.Pf, p.filter_alpha, p.filter_s, p.filter_ic);
  {
    std::lock_guard<std::mutex> lk(g_ct_mu);
    auto it = g_ct.find(key);
    if (it != g_ct.end()) { *out = it->second; return SEM_OK; }
  }
  auto t = std::make_shared<ColumnTables>();
  const int P = p.P, Q = P + 1, Nz = p.Nz, nrow = Nz * P + 1, Qf = p.Pf + 1, Pm = P - 1;
  Line Lf;
  try {
    t->L = make_line(P);
    Lf = make_line(p.Pf);
  } catch (const std::exception& e) {
    return fail(SEM_ERR_INVALID_ARG, e.what());
  }
  const Line& L = t->L;
  t->dsl.assign(Nz, 1.0 / Nz);
  const std::vector<double>& dsl = t->dsl;
  t->sig.resize(nrow);
  for (int iz = 0; iz < nrow; ++iz) {
    int l = iz / P; if (l >= Nz) l = Nz - 1;
    const int b = iz - l * P;
    t->sig[iz] = (double)l / Nz + 0.5 * (L.r[b] + 1.0) * dsl[l];
  }
  t->sig[nrow - 1] = 1.0;
  t->MD = matmul(L.M, L.D, Q, Q, Q);
  t->I = interpolation(L, Lf);                                        // Qf×Q
  std::vector<double> It(Q * Qf);
  for (int q = 0; q < Qf; ++q) for (int c = 0; c < Q; ++c) It[c * Qf + q] = t->I[q * Q + c];
  t->B = matmul(It, Lf.M, Q, Qf, Qf);                                 // Q×Qf = Iᵀ M_f
  t->F = filter_matrix(L, p.filter_alpha, p.filter_s, p.filter_ic);
  // w̃ weights: v = M_σ⁻¹ e_top, c_l = (Δσ_l/2) M v|_l, contracted with the layer's σ-derivative
  // (2/Δσ_l) D into one weight per row: w̃ d = Σ_iz wrow_iz Φ_iz
  t->wrow.assign((size_t)nrow, 0.0);
  {
    std::vector<long double> wr((size_t)nrow, 0.0L);
    std::vector<long double> Ms((size_t)nrow * nrow, 0.0L);
    for (int l = 0; l < Nz; ++l)
      for (int a = 0; a < Q; ++a)
        for (int b = 0; b < Q; ++b) Ms[(size_t)(l * P + a) * nrow + l * P + b] += 0.5L * dsl[l] * L.M[a * Q + b];
    if (!invert(Ms, nrow)) return fail(SEM_ERR_INVALID_ARG, "sigma mass is singular");
    for (int l = 0; l < Nz; ++l)
      for (int b = 0; b < Q; ++b) {
        long double s = 0.0L;
        for (int c = 0; c < Q; ++c) s += 0.5L * dsl[l] * L.M[b * Q + c] * Ms[(size_t)(l * P + c) * nrow + (nrow - 1)];
        for (int c = 0; c < Q; ++c) wr[(size_t)l * P + c] += s * (2.0L / dsl[l]) * L.D[b * Q + c];
      }
    for (int iz = 0; iz < nrow; ++iz) t->wrow[iz] = (double)wr[iz];
  }
  // static condensation of M' (element scale Δx/2 · M)
  t->Aii.assign((size_t)Pm * Pm, 0.0);
  t->Z.assign((size_t)2 * Pm, 0.0);
  {
    std::vector<long double> Mii((size_t)Pm * Pm);
    for (int i = 0; i < Pm; ++i) for (int k = 0; k < Pm; ++k) Mii[i * Pm + k] = L.M[(i + 1) * Q + (k + 1)];
    if (!invert(Mii, Pm)) return fail(SEM_ERR_INVALID_ARG, "interior mass is singular");
    for (int i = 0; i < Pm * Pm; ++i) t->Aii[i] = (double)Mii[i];
    const int bn[2] = {0, P};
    long double Zl[2][kMaxP];
    for (int s2 = 0; s2 < 2; ++s2)
      for (int i = 0; i < Pm; ++i) {
        long double acc = 0.0L;
        for (int k = 0; k < Pm; ++k) acc += (long double)L.M[bn[s2] * Q + (k + 1)] * Mii[k * Pm + i];
        Zl[s2][i] = acc;
        t->Z[s2 * Pm + i] = (double)acc;
      }
    auto sch = [&](int s1, int s2) {
      long double acc = L.M[bn[s1] * Q + bn[s2]];
      for (int i = 0; i < Pm; ++i) acc -= Zl[s1][i] * (long double)L.M[(i + 1) * Q + bn[s2]];
      return acc;
    };
    t->S00 = sch(0, 0); t->S01 = sch(0, 1); t->S11 = sch(1, 1);
  }
  // σ-separable preconditioner: Kσ S = Mσ S Λ on the interior rows (Dirichlet at the surface),
  // Kσ = Σ_l (2/Δσ_l) Dᵀ W D, Mσ = Σ_l (Δσ_l/2) W (GLL-lumped, as in the stiffness quadrature).
  const int nr = nrow - 1;
  t->Sg.assign((size_t)nr * nr, 0.0);
  t->lam.assign(nr, 0.0);
  {
    std::vector<long double> Ks((size_t)nrow * nrow, 0.0L), Ms(nrow, 0.0L);
    for (int l = 0; l < Nz; ++l)
      for (int a = 0; a < Q; ++a) {
        Ms[l * P + a] += 0.5L * dsl[l] * L.w[a];
        for (int b = 0; b < Q; ++b) {
          long double s2 = 0.0L;
          for (int c = 0; c < Q; ++c) s2 += (long double)L.D[c * Q + a] * L.w[c] * L.D[c * Q + b];
          Ks[(size_t)(l * P + a) * nrow + l * P + b] += (2.0L / dsl[l]) * s2;
        }
      }
    std::vector<long double> Bm((size_t)nr * nr), ev, V;
    for (int i = 0; i < nr; ++i)
      for (int j = 0; j < nr; ++j) Bm[(size_t)i * nr + j] = Ks[(size_t)i * nrow + j] / std::sqrt(Ms[i] * Ms[j]);
    sym_eig(Bm, nr, ev, V);
    for (int k = 0; k < nr; ++k) t->lam[k] = (double)ev[k];
    for (int j = 0; j < nr; ++j)
      for (int k = 0; k < nr; ++k) t->Sg[(size_t)j * nr + k] = (double)(V[(size_t)j * nr + k] / std::sqrt(Ms[j]));
  }
  std::lock_guard<std::mutex> lk(g_ct_mu);
  auto ins = g_ct.emplace(key, std::shared_ptr<const ColumnTables>(t));
  *out = ins.first->second;
  return SEM_OK;
}

static int mesh_create_impl(const sem_params* pin, const double* x_edges_h, const double* h_h, sem_mesh** out,
                            size_t* footprint_only);

int sem_mesh_create(const sem_params* pin, const double* x_edges_h, const double* h_h, sem_mesh** out) {
  if (!out) return fail(SEM_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  return mesh_create_impl(pin, x_edges_h, h_h, out, nullptr);
}

int sem_mesh_footprint(const sem_params* p, const double* x_edges_h, const double* h_h, int64_t* bytes) {
  if (!bytes) return fail(SEM_ERR_INVALID_ARG, "bytes is NULL");
  size_t b = 0;
  sem_mesh* unused = nullptr;
  const int rc = mesh_create_impl(p, x_edges_h, h_h, &unused, &b);
  *bytes = (int64_t)b;
  return rc;
}

static int mesh_create_impl(const sem_params* pin, const double* x_edges_h, const double* h_h, sem_mesh** out,
                            size_t* footprint_only) {
  if (!pin || !x_edges_h || !h_h) return fail(SEM_ERR_INVALID_ARG, "NULL argument");
  sem_params p = *pin;
  const int Nx_in = p.Nx > 0 ? p.Nx : 0;
  if (p.P < 2 || p.P > SEM_MAX_P) return fail(SEM_ERR_INVALID_ARG, "P must be in [2, 12]");
  if (p.Nz < 1 || p.Nz > kMaxNz) return fail(SEM_ERR_INVALID_ARG, "Nz must be in [1, 16]");
  if (p.periodic ? p.Nx < 3 : p.Nx < 1) return fail(SEM_ERR_INVALID_ARG, "Nx too small (periodic needs >= 3)");
  if (p.Pf == 0) p.Pf = p.P;
  if (p.Pf < p.P || p.Pf > 3 * p.P) return fail(SEM_ERR_INVALID_ARG, "Pf must be in [P, 3P]");
  if (p.precision != SEM_PREC_FP64 && p.precision != SEM_PREC_MIXED)
    return fail(SEM_ERR_INVALID_ARG, "unknown precision");
  if (p.precond != SEM_PRECOND_SEPARABLE && p.precond != SEM_PRECOND_JACOBI)
    return fail(SEM_ERR_INVALID_ARG, "unknown preconditioner");
  if (p.relax_left < 0.0 || p.relax_right < 0.0 || p.relax_tau < 0.0 ||
      p.relax_left + p.relax_right > x_edges_h[Nx_in] - x_edges_h[0])
    return fail(SEM_ERR_INVALID_ARG, "relaxation zones must be non-negative and fit in the tank");
  if (p.tol <= 0.0) p.tol = 1e-13;
  if (p.max_iter <= 0) p.max_iter = 5000;
  const int P = p.P, Q = P + 1, Nx = p.Nx, Nz = p.Nz;
  const int ncol = p.periodic ? Nx * P : Nx * P + 1;
  const int nrow = Nz * P + 1;
  const long long n = (long long)ncol * nrow;
  for (int i = 0; i < Nx; ++i)
    if (!(x_edges_h[i + 1] > x_edges_h[i])) return fail(SEM_ERR_INVALID_ARG, "x_edges must increase");
  for (int i = 0; i < ncol; ++i)
    if (!(h_h[i] > 0.0) || !std::isfinite(h_h[i])) return fail(SEM_ERR_INVALID_ARG, "h must be positive");

  int dev = 0;
  CUDA_TRY(cudaGetDevice(&dev));
  int rc = ensure_device_tables(dev);
  if (rc) return rc;

  // ---- host tables --------------------------------------------------------------
  // Tables that depend only on (P, Nz, Pf, filter) come from a per-process cache (they are
  // built in long double, which is software-emulated on some hosts); the x-dependent ones
  // below are O(Nx) in double.
  std::shared_ptr<const ColumnTables> ct;
  rc = column_tables(p, &ct);
  if (rc) return rc;
  const Line& L = ct->L;
  const std::vector<double>& MD = ct->MD;
  const std::vector<double>& I = ct->I;
  const std::vector<double>& B = ct->B;
  const std::vector<double>& F = ct->F;
  const std::vector<double>& wrow = ct->wrow;
  const std::vector<double>& Aii = ct->Aii;
  const std::vector<double>& Z = ct->Z;
  const std::vector<double>& Sg = ct->Sg;
  const std::vector<double>& lam = ct->lam;
  const std::vector<double>& dsl = ct->dsl;
  const std::vector<double>& sig = ct->sig;
  const int Qf = p.Pf + 1, Pm = P - 1;
  std::vector<double> dxe(Nx), hx_loc((size_t)Nx * Q), se(Nx);
  for (int e = 0; e < Nx; ++e) { dxe[e] = x_edges_h[e + 1] - x_edges_h[e]; se[e] = 0.5 * dxe[e]; }
  for (int e = 0; e < Nx; ++e)
    for (int a = 0; a < Q; ++a) {
      double s = 0.0;
      for (int c = 0; c < Q; ++c) {
        int col = e * P + c; if (col >= ncol) col -= ncol;
        s = std::fma(L.D[a * Q + c], h_h[col], s);
      }
      hx_loc[(size_t)e * Q + a] = s * 2.0 / dxe[e];
    }
  // M' interface tridiagonal (Thomas factors; Sherman–Morrison closure when periodic)
  const int N = p.periodic ? Nx : Nx + 1;
  std::vector<double> th_e(N, 0.0), th_m(N, 0.0), th_cp(N, 0.0), th_z(N, 0.0);
  double th_vlast = 0.0, th_fac = 0.0;
  {
    const double S00 = ct->S00, S01 = ct->S01, S11 = ct->S11;
    std::vector<double> d(N, 0.0), e(N, 0.0);
    for (int j = 0; j < Nx; ++j) {
      const int jr = (j + 1) % N;
      d[j] += se[j] * S00;
      d[jr] += se[j] * S11;
      e[j] = se[j] * S01;            // coupling j ↔ j+1 (periodic: e[N−1] is the corner)
    }
    double gamma = 0.0, corner = 0.0;
    if (p.periodic) {
      corner = e[N - 1];
      gamma = -d[0];
      d[0] -= gamma;
      d[N - 1] -= corner * corner / gamma;
    }
    std::vector<double> m(N), cp(N, 0.0);
    for (int j = 0; j < N; ++j) {
      const double piv = j == 0 ? d[0] : d[j] - e[j - 1] * cp[j - 1];
      m[j] = 1.0 / piv;
      if (j < N - 1) cp[j] = e[j] * m[j];
    }
    th_e = e; th_m = m; th_cp = cp;
    if (p.periodic) {
      std::vector<double> u(N, 0.0), y(N);
      u[0] = gamma;
      u[N - 1] = corner;
      for (int j = 0; j < N; ++j) y[j] = (j == 0 ? u[0] : u[j] - e[j - 1] * y[j - 1]) * m[j];
      for (int j = N - 2; j >= 0; --j) y[j] -= cp[j] * y[j + 1];
      const double vl = corner / gamma;
      th_z = y;
      th_vlast = vl;
      th_fac = 1.0 / (1.0 + y[0] + vl * y[N - 1]);
    }
  }
  const int nr = nrow - 1;

  // ---- device allocation -------------------------------------------------------
  sem_mesh* m = new sem_mesh;
  m->p = p; m->device = dev; m->ncol = ncol; m->nrow = nrow; m->n = n; m->Pf = p.Pf; m->nif = N;
  const int chunk = chunk_width(P, Nz);
  cudaError_t ge = pcg_grid_size(P, Nz, nrow, Nx, chunk, p.precision == SEM_PREC_MIXED, &m->grid, &m->smem);
  if (ge != cudaSuccess) { delete m; return fail(SEM_ERR_CUDA, std::string("Krylov kernel occupancy: ") + cudaGetErrorString(ge)); }
  if (const char* lim = std::getenv("SEM_GRID_LIMIT")) {   // tuning/testing knob: cap the Krylov grid
    const int v = std::atoi(lim);
    if (v >= 1 && v < m->grid) m->grid = v;
  }

  Carve cv;
  const size_t nE = (size_t)Nx * nrow;
  // the arrays filled on the host come first: one copy uploads all of them ([0, up_end) of the block)
  const size_t o_cxz = cv.take<double>((size_t)Nx * Nz * 2), o_r2dx = cv.take<double>(Nx);
  const size_t o_h = cv.take<double>(ncol), o_hx = cv.take<double>((size_t)Nx * Q), o_dxe = cv.take<double>(Nx),
               o_dsl = cv.take<double>(Nz), o_sig = cv.take<double>(nrow);
  const size_t o_S32 = cv.take<float>((size_t)nr * nr), o_ST32 = cv.take<float>((size_t)nr * nr),
               o_lam = cv.take<double>(nr), o_xcol = cv.take<double>(ncol);
  // surface tables
  const size_t o_tD = cv.take<double>(Q * Q), o_tMD = cv.take<double>(Q * Q), o_tB = cv.take<double>((size_t)Q * Qf),
               o_tI = cv.take<double>((size_t)Qf * Q), o_tF = cv.take<double>(Q * Q), o_twr = cv.take<double>((size_t)nrow),
               o_tAii = cv.take<double>((size_t)Pm * Pm + 1), o_tZ = cv.take<double>((size_t)2 * Pm + 1),
               o_tse = cv.take<double>(Nx), o_te = cv.take<double>(N), o_tm = cv.take<double>(N),
               o_tcp = cv.take<double>(N), o_tz = cv.take<double>(N);
  const size_t up_end = cv.off;
  const size_t o_geo64 = cv.take<double>((size_t)Nx * Q * 4),
               o_geo32 = cv.take<float>((size_t)Nx * Q * 4), o_id64 = cv.take<double>(n), o_id32 = cv.take<float>(n),
               o_status = cv.take<int>(4), o_rec = cv.take<SolveRecord>(1), o_bar = cv.take<unsigned>(4),
               o_part = cv.take<double>((size_t)16 * m->grid);
  const size_t o_r64 = cv.take<double>(n), o_z64 = cv.take<double>(n), o_p64a = cv.take<double>(n),
               o_p64b = cv.take<double>(n), o_q64 = cv.take<double>(n), o_q64b = cv.take<double>(n),
               o_e64 = cv.take<double>(nE), o_e64b = cv.take<double>(nE);
  const size_t o_d32 = cv.take<float>(n), o_r32 = cv.take<float>(n), o_z32 = cv.take<float>(n),
               o_p32a = cv.take<float>(n), o_p32b = cv.take<float>(n), o_q32 = cv.take<float>(n),
               o_e32 = cv.take<float>(nE);
  const size_t o_Phi = cv.take<double>(n), o_qtmp = cv.take<double>(n), o_etmp = cv.take<double>(nE);
  const size_t o_r64b = cv.take<double>(n), o_r32b = cv.take<float>(n);
  const size_t o_s64b = cv.take<double>(n), o_s32b = cv.take<float>(n);
  const size_t o_uh64 = cv.take<double>((size_t)m->grid * nrow), o_uh32 = cv.take<float>((size_t)m->grid * nrow);
  const size_t nEl = (size_t)nr * Nx, nIf = (size_t)nr * N;
  const size_t o_schur = cv.take<double>(nEl * 3),
               o_A32 = cv.take<float>(nEl * Pm * Pm + 1), o_Z32 = cv.take<float>(nEl * 2 * Pm + 1),
               o_te32 = cv.take<float>(nIf), o_tm32 = cv.take<float>(nIf),
               o_tcp32 = cv.take<float>(nIf), o_tz32 = cv.take<float>(nIf),
               o_tvl32 = cv.take<float>(nr), o_tfac32 = cv.take<float>(nr),
               o_gL32 = cv.take<float>(nEl), o_gR32 = cv.take<float>(nEl), o_zb32 = cv.take<float>(nIf),
               o_rh32 = cv.take<float>((size_t)ncol * nr);
  const size_t o_wave = cv.take<double>(4 * kMaxWaveComp);
  const bool zones = p.relax_left > 0.0 || p.relax_right > 0.0;
  const size_t o_wA = cv.take<double>(zones ? 4 * kMaxWaveComp : 0), o_wEP = cv.take<double>(zones ? 2 * ncol : 0);
  const size_t o_wt = cv.take<double>(ncol), o_etax = cv.take<double>(ncol), o_phisx = cv.take<double>(ncol),
               o_R = cv.take<double>((size_t)2 * Nx * Q), o_scr = cv.take<double>((size_t)4 * Nx + 2 * (N + 1)),
               o_ke = cv.take<double>(ncol), o_kp = cv.take<double>(ncol), o_ae = cv.take<double>(ncol),
               o_ap = cv.take<double>(ncol), o_se = cv.take<double>(ncol), o_sp = cv.take<double>(ncol),
               o_etad = cv.take<double>(ncol), o_phisd = cv.take<double>(ncol),
               o_s1e = cv.take<double>(ncol), o_s1p = cv.take<double>(ncol),
               o_P1 = cv.take<double>(n), o_P2 = cv.take<double>(n), o_P3 = cv.take<double>(n),
               o_D32 = cv.take<double>(n);
  const size_t o_gglob = cv.take<double>((size_t)3 * Nx * Nz * Q * Q);
  const size_t o_inst = cv.take<Instance>(1), o_ctai = cv.take<int>((size_t)m->grid), o_sbar = cv.take<unsigned>(4);
  const size_t total = cv.off + 256;
  if (footprint_only) {
    *footprint_only = total;
    delete m;
    return SEM_OK;
  }
  m->pool_bytes = total;
  cudaError_t ae = dev_alloc(dev, total, reinterpret_cast<void**>(&m->pool));
  if (ae != cudaSuccess) { delete m; return fail(SEM_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(ae)); }
  auto D_ = [&](size_t o) { return reinterpret_cast<double*>(m->pool + o); };
  auto F_ = [&](size_t o) { return reinterpret_cast<float*>(m->pool + o); };
  int code = SEM_OK;
  // host image of [0, up_end): the arrays are written into it and go up in one copy (zero padding
  // between them); the rest of the block is zeroed on the device
  std::vector<unsigned char> stage(up_end, 0);
  auto up = [&](size_t o, const std::vector<double>& v) {
    if (!v.empty()) std::memcpy(stage.data() + o, v.data(), v.size() * sizeof(double));
  };
  {
    cudaError_t e = cudaMemset(m->pool + up_end, 0, total - up_end);
    if (e != cudaSuccess) code = fail(SEM_ERR_CUDA, std::string("memset: ") + cudaGetErrorString(e));
  }
  up(o_h, std::vector<double>(h_h, h_h + ncol));
  up(o_hx, hx_loc); up(o_dxe, dxe); up(o_dsl, dsl); up(o_sig, sig);
  {
    std::vector<double> cxz((size_t)Nx * Nz * 2);
    for (int e = 0; e < Nx; ++e)
      for (int l = 0; l < Nz; ++l) {
        cxz[((size_t)e * Nz + l) * 2] = dsl[l] / dxe[e];
        cxz[((size_t)e * Nz + l) * 2 + 1] = dxe[e] / dsl[l];
      }
    up(o_cxz, cxz);
    std::vector<double> r2dx(Nx);
    for (int e = 0; e < Nx; ++e) r2dx[e] = 2.0 / dxe[e];
    up(o_r2dx, r2dx);
  }
  up(o_tD, L.D); up(o_tMD, MD); up(o_tB, B); up(o_tI, I); up(o_tF, F); up(o_twr, wrow);
  up(o_tAii, Aii); up(o_tZ, Z); up(o_tse, se); up(o_te, th_e); up(o_tm, th_m); up(o_tcp, th_cp); up(o_tz, th_z);
  up(o_lam, lam);
  {
    std::vector<double> xc(ncol);
    for (int c = 0; c < ncol; ++c) {
      const int e = std::min(c / P, Nx - 1), a = c - e * P;
      xc[c] = x_edges_h[e] + 0.5 * (L.r[a] + 1.0) * dxe[e];
    }
    up(o_xcol, xc);
    m->xcol_h = xc;
  }
  {
    std::vector<float> S32(Sg.begin(), Sg.end()), ST32(S32.size());
    for (int j = 0; j < nr; ++j)
      for (int k = 0; k < nr; ++k) ST32[(size_t)k * nr + j] = S32[(size_t)j * nr + k];
    std::memcpy(stage.data() + o_S32, S32.data(), S32.size() * sizeof(float));
    std::memcpy(stage.data() + o_ST32, ST32.data(), ST32.size() * sizeof(float));
  }
  if (code == SEM_OK) {
    cudaError_t e = cudaMemcpy(m->pool, stage.data(), up_end, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) code = fail(SEM_ERR_CUDA, std::string("upload: ") + cudaGetErrorString(e));
  }
  if (code != SEM_OK) { dev_free(dev, m->pool); delete m; return code; }

  DevGeom& g = m->g;
  g.P = P; g.Nx = Nx; g.Nz = Nz; g.ncol = ncol; g.nrow = nrow; g.periodic = p.periodic ? 1 : 0; g.chunk = chunk;
  g.h = D_(o_h); g.hx_loc = D_(o_hx); g.dxe = D_(o_dxe); g.dsl = D_(o_dsl); g.sig = D_(o_sig); g.cxz = D_(o_cxz);
  g.r2dx = D_(o_r2dx);
  g.geo64 = D_(o_geo64); g.geo32 = F_(o_geo32); g.invdiag64 = D_(o_id64); g.invdiag32 = F_(o_id32);
  g.status = reinterpret_cast<int*>(m->pool + o_status);
  g.gglob = D_(o_gglob);
  g.dv_nrow = FastDiv::make(nrow);
  g.dv_nr = FastDiv::make(nrow - 1);
  g.dv_colsz = FastDiv::make(Q * nrow);
  g.dv_elsz = FastDiv::make(Nz * Q * Q);
  g.dv_qn = FastDiv::make(Q * (nrow - 1));
  g.bar_timeout_ns = kBarrierTimeoutNs;
  g.drop_rank = -1;
  g.trace = nullptr;
#ifdef SEM_TRACE
  if (cudaMalloc(reinterpret_cast<void**>(&g.trace), sizeof(unsigned long long) * (1 + 2 * kTraceMax)) != cudaSuccess ||
      cudaMemset(g.trace, 0, sizeof(unsigned long long)) != cudaSuccess)
    g.trace = nullptr;
#endif
  m->rec = reinterpret_cast<SolveRecord*>(m->pool + o_rec);

  PcgArgs& a = m->pa;
  a.r64 = D_(o_r64); a.z64 = D_(o_z64); a.p64a = D_(o_p64a); a.p64b = D_(o_p64b);
  a.q64 = D_(o_q64); a.q64b = D_(o_q64b); a.edge64 = D_(o_e64); a.edge64b = D_(o_e64b);
  a.d32 = F_(o_d32); a.r32 = F_(o_r32); a.z32 = F_(o_z32); a.p32a = F_(o_p32a); a.p32b = F_(o_p32b);
  a.q32 = F_(o_q32); a.edge32 = F_(o_e32);
  a.part = D_(o_part); a.part_stride = m->grid;
  a.bar = reinterpret_cast<unsigned int*>(m->pool + o_bar);
  a.rec = m->rec;
  a.tol = p.tol; a.inner_rtol = 1e-6; a.max_iter = p.max_iter; a.mixed = p.precision == SEM_PREC_MIXED;
  a.r64b = D_(o_r64b); a.r32b = F_(o_r32b);
  a.s64b = D_(o_s64b); a.s32b = F_(o_s32b);
  a.uh64 = D_(o_uh64); a.uh32 = F_(o_uh32);
  a.precond = p.precond == SEM_PRECOND_JACOBI ? PREC_JACOBI : PREC_SEPARABLE;
  PrecSetup& ps = m->ps;
  ps.nr = nr; ps.nif = N; ps.lam = D_(o_lam); ps.schur = D_(o_schur);
  ps.Aii32 = F_(o_A32); ps.Z32 = F_(o_Z32); ps.te32 = F_(o_te32); ps.tm32 = F_(o_tm32); ps.tcp32 = F_(o_tcp32);
  ps.tz32 = F_(o_tz32); ps.tvl32 = F_(o_tvl32); ps.tfac32 = F_(o_tfac32);
  ps.v32 = PrecView<float>{nr, N, F_(o_S32), F_(o_ST32), ps.Aii32, ps.Z32, ps.te32, ps.tm32, ps.tcp32, ps.tz32, ps.tvl32,
                           ps.tfac32, F_(o_gL32), F_(o_gR32), F_(o_zb32), F_(o_rh32)};
  a.pv32 = ps.v32;

  m->Phi = D_(o_Phi); m->qtmp = D_(o_qtmp); m->edgetmp = D_(o_etmp);
  m->wt = D_(o_wt); m->etax = D_(o_etax); m->phisx = D_(o_phisx); m->R = D_(o_R); m->scr = D_(o_scr);
  m->ke = D_(o_ke); m->kp = D_(o_kp); m->ae = D_(o_ae); m->ap = D_(o_ap); m->se = D_(o_se); m->sp = D_(o_sp);
  m->eta_dev = D_(o_etad); m->phis_dev = D_(o_phisd);
  m->s1e = D_(o_s1e); m->s1p = D_(o_s1p);
  m->Phi1 = D_(o_P1); m->Phi2 = D_(o_P2); m->Phi3 = D_(o_P3); m->D32 = D_(o_D32);
  m->inst_d = reinterpret_cast<Instance*>(m->pool + o_inst);
  m->cta_inst_d = reinterpret_cast<int*>(m->pool + o_ctai);
  m->stage_bars = reinterpret_cast<unsigned int*>(m->pool + o_sbar);

  SurfTables& t = m->st;
  t.P = P; t.Pf = p.Pf; t.Nx = Nx; t.Nz = Nz; t.ncol = ncol; t.nrow = nrow; t.periodic = g.periodic; t.g = p.g;
  t.D = D_(o_tD); t.MD = D_(o_tMD); t.B = D_(o_tB); t.I = D_(o_tI); t.F = D_(o_tF); t.wrow = D_(o_twr);
  t.Aii = D_(o_tAii); t.Z = D_(o_tZ); t.se = D_(o_tse); t.dsl = g.dsl; t.h = g.h;
  t.th_e = D_(o_te); t.th_m = D_(o_tm); t.th_cp = D_(o_tcp); t.th_z = D_(o_tz);
  t.th_vlast = th_vlast; t.th_fac = th_fac; t.nif = N; t.filter_on = (p.filter_ic >= 0 && p.filter_ic < P) ? 1 : 0;
  t.xcol = D_(o_xcol); t.x0 = x_edges_h[0]; t.x1 = x_edges_h[Nx];
  t.relax_left = p.relax_left; t.relax_right = p.relax_right; t.ncomp = 0; t.wave = D_(o_wave);
  t.nzl = 0; t.wkx = nullptr;
  t.wA = zones ? D_(o_wA) : nullptr;
  t.wEP = zones ? D_(o_wEP) : nullptr;
  // the fused RK stage runs this mesh with one team of CTAs (at most its Krylov grid)
  {
    const char* fz = std::getenv("SEM_FUSED_STAGE");
    m->fused = !(fz && fz[0] == '0') && p.precond == SEM_PRECOND_SEPARABLE;
    m->stage_smem = stage_smem_bytes(P, nrow, Nz, chunk);
    int per_sm = 0, sms = 0;
    cudaError_t e = stage_occupancy(P, p.precision == SEM_PREC_MIXED, 0, m->stage_smem, &per_sm);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess || per_sm < 1) {
      dev_free(dev, m->pool);
      delete m;
      return fail(SEM_ERR_CUDA, "fused stage kernel does not fit on this device");
    }
    m->stage_team = std::min(m->grid, per_sm * sms);
    m->stage_smem_batch = m->stage_smem;
    m->own_chunk = chunk;
    // The own launch: all of a CTA's element columns in one pass (instead of passes of `chunk`,
    // each paying its own round trips to L2 and CTA barriers), and room for the solve's
    // geometric factors (3 per element-local node) after the apply's buffers, each if the
    // launch keeps its occupancy.
    {
      const int Qd = P + 1;
      const int ne_max = (Nx + m->stage_team - 1) / m->stage_team;
      const int mixed = p.precision == SEM_PREC_MIXED;
      int per2 = 0;
      const size_t smem_wide = stage_smem_bytes(P, nrow, Nz, ne_max);
      if (ne_max > chunk && smem_wide <= (size_t)kMaxDynSmem &&
          stage_occupancy(P, mixed, 0, smem_wide, &per2) == cudaSuccess && per2 >= per_sm) {
        m->own_chunk = ne_max;
        m->stage_smem = smem_wide;
      }
      const size_t need = (size_t)3 * ne_max * Nz * Qd * Qd;
      const size_t smem2 = m->stage_smem + need * sizeof(double);
      if (smem2 <= (size_t)kMaxDynSmem &&
          stage_occupancy(P, mixed, 0, smem2, &per2) == cudaSuccess && per2 >= per_sm) {
        m->stage_smem = smem2;
        m->gcache = (int)need;
      }
    }
    std::vector<int> zeros(m->grid, 0);
    cudaError_t e2 = cudaMemcpy(m->cta_inst_d, zeros.data(), sizeof(int) * m->grid, cudaMemcpyHostToDevice);
    if (e2 != cudaSuccess) {
      dev_free(dev, m->pool);
      delete m;
      return fail(SEM_ERR_CUDA, std::string("upload: ") + cudaGetErrorString(e2));
    }
  }
  *out = m;
  return SEM_OK;
}

void sem_mesh_destroy(sem_mesh* m) {
  if (!m) return;
  DeviceGuard dg(m->device);
  for (auto& pr : m->events) { cudaEventDestroy(pr.first); cudaEventDestroy(pr.second); }
  for (auto e : m->spare) cudaEventDestroy(e);
  cudaDeviceSynchronize();   // no work of this mesh may still run when its memory is reused
  if (m->wkx) dev_free(m->device, m->wkx);
  dev_free(m->device, m->pool);
  delete m;
}

int sem_mesh_info(const sem_mesh* m, sem_info* info) {
  if (!m || !info) return fail(SEM_ERR_INVALID_ARG, "NULL argument");
  info->n_nodes = m->n;
  info->n_unknowns = (int64_t)m->ncol * (m->nrow - 1);
  info->ncol = m->ncol; info->nrow = m->nrow;
  info->n_elements = m->p.Nx * m->p.Nz;
  info->P = m->p.P; info->Pf = m->Pf; info->Nx = m->p.Nx; info->Nz = m->p.Nz;
  info->periodic = m->p.periodic; info->precision = m->p.precision;
  info->grid_ctas = m->grid;
  info->stage_ctas = m->stage_team;
  info->device_bytes = (int64_t)m->pool_bytes;
  return SEM_OK;
}

int sem_mesh_l2g(sem_mesh* m, int32_t* l2g_d, void* stream) {
  if (!m || !l2g_d) return fail(SEM_ERR_INVALID_ARG, "NULL argument");
  DeviceGuard dg(m->device);
  CUDA_TRY(launch_l2g(m->g, l2g_d, (cudaStream_t)stream));
  return SEM_OK;
}

int sem_update_geometry(sem_mesh* m, const double* eta_d, void* stream) {
  if (!m || !eta_d) return fail(SEM_ERR_INVALID_ARG, "NULL argument");
  DeviceGuard dg(m->device);
  return do_geometry(m, eta_d, (cudaStream_t)stream);
}

int sem_laplace_apply(sem_mesh* m, const double* x_d, double* y_d, void* stream) {
  if (!m || !x_d || !y_d || x_d == y_d) return fail(SEM_ERR_INVALID_ARG, "bad pointer");
  DeviceGuard dg(m->device);
  const char* k = std::getenv("SEM_APPLY_KERNEL");   // "column": the element-column kernel, else tiled
  cudaError_t e = cudaErrorInvalidValue;
  if (!(k && std::strcmp(k, "column") == 0)) e = launch_apply_tile(0, m->g, x_d, y_d, (cudaStream_t)stream);
  // the element-column kernel when asked for, or when the FP64 tile does not fit in shared memory
  // (largest orders with many layers); the tile launcher checks that before launching anything
  if (e == cudaErrorInvalidValue) e = launch_apply(m->g, x_d, y_d, m->qtmp, m->edgetmp, (cudaStream_t)stream);
  if (e != cudaSuccess) return fail(SEM_ERR_CUDA, std::string("apply: ") + cudaGetErrorString(e));
  return SEM_OK;
}

int sem_laplace_apply_f32(const sem_mesh* m, const float* x_d, float* y_d, void* stream) {
  if (!m || !x_d || !y_d || x_d == y_d) return fail(SEM_ERR_INVALID_ARG, "bad pointer");
  DeviceGuard dg(m->device);
  // "tc": the tensor-core kernel for orders 4..7 (measured slower than the CUDA-core kernel on
  // GB300; kept for comparison), else the CUDA-core kernel
  const char* k = std::getenv("SEM_APPLY_F32");
  CUDA_TRY(launch_apply_tile(k && std::strcmp(k, "tc") == 0 ? 3 : 1, m->g, x_d, y_d, (cudaStream_t)stream));
  return SEM_OK;
}

int sem_laplace_apply_noalloc(const sem_mesh* m, const double* x_d, double* y_d, void* stream) {
  if (!m || !x_d || !y_d || x_d == y_d) return fail(SEM_ERR_INVALID_ARG, "bad pointer");
  if ((size_t)m->p.Nx * (size_t)m->nrow > kNoAllocEdgeMax)
    return fail(SEM_ERR_INVALID_ARG, "sem_laplace_apply_noalloc: Nx*Nrow = " +
                                         std::to_string((size_t)m->p.Nx * m->nrow) + " exceeds the static scratch of " +
                                         std::to_string(kNoAllocEdgeMax) + " values");
  DeviceGuard dg(m->device);
  CUDA_TRY(launch_apply_noalloc(m->g, x_d, y_d, (cudaStream_t)stream));
  return SEM_OK;
}

int sem_laplace_solve(sem_mesh* m, const double* phis_d, double* Phi_d, sem_solve_stats* st, void* stream) {
  if (!m || !phis_d || !Phi_d) return fail(SEM_ERR_INVALID_ARG, "NULL argument");
  DeviceGuard dg(m->device);
  cudaStream_t s = (cudaStream_t)stream;
  int rc = do_solve(m, phis_d, Phi_d, s);
  if (rc) return rc;
  if (st) {
    SolveRecord r{};
    CUDA_TRY(cudaMemcpyAsync(&r, m->rec, sizeof(r), cudaMemcpyDeviceToHost, s));
    rc = read_status(m, s);
    st->iterations = r.iterations;
    st->refinements = r.refinements;
    st->rel_residual = r.rel_residual;
    return rc;
  }
  return SEM_OK;
}

int sem_recover_gradient(sem_mesh* m, const double* Phi_d, const double* eta_d, const double* phis_d,
                         double* w_surf_d, double* etax_d, double* phisx_d, void* stream) {
  if (!m || !Phi_d || !eta_d || !phis_d || !w_surf_d || !etax_d || !phisx_d)
    return fail(SEM_ERR_INVALID_ARG, "NULL argument");
  DeviceGuard dg(m->device);
  cudaStream_t s = (cudaStream_t)stream;
  CUDA_TRY(launch_wsurf(m->st, Phi_d, eta_d, w_surf_d, s));
  CUDA_TRY(launch_sx(m->st, eta_d, phis_d, m->R, s));
  CUDA_TRY(launch_mass1d(m->st, m->R, 2, etax_d, phisx_d, m->scr, s));
  return SEM_OK;
}

int sem_zakharov_rhs(sem_mesh* m, const double* eta_d, const double* phis_d, double t, double* deta_d,
                     double* dphis_d, void* stream) {
  if (!m || !eta_d || !phis_d || !deta_d || !dphis_d) return fail(SEM_ERR_INVALID_ARG, "NULL argument");
  if (has_zones(m) && !(m->p.relax_tau > 0.0))
    return fail(SEM_ERR_INVALID_ARG, "relaxation zones need relax_tau > 0 outside sem_rk4_step");
  DeviceGuard dg(m->device);
  return do_rhs(m, eta_d, phis_d, t, m->p.relax_tau, deta_d, dphis_d, (cudaStream_t)stream);
}

int sem_set_wave_input(sem_mesh* m, int ncomp, const double* amp_h, const double* omega_h,
                       const double* k_h, const double* phase_h) {
  if (!m || ncomp < 0 || ncomp > kMaxWaveComp) return fail(SEM_ERR_INVALID_ARG, "ncomp must be in [0, 4096]");
  if (ncomp > 0 && (!amp_h || !omega_h || !k_h || !phase_h)) return fail(SEM_ERR_INVALID_ARG, "NULL argument");
  for (int i = 0; i < ncomp; ++i)
    if (!(omega_h[i] > 0.0)) return fail(SEM_ERR_INVALID_ARG, "wave frequencies must be positive");
  DeviceGuard dg(m->device);
  double* w = const_cast<double*>(m->st.wave);
  const double* src[4] = {amp_h, omega_h, k_h, phase_h};
  for (int q = 0; q < 4 && ncomp > 0; ++q)
    CUDA_TRY(cudaMemcpy(w + (size_t)q * ncomp, src[q], sizeof(double) * ncomp, cudaMemcpyHostToDevice));
  m->st.ncomp = ncomp;
  // cos, sin of k x at the left-zone columns (the first nzl columns), for the fused stage's
  // angle-addition evaluation; left out when there is no left zone or the table would pass 512 MB
  CUDA_TRY(cudaDeviceSynchronize());
  if (m->wkx) { dev_free(m->device, m->wkx); m->wkx = nullptr; }
  m->st.wkx = nullptr;
  m->st.nzl = 0;
  int nzl = 0;
  if (m->p.relax_left > 0.0)
    while (nzl < m->ncol && m->xcol_h[nzl] < m->st.x0 + m->p.relax_left) ++nzl;
  const size_t entries = (size_t)nzl * (size_t)ncomp * 2;
  if (nzl > 0 && ncomp > 0 && m->st.wA && entries * sizeof(double) <= (size_t(512) << 20)) {
    std::vector<double> tab(entries);
    for (int c = 0; c < nzl; ++c)
      for (int i = 0; i < ncomp; ++i) {
        const double kx = k_h[i] * m->xcol_h[c];
        tab[((size_t)c * ncomp + i) * 2] = std::cos(kx);
        tab[((size_t)c * ncomp + i) * 2 + 1] = std::sin(kx);
      }
    void* d = nullptr;
    cudaError_t e = dev_alloc(m->device, entries * sizeof(double), &d);
    if (e != cudaSuccess) return fail(SEM_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    m->wkx = static_cast<double*>(d);
    CUDA_TRY(cudaMemcpy(m->wkx, tab.data(), entries * sizeof(double), cudaMemcpyHostToDevice));
    m->st.wkx = m->wkx;
    m->st.nzl = nzl;
  }
  return SEM_OK;
}

int sem_apply_filter(sem_mesh* m, double* q_d, void* stream) {
  if (!m || !q_d) return fail(SEM_ERR_INVALID_ARG, "NULL argument");
  DeviceGuard dg(m->device);
  CUDA_TRY(launch_filter(m->st, q_d, nullptr, (cudaStream_t)stream));
  return SEM_OK;
}

int sem_rk4_step(sem_mesh* m, double* eta_d, double* phis_d, double* t, double dt, int nsteps, void* stream) {
  if (!m || !eta_d || !phis_d || nsteps < 0 || !(dt > 0.0)) return fail(SEM_ERR_INVALID_ARG, "bad argument");
  DeviceGuard dg(m->device);
  cudaStream_t s = (cudaStream_t)stream;
  int rc = do_rk4(m, eta_d, phis_d, t ? *t : 0.0, dt, nsteps, s);
  if (rc) return rc;
  rc = read_status(m, s);
  if (t) *t += nsteps * dt;
  return rc;
}

int sem_rk4_step_host(sem_mesh* m, double* eta_h, double* phis_h, double* t, double dt, int nsteps,
                      void* stream) {
  if (!m || !eta_h || !phis_h || nsteps < 0 || !(dt > 0.0)) return fail(SEM_ERR_INVALID_ARG, "bad argument");
  DeviceGuard dg(m->device);
  cudaStream_t s = (cudaStream_t)stream;
  const size_t bytes = sizeof(double) * m->ncol;
  CUDA_TRY(cudaMemcpyAsync(m->eta_dev, eta_h, bytes, cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(m->phis_dev, phis_h, bytes, cudaMemcpyHostToDevice, s));
  int rc = do_rk4(m, m->eta_dev, m->phis_dev, t ? *t : 0.0, dt, nsteps, s);
  if (rc) return rc;
  CUDA_TRY(cudaMemcpyAsync(eta_h, m->eta_dev, bytes, cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaMemcpyAsync(phis_h, m->phis_dev, bytes, cudaMemcpyDeviceToHost, s));
  rc = read_status(m, s);
  if (t) *t += nsteps * dt;
  return rc;
}

// Cost of a team's barriers and cross-CTA round trips per stage, in element-local nodes of work
// (team sizing of the cooperative plan).
constexpr double kTeamSyncNodes = 256.0;
// Batch planning parameters (sem_set_batch_tuning; the defaults are the untuned rules).
static std::mutex g_tune_mu;
static sem_batch_tuning g_tune{0.5, 16, 8, -1};

static sem_batch_tuning batch_tuning() {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  return g_tune;
}
// Dynamic shared memory per CTA up to which batch members widen their passes (two CTAs per SM,
// or one).
constexpr size_t kBatchSmemWide = 88 * 1024, kBatchSmemNarrow = 176 * 1024;
// Largest thread-block cluster (the non-portable limit of this architecture).
constexpr int kMaxCluster = 16;

int sem_set_batch_tuning(const sem_batch_tuning* t) {
  sem_batch_tuning v{0.5, 16, 8, -1};
  if (t) {
    if (!(t->cluster_share > 0.0) || t->cluster_share > 64.0 || t->max_cluster < 1 || t->max_cluster > kMaxCluster ||
        (t->max_cluster & (t->max_cluster - 1)) != 0 || t->narrow_max < 0 || t->plan < -1 || t->plan > 1)
      return fail(SEM_ERR_INVALID_ARG, "batch tuning out of range");
    v = *t;
  }
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune = v;
  return SEM_OK;
}

int sem_get_batch_tuning(sem_batch_tuning* t) {
  if (!t) return fail(SEM_ERR_INVALID_ARG, "NULL argument");
  *t = batch_tuning();
  return SEM_OK;
}

int sem_set_apply_tile_width(int P, int Nz, int E) {
  if (P < 2 || P > kMaxP || Nz < 1 || Nz > kMaxNz || E < 0 || E > 16)
    return fail(SEM_ERR_INVALID_ARG, "tile width out of range");
  set_apply_tile_width(P, Nz, E);
  return SEM_OK;
}

}  // extern "C"

namespace {

int batch_wide(size_t group_size) {
  const char* wenv = std::getenv("SEM_BATCH_WIDE");
  return wenv ? (std::atoi(wenv) != 0) : (group_size > (size_t)batch_tuning().narrow_max ? 1 : 0);
}

int batch_limit(const sem_mesh* m) {   // ≤ grid: the halo and reduction buffers are sized by it
  return std::max(1, std::min(m->grid, (m->p.Nx + m->g.chunk - 1) / m->g.chunk));
}

// Each member's CTAs take their element columns in as few passes as the launch's shared memory
// allows: a budget per CTA that keeps the build's CTAs per SM.  Returns the launch's dynamic
// shared memory.
size_t widen_passes(BatchLaunch& L, sem_mesh* const* meshes, size_t smem) {
  const size_t budget = L.wide ? kBatchSmemWide : kBatchSmemNarrow;
  size_t smem_l = smem;
  L.chunk.clear();
  for (size_t k = 0; k < L.members.size(); ++k) {
    const sem_mesh* m = meshes[L.members[k]];
    const int ne = (m->p.Nx + L.nteam[k] - 1) / L.nteam[k];
    int E = m->g.chunk;
    while (E < ne && stage_smem_bytes(m->p.P, m->nrow, m->p.Nz, E + 1) <= budget) ++E;
    L.chunk.push_back(E);
    smem_l = std::max(smem_l, stage_smem_bytes(m->p.P, m->nrow, m->p.Nz, E));
  }
  return smem_l;
}

// Cooperative plan: instances grouped by (order, precision), each group split into launches of at
// most the co-resident CTA count; a launch lasts as long as its slowest team, so the CTAs go one at
// a time to the team whose estimated stage time is the largest, while that lowers it (the time of a
// team of c CTAs is taken as w/c element-local nodes per CTA, plus kTeamSyncNodes when c > 1).
int plan_cooperative(sem_batch* b, sem_mesh* const* meshes, int count, int sms) {
  std::vector<std::pair<std::pair<int, int>, std::vector<int>>> groups;
  for (int i = 0; i < count; ++i) {
    const std::pair<int, int> key(meshes[i]->p.P, meshes[i]->p.precision == SEM_PREC_MIXED ? 1 : 0);
    auto it = std::find_if(groups.begin(), groups.end(), [&](const auto& g) { return g.first == key; });
    if (it == groups.end()) groups.push_back({key, {i}});
    else it->second.push_back(i);
  }
  for (auto& grp : groups) {
    size_t smem = 0;
    for (int i : grp.second) smem = std::max(smem, meshes[i]->stage_smem_batch);
    int per_sm = 0;
    // Build of the stage kernel: two CTAs per SM (128 registers) for groups of many instances,
    // where more co-resident teams pay; one CTA per SM with the full register file (the
    // single-mesh build, faster per CTA) for a few instances.  SEM_BATCH_WIDE=0/1 forces either.
    const int wide = batch_wide(grp.second.size());
    cudaError_t e = stage_occupancy(grp.first.first, grp.first.second, wide, smem, &per_sm);
    if (e != cudaSuccess || per_sm < 1) return fail(SEM_ERR_CUDA, "fused stage kernel does not fit");
    const int cap = per_sm * sms;
    for (size_t first = 0; first < grp.second.size(); first += cap) {
      BatchLaunch L;
      L.P = grp.first.first;
      L.mixed = grp.first.second;
      L.wide = wide;
      const size_t last = std::min(grp.second.size(), first + (size_t)cap);
      L.members.assign(grp.second.begin() + first, grp.second.begin() + last);
      std::vector<double> w;
      for (int i : L.members) {
        const sem_mesh* m = meshes[i];
        w.push_back((double)m->p.Nx * m->p.Nz * (m->p.P + 1) * (m->p.P + 1));
      }
      std::vector<int> c(L.members.size(), 1), limit(L.members.size());
      for (size_t k = 0; k < L.members.size(); ++k) limit[k] = batch_limit(meshes[L.members[k]]);
      auto est = [&](size_t k, int ck) { return w[k] / ck + (ck > 1 ? kTeamSyncNodes : 0.0); };
      {
        std::priority_queue<std::pair<double, size_t>> pq;
        for (size_t k = 0; k < c.size(); ++k) pq.push({est(k, 1), k});
        int used = (int)c.size();
        while (used < cap && !pq.empty()) {
          const size_t k = pq.top().second;
          pq.pop();
          if (c[k] >= limit[k] || est(k, c[k] + 1) >= est(k, c[k])) continue;   // this team is done
          ++c[k];
          ++used;
          pq.push({est(k, c[k]), k});
        }
      }
      int acc = 0;
      for (size_t k = 0; k < c.size(); ++k) { L.team0.push_back(acc); L.nteam.push_back(c[k]); acc += c[k]; }
      L.grid = acc;
      size_t smem_l = widen_passes(L, meshes, smem);
      int per2 = 0;
      if (smem_l > smem && (stage_occupancy(L.P, L.mixed, wide, smem_l, &per2) != cudaSuccess || per2 < per_sm)) {
        for (size_t k = 0; k < L.members.size(); ++k) L.chunk[k] = meshes[L.members[k]]->g.chunk;
        smem_l = smem;
      }
      L.smem = smem_l;
      b->launches.push_back(std::move(L));
    }
  }
  return SEM_OK;
}

// Cluster plan: each member's team is one thread-block cluster, so no CTA waits on a CTA outside
// its cluster; the launches need no co-residency, the hardware starts clusters as CTA slots free
// up, and the launches of all groups run at the same time on streams of their own.  A step then
// lasts about the larger of the total work per CTA slot and the longest team's time, so a member's
// team is the smallest power of two c ≤ 16 (and ≤ its buffer limit) whose work per CTA is at most
// half the total work per CTA slot (work: element-local nodes × the apply's flops per node).
// Members are grouped by (order, precision, c), the largest first within a launch.  Returns
// false (and builds nothing) when some group's cluster does not fit on the device.
double member_work(const sem_mesh* m) {
  const int Q = m->p.P + 1;
  return (double)m->p.Nx * m->p.Nz * Q * Q * (8.0 * Q + 7.0);
}

// Estimated step time of each plan, in units of work per CTA: the cluster plan's launches share the
// GPU, so it takes about the larger of the total work per CTA slot and its longest team; the
// cooperative plan's launches run one after another, each as long as its slowest team.
double estimate_clusters(const sem_batch* b, double slots) {
  double total = 0.0, longest = 0.0;
  for (const auto& L : b->cl_launches)
    for (size_t k = 0; k < L.members.size(); ++k) {
      const double w = member_work(b->meshes[L.members[k]]);
      total += w;
      longest = std::max(longest, w / L.nteam[k]);
    }
  return std::max(total / slots, longest);
}

double estimate_cooperative(const sem_batch* b) {
  double t = 0.0;
  for (const auto& L : b->launches) {
    double worst = 0.0;
    for (size_t k = 0; k < L.members.size(); ++k)
      worst = std::max(worst, member_work(b->meshes[L.members[k]]) / L.nteam[k]);
    t += worst;
  }
  return t;
}

bool plan_clusters(sem_batch* b, sem_mesh* const* meshes, int count, int sms) {
  std::vector<double> w(count);
  double total = 0.0;
  for (int i = 0; i < count; ++i) {
    w[i] = member_work(meshes[i]);
    total += w[i];
  }
  const sem_batch_tuning tune = batch_tuning();
  const double slots = 2.0 * sms;
  const double per_cta = tune.cluster_share * total / slots;
  std::vector<std::pair<std::array<int, 3>, std::vector<int>>> groups;
  for (int i = 0; i < count; ++i) {
    const int cmax = std::min(tune.max_cluster, batch_limit(meshes[i]));
    const double want = per_cta > 0.0 ? w[i] / per_cta : 1.0;
    int c = 1;
    while (c < want && 2 * c <= cmax) c *= 2;
    const std::array<int, 3> key{meshes[i]->p.P, meshes[i]->p.precision == SEM_PREC_MIXED ? 1 : 0, c};
    auto it = std::find_if(groups.begin(), groups.end(), [&](const auto& g) { return g.first == key; });
    if (it == groups.end()) groups.push_back({key, {i}});
    else it->second.push_back(i);
  }
  std::vector<BatchLaunch> out;
  for (auto& grp : groups) {
    BatchLaunch L;
    L.P = grp.first[0];
    L.mixed = grp.first[1];
    L.csize = grp.first[2];
    L.wide = batch_wide(grp.second.size());
    L.members = grp.second;
    std::stable_sort(L.members.begin(), L.members.end(), [&](int a, int c) { return w[a] > w[c]; });
    size_t smem = 0;
    for (int i : L.members) smem = std::max(smem, meshes[i]->stage_smem_batch);
    for (size_t k = 0; k < L.members.size(); ++k) {
      L.team0.push_back((int)k * L.csize);
      L.nteam.push_back(L.csize);
    }
    L.grid = (int)L.members.size() * L.csize;
    int fit = 0;
    if (cluster_fit(L.P, L.mixed, L.wide, L.csize, smem, &fit) != cudaSuccess || fit < 1) {
      cudaGetLastError();
      return false;
    }
    size_t smem_l = widen_passes(L, meshes, smem);
    int fit2 = 0;
    if (smem_l > smem && (cluster_fit(L.P, L.mixed, L.wide, L.csize, smem_l, &fit2) != cudaSuccess || fit2 < fit)) {
      cudaGetLastError();
      for (size_t k = 0; k < L.members.size(); ++k) L.chunk[k] = meshes[L.members[k]]->g.chunk;
      smem_l = smem;
    }
    L.smem = smem_l;
    out.push_back(std::move(L));
  }
  b->cl_launches = std::move(out);
  return true;
}

// Streams and events of cluster launches are kept per device after a batch is destroyed and
// handed to later batches (the serving loop creates batches every tick).
std::mutex g_sp_mu;
std::vector<std::pair<cudaStream_t, cudaEvent_t>> g_stream_pool[64];

cudaError_t take_stream(int dev, cudaStream_t* st, cudaEvent_t* ev) {
  {
    std::lock_guard<std::mutex> lk(g_sp_mu);
    if (dev >= 0 && dev < 64 && !g_stream_pool[dev].empty()) {
      *st = g_stream_pool[dev].back().first;
      *ev = g_stream_pool[dev].back().second;
      g_stream_pool[dev].pop_back();
      return cudaSuccess;
    }
  }
  cudaError_t e = cudaStreamCreateWithFlags(st, cudaStreamNonBlocking);
  if (e != cudaSuccess) return e;
  return cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
}

void release_plan(std::vector<BatchLaunch>& plan, int dev) {
  std::lock_guard<std::mutex> lk(g_sp_mu);
  for (auto& L : plan) {
    if (L.stream && L.done && dev >= 0 && dev < 64) g_stream_pool[dev].emplace_back(L.stream, L.done);
    L.stream = nullptr;
    L.done = nullptr;
  }
}


// A plan's device arrays (descriptors, CTA map, barrier words, gathered status) from the pool.
int carve_plan(sem_batch* b, std::vector<BatchLaunch>& plan, size_t& off) {
  for (auto& L : plan) {
    L.inst_d = reinterpret_cast<Instance*>(b->pool + off);
    off += (sizeof(Instance) * L.members.size() + 255) & ~size_t(255);
    L.cta_d = reinterpret_cast<int*>(b->pool + off);
    off += (sizeof(int) * (size_t)L.grid + 255) & ~size_t(255);
    L.bars_d = reinterpret_cast<unsigned int*>(b->pool + off);
    off += (sizeof(unsigned) * 2 * L.members.size() + 255) & ~size_t(255);
    L.status_d = reinterpret_cast<int*>(b->pool + off);
    off += (sizeof(int) * L.members.size() + 255) & ~size_t(255);
    std::vector<int> map(L.grid);
    for (size_t k = 0; k < L.members.size(); ++k)
      for (int c = 0; c < L.nteam[k]; ++c) map[L.team0[k] + c] = (int)k;
    CUDA_TRY(cudaMemcpy(L.cta_d, map.data(), sizeof(int) * L.grid, cudaMemcpyHostToDevice));
    L.inst_h.resize(L.members.size());
    L.status_h.resize(L.members.size());
    if (L.csize > 0) CUDA_TRY(take_stream(b->device, &L.stream, &L.done));
  }
  return SEM_OK;
}

size_t plan_bytes(const std::vector<BatchLaunch>& plan) {
  size_t total = 0;
  for (const auto& L : plan)
    total += ((sizeof(Instance) * L.members.size() + 255) & ~size_t(255)) +
             ((sizeof(int) * (size_t)L.grid + 255) & ~size_t(255)) +
             ((sizeof(unsigned) * 2 * L.members.size() + 255) & ~size_t(255)) +
             ((sizeof(int) * L.members.size() + 255) & ~size_t(255));
  return total;
}

}  // namespace

extern "C" {

int sem_batch_create(sem_mesh* const* meshes, int count, sem_batch** out) {
  if (!out) return fail(SEM_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!meshes || count < 1) return fail(SEM_ERR_INVALID_ARG, "empty batch");
  for (int i = 0; i < count; ++i)
    if (!meshes[i]) return fail(SEM_ERR_INVALID_ARG, "NULL mesh in batch");
  const int dev = meshes[0]->device;
  for (int i = 0; i < count; ++i) {
    if (meshes[i]->device != dev) return fail(SEM_ERR_INVALID_ARG, "batch meshes must share one device");
    if (!meshes[i]->fused) return fail(SEM_ERR_INVALID_ARG, "batched meshes need the separable preconditioner");
    for (int j = 0; j < i; ++j)
      if (meshes[j] == meshes[i]) return fail(SEM_ERR_INVALID_ARG, "a mesh appears twice in the batch");
  }
  DeviceGuard dg(dev);
  int sms = 0;
  CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  sem_batch* b = new sem_batch;
  b->device = dev;
  b->meshes.assign(meshes, meshes + count);
  int rc = plan_cooperative(b, meshes, count, sms);
  if (rc) { delete b; return rc; }
  // The cluster plan is kept where it is estimated faster than the cooperative one (it is not
  // when a few large members would need more CTAs than a cluster holds); SEM_BATCH_CLUSTER=0 or 1
  // forces either plan.
  const char* cenv = std::getenv("SEM_BATCH_CLUSTER");
  const int force = cenv ? (std::atoi(cenv) != 0 ? 1 : 0) : batch_tuning().plan;
  if (force != 0 && plan_clusters(b, meshes, count, sms) && force < 0 &&
      estimate_clusters(b, 2.0 * sms) > estimate_cooperative(b))
    b->cl_launches.clear();
  for (int i = 0; i < count; ++i) {
    b->off.push_back(b->ncol_total);
    b->ncol_total += (size_t)meshes[i]->ncol;
  }
  const size_t state_bytes = (2 * b->ncol_total * sizeof(double) + 255) & ~size_t(255);
  const size_t total = state_bytes + plan_bytes(b->launches) + plan_bytes(b->cl_launches);
  cudaError_t ae = dev_alloc(dev, total + 256, reinterpret_cast<void**>(&b->pool));
  if (ae != cudaSuccess) { delete b; return fail(SEM_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(ae)); }
  b->state = reinterpret_cast<double*>(b->pool);
  size_t off = state_bytes;
  rc = carve_plan(b, b->launches, off);
  if (!rc) rc = carve_plan(b, b->cl_launches, off);
  if (!rc && !b->cl_launches.empty() && cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess)
    rc = fail(SEM_ERR_CUDA, "event creation failed");
  if (rc) {
    release_plan(b->cl_launches, dev);
    dev_free(dev, b->pool);
    delete b;
    return rc;
  }
  *out = b;
  return SEM_OK;
}

void sem_batch_destroy(sem_batch* b) {
  if (!b) return;
  DeviceGuard dg(b->device);
  cudaDeviceSynchronize();   // no work of this batch may still run when its memory is reused
  release_plan(b->cl_launches, b->device);
  if (b->fork) cudaEventDestroy(b->fork);
  for (auto& pr : b->events) { cudaEventDestroy(pr.first); cudaEventDestroy(pr.second); }
  for (cudaEvent_t e : b->spare) cudaEventDestroy(e);
  dev_free(b->device, b->pool);
  delete b;
}

void sem_trim_cache(void) {
  std::lock_guard<std::mutex> lk(g_cache_mu);
  int prev = -1;
  cudaGetDevice(&prev);
  for (int d = 0; d < 64; ++d) {
    BlockCache& c = g_cache[d];
    if (c.free.empty()) continue;
    cudaSetDevice(d);
    for (auto& kv : c.free) {
      cudaFree(kv.second);
      c.size_of.erase(kv.second);
    }
    c.free.clear();
    c.cached = 0;
  }
  if (prev >= 0) cudaSetDevice(prev);
}

int sem_batch_info(const sem_batch* b, int* launches_per_stage, int* ctas) {
  if (!b) return fail(SEM_ERR_INVALID_ARG, "NULL batch");
  const auto& plan = b->cl_launches.empty() ? b->launches : b->cl_launches;
  int tot = 0;
  for (const auto& L : plan) tot += L.grid;
  if (launches_per_stage) *launches_per_stage = (int)plan.size();
  if (ctas) *ctas = tot;
  return SEM_OK;
}

}  // extern "C"

namespace {
int batch_status(sem_batch* b, std::vector<BatchLaunch>& plan, cudaStream_t s);

// The cluster plan serves a call unless a member carries the barrier testing hook, whose early
// CTA exit only the cooperative launches' bounded barriers turn into an error.
bool use_clusters(const sem_batch* b) {
  if (b->cl_launches.empty()) return false;
  for (const sem_mesh* m : b->meshes)
    if (m->g.drop_rank >= 0 || m->g.bar_timeout_ns != kBarrierTimeoutNs) return false;
  return true;
}

cudaError_t take_batch_event(sem_batch* b, cudaEvent_t* ev) {
  if (!b->spare.empty()) { *ev = b->spare.back(); b->spare.pop_back(); return cudaSuccess; }
  return cudaEventCreate(ev);
}

// One stage launch of a batch group on stream s, bracketed by events while timing is on.
cudaError_t batch_launch(sem_batch* b, const BatchLaunch& L, const StageArgs& a, cudaStream_t s) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e;
  if (b->timing) {
    if ((e = take_batch_event(b, &e0)) != cudaSuccess) return e;
    if ((e = take_batch_event(b, &e1)) != cudaSuccess) return e;
    if ((e = cudaEventRecord(e0, s)) != cudaSuccess) return e;
  }
  if (L.csize > 0) e = launch_stage_cluster(L.P, L.mixed, L.wide, a, L.grid, L.csize, L.smem, s);
  else e = launch_stage(L.P, L.mixed, L.wide, a, L.grid, L.smem, s);
  if (e != cudaSuccess) return e;
  if (b->timing) {
    if ((e = cudaEventRecord(e1, s)) != cudaSuccess) return e;
    b->events.emplace_back(e0, e1);
  }
  return cudaSuccess;
}

// The cluster plan: each group's stage launches in order on the group's own stream, the streams
// forked from and joined back to s.  stage 0: the Laplace solve alone; else nsteps RK4 steps.
cudaError_t run_clusters(sem_batch* b, int stage, int nsteps, cudaStream_t s) {
  cudaError_t e;
  if ((e = cudaEventRecord(b->fork, s)) != cudaSuccess) return e;
  for (auto& L : b->cl_launches)
    if ((e = cudaStreamWaitEvent(L.stream, b->fork, 0)) != cudaSuccess) return e;
  for (int step = 0; step < (stage == 0 ? 1 : nsteps); ++step)
    for (int st = (stage == 0 ? 0 : 1); st <= (stage == 0 ? 0 : 4); ++st)
      for (auto& L : b->cl_launches) {
        const StageArgs a{L.inst_d, L.cta_d, nullptr, st, step, 1};
        if ((e = batch_launch(b, L, a, L.stream)) != cudaSuccess) return e;
      }
  for (auto& L : b->cl_launches) {
    if ((e = cudaEventRecord(L.done, L.stream)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(s, L.done, 0)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}
}  // namespace

extern "C" {

int sem_batch_rk4_step(sem_batch* b, double* const* eta_d, double* const* phis_d, double* t_h, const double* dt_h,
                       int nsteps, void* stream) {
  if (!b || !eta_d || !phis_d || !dt_h || nsteps < 0) return fail(SEM_ERR_INVALID_ARG, "bad argument");
  const int n = (int)b->meshes.size();
  for (int i = 0; i < n; ++i)
    if (!eta_d[i] || !phis_d[i] || !(dt_h[i] > 0.0)) return fail(SEM_ERR_INVALID_ARG, "bad instance state");
  DeviceGuard dg(b->device);
  cudaStream_t s = (cudaStream_t)stream;
  const bool cl = use_clusters(b);
  auto& plan = cl ? b->cl_launches : b->launches;
  for (auto& L : plan) {
    for (size_t k = 0; k < L.members.size(); ++k) {
      const int i = L.members[k];
      L.inst_h[k] = make_instance(b->meshes[i], eta_d[i], phis_d[i], t_h ? t_h[i] : 0.0, dt_h[i], L.team0[k],
                                  L.nteam[k], false, L.chunk[k]);
    }
    CUDA_TRY(cudaMemcpyAsync(L.inst_d, L.inst_h.data(), sizeof(Instance) * L.members.size(),
                             cudaMemcpyHostToDevice, s));
  }
  if (cl) {
    if (nsteps > 0) CUDA_TRY(run_clusters(b, 1, nsteps, s));
  } else {
    for (int step = 0; step < nsteps; ++step)
      for (int stage = 1; stage <= 4; ++stage)
        for (auto& L : plan) {
          CUDA_TRY(cudaMemsetAsync(L.bars_d, 0, 2 * sizeof(unsigned int) * L.members.size(), s));
          const StageArgs a{L.inst_d, L.cta_d, L.bars_d, stage, step, 0};
          CUDA_TRY(batch_launch(b, L, a, s));
        }
  }
  if (nsteps > 0)
    for (int i = 0; i < n; ++i) set_history(b->meshes[i], eta_d[i], phis_d[i], dt_h[i]);
  int rc = batch_status(b, plan, s);
  if (t_h)
    for (int i = 0; i < n; ++i) t_h[i] += nsteps * dt_h[i];
  return rc;
}

int sem_batch_laplace_solve(sem_batch* b, const double* const* eta_d, const double* const* phis_d,
                            double* const* Phi_d, void* stream) {
  if (!b || !eta_d || !phis_d || !Phi_d) return fail(SEM_ERR_INVALID_ARG, "bad argument");
  const int n = (int)b->meshes.size();
  for (int i = 0; i < n; ++i)
    if (!eta_d[i] || !phis_d[i] || !Phi_d[i]) return fail(SEM_ERR_INVALID_ARG, "bad instance state");
  DeviceGuard dg(b->device);
  cudaStream_t s = (cudaStream_t)stream;
  const bool cl = use_clusters(b);
  auto& plan = cl ? b->cl_launches : b->launches;
  for (auto& L : plan) {
    for (size_t k = 0; k < L.members.size(); ++k) {
      const int i = L.members[k];
      L.inst_h[k] = make_instance(b->meshes[i], const_cast<double*>(eta_d[i]), const_cast<double*>(phis_d[i]),
                                  0.0, 1.0, L.team0[k], L.nteam[k], false, L.chunk[k]);
      L.inst_h[k].pa.x = Phi_d[i];
    }
    CUDA_TRY(cudaMemcpyAsync(L.inst_d, L.inst_h.data(), sizeof(Instance) * L.members.size(),
                             cudaMemcpyHostToDevice, s));
  }
  if (cl) {
    CUDA_TRY(run_clusters(b, 0, 0, s));
  } else {
    for (auto& L : plan) {
      CUDA_TRY(cudaMemsetAsync(L.bars_d, 0, 2 * sizeof(unsigned int) * L.members.size(), s));
      const StageArgs a{L.inst_d, L.cta_d, L.bars_d, 0, 0, 0};
      CUDA_TRY(batch_launch(b, L, a, s));
    }
  }
  return batch_status(b, plan, s);
}

int sem_batch_rk4_step_host(sem_batch* b, double* eta_h, double* phis_h, double* t_h, const double* dt_h,
                            int nsteps, void* stream) {
  if (!b || !eta_h || !phis_h || !dt_h || nsteps < 0) return fail(SEM_ERR_INVALID_ARG, "bad argument");
  DeviceGuard dg(b->device);
  cudaStream_t s = (cudaStream_t)stream;
  const size_t n = b->meshes.size(), bytes = sizeof(double) * b->ncol_total;
  double* eta_d = b->state;
  double* phis_d = b->state + b->ncol_total;
  CUDA_TRY(cudaMemcpyAsync(eta_d, eta_h, bytes, cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(phis_d, phis_h, bytes, cudaMemcpyHostToDevice, s));
  std::vector<double*> ep(n), pp(n);
  for (size_t i = 0; i < n; ++i) { ep[i] = eta_d + b->off[i]; pp[i] = phis_d + b->off[i]; }
  const int rc = sem_batch_rk4_step(b, ep.data(), pp.data(), t_h, dt_h, nsteps, stream);
  if (rc != SEM_OK && rc != SEM_ERR_NOT_CONVERGED && rc != SEM_ERR_NONFINITE && rc != SEM_ERR_TIMEOUT) return rc;
  // every member's state comes back, failed members' included (their codes say which)
  const std::string err = t_err;
  CUDA_TRY(cudaMemcpyAsync(eta_h, eta_d, bytes, cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaMemcpyAsync(phis_h, phis_d, bytes, cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  if (rc != SEM_OK) t_err = err;
  return rc;
}

int sem_batch_enable_timing(sem_batch* b, int on) {
  if (!b) return fail(SEM_ERR_INVALID_ARG, "NULL batch");
  b->timing = on != 0;
  return SEM_OK;
}

int sem_batch_get_timing(sem_batch* b, sem_timing* t) {
  if (!b || !t) return fail(SEM_ERR_INVALID_ARG, "NULL argument");
  DeviceGuard dg(b->device);
  double total = 0.0;
  for (auto& pr : b->events) {
    CUDA_TRY(cudaEventSynchronize(pr.second));
    float ms = 0.f;
    CUDA_TRY(cudaEventElapsedTime(&ms, pr.first, pr.second));
    total += ms;
    b->spare.push_back(pr.first);
    b->spare.push_back(pr.second);
  }
  t->krylov_launches = (int64_t)b->events.size();
  t->krylov_ms = total;
  b->events.clear();
  return SEM_OK;
}

}  // extern "C"

namespace {
// One gather of every member's status word and one copy per launch group; returns the
// first failing instance's error.
int batch_status(sem_batch* b, std::vector<BatchLaunch>& plan, cudaStream_t s) {
  const int n = (int)b->meshes.size();
  for (auto& L : plan) {
    CUDA_TRY(launch_gather_status(L.inst_d, (int)L.members.size(), L.status_d, s));
    CUDA_TRY(cudaMemcpyAsync(L.status_h.data(), L.status_d, sizeof(int) * L.members.size(),
                             cudaMemcpyDeviceToHost, s));
  }
  CUDA_TRY(cudaStreamSynchronize(s));
  int rc = SEM_OK, first = n;
  b->codes.assign(n, SEM_OK);
  for (const auto& L : plan)
    for (size_t k = 0; k < L.members.size(); ++k) {
      b->codes[L.members[k]] = status_code(L.status_h[k]);
      if (L.status_h[k] && L.members[k] < first) {
        first = L.members[k];
        rc = L.status_h[k];
      }
    }
  if (rc != SEM_OK) {
    for (int i = 0; i < n; ++i)
      if (b->codes[i] != SEM_OK) CUDA_TRY(reset_warm_start(b->meshes[i], s));
    CUDA_TRY(cudaStreamSynchronize(s));
    rc = status_error(rc);
    t_err = "instance " + std::to_string(first) + ": " + t_err;
  }
  return rc;
}
}  // namespace

extern "C" {

int sem_batch_status(const sem_batch* b, int* codes_h) {
  if (!b || !codes_h) return fail(SEM_ERR_INVALID_ARG, "NULL argument");
  for (size_t i = 0; i < b->meshes.size(); ++i) codes_h[i] = i < b->codes.size() ? b->codes[i] : SEM_OK;
  return SEM_OK;
}

int sem_get_counters(sem_mesh* m, sem_counters* c, void* stream) {
  if (!m || !c) return fail(SEM_ERR_INVALID_ARG, "NULL argument");
  DeviceGuard dg(m->device);
  cudaStream_t s = (cudaStream_t)stream;
  SolveRecord r{};
  CUDA_TRY(cudaMemcpyAsync(&r, m->rec, sizeof(r), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  c->solves = r.solves;
  c->iterations = r.total_iterations;
  c->refinements = r.total_refinements;
  c->max_rel_residual = r.max_rel_residual;
  return SEM_OK;
}

int sem_enable_timing(sem_mesh* m, int on) {
  if (!m) return fail(SEM_ERR_INVALID_ARG, "NULL argument");
  m->timing = on != 0;
  return SEM_OK;
}

int sem_get_timing(sem_mesh* m, sem_timing* t) {
  if (!m || !t) return fail(SEM_ERR_INVALID_ARG, "NULL argument");
  DeviceGuard dg(m->device);
  double total = 0.0;
  for (auto& pr : m->events) {
    CUDA_TRY(cudaEventSynchronize(pr.second));
    float ms = 0.f;
    CUDA_TRY(cudaEventElapsedTime(&ms, pr.first, pr.second));
    total += ms;
    m->spare.push_back(pr.first);
    m->spare.push_back(pr.second);
  }
  t->krylov_launches = (int64_t)m->events.size();
  t->krylov_ms = total;
  m->events.clear();
  return SEM_OK;
}

#ifdef SEM_TRACE
// Diagnostic builds only (not part of sem.h): copies the phase trace of the mesh's last launches
// ([0] = marks, then (tag, ns) pairs) to out_h and clears it.
int sem_trace_read(sem_mesh* m, unsigned long long* out_h, int max_words) {
  if (!m || !out_h || !m->g.trace) return fail(SEM_ERR_INVALID_ARG, "no trace");
  DeviceGuard dg(m->device);
  CUDA_TRY(cudaDeviceSynchronize());
  const int words = std::min(max_words, 1 + 2 * kTraceMax);
  CUDA_TRY(cudaMemcpy(out_h, m->g.trace, sizeof(unsigned long long) * words, cudaMemcpyDeviceToHost));
  CUDA_TRY(cudaMemset(m->g.trace, 0, sizeof(unsigned long long)));
  return SEM_OK;
}
#endif

int sem_set_barrier_test(sem_mesh* m, int drop_rank, double timeout_ms) {
  if (!m) return fail(SEM_ERR_INVALID_ARG, "NULL mesh");
  if (drop_rank < -1) return fail(SEM_ERR_INVALID_ARG, "drop_rank must be -1 or a team rank");
  if (!(timeout_ms >= 0.0) || timeout_ms > 1e-6 * (double)kBarrierTimeoutNs)
    return fail(SEM_ERR_INVALID_ARG, "timeout_ms must be in [0, 2000]");
  m->g.drop_rank = drop_rank;
  m->g.bar_timeout_ns = timeout_ms > 0.0 ? (unsigned long long)(timeout_ms * 1e6) : kBarrierTimeoutNs;
  return SEM_OK;
}

int sem_reset_counters(sem_mesh* m, void* stream) {
  if (!m) return fail(SEM_ERR_INVALID_ARG, "NULL argument");
  DeviceGuard dg(m->device);
  CUDA_TRY(cudaMemsetAsync(m->rec, 0, sizeof(SolveRecord), (cudaStream_t)stream));
  return SEM_OK;
}

}  // extern "C"
