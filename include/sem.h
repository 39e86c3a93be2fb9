/*
 * sem.h — C ABI of the GB300 library for the stabilised nodal spectral
 * element method for fully nonlinear potential-flow water waves
 * (Engsig-Karup, Eskilsson & Bigoni, arXiv 1512.02548).
 *
 * The library solves, on one GPU, the free-surface problem of §2: find the
 * surface elevation η(x,t) and surface potential φ̃(x,t) evolving by the
 * Zakharov equations (eq. FSeqs), where the vertical surface velocity w̃ comes
 * from the Laplace problem (eq. laplaceproblem) solved in the σ-transformed
 * domain (eqs. sigtrans–symTransformedLaplace2) on a 2D x–σ mesh of
 * tensor-product Gauss–Lobatto–Legendre (GLL) quadrilaterals (§3.1).
 *
 * Conventions shared by every call
 * --------------------------------
 * Layout.  The mesh has Nx elements along x and Nz layers along σ ∈ [0,1],
 * order P in both directions.  Columns ix = 0..Ncol-1 with Ncol = Nx·P
 * (periodic) or Nx·P+1 (walls); rows iz = 0..Nrow-1, Nrow = Nz·P+1, from the
 * bottom (iz = 0) to the free surface (iz = Nrow-1).  A volume field is a
 * contiguous FP64 array of n = Ncol·Nrow values, node (ix,iz) at index
 * ix·Nrow + iz.  A surface field is a contiguous FP64 array of Ncol values.
 *
 * Pointers.  "_d" arguments are device pointers on the mesh's device, "_h"
 * arguments host pointers.  The caller owns every array it passes; the mesh
 * owns its own workspace (allocated once in sem_mesh_create).  Arrays passed
 * to one call must not overlap unless stated.
 *
 * Streams.  `stream` is a cudaStream_t (NULL = legacy default stream).  Work
 * is enqueued on it.  Calls marked "synchronises" wait for the stream at the
 * end to read the mesh's device status word; all others return as soon as
 * the work is enqueued.
 *
 * Environment (tuning and testing).  Read by sem_mesh_create: SEM_GRID_LIMIT caps the number
 * of CTAs of the persistent Krylov kernel and of a mesh's fused stage (default: all
 * co-resident); SEM_FUSED_STAGE=0 makes sem_rk4_step run the multi-kernel path instead of one
 * fused launch per RK stage.  Read by sem_laplace_apply: SEM_APPLY_KERNEL=column (see there);
 * by sem_laplace_apply_f32: SEM_APPLY_F32=tc (see there).
 * Read by sem_batch_create: SEM_BATCH_WIDE=1 (or 0) makes every group of the batch use the
 * two-CTAs-per-SM build of the fused stage (or the one-CTA-per-SM build); by default groups of
 * more than 8 instances use the former.  SEM_BATCH_CLUSTER=1 (or 0) makes the batch run its
 * instances as thread-block-cluster teams on concurrent streams (or as cooperative launches, one
 * per RK stage and (order, precision) group); by default the batch takes the plan it estimates
 * faster.  The cluster plan runs one stream per group of its launches (15 for 512 uneven tanks of
 * orders 4..8): a CUDA context with at least that many hardware work queues
 * (CUDA_DEVICE_MAX_CONNECTIONS, read when the context is created; default 8) keeps one group's
 * launch from waiting behind another's.
 *
 * Device memory.  Each mesh and batch owns one device block, taken at creation from a
 * per-device cache of blocks freed by earlier meshes and batches (or from cudaMalloc) and given
 * back to that cache at destruction; sem_trim_cache returns the cached blocks to CUDA.
 *
 * Errors.  Every call returns SEM_OK (0) or one of the codes below;
 * sem_last_error() gives a message for the calling thread's last failure.
 * A status raised on the device (no convergence, non-finite values, a
 * timed-out grid barrier) is reported by the next synchronising call.
 */
#ifndef SEM_GB300_H
#define SEM_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SEM_MAX_P 12

enum sem_status {
  SEM_OK = 0,
  SEM_ERR_INVALID_ARG = 1,   /* bad size, pointer or parameter            */
  SEM_ERR_OOM = 2,           /* device or host allocation failed          */
  SEM_ERR_CUDA = 3,          /* a CUDA runtime call failed                */
  SEM_ERR_NOT_CONVERGED = 4, /* Laplace solve hit max_iter above tol      */
  SEM_ERR_NONFINITE = 5,     /* NaN/Inf in a residual                     */
  SEM_ERR_TIMEOUT = 6        /* a device grid barrier gave up waiting     */
};

enum sem_precision {
  SEM_PREC_FP64 = 0,  /* every step in FP64                                      */
  SEM_PREC_MIXED = 1  /* FP32 inner Krylov iterations, FP64 residual refinement  */
};

enum sem_preconditioner {
  SEM_PRECOND_SEPARABLE = 0, /* exact inverse of the σ-separable part (slope terms dropped) */
  SEM_PRECOND_JACOBI = 1     /* diagonal                                                   */
};

/* Discretisation and solver parameters (§3.1, §3.3, §3.4). */
typedef struct sem_params {
  int P;               /* GLL order in x and σ, 2 ≤ P ≤ SEM_MAX_P                    */
  int Nx;              /* elements along x (periodic: Nx ≥ 3; walls: Nx ≥ 1)         */
  int Nz;              /* layers along σ, 1 ≤ Nz ≤ 16                                 */
  int periodic;        /* 1: periodic in x; 0: impermeable walls at both ends        */
  int Pf;              /* over-integration order of §3.3 (0 → P, i.e. none), ≤ 3P    */
  int filter_ic;       /* filter cut-off index i_c of §3.4; < 0 disables the filter  */
  double filter_alpha; /* filter strength α                                          */
  double filter_s;     /* filter order s (s = 0: constant factor e^-α above i_c)     */
  double g;            /* gravitational acceleration                                 */
  double tol;          /* Laplace solve: stop when ‖r‖₂ ≤ tol·‖b‖₂ (0 → 1e-13)       */
  int max_iter;        /* Laplace solve: Krylov iteration cap (0 → 5000)             */
  int precision;       /* enum sem_precision                                          */
  int precond;         /* enum sem_preconditioner                                     */
  double relax_left;   /* §2.2 generation zone length at the left end (0: none)           */
  double relax_right;  /* §2.2 absorption zone length at the right end (0: none)          */
  double relax_tau;    /* relaxation time τ (0: the RK4 step dt, as the paper chooses)     */
} sem_params;

typedef struct sem_info {
  int64_t n_nodes;     /* Ncol·Nrow                           */
  int64_t n_unknowns;  /* Ncol·(Nrow-1): Laplace unknowns      */
  int ncol, nrow;
  int n_elements;      /* Nx·Nz                               */
  int P, Pf, Nx, Nz, periodic, precision;
  int grid_ctas;       /* CTAs of the persistent Krylov kernel */
  int stage_ctas;      /* CTAs of the fused RK stage launch    */
  int64_t device_bytes;/* device memory owned by the mesh      */
} sem_info;

typedef struct sem_solve_stats {
  int iterations;        /* Krylov iterations of the last solve (inner, all refinements) */
  int refinements;       /* FP64 residual refinements (mixed precision), else 0          */
  double rel_residual;   /* final ‖r‖₂/‖b‖₂ in FP64                                       */
} sem_solve_stats;

typedef struct sem_counters {
  int64_t solves;            /* Laplace solves since creation / last reset    */
  int64_t iterations;        /* total Krylov iterations over those solves     */
  int64_t refinements;       /* total FP64 refinements (mixed precision)      */
  double max_rel_residual;   /* worst final relative residual                  */
} sem_counters;

typedef struct sem_mesh sem_mesh;

/* Create a mesh on the current CUDA device (§3.1): element edges x_edges_h[Nx+1]
 * (strictly increasing, host), still-water depth h_h[Ncol] at the columns (host,
 * > 0).  Builds the GLL tables, the surface-mass factorisation and all workspace
 * (owned by the mesh).  On failure *out is NULL. */
int sem_mesh_create(const sem_params* p, const double* x_edges_h, const double* h_h,
                    sem_mesh** out);
/* Waits for the device to be idle, then returns the mesh's memory to a per-device cache that
 * later sem_mesh_create / sem_batch_create calls reuse (at most 8 GiB per device is kept;
 * beyond that, blocks go back to CUDA). */
void sem_mesh_destroy(sem_mesh* m);
/* Returns every cached device block to CUDA (see sem_mesh_destroy). */
void sem_trim_cache(void);
/* Device memory sem_mesh_create would allocate for these arguments, without allocating
 * (for admission control); same validation and errors as sem_mesh_create. */
int sem_mesh_footprint(const sem_params* p, const double* x_edges_h, const double* h_h, int64_t* bytes);
int sem_mesh_info(const sem_mesh* m, sem_info* info);

/* Element-to-global map used by every gather/scatter (§3.1.2, assembly over
 * elements): l2g_d[((ex·Nz + l)·(P+1) + a)·(P+1) + b] = global id of local node
 * (a,b) of element (ex,l), written by a device kernel.  l2g_d: device, int32,
 * Nx·Nz·(P+1)² entries. */
int sem_mesh_l2g(sem_mesh* m, int32_t* l2g_d, void* stream);

/* σ-geometry for the current surface (§2, eqs. sigtrans, jacobian,
 * symTransformedLaplace2): d = η + h, element-local ∂x d, and the Jacobi
 * diagonal of the Laplace operator.  eta_d: device, Ncol.  Must precede
 * sem_laplace_apply / sem_laplace_solve for that η. */
int sem_update_geometry(sem_mesh* m, const double* eta_d, void* stream);

/* y = 𝓛 x with 𝓛_ij = −Σ_k ∫ (K∇N_j)·∇N_i over the mesh (§3.1.2), matrix-free,
 * all n rows (no Dirichlet modification), for the last sem_update_geometry.
 * x_d, y_d: device, n values, must not overlap.  Runs the tiled kernel of
 * sem_laplace_apply_f32 in FP64; the environment variable SEM_APPLY_KERNEL=column selects the
 * element-column kernel with the mesh's edge workspace instead (same result up to rounding
 * order). */
int sem_laplace_apply(sem_mesh* m, const double* x_d, double* y_d, void* stream);

/* The same operator in FP32 (the arithmetic of the mixed-precision inner solve): y = 𝓛 x
 * with the FP32 copy of the geometry of the last sem_update_geometry.  One kernel, tiles of
 * consecutive x-elements with the element left of each tile recomputed, so every output
 * column is complete in one CTA and written once; uses no workspace.  x_d, y_d: device,
 * float, n values, must not overlap.  The environment variable SEM_APPLY_F32=tc selects, for
 * orders 4..7, a kernel whose element contractions run on the tensor cores (TF32 products
 * split three ways for FP32 accuracy; same result up to rounding, and slower on GB300). */
int sem_laplace_apply_f32(const sem_mesh* m, const float* x_d, float* y_d, void* stream);

/* Allocation-free form of sem_laplace_apply (the paper has no counterpart; this is a
 * service of the library).  For callers that must not allocate device memory at the time
 * of the call: real-time or latency-bound loops that forbid allocator calls (cudaMalloc
 * and cudaFree can synchronise the device and take unbounded time), and hosts whose own
 * memory manager owns the device's memory (a caching allocator that has reserved it, so a
 * raw cudaMalloc fails or fragments its pool).  It computes y = 𝓛x exactly as
 * sem_laplace_apply does, for the last sem_update_geometry, but touches no workspace of the
 * mesh and calls no allocator: y receives partial sums first, and the one temporary the
 * apply needs (the shared x-interface column of every element column, Nx·Nrow values) lives
 * in a static device array of 2^20 doubles (8 MiB) that every device which loads the library
 * holds until the process exits.  Nx·Nrow above 2^20 is rejected with SEM_ERR_INVALID_ARG.
 * The first call on a device (and the first after that device's context was reset) looks up
 * the array's device address.  All calls on a device share the array and it keeps the last
 * call's contents (every entry a call reads is written earlier in that call, so nothing needs
 * clearing); calls that can overlap on the GPU (other streams, other meshes) race on it and
 * must be serialised by the caller.  x_d, y_d: device, n values, must not overlap. */
int sem_laplace_apply_noalloc(const sem_mesh* m, const double* x_d, double* y_d, void* stream);

/* Laplace problem of eq. (laplaceproblem) for the last sem_update_geometry:
 * 𝓛Φ = 0 at interior nodes, Φ = φ̃ at the surface (eq. FSeqs BC), solved by
 * preconditioned conjugate gradients on the Dirichlet-eliminated SPD system
 * (§3.1.2 names PCG for large systems).  phis_d: device, Ncol.  Phi_d: device,
 * n; on entry its interior values are the initial guess, on exit the solution
 * (surface rows set to φ̃).  If st is non-NULL the call synchronises and fills
 * it; otherwise device status is reported by the next synchronising call. */
int sem_laplace_solve(sem_mesh* m, const double* phis_d, double* Phi_d,
                      sem_solve_stats* st, void* stream);

/* Gradient recovery (§3.1.3): w̃ = w at the surface from 𝓜w = 𝓢_zΦ
 * (eq. velocpot2), and the C⁰ derivatives from M'u = S_x f (eq.
 * representationU) for f = η and f = φ̃.  Uses the geometry of the last
 * sem_update_geometry (for 1/d).  Inputs Phi_d (n), eta_d, phis_d (Ncol);
 * outputs w_surf_d, etax_d, phisx_d (Ncol each); all device. */
int sem_recover_gradient(sem_mesh* m, const double* Phi_d, const double* eta_d,
                         const double* phis_d, double* w_surf_d, double* etax_d,
                         double* phisx_d, void* stream);

/* Right-hand side of the semi-discrete free-surface equations (§3.1.1 with
 * the PDE form of eq. FSeqs, over-integrated at order Pf per §3.3):
 * M' ∂tη = ∫(−ηxφ̃x + w̃(1+ηx²))N_i,  M' ∂tφ̃ = ∫(−gη − ½(φ̃x² − w̃²(1+ηx²)))N_i,
 * plus the relaxation source of §2.2 at time t when zones are configured (then
 * relax_tau must be > 0).  Runs geometry, the Laplace solve (warm-started from the
 * mesh's previous potential), recovery and the projection.
 * eta_d, phis_d in; deta_d, dphis_d out; device, Ncol each. */
int sem_zakharov_rhs(sem_mesh* m, const double* eta_d, const double* phis_d, double t,
                     double* deta_d, double* dphis_d, void* stream);

/* Wave input of the generation zone (§2.2): the left zone relaxes (η, φ̃) towards the
 * linear superposition η_a = Σ a_i cos(ω_i t − k_i x + θ_i), φ̃_a = −Σ (g a_i/ω_i)
 * sin(ω_i t − k_i x + θ_i); the right zone relaxes towards rest.  The relaxation source
 * (1 − γ(x))(q_a − q)/τ is added at the surface nodes, with γ a smooth step ξ²(3−2ξ) across
 * each zone.  Arrays are host, ncomp ≤ 4096 entries each; ncomp = 0 clears the signal.
 * The copy is synchronous and not ordered with `stream` work: call it while no step of
 * this mesh is in flight.  It also tabulates cos, sin of k_i x at the left-zone columns
 * (one more device block of 16·ncomp bytes per zone column, up to 512 MB; larger tables are
 * skipped): the fused RK stage then evaluates the signal by angle addition, with per-stage
 * sines of ω_i t + θ_i, spread over all CTAs of the team.  Returns SEM_ERR_OOM if that block
 * cannot be allocated. */
int sem_set_wave_input(sem_mesh* m, int ncomp, const double* amp_h, const double* omega_h,
                       const double* k_h, const double* phase_h);

/* Per-element modal filter F = V̂SV̂⁻¹ of §3.4 applied in place to a surface
 * field (no-op if filter_ic < 0).  q_d: device, Ncol. */
int sem_apply_filter(sem_mesh* m, double* q_d, void* stream);

/* nsteps classical RK4 steps of size dt on (η, φ̃) in place, each followed by
 * the filter (§3.1.1, §3.4); *t advances by nsteps·dt.  eta_d, phis_d: device,
 * Ncol.  Synchronises once at the end.  Each stage's Laplace solve starts from an
 * extrapolation of earlier stage potentials kept by the mesh; stages 2 and 3 of the
 * first step use the previous call's potentials when this call steps the same eta_d,
 * phis_d with the same dt (a continuing trajectory).  The starting point does not change
 * the converged result, only the iteration count; a failed step clears the history. */
int sem_rk4_step(sem_mesh* m, double* eta_d, double* phis_d, double* t, double dt,
                 int nsteps, void* stream);

/* As sem_rk4_step for callers holding the state in host memory: copies eta_h,
 * phis_h (host, Ncol each; pinned memory recommended) to the device, steps,
 * and copies the result back.  Synchronises. */
int sem_rk4_step_host(sem_mesh* m, double* eta_h, double* phis_h, double* t, double dt,
                      int nsteps, void* stream);

/* Batched instances (many tanks stepped together).  Each instance is served by its own team of
 * CTAs, sized to its work, with its own barriers and reductions, so results equal the instance
 * run alone up to the summation order of the team's reductions.  Two execution plans: every
 * team one thread-block cluster (at most 16 CTAs), the launches of all (order, precision, team
 * size) groups on streams of their own that run at the same time; or one cooperative launch per
 * RK stage and (order P, precision) group, teams sized to fill the co-resident CTAs.  A batch
 * takes the plan it estimates faster (the cooperative one when a few large instances would need
 * more CTAs than a cluster holds); instances carrying the barrier testing hook force the
 * cooperative plan.  The meshes stay owned by the caller and must outlive the batch; they
 * must share one device and use the separable preconditioner.  Stepping a batch uses each
 * mesh's workspace, so a mesh may not be stepped elsewhere concurrently. */
typedef struct sem_batch sem_batch;
int sem_batch_create(sem_mesh* const* meshes, int count, sem_batch** out);
void sem_batch_destroy(sem_batch* b);
/* Launches per RK stage and total CTAs of one stage (for reporting). */
int sem_batch_info(const sem_batch* b, int* launches_per_stage, int* ctas);
/* nsteps RK4 steps (with filter and relaxation as configured per mesh) on every instance:
 * eta_d[i], phis_d[i] device arrays of instance i (Ncol_i values), dt_h[i] its step, t_h[i]
 * (host, may be NULL) its time, advanced by nsteps·dt_h[i].  Synchronises; the first failing
 * instance's error is returned (its index in the message). */
int sem_batch_rk4_step(sem_batch* b, double* const* eta_d, double* const* phis_d, double* t_h,
                       const double* dt_h, int nsteps, void* stream);
/* One Laplace solve per instance in one cooperative launch per (order, precision) group:
 * the σ-geometry and preconditioner of mesh i are rebuilt for eta_d[i] (as sem_update_geometry
 * does), then 𝓛Φ = 0 with Φ = φ̃ = phis_d[i] at the surface is solved as sem_laplace_solve
 * does.  Phi_d[i]: device, n_i values; on entry its interior values are the initial guess, on
 * exit the solution.  eta_d[i], phis_d[i]: device, Ncol_i.  Synchronises; the first failing
 * instance's error is returned (its index in the message). */
int sem_batch_laplace_solve(sem_batch* b, const double* const* eta_d, const double* const* phis_d,
                            double* const* Phi_d, void* stream);
/* As sem_batch_rk4_step for callers holding every instance's state in host memory (pinned
 * memory recommended): eta_h and phis_h are packed, instance i's Ncol_i values following those
 * of instances 0..i-1 (Σ Ncol_i values each).  Two host→device copies, the steps, two
 * device→host copies, on `stream`, into a packed device copy that the batch owns.  Synchronises.
 * The state of every instance comes back, a failed instance's included (sem_batch_status says
 * which failed); the first failing instance's error is returned. */
int sem_batch_rk4_step_host(sem_batch* b, double* eta_h, double* phis_h, double* t_h, const double* dt_h,
                            int nsteps, void* stream);
/* Planning parameters of later sem_batch_create calls (process-wide; written by the autotuner
 * paper_1512_02548_gb300/autotune.py from measurements on the device, NULL restores the defaults).
 * The environment variables SEM_BATCH_WIDE and SEM_BATCH_CLUSTER still take precedence. */
typedef struct sem_batch_tuning {
  double cluster_share;  /* cluster plan: a team is the smallest power of two of CTAs whose work per
                            CTA is at most this fraction of the batch's work per CTA slot (0.5)   */
  int max_cluster;       /* largest cluster team, a power of two in 1..16 (16)                   */
  int narrow_max;        /* groups of at most this many instances use the one-CTA-per-SM build (8) */
  int plan;              /* -1: the plan estimated faster; 0: cooperative; 1: clusters (-1)       */
} sem_batch_tuning;
int sem_set_batch_tuning(const sem_batch_tuning* t);
int sem_get_batch_tuning(sem_batch_tuning* t);
/* Tile width (elements per tile, 1..16) of the FP32 tiled apply (sem_laplace_apply_f32, CUDA-core
 * kernel) for order P and Nz layers, as measured by the autotuner; 0 restores the default (the widest
 * tile up to 16 that keeps three CTAs per SM).  The FP64 apply takes the widest tile up to 16 that
 * fits in shared memory.  Process-wide. */
int sem_set_apply_tile_width(int P, int Nz, int E);

/* Per-instance result of the last sem_batch_rk4_step or sem_batch_laplace_solve:
 * codes_h[i] (host, one per instance) = SEM_OK or the instance's own error code, so a caller
 * can fail one instance and keep the others (each instance's state is advanced or solved
 * independently of the others' outcome).  All SEM_OK before the first call. */
int sem_batch_status(const sem_batch* b, int* codes_h);

/* Solver counters accumulated on the device; reading synchronises the stream. */
int sem_get_counters(sem_mesh* m, sem_counters* c, void* stream);
int sem_reset_counters(sem_mesh* m, void* stream);

/* Kernel timing.  While enabled, every launch of the persistent Krylov kernel is
 * bracketed by CUDA events recorded on its stream.  sem_get_timing waits for the
 * recorded events, returns the number of those launches and their summed device
 * time in milliseconds, and clears the record. */
typedef struct sem_timing {
  int64_t krylov_launches;
  double krylov_ms;
} sem_timing;
int sem_enable_timing(sem_mesh* m, int on);
int sem_get_timing(sem_mesh* m, sem_timing* t);

/* The same timing for the fused stage launches of a batch (one record per (order, precision)
 * group and stage). */
int sem_batch_enable_timing(sem_batch* b, int on);
int sem_batch_get_timing(sem_batch* b, sem_timing* t);

/* Testing hook for the bounded team barriers (a barrier that gives up reports
 * SEM_ERR_TIMEOUT).  Every wait of a team barrier is limited to timeout_ms of wall-clock
 * time (0: the default, 2000 ms; at most 2000).  drop_rank ≥ 0 makes the CTA of that rank in the
 * mesh's team return at the start of each later Krylov or fused stage launch of this mesh (alone
 * or in a batch), before its first barrier, so that the other CTAs' waits run out: the launch
 * ends within about timeout_ms, the status word carries the timeout and the next synchronising
 * call returns SEM_ERR_TIMEOUT.  A team of one CTA has no barrier to miss (drop_rank 0 then
 * skips the work, with no error).  drop_rank = -1 restores normal launches. */
int sem_set_barrier_test(sem_mesh* m, int drop_rank, double timeout_ms);

/* Number of kernels this library has launched in the calling process. */
int64_t sem_launch_count(void);

/* Message for the calling thread's last error ("" if none). */
const char* sem_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* SEM_GB300_H */
