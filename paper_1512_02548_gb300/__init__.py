"""GB300 library for the stabilised nodal SEM water-wave model (arXiv 1512.02548).

Thin ctypes binding of the C ABI in ``include/sem.h``: argument marshalling only.
Every step of the method runs in the CUDA kernels of ``libsem_gb300.so``; there is
no CPU fallback, and using the binding without the built library raises.

Device arrays are ``torch.Tensor`` objects on the mesh's CUDA device (FP64,
contiguous); the current torch stream is passed to every call.  PyTorch is used
only for device memory and streams.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsem_gb300.so")

SEM_OK = 0
(SEM_ERR_INVALID_ARG, SEM_ERR_OOM, SEM_ERR_CUDA, SEM_ERR_NOT_CONVERGED, SEM_ERR_NONFINITE,
 SEM_ERR_TIMEOUT) = range(1, 7)
SEM_ERRORS = {1: "SEM_ERR_INVALID_ARG", 2: "SEM_ERR_OOM", 3: "SEM_ERR_CUDA",
              4: "SEM_ERR_NOT_CONVERGED", 5: "SEM_ERR_NONFINITE", 6: "SEM_ERR_TIMEOUT"}
SEM_PREC_FP64, SEM_PREC_MIXED = 0, 1
SEM_PRECOND_SEPARABLE, SEM_PRECOND_JACOBI = 0, 1

EXPORTED = ("sem_mesh_create", "sem_mesh_destroy", "sem_trim_cache", "sem_mesh_footprint", "sem_mesh_info", "sem_mesh_l2g",
            "sem_update_geometry", "sem_laplace_apply", "sem_laplace_apply_f32", "sem_laplace_apply_noalloc", "sem_laplace_solve",
            "sem_recover_gradient", "sem_zakharov_rhs", "sem_set_wave_input", "sem_apply_filter", "sem_rk4_step",
            "sem_rk4_step_host", "sem_get_counters", "sem_reset_counters", "sem_enable_timing",
            "sem_get_timing", "sem_batch_create", "sem_batch_destroy", "sem_batch_info",
            "sem_batch_rk4_step", "sem_batch_rk4_step_host", "sem_batch_laplace_solve", "sem_batch_status",
            "sem_batch_enable_timing", "sem_batch_get_timing", "sem_set_batch_tuning", "sem_get_batch_tuning",
            "sem_set_apply_tile_width", "sem_set_barrier_test", "sem_launch_count", "sem_last_error")


class sem_params(ctypes.Structure):
    _fields_ = [("P", ctypes.c_int), ("Nx", ctypes.c_int), ("Nz", ctypes.c_int),
                ("periodic", ctypes.c_int), ("Pf", ctypes.c_int), ("filter_ic", ctypes.c_int),
                ("filter_alpha", ctypes.c_double), ("filter_s", ctypes.c_double),
                ("g", ctypes.c_double), ("tol", ctypes.c_double), ("max_iter", ctypes.c_int),
                ("precision", ctypes.c_int), ("precond", ctypes.c_int),
                ("relax_left", ctypes.c_double), ("relax_right", ctypes.c_double),
                ("relax_tau", ctypes.c_double)]


class sem_info(ctypes.Structure):
    _fields_ = [("n_nodes", ctypes.c_int64), ("n_unknowns", ctypes.c_int64),
                ("ncol", ctypes.c_int), ("nrow", ctypes.c_int), ("n_elements", ctypes.c_int),
                ("P", ctypes.c_int), ("Pf", ctypes.c_int), ("Nx", ctypes.c_int), ("Nz", ctypes.c_int),
                ("periodic", ctypes.c_int), ("precision", ctypes.c_int), ("grid_ctas", ctypes.c_int),
                ("stage_ctas", ctypes.c_int), ("device_bytes", ctypes.c_int64)]


class sem_solve_stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("refinements", ctypes.c_int),
                ("rel_residual", ctypes.c_double)]


class sem_batch_tuning(ctypes.Structure):
    _fields_ = [("cluster_share", ctypes.c_double), ("max_cluster", ctypes.c_int), ("narrow_max", ctypes.c_int),
                ("plan", ctypes.c_int)]


class sem_counters(ctypes.Structure):
    _fields_ = [("solves", ctypes.c_int64), ("iterations", ctypes.c_int64),
                ("refinements", ctypes.c_int64), ("max_rel_residual", ctypes.c_double)]


class sem_timing(ctypes.Structure):
    _fields_ = [("krylov_launches", ctypes.c_int64), ("krylov_ms", ctypes.c_double)]


_lib = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libsem_gb300.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it first (python -m paper_1512_02548_gb300.build)")
    lib = ctypes.CDLL(path)
    vp, dp, ip = ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int
    lib.sem_mesh_create.argtypes = [ctypes.POINTER(sem_params), dp, dp, ctypes.POINTER(vp)]
    lib.sem_mesh_footprint.argtypes = [ctypes.POINTER(sem_params), dp, dp, ctypes.POINTER(ctypes.c_int64)]
    lib.sem_mesh_destroy.argtypes = [vp]
    lib.sem_mesh_destroy.restype = None
    lib.sem_trim_cache.argtypes = []
    lib.sem_trim_cache.restype = None
    lib.sem_mesh_info.argtypes = [vp, ctypes.POINTER(sem_info)]
    lib.sem_mesh_l2g.argtypes = [vp, dp, vp]
    lib.sem_update_geometry.argtypes = [vp, dp, vp]
    lib.sem_laplace_apply.argtypes = [vp, dp, dp, vp]
    lib.sem_laplace_apply_noalloc.argtypes = [vp, dp, dp, vp]
    lib.sem_laplace_apply_f32.argtypes = [vp, vp, vp, vp]
    lib.sem_laplace_solve.argtypes = [vp, dp, dp, ctypes.POINTER(sem_solve_stats), vp]
    lib.sem_recover_gradient.argtypes = [vp, dp, dp, dp, dp, dp, dp, vp]
    lib.sem_zakharov_rhs.argtypes = [vp, dp, dp, ctypes.c_double, dp, dp, vp]
    lib.sem_apply_filter.argtypes = [vp, dp, vp]
    lib.sem_set_wave_input.argtypes = [vp, ip, dp, dp, dp, dp]
    lib.sem_rk4_step.argtypes = [vp, dp, dp, ctypes.POINTER(ctypes.c_double), ctypes.c_double, ip, vp]
    lib.sem_rk4_step_host.argtypes = [vp, dp, dp, ctypes.POINTER(ctypes.c_double), ctypes.c_double, ip, vp]
    lib.sem_get_counters.argtypes = [vp, ctypes.POINTER(sem_counters), vp]
    lib.sem_reset_counters.argtypes = [vp, vp]
    lib.sem_enable_timing.argtypes = [vp, ip]
    lib.sem_get_timing.argtypes = [vp, ctypes.POINTER(sem_timing)]
    lib.sem_batch_create.argtypes = [ctypes.POINTER(vp), ip, ctypes.POINTER(vp)]
    lib.sem_batch_destroy.argtypes = [vp]
    lib.sem_batch_destroy.restype = None
    lib.sem_batch_info.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
    lib.sem_batch_rk4_step.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_double), ip, vp]
    lib.sem_batch_rk4_step_host.argtypes = [vp, dp, dp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                            ip, vp]
    lib.sem_batch_laplace_solve.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp), vp]
    lib.sem_batch_enable_timing.argtypes = [vp, ip]
    lib.sem_batch_get_timing.argtypes = [vp, ctypes.POINTER(sem_timing)]
    lib.sem_set_barrier_test.argtypes = [vp, ip, ctypes.c_double]
    lib.sem_set_batch_tuning.argtypes = [ctypes.POINTER(sem_batch_tuning)]
    lib.sem_get_batch_tuning.argtypes = [ctypes.POINTER(sem_batch_tuning)]
    lib.sem_set_apply_tile_width.argtypes = [ip, ip, ip]
    lib.sem_batch_status.argtypes = [vp, ctypes.POINTER(ctypes.c_int)]
    lib.sem_launch_count.restype = ctypes.c_int64
    lib.sem_launch_count.argtypes = []
    lib.sem_last_error.restype = ctypes.c_char_p
    lib.sem_last_error.argtypes = []
    for name in EXPORTED:
        if name not in ("sem_mesh_destroy", "sem_batch_destroy", "sem_launch_count", "sem_last_error"):
            getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


class SemError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{SEM_ERRORS.get(code, code)}: {msg}")
        self.code = code


def _check(code: int):
    if code != SEM_OK:
        raise SemError(code, load_library().sem_last_error().decode())


def _stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t, dtype=None):
    if t is None:
        return None
    if not (t.is_cuda and t.is_contiguous()):
        raise ValueError("expected a contiguous CUDA tensor")
    import torch
    if dtype is not None:
        if t.dtype != dtype:
            raise ValueError(f"expected {dtype}")
    elif t.dtype not in (torch.float64, torch.int32):
        raise ValueError("expected float64 (or int32 for l2g)")
    return ctypes.c_void_p(t.data_ptr())


def launch_count() -> int:
    return int(load_library().sem_launch_count())


def set_batch_tuning(cluster_share: float | None = None, max_cluster: int | None = None,
                     narrow_max: int | None = None, plan: int | None = None, reset: bool = False):
    """Process-wide batch planning parameters (sem_set_batch_tuning); unset fields keep their value,
    reset=True restores the defaults first."""
    lib = load_library()
    if reset:
        _check(lib.sem_set_batch_tuning(None))
    t = sem_batch_tuning()
    _check(lib.sem_get_batch_tuning(ctypes.byref(t)))
    for name, v in (("cluster_share", cluster_share), ("max_cluster", max_cluster), ("narrow_max", narrow_max),
                    ("plan", plan)):
        if v is not None:
            setattr(t, name, v)
    _check(lib.sem_set_batch_tuning(ctypes.byref(t)))
    return t


def get_batch_tuning() -> dict:
    t = sem_batch_tuning()
    _check(load_library().sem_get_batch_tuning(ctypes.byref(t)))
    return {"cluster_share": t.cluster_share, "max_cluster": t.max_cluster, "narrow_max": t.narrow_max, "plan": t.plan}


def set_apply_tile_width(P: int, Nz: int, E: int):
    """Tile width of the tiled apply for (P, Nz) (sem_set_apply_tile_width); 0 = default."""
    _check(load_library().sem_set_apply_tile_width(int(P), int(Nz), int(E)))


def mesh_params(P, Nx, Nz, periodic=True, Pf=0, filter_alpha=0.0, filter_s=0.0, filter_ic=-1, g=9.81,
                tol=1e-13, max_iter=5000, precision="fp64", precond="separable", relax_left=0.0,
                relax_right=0.0, relax_tau=0.0) -> sem_params:
    if precision not in ("fp64", "mixed") or precond not in ("separable", "jacobi"):
        raise ValueError("precision must be fp64|mixed and precond separable|jacobi")
    return sem_params(P=P, Nx=Nx, Nz=Nz, periodic=int(bool(periodic)), Pf=Pf, filter_ic=filter_ic,
                      filter_alpha=filter_alpha, filter_s=filter_s, g=g, tol=tol, max_iter=max_iter,
                      precision=SEM_PREC_MIXED if precision == "mixed" else SEM_PREC_FP64,
                      precond=SEM_PRECOND_JACOBI if precond == "jacobi" else SEM_PRECOND_SEPARABLE,
                      relax_left=relax_left, relax_right=relax_right, relax_tau=relax_tau)


def mesh_footprint(prm: sem_params, x_edges, h) -> int:
    """Device bytes a mesh with these parameters would own (sem_mesh_footprint)."""
    xe = np.ascontiguousarray(x_edges, dtype=np.float64)
    hh = np.ascontiguousarray(h, dtype=np.float64)
    b = ctypes.c_int64()
    _check(load_library().sem_mesh_footprint(ctypes.byref(prm), xe.ctypes.data_as(ctypes.c_void_p),
                                             hh.ctypes.data_as(ctypes.c_void_p), ctypes.byref(b)))
    return int(b.value)


class Mesh:
    """One σ-mesh on the current CUDA device; wraps ``sem_mesh``.

    Method names follow the C ABI (``sem_<name>``); arrays are torch CUDA tensors.
    """

    def __init__(self, P: int, Nx: int, Nz: int, x_edges, h, periodic: bool = True, Pf: int = 0,
                 filter_alpha: float = 0.0, filter_s: float = 0.0, filter_ic: int = -1,
                 g: float = 9.81, tol: float = 1e-13, max_iter: int = 5000, precision: str = "fp64",
                 precond: str = "separable", relax_left: float = 0.0, relax_right: float = 0.0,
                 relax_tau: float = 0.0, wave=None):
        lib = load_library()
        from .autotune import apply_tuning
        apply_tuning(batch=False)   # the measured tile widths of the tiled apply, once per process
        prm = mesh_params(P, Nx, Nz, periodic, Pf, filter_alpha, filter_s, filter_ic, g, tol, max_iter, precision,
                          precond, relax_left, relax_right, relax_tau)
        xe = np.ascontiguousarray(x_edges, dtype=np.float64)
        hh = np.ascontiguousarray(h, dtype=np.float64)
        handle = ctypes.c_void_p()
        _check(lib.sem_mesh_create(ctypes.byref(prm), xe.ctypes.data_as(ctypes.c_void_p),
                                   hh.ctypes.data_as(ctypes.c_void_p), ctypes.byref(handle)))
        self._h = handle
        self.info = sem_info()
        _check(lib.sem_mesh_info(self._h, ctypes.byref(self.info)))
        self.ncol, self.nrow = self.info.ncol, self.info.nrow
        self.n = int(self.info.n_nodes)
        self.n_unknowns = int(self.info.n_unknowns)
        if wave is not None:
            self.set_wave_input(*wave)

    @classmethod
    def from_workload(cls, wl, h=None, precision: str = "fp64", tol: float = 1e-13, max_iter: int = 5000,
                      precond: str = "separable"):
        edges = wl.element_edges()
        if h is None:
            h = np.full(wl.ncol, wl.depth)
        return cls(wl.P, wl.Nx, wl.Nz, edges, h, periodic=wl.periodic, Pf=wl.Pf,
                   filter_alpha=wl.filter_alpha, filter_s=wl.filter_s, filter_ic=wl.filter_ic,
                   g=wl.g, tol=tol, max_iter=max_iter, precision=precision, precond=precond,
                   relax_left=wl.relax_left, relax_right=wl.relax_right, relax_tau=wl.relax_tau,
                   wave=wl.wave)

    def close(self):
        if getattr(self, "_h", None):
            load_library().sem_mesh_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- C ABI calls -----------------------------------------------------------------
    def l2g(self, out):
        _check(load_library().sem_mesh_l2g(self._h, _ptr(out), _stream()))
        return out

    def update_geometry(self, eta):
        _check(load_library().sem_update_geometry(self._h, _ptr(eta), _stream()))

    def laplace_apply(self, x, y):
        _check(load_library().sem_laplace_apply(self._h, _ptr(x), _ptr(y), _stream()))
        return y

    def laplace_apply_f32(self, x, y):
        """y = 𝓛x in FP32 (float32 tensors), tiled kernel (sem_laplace_apply_f32)."""
        import torch
        _check(load_library().sem_laplace_apply_f32(self._h, _ptr(x, torch.float32), _ptr(y, torch.float32),
                                                     _stream()))
        return y

    def laplace_apply_noalloc(self, x, y):
        """y = 𝓛x without any allocation by the library (static device scratch, see sem.h)."""
        _check(load_library().sem_laplace_apply_noalloc(self._h, _ptr(x), _ptr(y), _stream()))
        return y

    def laplace_solve(self, phis, Phi, stats: bool = True):
        st = sem_solve_stats()
        _check(load_library().sem_laplace_solve(self._h, _ptr(phis), _ptr(Phi),
                                                ctypes.byref(st) if stats else None, _stream()))
        return st if stats else None

    def recover_gradient(self, Phi, eta, phis, w, etax, phisx):
        _check(load_library().sem_recover_gradient(self._h, _ptr(Phi), _ptr(eta), _ptr(phis),
                                                   _ptr(w), _ptr(etax), _ptr(phisx), _stream()))

    def zakharov_rhs(self, eta, phis, deta, dphis, t: float = 0.0):
        _check(load_library().sem_zakharov_rhs(self._h, _ptr(eta), _ptr(phis), ctypes.c_double(t),
                                               _ptr(deta), _ptr(dphis), _stream()))

    def set_wave_input(self, amp, omega, k, phase):
        arrs = [np.ascontiguousarray(v, dtype=np.float64) for v in (amp, omega, k, phase)]
        n = len(arrs[0])
        _check(load_library().sem_set_wave_input(self._h, n, *(a.ctypes.data_as(ctypes.c_void_p) for a in arrs)))

    def apply_filter(self, q):
        _check(load_library().sem_apply_filter(self._h, _ptr(q), _stream()))

    def rk4_step(self, eta, phis, dt: float, nsteps: int = 1, t: float = 0.0) -> float:
        tt = ctypes.c_double(t)
        _check(load_library().sem_rk4_step(self._h, _ptr(eta), _ptr(phis), ctypes.byref(tt),
                                           ctypes.c_double(dt), int(nsteps), _stream()))
        return tt.value

    def rk4_step_host(self, eta, phis, dt: float, nsteps: int = 1, t: float = 0.0) -> float:
        """eta, phis: host float64 arrays (numpy or pinned CPU tensors), updated in place."""
        def hp(a):
            if isinstance(a, np.ndarray):
                if a.dtype != np.float64 or not a.flags.c_contiguous:
                    raise ValueError("expected a contiguous float64 array")
                return a.ctypes.data_as(ctypes.c_void_p)
            return ctypes.c_void_p(a.data_ptr())
        tt = ctypes.c_double(t)
        _check(load_library().sem_rk4_step_host(self._h, hp(eta), hp(phis), ctypes.byref(tt),
                                                ctypes.c_double(dt), int(nsteps), _stream()))
        return tt.value

    def counters(self) -> sem_counters:
        c = sem_counters()
        _check(load_library().sem_get_counters(self._h, ctypes.byref(c), _stream()))
        return c

    def reset_counters(self):
        _check(load_library().sem_reset_counters(self._h, _stream()))

    def enable_timing(self, on: bool = True):
        _check(load_library().sem_enable_timing(self._h, int(bool(on))))

    def timing(self) -> sem_timing:
        t = sem_timing()
        _check(load_library().sem_get_timing(self._h, ctypes.byref(t)))
        return t

    def set_barrier_test(self, drop_rank: int = -1, timeout_ms: float = 0.0):
        """Testing hook (sem_set_barrier_test): shorten the team barrier limit and make one CTA
        leave the next launches before its first barrier; (-1, 0) restores normal launches."""
        _check(load_library().sem_set_barrier_test(self._h, int(drop_rank), ctypes.c_double(timeout_ms)))


class Batch:
    """Many meshes stepped or solved together (``sem_batch``): one fused launch per RK stage and order."""

    def __init__(self, meshes, tuned: bool = True):
        """tuned: hand the autotuner's measured planning parameters (tuning.json, if measured on
        this GPU) to the library before the first batch of the process."""
        lib = load_library()
        if tuned:
            from .autotune import apply_tuning
            apply_tuning(tiles=False)
        self.meshes = list(meshes)
        arr = (ctypes.c_void_p * len(self.meshes))(*[m._h.value for m in self.meshes])
        handle = ctypes.c_void_p()
        _check(lib.sem_batch_create(arr, len(self.meshes), ctypes.byref(handle)))
        self._h = handle

    def info(self):
        a, b = ctypes.c_int(), ctypes.c_int()
        _check(load_library().sem_batch_info(self._h, ctypes.byref(a), ctypes.byref(b)))
        return {"launches_per_stage": a.value, "ctas": b.value}

    def rk4_step(self, etas, phises, dts, nsteps: int = 1, ts=None):
        n = len(self.meshes)
        e = (ctypes.c_void_p * n)(*[_ptr(x).value for x in etas])
        p = (ctypes.c_void_p * n)(*[_ptr(x).value for x in phises])
        d = (ctypes.c_double * n)(*dts)
        t = (ctypes.c_double * n)(*(ts if ts is not None else [0.0] * n))
        _check(load_library().sem_batch_rk4_step(self._h, e, p, t, d, int(nsteps), _stream()))
        return list(t)

    def rk4_step_host(self, eta_h, phis_h, dts, nsteps: int = 1, ts=None):
        """sem_batch_rk4_step_host: eta_h, phis_h are packed host float64 arrays (instance i's
        columns after those of instances 0..i-1), numpy or pinned CPU tensors, updated in place."""
        def hp(a):
            if isinstance(a, np.ndarray):
                if a.dtype != np.float64 or not a.flags.c_contiguous:
                    raise ValueError("expected a contiguous float64 array")
                return a.ctypes.data_as(ctypes.c_void_p)
            return ctypes.c_void_p(a.data_ptr())
        n = len(self.meshes)
        d = (ctypes.c_double * n)(*dts)
        t = (ctypes.c_double * n)(*(ts if ts is not None else [0.0] * n))
        _check(load_library().sem_batch_rk4_step_host(self._h, hp(eta_h), hp(phis_h), t, d, int(nsteps),
                                                      _stream()))
        return list(t)

    def enable_timing(self, on: bool = True):
        _check(load_library().sem_batch_enable_timing(self._h, int(bool(on))))

    def timing(self) -> sem_timing:
        """Launches and summed device time (ms) of the stage launches since the last call."""
        t = sem_timing()
        _check(load_library().sem_batch_get_timing(self._h, ctypes.byref(t)))
        return t

    def laplace_solve(self, etas, phises, Phis):
        """One Laplace solve per instance (geometry rebuilt for etas[i]); Phis[i] in/out."""
        n = len(self.meshes)
        e = (ctypes.c_void_p * n)(*[_ptr(x).value for x in etas])
        p = (ctypes.c_void_p * n)(*[_ptr(x).value for x in phises])
        f = (ctypes.c_void_p * n)(*[_ptr(x).value for x in Phis])
        _check(load_library().sem_batch_laplace_solve(self._h, e, p, f, _stream()))
        return Phis

    def status(self) -> list[int]:
        """Per-instance SEM error codes of the last step or solve (0 = ok)."""
        c = (ctypes.c_int * len(self.meshes))()
        _check(load_library().sem_batch_status(self._h, c))
        return list(c)

    def close(self):
        if getattr(self, "_h", None):
            load_library().sem_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
