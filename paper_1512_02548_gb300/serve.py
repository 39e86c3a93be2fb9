"""Continuous-batching request loop for wave-tank simulations and Laplace solves.

Requests arrive over time.  Each admitted request keeps its instance resident on the device
(mesh, σ-geometry, preconditioner, state and warm-start potential).  Waiting requests are
admitted in arrival order whenever the device-memory budget has room, so requests that arrive
while others run join the next tick.  One tick runs

* every newly admitted Laplace request: one fused launch per (order, precision) group
  (``sem_batch_laplace_solve``), after which the request completes;
* one RK4 step of every admitted RK4 request: one fused launch per RK stage and group
  (``sem_batch_rk4_step``); a request completes after its last step.

An instance's result does not depend on what else is in its batch (each instance has its own
CTA team, barriers and reductions).  A failing instance fails its own request only
(``sem_batch_status``); the others go on.  Latency = completion − arrival.

The scheduling core (:class:`Server`) does not touch the device: an executor owns the work
(:class:`GpuExecutor` runs it through the C ABI).
"""
from __future__ import annotations

import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Request:
    rid: int
    kind: str                 # "rk4" (nsteps RK4 steps of size wl.dt) or "laplace" (one solve)
    wl: object                # workload: mesh sizes, depth, filter, dt
    eta0: np.ndarray
    phis0: np.ndarray
    nsteps: int = 10
    arrival: float = 0.0      # seconds after the start of the run
    admitted: float | None = None
    finished: float | None = None
    error: str | None = None
    result: dict = field(default_factory=dict)


class GpuExecutor:
    """Device side of the loop: resident instances and batched calls through the C ABI.

    solo_nodes (off by default): a tick's requests of at least that many nodes, and a tick's only
    request, run on their mesh's own single-instance path (sem_rk4_step / sem_laplace_solve: one
    fused launch per RK stage over all SMs), one after another, and the rest as one batch.
    Measured on the C5 stream (two runs each, host tables warm), solo_nodes = 50 000 raised the p99
    latency at 100 requests/s (228–236 against 181–200 ms) and cut the throughput at 1000 requests/s
    (153 against 272 M DOF/s): the requests run alone no longer overlap with the batch."""

    def __init__(self, precision: str = "mixed", device: str = "cuda:0", tol: float | None = None,
                 solo_nodes: int | None = None):
        import torch
        import paper_1512_02548_gb300 as sem
        self.sem, self.torch = sem, torch
        self.dev = torch.device(device)
        self.precision = precision
        self.tol = tol if tol is not None else (1e-12 if precision == "mixed" else 1e-13)
        self.solo_nodes = solo_nodes
        self.slots: dict[int, dict] = {}
        self._batch = None
        self._batch_key = None
        self.stats = {"batch_create_s": 0.0, "batches_created": 0}   # host time spent building batches

    def _new_batch(self, meshes):
        t = time.perf_counter()
        b = self.sem.Batch(meshes)
        self.stats["batch_create_s"] += time.perf_counter() - t
        self.stats["batches_created"] += 1
        return b

    @staticmethod
    def _h(wl):
        return np.full(wl.ncol, wl.depth)

    def footprint(self, req: Request) -> int:
        """Mesh bytes (sem_mesh_footprint) plus the request's resident state."""
        sem, wl = self.sem, req.wl
        prm = sem.mesh_params(wl.P, wl.Nx, wl.Nz, wl.periodic, wl.Pf, wl.filter_alpha, wl.filter_s,
                              wl.filter_ic, wl.g, tol=self.tol, precision=self.precision)
        state = 2 * wl.ncol + (wl.n_nodes if req.kind == "laplace" else 0)
        return sem.mesh_footprint(prm, wl.element_edges(), self._h(wl)) + 8 * state

    def warm(self, requests) -> int:
        """Build the per-process host tables of every (order, layers, over-integration order,
        filter) combination among `requests` (a server's start-up step): the first mesh of a
        combination otherwise builds them at admission, in long double, which stalls the loop for
        up to tens of milliseconds on some hosts.  Returns the number of combinations."""
        seen = set()
        for r in requests:
            wl = r.wl
            key = (wl.P, wl.Nz, wl.Pf, wl.filter_alpha, wl.filter_s, wl.filter_ic)
            if key not in seen:
                seen.add(key)
                self.footprint(r)
        return len(seen)

    def admit(self, req: Request):
        torch, wl = self.torch, req.wl
        m = self.sem.Mesh.from_workload(wl, h=self._h(wl), precision=self.precision, tol=self.tol)
        slot = {"mesh": m, "eta": torch.as_tensor(req.eta0, dtype=torch.float64).to(self.dev),
                "phis": torch.as_tensor(req.phis0, dtype=torch.float64).to(self.dev),
                "t": 0.0, "left": req.nsteps, "dt": wl.dt}
        if req.kind == "laplace":
            slot["Phi"] = torch.zeros(m.n, dtype=torch.float64, device=self.dev)
        self.slots[req.rid] = slot

    def _batch_for(self, rids):
        key = tuple(rids)
        if key != self._batch_key:
            self._drop_batch()
            self._batch = self._new_batch([self.slots[r]["mesh"] for r in rids])
            self._batch_key = key
        return self._batch

    def _drop_batch(self):
        if self._batch is not None:
            self._batch.close()
        self._batch, self._batch_key = None, None

    def _run(self, b, call) -> list[int]:
        try:
            call()
        except self.sem.SemError:
            pass                     # per-instance codes below say which instances failed
        return b.status()

    def _split(self, rids) -> tuple[list[int], list[int]]:
        """(requests that run alone, requests that run as one batch)."""
        if self.solo_nodes is None:
            return [], list(rids)
        if len(rids) == 1:
            return list(rids), []
        solo = [r for r in rids if self.slots[r]["mesh"].n >= self.solo_nodes]
        rest = [r for r in rids if self.slots[r]["mesh"].n < self.solo_nodes]
        if len(rest) == 1:
            solo, rest = solo + rest, []
        return solo, rest

    def _alone(self, call) -> int:
        try:
            call()
            return 0
        except self.sem.SemError as ex:
            return ex.code

    def solve(self, rids) -> dict[int, int]:
        """Laplace solve of every listed request (large ones alone, the rest in one batched
        call); rid → error code."""
        solo, rest = self._split(rids)
        codes = {}
        for r in solo:
            s = self.slots[r]
            codes[r] = self._alone(lambda: (s["mesh"].update_geometry(s["eta"]),
                                            s["mesh"].laplace_solve(s["phis"], s["Phi"], stats=False)))
        if rest:
            b = self._new_batch([self.slots[r]["mesh"] for r in rest])
            try:
                sl = [self.slots[r] for r in rest]
                codes.update(zip(rest, self._run(b, lambda: b.laplace_solve(
                    [s["eta"] for s in sl], [s["phis"] for s in sl], [s["Phi"] for s in sl]))))
            finally:
                b.close()
        return codes

    def step(self, rids, nsteps: int = 1) -> dict[int, int]:
        """`nsteps` RK4 steps of every listed request (large ones alone, the rest in one batched
        call); rid → error code."""
        solo, rest = self._split(rids)
        codes = {}
        for r in solo:
            s = self.slots[r]
            codes[r] = self._alone(lambda: s["mesh"].rk4_step(s["eta"], s["phis"], s["dt"], nsteps, t=s["t"]))
        if rest:
            b = self._batch_for(rest)
            sl = [self.slots[r] for r in rest]
            codes.update(zip(rest, self._run(b, lambda: b.rk4_step(
                [s["eta"] for s in sl], [s["phis"] for s in sl], [s["dt"] for s in sl], nsteps,
                ts=[s["t"] for s in sl]))))
        for r in rids:
            s = self.slots[r]
            s["t"] += nsteps * s["dt"]
            s["left"] -= nsteps
        return codes

    def steps_left(self, rid) -> int:
        return self.slots[rid]["left"]

    def release(self, req: Request, keep_result: bool = True) -> dict:
        s = self.slots.pop(req.rid)
        if self._batch_key is not None and req.rid in self._batch_key:
            self._drop_batch()
        out = {}
        if keep_result:
            if req.kind == "laplace":
                out = {"Phi": s["Phi"].cpu().numpy()}
            else:
                out = {"eta": s["eta"].cpu().numpy(), "phis": s["phis"].cpu().numpy(), "t": s["t"]}
        s["mesh"].close()
        return out


class Server:
    """Budgeted admission in arrival order and one batched tick at a time."""

    def __init__(self, executor, hbm_budget: int, clock=time.perf_counter, sleep=time.sleep,
                 keep_results=True, max_steps_per_tick: int = 1):
        """keep_results: True (every request's result is copied back), False, or a set of
        request ids whose results are kept.  max_steps_per_tick > 1: while no request waits for
        admission, a tick may advance the RK4 requests by several steps in one batched call, up
        to the fewest steps any of them has left and to the steps that fit before the next
        arrival (at the measured time per step), so that a lightly loaded loop does not pay a
        tick per step; requests that arrive meanwhile join the next tick as before."""
        self.ex = executor
        self.budget = int(hbm_budget)
        self.clock = clock
        self.sleep = sleep
        self.keep = keep_results
        self.max_steps = max(1, int(max_steps_per_tick))

    def run(self, requests: list[Request], cancel: dict[int, float] | None = None) -> dict:
        """Serve ``requests``; ``cancel`` maps rid → time after which the request is dropped
        (waiting or running).  Returns latency and throughput figures; each request's
        ``result``, ``error`` and times are filled in."""
        reqs = sorted(requests, key=lambda r: (r.arrival, r.rid))
        cancel = dict(cancel or {})
        pending = deque(reqs)
        waiting: deque[Request] = deque()
        active: dict[int, Request] = {}
        fresh: list[int] = []          # admitted Laplace requests not yet solved
        used = 0
        fp: dict[int, int] = {}
        t0 = self.clock()
        ticks = peak_active = peak_bytes = 0
        per_step = 0.0                  # measured time of one RK4 step of a tick (running mean)
        phase = {"admit_s": 0.0, "solve_s": 0.0, "step_s": 0.0, "release_s": 0.0, "idle_s": 0.0}

        def finish(r: Request, error: str | None = None):
            nonlocal used
            tf = self.clock()
            r.error = error
            keep = self.keep if isinstance(self.keep, bool) else r.rid in self.keep
            r.result = self.ex.release(r, keep_result=keep and error is None)
            phase["release_s"] += self.clock() - tf
            r.finished = self.clock() - t0
            used -= fp[r.rid]
            del active[r.rid]

        while pending or waiting or active:
            now = self.clock() - t0
            while pending and pending[0].arrival <= now:
                waiting.append(pending.popleft())
            for rid, tc in list(cancel.items()):
                if tc > now:
                    continue
                del cancel[rid]
                if rid in active:
                    if rid in fresh:
                        fresh.remove(rid)
                    finish(active[rid], "cancelled")
                else:
                    for q in (waiting, pending):
                        for r in list(q):
                            if r.rid == rid:
                                q.remove(r)
                                r.error, r.finished = "cancelled", now
            ta = self.clock()
            while waiting:
                r = waiting[0]
                if r.rid not in fp:
                    fp[r.rid] = self.ex.footprint(r)
                if fp[r.rid] > self.budget:
                    waiting.popleft()
                    r.error, r.finished = "rejected: needs more device memory than the whole budget", now
                    continue
                if used + fp[r.rid] > self.budget:
                    break               # no overtaking: keeps arrival order fair
                waiting.popleft()
                self.ex.admit(r)
                r.admitted = self.clock() - t0
                used += fp[r.rid]
                active[r.rid] = r
                if r.kind == "laplace":
                    fresh.append(r.rid)
            phase["admit_s"] += self.clock() - ta
            peak_bytes = max(peak_bytes, used)
            if not active:
                if pending:
                    ti = self.clock()
                    self.sleep(max(0.0, min(pending[0].arrival - (self.clock() - t0), 0.05)))
                    phase["idle_s"] += self.clock() - ti
                continue
            peak_active = max(peak_active, len(active))
            if fresh:
                ts = self.clock()
                codes = self.ex.solve(fresh)
                phase["solve_s"] += self.clock() - ts
                for rid in fresh:
                    finish(active[rid], None if codes[rid] == 0 else f"error code {codes[rid]}")
                fresh = []
            rk = [rid for rid, r in active.items() if r.kind == "rk4"]
            if rk:
                k = 1
                if self.max_steps > 1 and not waiting:
                    k = min([self.max_steps] + [self.ex.steps_left(rid) for rid in rk])
                    if pending:
                        gap = pending[0].arrival - (self.clock() - t0)
                        k = max(1, min(k, int(gap / per_step))) if per_step > 0 else 1
                tk = self.clock()
                codes = self.ex.step(rk, k) if k > 1 else self.ex.step(rk)
                phase["step_s"] += self.clock() - tk
                dt_step = (self.clock() - tk) / k
                per_step = dt_step if per_step <= 0 else 0.5 * (per_step + dt_step)
                for rid in rk:
                    if codes[rid] != 0:
                        finish(active[rid], f"error code {codes[rid]}")
                    elif self.ex.steps_left(rid) <= 0:
                        finish(active[rid])
            ticks += 1
        wall = self.clock() - t0
        phase.update(getattr(self.ex, "stats", {}))
        return summarize(reqs, wall) | {"ticks": ticks, "peak_active": peak_active, "peak_bytes": peak_bytes,
                                        "host_phases": phase}


def laplace_dofs(r: Request) -> int:
    """Unknowns solved for a request: one solve, or four per RK4 step."""
    return r.wl.n_unknowns * (4 * r.nsteps if r.kind == "rk4" else 1)


def summarize(reqs: list[Request], wall: float) -> dict:
    ok = [r for r in reqs if r.error is None and r.finished is not None]
    lat = np.array([r.finished - r.arrival for r in ok]) if ok else np.zeros(1)
    return {"requests": len(reqs), "completed": len(ok), "failed": len(reqs) - len(ok), "wall_s": wall,
            "p50_ms": 1e3 * float(np.percentile(lat, 50)), "p99_ms": 1e3 * float(np.percentile(lat, 99)),
            "laplace_dof_per_s": sum(laplace_dofs(r) for r in ok) / wall,
            "rk4_steps_per_s": sum(r.nsteps for r in ok if r.kind == "rk4") / wall,
            "requests_per_s": len(ok) / wall}


def run_alone(req: Request, precision: str = "fp64", tol: float | None = None, device: str = "cuda:0") -> dict:
    """One request on the plain single-instance path (sem_update_geometry + sem_laplace_solve,
    or sem_rk4_step), with nothing else on the device."""
    import torch
    import paper_1512_02548_gb300 as sem
    wl = req.wl
    tol = tol if tol is not None else (1e-12 if precision == "mixed" else 1e-13)
    m = sem.Mesh.from_workload(wl, h=GpuExecutor._h(wl), precision=precision, tol=tol)
    try:
        eta = torch.as_tensor(req.eta0, dtype=torch.float64).to(device)
        phis = torch.as_tensor(req.phis0, dtype=torch.float64).to(device)
        if req.kind == "laplace":
            Phi = torch.zeros(m.n, dtype=torch.float64, device=device)
            m.update_geometry(eta)
            m.laplace_solve(phis, Phi)
            return {"Phi": Phi.cpu().numpy()}
        t = m.rk4_step(eta, phis, wl.dt, req.nsteps)
        return {"eta": eta.cpu().numpy(), "phis": phis.cpu().numpy(), "t": t}
    finally:
        m.close()


def sequential(requests: list[Request], precision: str = "fp64", clock=time.perf_counter,
               sleep=time.sleep) -> dict:
    """Baseline: the same requests one after another in arrival order on the plain
    single-instance path (no batching, no overlap across requests)."""
    reqs = sorted(requests, key=lambda r: (r.arrival, r.rid))
    t0 = clock()
    for r in reqs:
        now = clock() - t0
        if r.arrival > now:
            sleep(r.arrival - now)
        try:
            run_alone(r, precision)
            r.error = None
        except Exception as exc:        # a failed request is reported, not fatal
            r.error = str(exc)
        r.finished = clock() - t0
    return summarize(reqs, clock() - t0)
