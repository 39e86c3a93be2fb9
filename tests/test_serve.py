"""Scheduling logic of the continuous-batching loop, on the host with a stand-in executor.

The stand-in charges a fixed time per call on a simulated clock, so arrival, admission and
completion times are exact.  Checked: every request completes once; admission follows arrival
order and never overtakes; device bytes in use never exceed the budget; requests that arrive
while others run join the next tick (continuous batching, not a queue); a request above the
whole budget is rejected without blocking the others; a failure or a cancellation ends one
request only.
"""
import math

import numpy as np
import pytest

from paper_1512_02548_gb300.serve import Request, Server, summarize
from sem_workloads import c5_requests


class Clock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def sleep(self, dt):
        self.t += max(dt, 1e-6)


class FakeExecutor:
    """Charges tick_s per batched call; an instance whose η holds a NaN fails."""

    def __init__(self, clock, tick_s=1e-3, bytes_per_node=1000):
        self.clock, self.tick_s, self.bpn = clock, tick_s, bytes_per_node
        self.slots, self.admitted, self.batches, self.calls = {}, [], [], []

    def footprint(self, r):
        return r.wl.n_nodes * self.bpn

    def admit(self, r):
        self.slots[r.rid] = {"left": r.nsteps, "bad": bool(np.isnan(r.eta0).any()), "steps": 0}
        self.admitted.append(r.rid)

    def solve(self, rids):
        self.clock.t += self.tick_s
        self.calls.append(("solve", tuple(rids)))
        return {r: (5 if self.slots[r]["bad"] else 0) for r in rids}

    def step(self, rids, nsteps=1):
        self.clock.t += self.tick_s * nsteps
        self.calls.append(("step", tuple(rids), nsteps))
        out = {}
        for r in rids:
            s = self.slots[r]
            assert s["left"] >= nsteps           # no request is stepped past its end
            s["left"] -= nsteps
            s["steps"] += nsteps
            out[r] = 5 if s["bad"] else 0
        return out

    def steps_left(self, rid):
        return self.slots[rid]["left"]

    def release(self, r, keep_result=True):
        s = self.slots.pop(r.rid)
        return {"steps": s["steps"]} if keep_result else {}


def requests(rate=2000.0, count=60, seed=0, nsteps=10):
    out = []
    for i, (kind, t, wl, ns) in enumerate(c5_requests(rate, count, seed, nmin=1e3, nmax=2e4, nsteps=nsteps)):
        eta = np.zeros(wl.ncol)
        out.append(Request(i, kind, wl, eta, eta.copy(), ns, t))
    return out


def serve(reqs, budget, tick_s=1e-3, cancel=None):
    clk = Clock()
    ex = FakeExecutor(clk, tick_s)
    srv = Server(ex, budget, clock=clk, sleep=clk.sleep)
    summary = srv.run(reqs, cancel=cancel)
    return ex, summary


def test_c5_request_stream_matches_its_recipe():
    r = c5_requests(100.0, 2000, 0)
    assert len(r) == 2000
    t = np.array([x[1] for x in r])
    assert np.all(np.diff(t) > 0)
    gaps = np.diff(np.r_[0.0, t])
    assert abs(gaps.mean() - 1 / 100.0) < 0.1 / 100.0       # Poisson at 100/s
    kinds = [x[0] for x in r]
    assert 900 < kinds.count("laplace") < 1100
    for kind, _, wl, ns in r:
        assert 4 <= wl.P <= 10 and wl.Nz in (1, 2, 4) and wl.Nx >= 2 and wl.periodic
        assert ns == (10 if kind == "rk4" else 0)
        assert 0.5 <= wl.depth <= 3.0 and wl.Pf == (3 * wl.P + 1) // 2
        # stable explicit step: at most T/200, and short waves on the finest GLL spacing
        # resolved within half of RK4's imaginary-axis limit
        T = 2 * math.pi / math.sqrt(9.81 * math.tanh(wl.depth))
        dx_min = 0.5 * (wl.length / wl.Nx) * (1 - math.cos(math.pi / wl.P))
        assert wl.dt <= T / 200 * (1 + 1e-12)
        assert math.sqrt(9.81 * math.pi / dx_min) * wl.dt <= 1.4 * (1 + 1e-12)
        # Courant number ≤ ½ for the surface velocity of linear theory at the crest
        H, k, h = wl.wave_height, wl.wavenumber, wl.depth
        om = math.sqrt(9.81 * k * math.tanh(k * h))
        u = 9.81 * H * k / (2 * om) * math.cosh(k * (h + H / 2)) / math.cosh(k * h)
        assert u * wl.dt / dx_min <= 0.5
    n = np.array([x[2].n_nodes for x in r])
    assert n.min() > 500 and n.max() < 2.5e5
    # node counts log-uniform: median near the geometric mean of the range
    assert abs(math.log(np.median(n)) - 0.5 * (math.log(1e3) + math.log(2e5))) < 0.3


def test_every_request_completes_once_in_arrival_order():
    reqs = requests()
    ex, s = serve(reqs, budget=1 << 60)
    assert s["completed"] == len(reqs) and s["failed"] == 0
    assert ex.admitted == [r.rid for r in sorted(reqs, key=lambda r: r.arrival)]
    for r in reqs:
        assert r.admitted >= r.arrival and r.finished >= r.admitted
        if r.kind == "rk4":
            assert r.result["steps"] == r.nsteps
    # each Laplace request is in exactly one solve call, each RK4 request in exactly nsteps steps
    solved = [rid for c in ex.calls if c[0] == "solve" for rid in c[1]]
    stepped = [rid for c in ex.calls if c[0] == "step" for rid in c[1]]
    assert sorted(solved) == sorted(r.rid for r in reqs if r.kind == "laplace")
    for r in reqs:
        if r.kind == "rk4":
            assert stepped.count(r.rid) == r.nsteps


def test_requests_arriving_while_others_run_join_the_next_tick():
    reqs = requests(rate=5000.0, count=40)
    ex, s = serve(reqs, budget=1 << 60, tick_s=2e-3)
    steps = [c[1] for c in ex.calls if c[0] == "step"]
    assert max(len(x) for x in steps) > 1           # batched across requests
    # some RK4 request was admitted while another RK4 request was part-way through its steps
    joined = False
    for i in range(1, len(steps)):
        new = set(steps[i]) - set(steps[i - 1])
        if new and set(steps[i]) & set(steps[i - 1]):
            joined = True
    assert joined
    # with an idle device, a request waits at most one tick before admission
    for r in reqs:
        assert r.admitted - r.arrival <= 2e-3 * 2 + 1e-9


def test_budget_is_never_exceeded_and_limits_concurrency():
    reqs = requests(rate=20000.0, count=50)
    biggest = max(r.wl.n_nodes for r in reqs) * 1000
    budget = 2 * biggest
    clk = Clock()
    ex = FakeExecutor(clk)
    in_use = []
    orig_admit, orig_release = ex.admit, ex.release

    def admit(r):
        orig_admit(r)
        in_use.append(sum(ex.footprint(q) for q in reqs if q.rid in ex.slots))

    ex.admit = admit
    s = Server(ex, budget, clock=clk, sleep=clk.sleep).run(reqs)
    assert s["completed"] == len(reqs)
    assert max(in_use) <= budget and s["peak_bytes"] <= budget
    # the order of admission is still the order of arrival (no overtaking by small requests)
    assert ex.admitted == [r.rid for r in sorted(reqs, key=lambda r: r.arrival)]
    del orig_release


def test_request_above_the_whole_budget_is_rejected_alone():
    reqs = requests(count=20)
    big = max(reqs, key=lambda r: r.wl.n_nodes)
    budget = big.wl.n_nodes * 1000 - 1
    small = [r for r in reqs if r.wl.n_nodes * 1000 <= budget]
    ex, s = serve(reqs, budget)
    assert big.error and big.error.startswith("rejected")
    assert all(r.error is None for r in small)
    assert s["completed"] == len(reqs) - sum(1 for r in reqs if r.wl.n_nodes * 1000 > budget)


def test_failed_instance_fails_only_its_request():
    reqs = requests(count=30)
    bad = [r for r in reqs if r.kind == "rk4"][2]
    bad.eta0 = bad.eta0.copy()
    bad.eta0[0] = np.nan
    ex, s = serve(reqs, budget=1 << 60)
    assert bad.error == "error code 5"
    assert all(r.error is None for r in reqs if r is not bad)
    assert s["failed"] == 1


def test_cancellation_of_a_running_and_a_waiting_request():
    reqs = requests(rate=50000.0, count=12)
    rk = [r for r in reqs if r.kind == "rk4"]
    running, waiting = rk[0], rk[-1]
    budget = sum(r.wl.n_nodes * 1000 for r in reqs if r.rid <= running.rid)
    cancel = {running.rid: running.arrival + 2.5e-3, waiting.rid: 0.0}
    ex, s = serve(reqs, budget, cancel=cancel)
    assert running.error == "cancelled" and waiting.error == "cancelled"
    assert waiting.rid not in ex.admitted
    assert all(r.error is None for r in reqs if r not in (running, waiting))
    assert s["completed"] == len(reqs) - 2


def test_summary_latency_and_throughput():
    reqs = requests(count=10)
    for k, r in enumerate(reqs):
        r.arrival, r.finished, r.error = 0.0, 0.01 * (k + 1), None
    s = summarize(reqs, wall=0.1)
    assert s["p50_ms"] == pytest.approx(1e3 * np.percentile(0.01 * np.arange(1, 11), 50))
    assert s["p99_ms"] == pytest.approx(1e3 * np.percentile(0.01 * np.arange(1, 11), 99))
    dofs = sum(r.wl.n_unknowns * (40 if r.kind == "rk4" else 1) for r in reqs)
    assert s["laplace_dof_per_s"] == pytest.approx(dofs / 0.1)


def test_multi_step_ticks_when_nothing_waits():
    """With max_steps_per_tick, a lightly loaded loop advances its RK4 requests by several steps
    per call, never past a request's last step, and only while no request waits for admission;
    every request still gets exactly its steps."""
    reqs = requests(rate=50.0, count=40)
    clk = Clock()
    ex = FakeExecutor(clk, 1e-3)
    s = Server(ex, 1 << 60, clock=clk, sleep=clk.sleep, max_steps_per_tick=8).run(reqs)
    assert s["completed"] == len(reqs) and s["failed"] == 0
    for r in reqs:
        if r.kind == "rk4":
            assert r.result["steps"] == r.nsteps
    multi = [c for c in ex.calls if c[0] == "step" and c[2] > 1]
    assert multi and all(c[2] <= 8 for c in multi)
    one = serve(requests(rate=50.0, count=40), budget=1 << 60)[0]
    assert sum(1 for c in ex.calls if c[0] == "step") < sum(1 for c in one.calls if c[0] == "step")


def test_host_phase_times_add_up_to_at_most_the_wall_time():
    """The loop reports where its host time went (admission, solves, steps, release, idle); with a
    simulated clock the phases are non-negative and their sum does not exceed the wall time."""
    reqs = requests(rate=200.0, count=30)
    clk = Clock()
    ex = FakeExecutor(clk, 2e-3)
    s = Server(ex, 1 << 60, clock=clk, sleep=clk.sleep).run(reqs)
    ph = s["host_phases"]
    keys = ("admit_s", "solve_s", "step_s", "release_s", "idle_s")
    assert all(ph[k] >= 0.0 for k in keys)
    assert ph["step_s"] > 0.0 and ph["solve_s"] > 0.0
    assert sum(ph[k] for k in keys) <= s["wall_s"] + 1e-9
