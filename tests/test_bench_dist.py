"""Multi-rank timing harness of bench.py on CPU (gloo, world size 2).

The benchmark runs one independent replica of the tank per rank (weak scaling, no
collective on the data path); the only communication is the barrier and the max of the
per-rank times.  These tests run that harness on two gloo ranks and check that rank 0
reports the whole-job throughput from the slowest rank, and that the reference arm exits
without work on ranks other than 0.
"""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    dist.barrier()
    local_ms = 100.0 + 50.0 * rank          # rank 1 is the slow one
    t_max = bench.max_over_ranks(local_ms)
    value = bench.job_throughput(world, 10, 4 * 9216, t_max)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, t_max, value))


def test_two_rank_max_time_and_job_throughput():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = dict((r, (t, v)) for r, t, v in (q.get(timeout=10) for _ in range(2)))
    for r in (0, 1):
        assert res[r][0] == 150.0
        assert res[r][1] == pytest.approx(2 * 10 * 4 * 9216 / 0.150)


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "3"], env=env, capture_output=True, text=True, timeout=120)
    assert out.returncode == 0 and out.stdout.strip() == ""


def test_c3_sample_is_seeded_and_distinct():
    sys.path.insert(0, ROOT)
    import bench
    a, b = bench.c3_sample(32), bench.c3_sample(32)
    assert a == b and len(set(a)) == 32 and all(0 <= i < 512 for i in a)
    assert bench.c3_sample(8) == a[:8]


def test_oracle_pool_runs_one_step_per_tank():
    """The spawned oracle pool of the cpu_baseline and the reference arm: one RK4 step of two small
    C3 tanks, each equal to the oracle run in this process, with four Laplace solves per tank."""
    import numpy as np
    sys.path.insert(0, ROOT)
    import bench
    from oracle import sem as osem
    from sem_workloads import c3_instances
    wls = c3_instances(512)
    small = sorted(range(512), key=lambda i: wls[i].n_unknowns)[:2]
    pool = bench.oracle_pool(2)
    try:
        res = pool.map(bench.oracle_job, [("c3", i, *bench.c3_initial(i), 1, 0.0) for i in small])
    finally:
        pool.close()
        pool.join()
    for i, (key, (eta, phis), secs, dof) in zip(small, res):
        wl = wls[i]
        assert key == i and dof == 4 * wl.n_unknowns and secs > 0
        om = osem.mesh_for(wl, h_col=np.full(wl.ncol, wl.depth))
        e, p = om.rk4_step(*bench.c3_initial(i), wl.dt)
        assert np.array_equal(e, eta) and np.array_equal(p, phis)
