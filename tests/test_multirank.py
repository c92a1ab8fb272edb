"""The multi-GPU path of bench.py on CPU: two gloo ranks (world size 2) run the rank logic of
the replicas-only scaling (one bias point per rank, no data-path collective, the job's step
time is the slowest rank's).  No GPU is touched."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        ms = 100.0 + 10.0 * rank          # ranks finish at different times
        t_max = bench.max_over_ranks(ms, world)
        value = bench.job_value(1000, world, t_max)
        out[rank] = (bench.rank_gate_voltage(rank), t_max, value)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_step_and_distinct_bias_points():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert set(res) == {0, 1}
    vgs = [res[r][0] for r in range(world)]
    assert len(set(vgs)) == world                      # independent problems per rank
    assert all(res[r][1] == 110.0 for r in range(world))   # the slowest rank's time
    assert all(abs(res[r][2] - world * 1000 / 0.110) < 1e-6 for r in range(world))


def _evaluate(V_GS):
    """One NEGF evaluation of a small mode-space tube whose channel the gate lowers by V_GS
    (the oracle, since no GPU is touched here)."""
    import numpy as np
    from oracle import charge as ochg
    from oracle import model as omdl
    from oracle import quadrature as oq
    N = 16
    dev = omdl.cnt_build("mode", 17, -2.7, N, 0.0, -0.1, modes=(6,))
    U = np.linspace(0.0, -0.1, N) - V_GS * np.sin(np.pi * (np.arange(N) + 0.5) / N)
    grid = oq.bias_grid(0.0, -0.1, 0.025, 24, 8, -10.0, 1e-6)
    return ochg.negf_evaluate(dev, U, grid)


def _rank_eval(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import time
        import bench
        V_GS = bench.rank_gate_voltage(rank)
        t0 = time.perf_counter()
        r = _evaluate(V_GS)
        ms = (time.perf_counter() - t0) * 1e3
        out[rank] = (V_GS, list(r["n"]), r["I"], ms, bench.max_over_ranks(ms, world))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_each_evaluate_their_own_bias_point():
    """Each rank evaluates the problem of its own gate voltage with nothing exchanged but the
    step time: its results are those of the same evaluation in one process, the ranks' results
    differ, and both ranks report the slower rank's time."""
    import numpy as np
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_eval, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert set(res) == {0, 1}
    for r in range(world):
        V_GS, n, I, ms, t_max = res[r]
        alone = _evaluate(V_GS)
        assert np.array_equal(np.asarray(n), alone["n"]) and I == alone["I"]
        assert t_max == max(res[q][3] for q in range(world))
    assert not np.array_equal(np.asarray(res[0][1]), np.asarray(res[1][1]))


def test_single_rank_needs_no_collective():
    import bench
    assert bench.max_over_ranks(12.5, 1) == 12.5
    assert bench.job_value(10, 1, 1000.0) == 10.0
