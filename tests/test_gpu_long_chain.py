"""GPU parity of the sweep split along the channel (1 x 1 chains of many layers and few
energies): the CUDA path through the C ABI against the FP64 oracle on long and ragged chains,
against the unsplit sweep, and its invariances (batch, waves under a memory budget, the
self-consistent loop replayed from a captured graph)."""
import numpy as np
import pytest

from paper_2407_14633_gb300 import synth
from tests.cases import case_params, current_err, rel_inf, run_lib, run_oracle, lib_device, lib_grid

pytestmark = pytest.mark.gpu
TOL = 1e-10


def _ctx(**kw):
    from paper_2407_14633_gb300 import negf
    return negf.Context(**kw)


def run_counted(ctx, p):
    """run_lib with the kernel launches of the evaluation itself counted."""
    dev = lib_device(ctx, p["kind"], p["n_tube"], p["t"], p["N"], p["U_S"], p["U_D"], p["modes"], p["cells"])
    ctx.set_potential(dev, p["U"])
    lib_grid(ctx, dev, p)
    n0 = ctx.launch_count()
    r = ctx.compute([dev])[0]
    return r, ctx.launch_count() - n0


def check(p, r, o, tol=TOL):
    assert rel_inf(r["n"], o["n"]) < tol, rel_inf(r["n"], o["n"])
    assert rel_inf(r["n_cont"], o["n_cont"]) < tol, rel_inf(r["n_cont"], o["n_cont"])
    if p["n_real"]:
        assert rel_inf(r["T"], o["T"]) < tol, rel_inf(r["T"], o["T"])
        g = 2.0 * 2.0 * len(p["modes"])
        assert current_err(r["I"], o["I"], g, p["mu_S"] - p["mu_D"]) < tol


@pytest.mark.parametrize("N,modes,n_real,n_cont", [(20000, (6,), 40, 20), (16384 + 300, (6, 5), 45, 7)])
def test_long_chain_matches_oracle(N, modes, n_real, n_cont):
    # long enough and few enough energies for the split sweep under the default rule; the
    # second case ends on a ragged segment of 300 layers and a ragged 13-energy item
    U = synth.ramp_barrier(N)
    p = case_params("mode", N, n_real, n_cont, U, modes=modes)
    with _ctx() as ctx:
        r, launches = run_counted(ctx, p)
    # prep, five launches of the one wave of split items, second stage: no thread-per-lane sweep
    assert launches == 7
    check(p, r, run_oracle(p))


@pytest.mark.parametrize("N,n_real,n_cont", [(1, 33, 5), (2, 31, 1), (37, 45, 7), (512, 64, 0), (513, 20, 3),
                                             (1100, 97, 32)])
def test_forced_split_ragged_sizes(N, n_real, n_cont):
    # every 1 x 1 chain split: one layer, one partial segment, a full segment plus one layer
    U = synth.ramp_barrier(N) if N > 1 else np.array([0.05])
    p = case_params("mode", N, n_real, n_cont, U, modes=(6,))
    if n_cont == 0:
        p["n_cont"] = 0
    with _ctx(long_chain_split=1) as ctx:
        _, r = run_lib(ctx, p)
    check(p, r, run_oracle(p))


def test_split_agrees_with_unsplit_sweep():
    N = 20000
    U = synth.ramp_barrier(N, drop=0.3, height=0.15)
    p = case_params("mode", N, 64, 32, U, mu_D=-0.3, modes=(6, 5))
    out = []
    for mode in (0, -1):
        with _ctx(long_chain_split=mode) as ctx:
            _, r = run_lib(ctx, p)
            out.append(r)
    a, b = out
    assert rel_inf(a["n"], b["n"]) < TOL
    assert rel_inf(a["T"], b["T"]) < TOL
    assert abs(a["I"] - b["I"]) <= TOL * abs(b["I"])


def test_split_device_is_bitwise_alone_and_in_a_batch():
    # the split rule looks at the device alone: batching it with a short device changes nothing
    N = 17000
    p = case_params("mode", N, 40, 16, synth.ramp_barrier(N), modes=(6,))
    q = case_params("mode", 300, 70, 20, synth.ramp_barrier(300), modes=(5,))
    with _ctx() as ctx:
        d1, r1 = run_lib(ctx, p)
        d2, r2 = run_lib(ctx, q)
        both = ctx.compute([d2, d1])
    for k in ("n", "T"):
        assert np.array_equal(both[1][k], r1[k])
        assert np.array_equal(both[0][k], r2[k])
    assert both[1]["I"] == r1["I"] and both[0]["I"] == r2["I"]


def test_waves_under_a_budget_are_bitwise_equal():
    # a budget too small for the staging of all split items at once runs them in waves
    N = 20000
    p = case_params("mode", N, 64, 32, synth.ramp_barrier(N), modes=(6,))
    with _ctx() as ctx:
        ref, one_wave = run_counted(ctx, p)
    from paper_2407_14633_gb300 import negf
    done = False
    for mb in range(24, 48, 2):
        try:
            with _ctx(hbm_budget=mb * 1000 * 1000) as ctx:
                r, launches = run_counted(ctx, p)
        except negf.NegfError as e:
            assert e.status == negf.ENOMEM
            continue
        if launches > one_wave:
            done = True
            assert (launches - one_wave) % 5 == 0
            for k in ("n", "T", "n_cont"):
                assert np.array_equal(r[k], ref[k])
            assert r["I"] == ref["I"]
            break
    assert done


def test_budget_below_one_split_item_is_refused():
    from paper_2407_14633_gb300 import negf
    N = 20000
    p = case_params("mode", N, 64, 32, synth.ramp_barrier(N), modes=(6,))
    with _ctx(hbm_budget=8 * 1000 * 1000) as ctx:
        with pytest.raises(negf.NegfError) as e:
            run_lib(ctx, p)
        assert e.value.status == negf.ENOMEM


def test_split_self_consistent_loop_matches_oracle():
    # the self-consistent loop replays its iteration from a captured graph, split launches included
    from tests.test_gpu_selfconsistent import oracle_solve
    from paper_2407_14633_gb300 import negf
    N, V_DS, V_GS = 40, 0.2, 0.1
    n_real, n_cont, E_B = 48, 16, -10.0
    U0 = np.linspace(0.0, -V_DS, N) + 0.02 * np.sin(np.arange(N))
    with _ctx(long_chain_split=1) as ctx:
        dev = lib_device(ctx, "mode", 17, -2.7, N, 0.0, -V_DS, (6, 5))
        ctx.set_grid_spec(dev, 0.0, -V_DS, 0.025, 1e-6, E_B, n_real, n_cont)
        r = ctx.sc_solve(dev, V_DS, V_GS, U0, negf.poisson_kappa(), zeta=0.1, M=64, tol=1e-9)
    o = oracle_solve("mode", 17, (6, 5), N, V_DS, V_GS, U0, n_real, n_cont, E_B, 0.1, 64, 1e-9)
    assert r["converged"] and o["converged"]
    assert r["iterations"] == o["iterations"]
    assert rel_inf(r["n"], o["n"]) < 1e-9
    assert rel_inf(r["U"], o["U"]) < 1e-9


def test_split_ring_integrand_and_conductance():
    # the refinement ring's integrand (captured inside the backward re-run) and the zero-bias
    # conductance (real-axis lanes only) against the unsplit sweep
    N = 1100
    U = synth.ramp_barrier(N)
    out = []
    for mode in (1, -1):
        with _ctx(long_chain_split=mode) as ctx:
            dev = lib_device(ctx, "mode", 17, -2.7, N, float(U[0]), float(U[-1]), (6,))
            ctx.set_potential(dev, U)
            ctx.set_grid_spec(dev, 0.0, -0.1, 0.025, 1e-6, -10.0, 96, 16)
            ring = ctx.ring_integrand(dev, 700)
            G = ctx.conductance([dev], -1.0, 0.025)
            out.append((np.asarray(ring), np.asarray(G)))
    assert rel_inf(out[0][0], out[1][0]) < TOL
    assert rel_inf(out[0][1], out[1][1]) < TOL


def test_invalid_split_option_rejected():
    from paper_2407_14633_gb300 import negf
    for bad in (2, -2):
        with pytest.raises(negf.NegfError):
            _ctx(long_chain_split=bad)
