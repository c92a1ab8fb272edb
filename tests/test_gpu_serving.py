"""Continuous batching of self-consistent solves: results alone vs in the mix, admission
under an HBM budget, cancellation, timeouts, and agreement with the single-solve loop."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

REQS = [(120, (6, 5), 0.1, 0.0), (200, (6, 5), 0.3, -0.2), (90, (6, 5), 0.0, 0.3), (150, (6,), 0.5, 0.1)]
TOL = 1e-6


def submit_all(ctx, reqs):
    return [ctx.submit(n, list(m), vds, vgs, n_real=192, n_cont=32, tol=TOL) for n, m, vds, vgs in reqs]


def test_mix_equals_alone_bitwise():
    from paper_2407_14633_gb300 import negf
    with negf.Context() as ctx:
        tks = submit_all(ctx, REQS)
        while any(ctx.poll(t) is None for t in tks):
            ctx.serve_step()
        mix = [ctx.poll(t) for t in tks]
    with negf.Context() as ctx:
        alone = [ctx.wait(ctx.submit(n, list(m), vds, vgs, n_real=192, n_cont=32, tol=TOL))
                 for n, m, vds, vgs in REQS]
    assert sum(a["converged"] for a in mix) >= 3
    for a, b in zip(mix, alone):
        assert a["status"] == b["status"] and a["converged"] == b["converged"]
        assert a["iterations"] == b["iterations"]
        assert np.array_equal(a["n"], b["n"]) and np.array_equal(a["U"], b["U"])
        assert a["I"] == b["I"]


def test_served_equals_single_solve_loop():
    from paper_2407_14633_gb300 import negf
    n, modes, vds, vgs = REQS[0]
    U0 = np.linspace(0.0, -vds, n) + 0.01 * np.sin(np.arange(n))
    with negf.Context() as ctx:
        r = ctx.wait(ctx.submit(n, list(modes), vds, vgs, n_real=192, n_cont=32, tol=TOL, U0=U0))
        dev = ctx.device_create(n, n_chains=len(modes))
        ctx.build_cnt_modespace(dev, 17, -2.7, list(modes), 0.0, -vds)
        E_B = -vds - 3 * 2.7 - 1.0
        ctx.set_grid_spec(dev, 0.0, -vds, 0.025, 1e-6, E_B, 192, 32)
        s = ctx.sc_solve(dev, vds, vgs, U0, negf.poisson_kappa(), M=64, tol=TOL, check=False)
    assert r["converged"] and s["converged"]
    assert r["status"] == s["status"] and r["iterations"] == s["iterations"]
    assert np.array_equal(r["n"], s["n"]) and np.array_equal(r["U"], s["U"])


def test_served_requests_match_oracle():
    """Two requests served together by continuous batching, each against the oracle's own loop
    (Alg. 3 with the 1D Poisson stand-in, Eq. GR leads, Alg. 1 / Alg. 2 as read) on the same
    inputs: the same iteration count, n and U within 1e-9, the current within 1e-9."""
    from paper_2407_14633_gb300 import negf
    from oracle import charge as ochg
    from oracle import model as omdl
    from oracle import quadrature as oq
    from oracle import selfconsistent as osc
    from tests.cases import rel_inf
    reqs = [(24, (6,), 0.2, 0.1), (30, (6, 5), 0.1, -0.1)]
    n_real, n_cont, E_B, tol = 48, 16, -10.0, 1e-9
    U0s = [np.linspace(0.0, -vds, n) + 0.02 * np.sin(np.arange(n)) for n, _, vds, _ in reqs]
    with negf.Context() as ctx:
        tks = [ctx.submit(n, list(m), vds, vgs, n_real=n_real, n_cont=n_cont, E_B=E_B, tol=tol, U0=U0)
               for (n, m, vds, vgs), U0 in zip(reqs, U0s)]
        while any(ctx.poll(t) is None for t in tks):
            ctx.serve_step()
        res = [ctx.poll(t) for t in tks]
    for (n, m, vds, vgs), U0, r in zip(reqs, U0s, res):
        dev = omdl.cnt_build("mode", 17, -2.7, n, 0.0, -vds, modes=m)
        grid = oq.bias_grid(0.0, -vds, 0.025, n_real, n_cont, E_B, 1e-6)
        n0 = ochg.neutral_charge(dev, n_cont, E_B)
        pp = osc.PoissonParams(kappa=osc.kappa_from_geometry(), U_G=-vgs, U_S=0.0, U_D=-vds)
        o = osc.sc_solve(lambda U: ochg.negf_evaluate(dev, U, grid), U0, n0, pp, zeta=0.1, M=64, tol=tol)
        assert r["converged"] and o["converged"]
        assert r["iterations"] == o["iterations"]
        assert rel_inf(r["n"], o["n"]) < 1e-9 and rel_inf(r["U"], o["U"]) < 1e-9
        assert abs(r["I"] - o["I"]) <= 1e-9 * max(abs(o["I"]), 1e-15)


def test_budget_admission_limits_active_slots():
    from paper_2407_14633_gb300 import negf
    # ~7 MB of per-request buffers and ~31 MB of sweep staging per resident block at N = 3000:
    # a 64 MB budget admits at most four at a time
    with negf.Context(hbm_budget=64 << 20) as ctx:
        tks = [ctx.submit(3000, [6, 5], 0.05 * i, 0.0, n_real=2048, n_cont=32, tol=1e-5) for i in range(6)]
        peak = 0
        while any(ctx.poll(t) is None for t in tks):
            peak = max(peak, ctx.serve_step())
        assert 1 <= peak < 6
        res = [ctx.poll(t) for t in tks]
        assert all(r is not None for r in res)
        # admission is in arrival order
        starts = [ctx.request_times(t)[1] for t in tks]
        assert starts == sorted(starts)


def test_cancel_and_timeout():
    from paper_2407_14633_gb300 import negf
    with negf.Context() as ctx:
        a = ctx.submit(200, [6], 0.2, 0.0, n_real=128, n_cont=16, tol=1e-12, M=64)
        b = ctx.submit(100, [6], 0.1, 0.0, n_real=128, n_cont=16, tol=TOL)
        ctx.serve_step()
        ctx.cancel(a)
        rb = ctx.wait(b)
        assert rb["converged"]
        with pytest.raises(negf.NegfError):
            ctx.poll(a)
        c = ctx.submit(300, [6, 5], 0.2, 0.0, n_real=256, n_cont=32, tol=1e-12, M=64)
        with pytest.raises(negf.NegfError) as e:
            ctx.wait(c, timeout_ms=1)
        assert e.value.status == negf.ETIMEDOUT
        ctx.cancel(c)
        ctx.serve_step()


def test_injected_allocation_failure_fails_one_request():
    from paper_2407_14633_gb300 import negf
    # host-side fault injection: an early arena allocation fails; the request reports an
    # error status and the context keeps serving
    with negf.Context(fault_alloc_after=3) as ctx:
        t1 = ctx.submit(100, [6], 0.1, 0.0, n_real=64, n_cont=16)
        ctx.serve_step()
        with pytest.raises(negf.NegfError) as e:
            ctx.wait(t1)
        assert e.value.status == negf.ENOMEM
        t2 = ctx.submit(100, [6], 0.1, 0.0, n_real=64, n_cont=16)
        assert ctx.wait(t2)["converged"]


def test_batched_uneven_devices_bitwise_and_parity():
    # uneven devices (ring counts, modes, 1x1 and 2x2 blocks, grid sizes) in one compute
    from paper_2407_14633_gb300 import negf, synth
    from tests.cases import rel_inf
    from oracle import charge as ochg
    from oracle import model as omdl
    from oracle import quadrature as oq
    w = synth.batched_uneven(n_devices=6, seed=3)
    with negf.Context() as ctx:
        devs = []
        for d in w["devices"]:
            N = min(d["N"], 160) // 2 * 2
            cells = d["block"] == 2
            dev = ctx.device_create(N, block=2 if cells else 1, rings_per_block=2 if cells else 1,
                                    n_chains=len(d["modes"]))
            ctx.build_cnt_modespace(dev, 17, w["t"], list(d["modes"]), 0.0, -d["V_DS"])
            ctx.set_potential(dev, d["U"][:N])
            ctx.set_grid_spec(dev, 0.0, -d["V_DS"], w["kT"], w["eta"], d["E_B"], min(d["n_real"], 97), 33)
            devs.append((dev, d, N, cells))
        batch = ctx.compute([x[0] for x in devs])
        for (dev, d, N, cells), rb in zip(devs, batch):
            ra = ctx.compute([dev])[0]
            assert np.array_equal(ra["n"], rb["n"]) and np.array_equal(ra["T"], rb["T"])
            od = omdl.cnt_build("mode", 17, w["t"], N, 0.0, -d["V_DS"], modes=d["modes"], cells=cells)
            g = oq.bias_grid(0.0, -d["V_DS"], w["kT"], min(d["n_real"], 97), 33, d["E_B"], w["eta"])
            o = ochg.negf_evaluate(od, d["U"][:N], g)
            assert rel_inf(rb["n"], o["n"]) < 1e-10
            assert rel_inf(rb["T"], o["T"]) < 1e-10
