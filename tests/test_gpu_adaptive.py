"""GPU parity of the semi-adaptive real-axis grid (Sec. 3.3) against the oracle: the charge
integrand of one ring, the located peak and the refined grid, and the self-consistent loop
that refines its grid at the first iteration and every `period` iterations."""
import numpy as np
import pytest

from paper_2407_14633_gb300 import synth
from tests.cases import lib_device, oracle_device, rel_inf
from oracle import charge as ochg
from oracle import quadrature as oq
from oracle import selfconsistent as osc

pytestmark = pytest.mark.gpu

KT, ETA, E_B = 0.025, 1e-6, -10.0


@pytest.fixture(scope="module")
def ctx():
    from paper_2407_14633_gb300 import negf
    c = negf.Context()
    yield c
    c.close()


CASES = [("mode", 17, (6, 5), 36, False), ("mode", 17, (6,), 20, True), ("real", 17, (1,), 8, False)]


def _setup(ctx, kind, n_tube, modes, N, cells, limits, dens, V_DS=0.3):
    U = synth.ramp_barrier(N, drop=V_DS, height=0.15, width=N / 6.0)
    dev = lib_device(ctx, kind, n_tube, -2.7, N, 0.0, -V_DS, modes, cells)
    ctx.set_potential(dev, U)
    ctx.set_grid_adaptive(dev, 0.0, -V_DS, KT, ETA, E_B, 8, limits[0], limits[1], dens)
    od = oracle_device(kind, n_tube, -2.7, N, 0.0, -V_DS, modes, cells)
    g = oq.adaptive_grid(0.0, -V_DS, KT, limits[0], limits[1], dens, 8, E_B, ETA)
    return dev, od, U, g


@pytest.mark.parametrize("kind,n_tube,modes,N,cells", CASES)
def test_ring_integrand_matches_oracle(ctx, kind, n_tube, modes, N, cells):
    dev, od, U, g = _setup(ctx, kind, n_tube, modes, N, cells, (-0.45, -0.35), (1.0, 6.0, 0.5))
    assert ctx.grid_info(dev)["n_real"] == g["E"].size
    for ring in (0, N // 2, N - 1):
        I = ctx.ring_integrand(dev, ring)
        Iref = ochg.ring_integrand(od, U, g, ring)
        assert rel_inf(I, Iref) < 1e-10


@pytest.mark.parametrize("kind,n_tube,modes,N,cells", CASES)
def test_refined_grid_matches_oracle(ctx, kind, n_tube, modes, N, cells):
    dev, od, U, g = _setup(ctx, kind, n_tube, modes, N, cells, (-0.6, -0.1), (1.5, 6.0, 0.5))
    E_s = ctx.refine_grid(dev)
    Es_ref, k = ochg.singularity_peak(g["E"], ochg.ring_integrand(od, U, g, N // 2))
    assert abs(E_s - Es_ref) < 1e-12
    l1, l2 = oq.refined_limits(Es_ref, 3.0, 1.0, KT)
    g2 = oq.adaptive_grid(0.0, -0.3, KT, l1, l2, (1.5, 6.0, 0.5), 8, E_B, ETA)
    info = ctx.grid_info(dev)
    assert info["n_real"] == g2["E"].size
    assert abs(info["E_l1"] - g2["E_l1"]) < 1e-12 and abs(info["E_l2"] - g2["E_l2"]) < 1e-12
    # the refined grid evaluates like the oracle's
    r = ctx.compute([dev])[0]
    o = ochg.negf_evaluate(od, U, g2)
    assert rel_inf(r["n"], o["n"]) < 1e-10 and rel_inf(r["T"], o["T"]) < 1e-10


@pytest.mark.parametrize("period,M,tol", [(0, 64, 1e-9), (4, 14, 1e-12)])
def test_adaptive_sc_matches_oracle(ctx, period, M, tol):
    from paper_2407_14633_gb300 import negf
    N, V_DS, V_GS = 20, 0.3, 0.1
    dens, limits = (1.0, 8.0, 0.5), (-0.3, -0.2)
    dev = lib_device(ctx, "mode", 17, -2.7, N, 0.0, -V_DS, (6,))
    ctx.set_grid_adaptive(dev, 0.0, -V_DS, KT, ETA, E_B, 16, limits[0], limits[1], dens, period=period)
    U0 = np.linspace(0.0, -V_DS, N) + 0.05 * np.sin(np.arange(N))
    r = ctx.sc_solve(dev, V_DS, V_GS, U0, negf.poisson_kappa(), M=M, tol=tol, check=False)
    od = oracle_device("mode", 17, -2.7, N, 0.0, -V_DS, (6,))
    n0 = ochg.neutral_charge(od, 16, E_B)
    p = osc.PoissonParams(kappa=osc.kappa_from_geometry(), U_G=-V_GS, U_S=0.0, U_D=-V_DS)
    make = lambda l1, l2: oq.adaptive_grid(0.0, -V_DS, KT, l1, l2, dens, 16, E_B, ETA)
    o = osc.sc_solve_adaptive(lambda U, g: ochg.negf_evaluate(od, U, g),
                              lambda U, g: ochg.ring_integrand(od, U, g, N // 2),
                              make, U0, n0, p, limits, 3.0, 1.0, KT, period, M=M, tol=tol)
    assert r["converged"] == o["converged"] and r["iterations"] == o["iterations"]
    if period == 0:
        assert r["converged"]
    info = ctx.grid_info(dev)
    assert info["n_real"] == o["grid"]["E"].size
    assert abs(info["E_l1"] - o["grid"]["E_l1"]) < 1e-12 and abs(info["E_l2"] - o["grid"]["E_l2"]) < 1e-12
    assert rel_inf(r["n"], o["n"]) < 1e-9
    assert rel_inf(r["U"], o["U"]) < 1e-9
    assert rel_inf(r["T"], o["T"]) < 1e-8
    assert rel_inf(r["history"], np.array(o["history"])) < 1e-6


def test_adaptive_arguments_rejected(ctx):
    from paper_2407_14633_gb300 import negf
    dev = lib_device(ctx, "mode", 17, -2.7, 12, 0.0, 0.0, (6,))
    ctx.set_potential(dev, np.zeros(12))
    ctx.set_grid_spec(dev, 0.0, 0.0, KT, ETA, E_B, 16, 4)
    with pytest.raises(negf.NegfError) as e:
        ctx.refine_grid(dev)        # not a semi-adaptive grid
    assert e.value.status == negf.EINVAL
    for dens in ((0.0, 1.0, 1.0), (1.0, -2.0, 1.0), (1.0, float("nan"), 1.0)):
        with pytest.raises(negf.NegfError) as e:
            ctx.set_grid_adaptive(dev, 0.0, 0.0, KT, ETA, E_B, 4, -0.1, 0.0, dens)
        assert e.value.status == negf.EINVAL
    with pytest.raises(negf.NegfError) as e:
        ctx.set_grid_adaptive(dev, 0.0, 0.0, KT, ETA, E_B, 4, -0.1, 0.0, (1.0, 1.0, 1.0), ring=12)
    assert e.value.status == negf.EINVAL
    assert np.isnan(ctx.grid_info(dev)["E_l1"])
