"""GPU parity of the zero-bias conductance (Eq. zeroBiasG) against the oracle, on the same
seeded devices: single evaluations (mode space, 2 x 2 cells, real space), batch invariance,
and a warm-started gate sweep of self-consistent solves."""
import numpy as np
import pytest

from paper_2407_14633_gb300 import synth
from tests.cases import lib_device, oracle_device, rel_inf
from oracle import charge as ochg
from oracle import quadrature as oq
from oracle import selfconsistent as osc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2407_14633_gb300 import negf
    c = negf.Context()
    yield c
    c.close()


CASES = [("mode", 17, (6, 5), 40, False), ("mode", 17, (6,), 24, True), ("real", 17, (1,), 9, False)]


@pytest.mark.parametrize("kind,n_tube,modes,N,cells", CASES)
@pytest.mark.parametrize("mu", [0.0, 0.31, -0.55])
def test_conductance_matches_oracle(ctx, kind, n_tube, modes, N, cells, mu):
    kT, n_real = 0.025, 72
    U = synth.ramp_barrier(N, drop=0.0, height=0.15, width=N / 6.0)
    dev = lib_device(ctx, kind, n_tube, -2.7, N, 0.0, 0.0, modes, cells)
    ctx.set_potential(dev, U)
    ctx.set_grid_spec(dev, mu, mu, kT, 1e-6, -10.0, n_real, 8)
    G, (T,) = ctx.conductance([dev], mu, kT, want_T=True)
    od = oracle_device(kind, n_tube, -2.7, N, 0.0, 0.0, modes, cells)
    g = oq.bias_grid(mu, mu, kT, n_real, 8, -10.0, 1e-6)
    r = ochg.negf_evaluate(od, U, g)
    G_ref = ochg.zero_bias_conductance(r["T"], g["E"], g["w"], mu, kT)
    assert rel_inf(T, r["T"]) < 1e-10
    assert abs(G[0] - G_ref) <= 1e-10 * abs(G_ref)


def test_conductance_batch_is_bitwise_alone(ctx):
    devs = []
    for kind, n_tube, modes, N, cells in CASES:
        d = lib_device(ctx, kind, n_tube, -2.7, N, 0.0, 0.0, modes, cells)
        ctx.set_potential(d, synth.ramp_barrier(N, drop=0.0, height=0.1, width=3.0))
        ctx.set_grid_spec(d, 0.2, 0.2, 0.025, 1e-6, -10.0, 40, 8)
        devs.append(d)
    batch = ctx.conductance(devs, 0.2, 0.025)
    for i, d in enumerate(devs):
        alone = ctx.conductance([d], 0.2, 0.025)
        assert alone[0] == batch[i]


def test_gate_sweep_matches_oracle(ctx):
    # warm-started sweep of zero-bias solves, then G on each converged state
    from paper_2407_14633_gb300 import negf
    w = synth.gate_sweep(N=24, n_points=3, v_lo=-0.5, v_hi=1.5, n_real=48, n_cont=16)
    N, kT, mu = w["N"], w["kT"], w["mu"]
    dev = lib_device(ctx, "mode", w["n_tube"], w["t"], N, 0.0, 0.0, w["modes"])
    ctx.set_grid_spec(dev, mu, mu, kT, w["eta"], w["E_B"], w["n_real"], w["n_cont"])
    od = oracle_device("mode", w["n_tube"], w["t"], N, 0.0, 0.0, w["modes"])
    g = oq.bias_grid(mu, mu, kT, w["n_real"], w["n_cont"], w["E_B"], w["eta"])
    n0 = ochg.neutral_charge(od, w["n_cont"], w["E_B"])
    U_lib = np.zeros(N)
    U_ora = np.zeros(N)
    Gs = []
    for v in w["V_GS"]:
        r = ctx.sc_solve(dev, 0.0, float(v), U_lib, negf.poisson_kappa(), M=64, tol=1e-10)
        G = ctx.conductance([dev], mu, kT)[0]
        p = osc.PoissonParams(kappa=osc.kappa_from_geometry(), U_G=-float(v), U_S=0.0, U_D=0.0)
        o = osc.sc_solve(lambda U: ochg.negf_evaluate(od, U, g), U_ora, n0, p, zeta=0.1, M=64, tol=1e-10)
        G_ref = ochg.zero_bias_conductance(o["T"], g["E"], g["w"], mu, kT)
        assert r["converged"] and o["converged"] and r["iterations"] == o["iterations"]
        assert rel_inf(r["U"], o["U"]) < 1e-9
        assert abs(G - G_ref) <= 1e-8 * abs(G_ref)
        Gs.append(G)
        U_lib, U_ora = r["U"], o["U"]
    # the gate moves the channel bands: every point gives its own conductance
    assert len(set(Gs)) == len(Gs)


def test_conductance_rejects_bad_arguments(ctx):
    from paper_2407_14633_gb300 import negf
    dev = lib_device(ctx, "mode", 17, -2.7, 12, 0.0, 0.0, (6,))
    ctx.set_potential(dev, np.zeros(12))
    ctx.set_grid_spec(dev, 0.0, 0.0, 0.025, 1e-6, -10.0, 16, 4)
    for bad in ((0.0, 0.0), (float("nan"), 0.025), (0.0, -0.01)):
        with pytest.raises(negf.NegfError) as e:
            ctx.conductance([dev], *bad)
        assert e.value.status == negf.EINVAL
    with pytest.raises(negf.NegfError) as e:
        ctx.conductance([dev, dev], 0.0, 0.025)
    assert e.value.status == negf.EINVAL
