"""GPU parity of the self-consistent loop (Alg. 3 with the 1D Poisson stand-in) against the
oracle's loop on the same inputs, and the session / checkpoint calls."""
import numpy as np
import pytest

from paper_2407_14633_gb300 import synth
from tests.cases import lib_device, rel_inf
from oracle import charge as ochg
from oracle import model as omdl
from oracle import quadrature as oq
from oracle import selfconsistent as osc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2407_14633_gb300 import negf
    c = negf.Context()
    yield c
    c.close()


def oracle_solve(kind, n_tube, modes, N, V_DS, V_GS, U0, n_real, n_cont, E_B, zeta, M, tol):
    dev = omdl.cnt_build(kind, n_tube, -2.7, N, 0.0, -V_DS, modes=modes)
    grid = oq.bias_grid(0.0, -V_DS, 0.025, n_real, n_cont, E_B, 1e-6)
    n0 = ochg.neutral_charge(dev, n_cont, E_B)
    p = osc.PoissonParams(kappa=osc.kappa_from_geometry(), U_G=-V_GS, U_S=0.0, U_D=-V_DS)
    return osc.sc_solve(lambda U: ochg.negf_evaluate(dev, U, grid), U0, n0, p, zeta=zeta, M=M, tol=tol)


@pytest.mark.parametrize("kind,n_tube,modes,N", [("mode", 17, (6,), 24), ("mode", 17, (6, 5), 40),
                                                  ("real", 5, (1,), 10)])
def test_sc_solve_matches_oracle(ctx, kind, n_tube, modes, N):
    from paper_2407_14633_gb300 import negf
    V_DS, V_GS = 0.2, 0.1
    n_real, n_cont, E_B = 48, 16, -10.0
    U0 = np.linspace(0.0, -V_DS, N) + 0.02 * np.sin(np.arange(N))
    dev = lib_device(ctx, kind, n_tube, -2.7, N, 0.0, -V_DS, modes)
    ctx.set_grid_spec(dev, 0.0, -V_DS, 0.025, 1e-6, E_B, n_real, n_cont)
    r = ctx.sc_solve(dev, V_DS, V_GS, U0, negf.poisson_kappa(), zeta=0.1, M=64, tol=1e-9)
    o = oracle_solve(kind, n_tube, modes, N, V_DS, V_GS, U0, n_real, n_cont, E_B, 0.1, 64, 1e-9)
    assert r["converged"] and o["converged"]
    assert r["iterations"] == o["iterations"]
    assert rel_inf(r["n"], o["n"]) < 1e-9
    assert rel_inf(r["U"], o["U"]) < 1e-9
    assert rel_inf(r["history"], np.array(o["history"])) < 1e-6
    assert abs(r["I"] - o["I"]) <= 1e-9 * max(abs(o["I"]), 1e-15)


def test_session_steps_and_checkpoint_roundtrip(ctx):
    from paper_2407_14633_gb300 import negf
    N, V_DS, V_GS = 20, 0.1, 0.0
    U0 = np.linspace(0.0, -V_DS, N)
    dev = lib_device(ctx, "mode", 17, -2.7, N, 0.0, -V_DS, (6,))
    ctx.set_grid_spec(dev, 0.0, -V_DS, 0.025, 1e-6, -10.0, 40, 12)
    kappa = negf.poisson_kappa()
    ref = ctx.sc_solve(dev, V_DS, V_GS, U0, kappa, M=64, tol=1e-10)
    # same loop driven step by step, with a checkpoint / restore in the middle
    ctx.sc_begin(dev, V_DS, V_GS, U0, kappa, M=64, tol=1e-10)
    with pytest.raises(negf.NegfError):
        ctx.set_potential(dev, U0)          # set-up calls refuse a device in a session
    ctx.sc_step(dev, 3)
    st = ctx.sc_get_state(dev)
    ctx.sc_step(dev, 2)
    ctx.sc_set_state(dev, st)               # roll back two iterations
    state = 0
    while state == 0:
        state = ctx.sc_step(dev, 1)
    r = ctx.sc_end(dev)
    assert r["converged"] and ref["converged"]
    assert np.array_equal(r["n"], ref["n"])
    assert np.array_equal(r["U"], ref["U"])


def test_not_converged_is_reported(ctx):
    from paper_2407_14633_gb300 import negf
    N = 16
    dev = lib_device(ctx, "mode", 17, -2.7, N, 0.0, -0.1, (6,))
    ctx.set_grid_spec(dev, 0.0, -0.1, 0.025, 1e-6, -10.0, 32, 8)
    r = ctx.sc_solve(dev, 0.1, 0.0, np.zeros(N), negf.poisson_kappa(), M=3, tol=1e-14, check=False)
    assert r["status"] == negf.ENOTCONVERGED and not r["converged"] and r["iterations"] == 3
