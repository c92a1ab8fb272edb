"""GPU parity of the self-consistent loop of several coupled channels with one Broyden vector
(Sec. 2.3) against the oracle's loop, and its reduction to one tube."""
import numpy as np
import pytest

from tests.cases import lib_device, oracle_device, rel_inf
from oracle import charge as ochg
from oracle import quadrature as oq
from oracle import selfconsistent as osc

pytestmark = pytest.mark.gpu

E_B, KT, ETA = -10.0, 0.025, 1e-6


@pytest.fixture(scope="module")
def ctx():
    from paper_2407_14633_gb300 import negf
    c = negf.Context()
    yield c
    c.close()


def test_multi_channel_solve_matches_oracle(ctx):
    N, V_DS, V_GS, n_real, n_cont = 16, 0.2, 0.1, 40, 12
    mode_sets = [(6,), (5,), (6, 5)]
    k = osc.kappa_from_geometry()
    K = np.array([[k, 2.0, 0.5], [2.0, k, 2.0], [0.5, 2.0, k]])
    U0 = np.array([np.linspace(0.0, -V_DS, N) + 0.02 * np.sin(np.arange(N) + c) for c in range(3)])
    devs = []
    for modes in mode_sets:
        d = lib_device(ctx, "mode", 17, -2.7, N, 0.0, -V_DS, modes)
        ctx.set_grid_spec(d, 0.0, -V_DS, KT, ETA, E_B, n_real, n_cont)
        devs.append(d)
    r = ctx.sc_solve_multi(devs, V_DS, V_GS, U0, K, M=64, tol=1e-10)
    g = oq.bias_grid(0.0, -V_DS, KT, n_real, n_cont, E_B, ETA)
    ods = [oracle_device("mode", 17, -2.7, N, 0.0, -V_DS, m) for m in mode_sets]
    evs = [(lambda od: (lambda U: ochg.negf_evaluate(od, U, g)))(od) for od in ods]
    n0 = np.array([ochg.neutral_charge(od, n_cont, E_B) for od in ods])
    p = osc.PoissonParams(kappa=0.0, U_G=-V_GS, U_S=0.0, U_D=-V_DS)
    o = osc.sc_solve_multi(evs, U0, n0, p, K, M=64, tol=1e-10)
    assert r["converged"] and o["converged"] and r["iterations"] == o["iterations"]
    assert rel_inf(r["history"], np.array(o["history"])) < 1e-6
    for c in range(3):
        assert rel_inf(r["n"][c], o["n"][c]) < 1e-9
        assert rel_inf(r["U"][c], o["U"][c]) < 1e-9
        assert rel_inf(r["T"][c], o["T"][c]) < 1e-8
        assert abs(r["I"][c] - o["I"][c]) <= 1e-8 * max(abs(o["I"][c]), 1e-15)


def test_two_identical_tubes_solve_like_one_tube(ctx):
    from paper_2407_14633_gb300 import negf
    N, V_DS, V_GS = 18, 0.25, -0.1
    k, kx = negf.poisson_kappa(), 4.0
    U0 = np.linspace(0.0, -V_DS, N)
    devs = []
    for _ in range(3):
        d = lib_device(ctx, "mode", 17, -2.7, N, 0.0, -V_DS, (6, 5))
        ctx.set_grid_spec(d, 0.0, -V_DS, KT, ETA, E_B, 48, 12)
        devs.append(d)
    two = ctx.sc_solve_multi(devs[:2], V_DS, V_GS, np.array([U0, U0]), [[k, kx], [kx, k]], M=64, tol=1e-10)
    one = ctx.sc_solve(devs[2], V_DS, V_GS, U0, k + kx, M=64, tol=1e-10)
    assert two["converged"] and one["converged"] and two["iterations"] == one["iterations"]
    for c in range(2):
        assert rel_inf(two["n"][c], one["n"]) < 1e-10
        assert rel_inf(two["U"][c], one["U"]) < 1e-10


def test_multi_channel_rejects_bad_arguments(ctx):
    from paper_2407_14633_gb300 import negf
    a = lib_device(ctx, "mode", 17, -2.7, 12, 0.0, -0.1, (6,))
    b = lib_device(ctx, "mode", 17, -2.7, 14, 0.0, -0.1, (6,))
    for d in (a, b):
        ctx.set_grid_spec(d, 0.0, -0.1, KT, ETA, E_B, 16, 4)
    k = negf.poisson_kappa()
    cases = [([a, b], np.zeros((2, 12)), [[k, 0.0], [0.0, k]]),        # unequal lengths
             ([a, a], np.zeros((2, 12)), [[k, 0.0], [0.0, k]]),        # listed twice
             ([a], np.zeros((1, 12)), [[0.0]]),                       # singular K
             ([a], np.zeros((1, 12)), [[float("nan")]])]
    for devs, U0, K in cases:
        with pytest.raises(negf.NegfError) as e:
            ctx.sc_solve_multi(devs, 0.1, 0.0, U0, K)
        assert e.value.status == negf.EINVAL
