"""Pins of the oracle's Green's functions: dense inverse vs the block recursion of
Alg. 1 / Alg. 2, sum rule, reciprocity, Hermiticity, plateaus, mode equivalences."""
import numpy as np
import pytest

from oracle import green as gr
from oracle import model as mdl
from oracle.leads import broadening

T_HOP = -2.7


def rel(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


def chains_under_test():
    U8 = 0.05 * np.sin(np.arange(8)) + np.linspace(0, -0.1, 8)
    return [
        ("mode1x1", mdl.mode_chain(17, 6, T_HOP, 8, U8[0], U8[-1]), U8),
        ("mode1x1_j1", mdl.mode_chain(17, 1, T_HOP, 8, 0.1, -0.1), U8),
        ("cells2x2", mdl.mode_chain_cells(17, 5, T_HOP, 8, 0.0, -0.2), U8),
        ("real5", mdl.realspace_chain(5, T_HOP, 6, 0.0, -0.1), U8[:6]),
        ("real17", mdl.realspace_chain(17, T_HOP, 4, 0.02, -0.1), U8[:4]),
        ("real26", mdl.realspace_chain(26, T_HOP, 3, 0.0, -0.1), U8[:3]),
        ("real34", mdl.realspace_chain(34, T_HOP, 3, 0.03, -0.05), U8[:3]),
    ]


@pytest.mark.parametrize("name,chain,U", chains_under_test())
def test_recursion_equals_dense_inverse(name, chain, U):
    E = np.array([-2.1, -0.9, -0.3, 0.05, 0.27, 0.8, 1.7])
    for eps in (E + 1e-6j, -4 + 3.5 * np.exp(1j * np.linspace(0.2, 2.9, 5))):
        d = gr.dense_lanes(chain, U, eps)
        r = gr.rgf_lanes(chain, U, eps)
        assert rel(r["Gdiag"], d["Gdiag"]) < 1e-12
        assert rel(r["AS"], d["AS"]) < 1e-11
        assert rel(r["AD"], d["AD"]) < 1e-11
        assert np.max(np.abs(r["T"] - d["T"])) < 1e-11 * max(1.0, np.max(np.abs(d["T"])))


@pytest.mark.parametrize("name,chain,U", chains_under_test())
def test_sum_rule_dense(name, chain, U):
    eta = 1e-3
    eps = np.array([-1.3, -0.2, 0.4, 2.2]) + 1j * eta
    d = gr.dense_lanes(chain, U, eps)
    G = d["G"]
    lhs = 1j * (G - np.conj(np.swapaxes(G, 1, 2)))
    n = G.shape[1]
    gam = d["GammaS_full"] + d["GammaD_full"] + 2 * eta * np.eye(n)
    rhs = G @ gam @ np.conj(np.swapaxes(G, 1, 2))
    assert rel(lhs, rhs) < 1e-12


@pytest.mark.parametrize("name,chain,U", chains_under_test())
def test_reciprocity_and_spectral_positivity(name, chain, U):
    eps = np.array([-2.3, -0.35, 0.31, 1.5]) + 1e-6j
    r = gr.rgf_lanes(chain, U, eps, blocks=True)
    assert np.max(np.abs(r["T"] - r["T_DS"])) < 1e-12 * max(1.0, np.max(r["T"]))
    for A in (r["AS_blocks"], r["AD_blocks"]):
        Ah = np.conj(np.swapaxes(A, -1, -2))
        assert np.max(np.abs(A - Ah)) < 1e-13 * max(1.0, np.max(np.abs(A)))
        ev = np.linalg.eigvalsh(0.5 * (A + Ah))
        assert ev.min() > -1e-12 * max(1.0, np.abs(ev).max())


def open_channels(E, U, t, bjs):
    e = abs(E - U)
    return sum(1 for b in bjs if abs(abs(t) - abs(b)) < e < abs(t) + abs(b))


def test_transmission_plateaus_mode_and_real_space():
    n, N = 7, 10
    U = np.zeros(N)
    bjs = [mdl.mode_hopping(n, j, T_HOP) for j in range(n)]
    edges = sorted({abs(abs(T_HOP) - abs(b)) for b in bjs} | {abs(T_HOP) + abs(b) for b in bjs})
    # off the band edges and off the zero-energy surface state of the zigzag leads
    E = np.array([e for e in np.linspace(-8, 8, 161)
                  if min(abs(abs(e) - x) for x in edges + [0.0]) > 1e-3])
    eps = E + 1e-9j
    real = gr.rgf_lanes(mdl.realspace_chain(n, T_HOP, N, 0.0, 0.0), U, eps)
    want = np.array([open_channels(e, 0.0, T_HOP, bjs) for e in E])
    assert np.max(np.abs(real["T"] - want)) < 1e-5
    for j in (1, 2, 3):
        m = gr.rgf_lanes(mdl.mode_chain(n, j, T_HOP, N, 0.0, 0.0), U, eps)
        wj = np.array([open_channels(e, 0.0, T_HOP, [bjs[j]]) for e in E])
        assert np.max(np.abs(m["T"] - wj)) < 1e-5


def test_realspace_equals_sum_of_modes():
    n, N = 5, 8
    U = 0.1 * np.cos(np.arange(N)) - 0.05
    eps = np.concatenate([np.linspace(-3, 3, 9) + 1e-6j,
                          -5 + 4 * np.exp(1j * np.linspace(0.3, 2.8, 4))])
    real = gr.rgf_lanes(mdl.realspace_chain(n, T_HOP, N, 0.03, -0.07), U, eps)
    T = 0
    AS = 0
    AD = 0
    G = 0
    for j in range(n):
        m = gr.rgf_lanes(mdl.mode_chain(n, j, T_HOP, N, 0.03, -0.07), U, eps)
        T = T + m["T"]
        AS = AS + m["AS"][..., 0]
        AD = AD + m["AD"][..., 0]
        G = G + m["Gdiag"][..., 0]
    assert rel(real["T"], T) < 1e-10
    assert rel(real["AS"].sum(-1), AS) < 1e-10
    assert rel(real["AD"].sum(-1), AD) < 1e-10
    assert rel(real["Gdiag"].sum(-1), G) < 1e-10


def test_cells_equal_single_sites():
    N = 12
    U = np.linspace(0.1, -0.2, N)
    eps = np.concatenate([np.linspace(-3, 3, 11) + 1e-6j, [-2 + 1j, -6 + 0.5j]])
    a = gr.rgf_lanes(mdl.mode_chain(17, 6, T_HOP, N, 0.1, -0.2), U, eps)
    b = gr.rgf_lanes(mdl.mode_chain_cells(17, 6, T_HOP, N, 0.1, -0.2), U, eps)
    assert rel(b["Gdiag"].reshape(-1, N), a["Gdiag"][..., 0]) < 1e-12
    assert rel(b["AS"].reshape(-1, N), a["AS"][..., 0]) < 1e-11
    assert rel(b["AD"].reshape(-1, N), a["AD"][..., 0]) < 1e-11
    assert np.max(np.abs(a["T"] - b["T"])) < 1e-12


def test_dense_matches_brute_force_solve():
    # tiny case: each column of G from a linear solve with a unit right-hand side
    ch = mdl.mode_chain(17, 6, T_HOP, 5, 0.0, 0.0)
    U = np.array([0.0, 0.1, 0.2, 0.1, 0.0])
    eps = np.array([0.5 + 1e-6j])
    d = gr.dense_lanes(ch, U, eps)
    sS, sD, _, _ = gr.contact_blocks(ch, eps)
    M = eps[0] * np.eye(5) - mdl.dense_hamiltonian(ch, U)
    M[0, 0] -= sS[0, 0, 0]
    M[4, 4] -= sD[0, 0, 0]
    for c in range(5):
        e = np.zeros(5)
        e[c] = 1
        col = np.linalg.solve(M, e)
        assert np.max(np.abs(col - d["G"][0][:, c])) < 1e-13
