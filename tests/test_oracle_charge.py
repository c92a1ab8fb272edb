"""Pins of the oracle's charge / current quadrature (Eq. Rho, Eq. deviceCharacteristics)."""
import numpy as np
import pytest

from oracle import charge as chg
from oracle import model as mdl
from oracle import quadrature as q

T_HOP = -2.7


def test_zero_bias_current_is_exactly_zero():
    dev = mdl.cnt_build("mode", 17, T_HOP, 12, 0.02, 0.02, modes=(6, 5))
    U = 0.02 + 0.1 * np.exp(-((np.arange(12) - 5.5) ** 2) / 8)
    g = q.bias_grid(0.1, 0.1, 0.025, 64, 16, E_B=-10.0, eta=1e-6)
    r = chg.negf_evaluate(dev, U, g)
    assert r["I"] == 0.0
    assert np.all(r["T"] >= 0)


@pytest.mark.parametrize("kind,modes,gb", [("mode", (6,), 2.0), ("mode", (1, 6), 2.0), ("real", None, 1.0)])
def test_neutral_charge_is_half_filling(kind, modes, gb):
    # bipartite chain, zero potential everywhere: particle-hole symmetry gives exactly
    # g_s g_b / 2 electrons per site and chain (Sec. 2.2.1 rho_0 reading)
    n = 17 if kind == "mode" else 7
    dev = mdl.cnt_build(kind, n, T_HOP, 10, 0.0, 0.0, modes=modes or (1,))
    n0 = chg.neutral_charge(dev, 96, E_B=-10.0)
    sites_per_ring = 1 if kind == "mode" else n
    want = 2.0 * gb / 2.0 * sites_per_ring * len(dev.chains)
    assert np.max(np.abs(n0 - want)) < 1e-9 * want


def test_dense_and_recursion_give_same_charge():
    dev = mdl.cnt_build("mode", 17, T_HOP, 8, 0.0, -0.1, modes=(6,), cells=True)
    U = np.linspace(0, -0.1, 8) + 0.05
    g = q.bias_grid(0.0, -0.1, 0.025, 40, 12, E_B=-10.0, eta=1e-6)
    a = chg.negf_evaluate(dev, U, g, lanes="rgf")
    b = chg.negf_evaluate(dev, U, g, lanes="dense")
    assert np.max(np.abs(a["n"] - b["n"])) < 1e-12 * np.max(np.abs(b["n"]))
    assert abs(a["I"] - b["I"]) < 1e-12 * max(abs(b["I"]), 1e-20)


def graded_rule(a, b, singular, levels=44, n=12):
    """Composite GL on [a, b], panels graded geometrically toward each inverse-square-root
    band-edge singularity listed in `singular` (independent of the oracle's rules)."""
    sing = set(singular)
    cuts = sorted({a, b} | {s for s in singular if a < s < b})
    bounds = []
    for p, r in zip(cuts[:-1], cuts[1:]):
        mid = 0.5 * (p + r)
        L = mid - p
        if p in sing:
            left = [p] + [p + L * 2.0 ** -k for k in range(levels, 0, -1)]
        else:
            left = list(np.linspace(p, mid, 9)[:-1])
        if r in sing:
            right = [mid] + [r - L * 2.0 ** -k for k in range(1, levels + 1)]
        else:
            right = list(np.linspace(mid, r, 9)[:-1])
        bounds += left + right
    bounds.append(b)
    Es, ws = [], []
    for x0, x1 in zip(bounds[:-1], bounds[1:]):
        e, w = q.real_axis_gauss(x0, x1, n)
        Es.append(e)
        ws.append(w)
    return np.concatenate(Es), np.concatenate(ws)


def test_contour_plus_window_equals_real_axis_integral():
    # equilibrium, flat device identical to its leads (no bound states): the contour part up
    # to E_min plus the real-axis window must equal the plain real-axis integral of
    # (A_S + A_D) f from below the band to E_max (up to O(eta) and quadrature error)
    N = 6
    dev = mdl.cnt_build("mode", 17, T_HOP, N, 0.0, 0.0, modes=(6,))
    U = np.zeros(N)
    mu, kT, eta = 0.1, 0.025, 1e-9
    c = abs(np.cos(6 * np.pi / 17))
    edges = [-abs(T_HOP) * (1 + 2 * c), -abs(T_HOP) * abs(1 - 2 * c), abs(T_HOP) * abs(1 - 2 * c)]
    g = q.bias_grid(mu, mu, kT, 400, 96, E_B=-9.0, eta=eta)
    # the window part on a graded rule too (a plain GL rule across the van Hove edge at
    # 0.293 eV is only good to ~1e-5 here, the sharpening discussed in Sec. 3.3)
    Ew, ww = graded_rule(g["E_min"], g["E_max"], edges)
    g.update(E=Ew, w=ww, fS=q.fermi(Ew - mu, kT), fD=q.fermi(Ew - mu, kT))
    split = chg.negf_evaluate(dev, U, g, chunk=4096)["n"]
    E, w = graded_rule(-9.0, g["E_max"], edges)
    f = q.fermi(E - mu, kT)
    full = dict(E=E, w=w, fS=f, fD=f, eta=eta, z=np.zeros(0, complex), c=np.zeros(0, complex))
    ref = chg.negf_evaluate(dev, U, full, chunk=4096)["n"]
    assert np.max(np.abs(split - ref)) < 1e-6 * np.max(ref)


def test_current_sign_and_units():
    # one open channel in a flat wire: I = g_s g_b (e^2/h) integral (f_S - f_D) dE
    N = 6
    dev = mdl.cnt_build("mode", 17, T_HOP, N, 0.0, 0.0, modes=(6,))
    U = np.zeros(N)
    mu_S, mu_D, kT = 0.9, 0.8, 0.005   # window inside the first subband (edge 0.293 eV)
    g = q.bias_grid(mu_S, mu_D, kT, 512, 8, E_B=-10.0, eta=1e-9)
    r = chg.negf_evaluate(dev, U, g)
    expect = 2.0 * 2.0 * chg.E2_OVER_H * (mu_S - mu_D)
    assert abs(r["I"] - expect) < 1e-6 * expect
    assert abs(chg.E2_OVER_H - 3.874045865e-5) < 1e-13


# ---- zero-bias conductance (Eq. zeroBiasG)

def test_conductance_of_constant_transmission_is_fermi_difference():
    # integral_a^b (-df/dE) dE = f(a - mu) - f(b - mu): with T == 3 on a Gauss-Legendre rule over
    # mu -+ 14 kT, G = 3 g_s (e^2/h) (f(-14 kT) - f(14 kT)) = 3 g_s (e^2/h) tanh(7)
    mu, kT = 0.13, 0.025
    E, w = q.real_axis_gauss(mu - 14 * kT, mu + 14 * kT, 200)
    G = chg.zero_bias_conductance(np.full(E.size, 3.0), E, w, mu, kT)
    expect = 3.0 * 2.0 * chg.E2_OVER_H * (1.0 / (1.0 + np.exp(-14.0)) - 1.0 / (1.0 + np.exp(14.0)))
    assert abs(G - expect) < 1e-13 * expect
    assert abs(expect / (6.0 * chg.E2_OVER_H) - np.tanh(7.0)) < 1e-15


@pytest.mark.parametrize("a", [-8.0, 3.0, 8.0])
def test_conductance_of_exponential_transmission_closed_form(a):
    # integral e^{a x} (-df/dx) dx over the real line = pi a kT / sin(pi a kT) (|a kT| < 1); the
    # window mu -+ 40 kT leaves tails below 1e-13 for |a kT| <= 0.2
    mu, kT = -0.07, 0.025
    E, w = q.real_axis_gauss(mu - 40 * kT, mu + 40 * kT, 400)
    G = chg.zero_bias_conductance(np.exp(a * (E - mu)), E, w, mu, kT)
    x = np.pi * a * kT
    assert abs(G / (2.0 * chg.E2_OVER_H) - x / np.sin(x)) < 1e-12


def test_conductance_ballistic_plateau_is_two_quanta_per_subband():
    # flat (17,0) mode-space wire, mode j = 6, mu inside its first subband (edge 0.293 eV):
    # one open spin-degenerate channel of band degeneracy 2, G = 2 G_0 = 4 e^2/h up to the
    # Fermi tails outside the window, and T(E) = 2 at every node
    N = 6
    dev = mdl.cnt_build("mode", 17, T_HOP, N, 0.0, 0.0, modes=(6,))
    mu, kT = 0.9, 0.005
    g = q.bias_grid(mu, mu, kT, 96, 4, E_B=-10.0, eta=1e-9)
    r = chg.negf_evaluate(dev, np.zeros(N), g)
    assert np.max(np.abs(r["T"] - 2.0)) < 1e-8
    G = chg.zero_bias_conductance(r["T"], g["E"], g["w"], mu, kT)
    expect = 2.0 * 2.0 * chg.E2_OVER_H * np.tanh(7.0)
    assert abs(G - expect) < 1e-8 * expect


# ---- charge integrand of one ring and its peak (semi-adaptive grid, Sec. 3.3)

def dimer_ldos(E, t1, t2):
    """Local density of states per site of the infinite chain with alternating bonds t1, t2:
    |E| / (pi sqrt(((t1+t2)^2 - E^2)(E^2 - (t1-t2)^2))) inside the bands, 0 in the gaps."""
    p = ((t1 + t2) ** 2 - E ** 2) * (E ** 2 - (t1 - t2) ** 2)
    out = np.zeros_like(E)
    ok = p > 0
    out[ok] = np.abs(E[ok]) / (np.pi * np.sqrt(p[ok]))
    return out


def test_ring_integrand_is_the_infinite_chain_ldos():
    # flat mode-space wire identical to its leads = the infinite dimerised chain: at every ring
    # A_S + A_D = 2 pi rho(E) (eta -> 0), so with f = 1 the integrand is g_s g_b rho(E)
    N = 8
    t1, t2 = abs(T_HOP), abs(2 * T_HOP * np.cos(6 * np.pi / 17))
    dev = mdl.cnt_build("mode", 17, T_HOP, N, 0.0, 0.0, modes=(6,))
    E = np.concatenate([np.linspace(-1.0, -0.4, 7), np.linspace(0.4, 1.0, 7), [0.1, -0.2]])
    g = dict(E=E, w=np.ones(E.size), fS=np.ones(E.size), fD=np.ones(E.size), eta=1e-9,
             z=np.zeros(0, complex), c=np.zeros(0, complex))
    for ring in (0, N // 2, N - 1):
        I = chg.ring_integrand(dev, np.zeros(N), g, ring)
        want = 2.0 * 2.0 * dimer_ldos(E, t1, t2)
        assert np.max(np.abs(I - want)) < 1e-6 * np.max(want)
    assert np.all(np.abs(I[-2:]) < 1e-6)   # gap energies


def test_singularity_peak_is_first_node_above_band_edge():
    N = 8
    t1, t2 = abs(T_HOP), abs(2 * T_HOP * np.cos(6 * np.pi / 17))
    edge = abs(t1 - t2)
    dev = mdl.cnt_build("mode", 17, T_HOP, N, 0.0, 0.0, modes=(6,))
    E, w = q.real_axis_gauss(0.2, 0.6, 120)
    g = dict(E=E, w=w, fS=q.fermi(E - 5.0, 0.025), fD=q.fermi(E - 5.0, 0.025), eta=1e-9,
             z=np.zeros(0, complex), c=np.zeros(0, complex))
    Es, k = chg.singularity_peak(E, chg.ring_integrand(dev, np.zeros(N), g, N // 2))
    assert k == int(np.argmax(E > edge)) and Es == E[k]


def test_ring_integrand_sums_to_real_axis_charge():
    N = 14
    dev = mdl.cnt_build("mode", 17, T_HOP, N, 0.0, -0.2, modes=(6, 5))
    U = np.linspace(0.0, -0.2, N) + 0.1 * np.exp(-((np.arange(N) - 6.5) ** 2) / 6)
    g = q.bias_grid(0.0, -0.2, 0.025, 64, 8, E_B=-10.0, eta=1e-6)
    r = chg.negf_evaluate(dev, U, g)
    for ring in (3, N // 2, N - 2):
        I = chg.ring_integrand(dev, U, g, ring)
        assert abs(np.sum(g["w"] * I) - r["n_real"][ring]) < 1e-12 * r["n_real"][ring]
