"""Pins of the oracle's quadrature rules and energy grids (Sec. 2.2.1, Eq. Rho)."""
import numpy as np
import pytest

from oracle import quadrature as q


@pytest.mark.parametrize("n", [1, 2, 3, 8, 64, 128, 2048])
def test_gauss_legendre_matches_library_rule(n):
    # numpy's leggauss uses an eigenvalue (Golub-Welsch type) method: an independent route
    x, w = q.gauss_legendre(n)
    xr, wr = np.polynomial.legendre.leggauss(n)
    assert np.max(np.abs(x - xr)) < 1e-14
    assert np.max(np.abs(w - wr)) < 1e-12 * max(1.0, n / 64)


@pytest.mark.parametrize("n", [1, 4, 7, 16])
def test_gauss_legendre_exact_on_polynomials(n):
    x, w = q.gauss_legendre(n)
    for k in range(2 * n):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.sum(w * x ** k) - exact) < 1e-14
    # degree 2n is not integrated exactly
    k = 2 * n
    assert abs(np.sum(w * x ** k) - 2.0 / (k + 1)) > 1e-12


def test_midpoint_rule_exact_for_linear():
    E, w = q.real_axis_midpoint(-1.0, 1.0, 256)
    assert abs(np.sum(w) - 2.0) < 1e-14
    assert abs(np.sum(w * (3 * E + 1))) - 2.0 < 1e-13
    assert E[0] > -1.0 and E[-1] < 1.0


def test_fermi_symmetry_and_limits():
    x = np.linspace(-3, 3, 101)
    f = q.fermi(x, 0.025)
    assert np.all(np.abs(f + q.fermi(-x, 0.025) - 1.0) < 1e-15)
    assert q.fermi(np.array([0.0]), 0.025)[0] == 0.5
    big = q.fermi(np.array([1e4, -1e4]), 0.025)
    assert big[0] == 0.0 and big[1] == 1.0


@pytest.mark.parametrize("pole", [0.3 - 0.05j, -4.0 - 1e-3j, -9.0 - 0.5j])
def test_contour_integrates_rational_function(pole):
    # F(E) = 1/(E - p) with Im p < 0 is analytic in the closed upper half plane:
    # integral_{E_B}^{E_min} F dE = log(E_min - p) - log(E_B - p) (no branch crossing)
    E_B, E_min = -10.0, -0.35
    z, zw = q.contour_semicircle(E_B, E_min, 64)
    approx = -np.sum(zw / (z - pole))
    exact = np.log(E_min - pole) - np.log(E_B - pole)
    if abs(pole.imag) > 0.01:
        assert abs(approx - exact) < 1e-12
    else:
        # a pole 1 meV below the real axis far from the arc: still converged
        assert abs(approx - exact) < 1e-10
    assert np.all(z.imag > 0)


def test_contour_polynomial_exact():
    E_B, E_min = -9.0, -1.0
    z, zw = q.contour_semicircle(E_B, E_min, 40)
    for k in range(6):
        exact = (E_min ** (k + 1) - E_B ** (k + 1)) / (k + 1)
        assert abs(-np.sum(zw * z ** k) - exact) < 1e-11 * max(1.0, abs(exact))


def test_bias_grid_window_and_weights():
    g = q.bias_grid(0.0, -0.4, 0.025, 2048, 128, E_B=-11.0, eta=1e-6)
    assert abs(g["E_min"] - (-0.4 - 14 * 0.025)) < 1e-15
    assert abs(g["E_max"] - (0.0 + 14 * 0.025)) < 1e-15
    assert abs(np.sum(g["w"]) - (g["E_max"] - g["E_min"])) < 1e-13
    # contour weights include f(z - mu_min), which is ~1 on the arc
    z, zw = q.contour_semicircle(-11.0, g["E_min"], 128)
    assert np.max(np.abs(g["c"] - zw)) < 1e-5 * np.max(np.abs(zw))


# ---- semi-adaptive real-axis rule (Sec. 3.3)

def test_semi_adaptive_segment_counts_and_exactness():
    kT = 0.025
    E, w, ns = q.semi_adaptive_rule(-0.75, 0.35, -0.5, -0.4, (20, 80, 5), kT)
    # 10 kT at 20 / kT, 4 kT at 80 / kT, 30 kT at 5 / kT
    assert ns == (200, 320, 150)
    assert E.size == 670 and np.all(np.diff(E) > 0)
    a, b = -0.75, 0.35
    for k in range(0, 40):
        exact = (b ** (k + 1) - a ** (k + 1)) / (k + 1)
        assert abs(np.sum(w * E ** k) - exact) < 1e-13 * max(1.0, abs(exact))


def test_semi_adaptive_limits_are_clipped():
    kT = 0.025
    _, _, ns = q.semi_adaptive_rule(-0.75, 0.35, -2.0, -0.7, (10, 10, 10), kT)
    assert ns[0] == 0 and ns[1] == 20 and ns[2] == 420
    _, _, ns = q.semi_adaptive_rule(-0.75, 0.35, 0.3, 9.0, (10, 10, 10), kT)
    assert ns[2] == 0 and ns[1] == 20
    _, _, ns = q.semi_adaptive_rule(-0.75, 0.35, -0.2, -0.4, (10, 10, 10), kT)
    assert ns[1] == 0 and sum(ns) == 220 + 220
    assert q.refined_limits(-0.45, 3.0, 1.0, kT) == (-0.45 - 3 * kT, -0.45 + kT)


def test_semi_adaptive_rule_resolves_a_sharp_peak():
    # a Lorentzian of width 1 meV (closed-form integral): dense points around the peak get it
    # to rounding, one Gauss-Legendre rule with the same point count over the whole window does not
    kT, Es, gam = 0.025, -0.45, 1e-3
    a, b = -0.75, 0.35
    exact = np.arctan((b - Es) / gam) - np.arctan((a - Es) / gam)
    l1, l2 = q.refined_limits(Es, 3.0, 1.0, kT)
    E, w, ns = q.semi_adaptive_rule(a, b, l1, l2, (10, 400, 10), kT)
    f = lambda x: gam / ((x - Es) ** 2 + gam ** 2)
    assert abs(np.sum(w * f(E)) - exact) < 1e-10 * exact
    Eu, wu = q.real_axis_gauss(a, b, E.size)
    assert abs(np.sum(wu * f(Eu)) - exact) > 1e-6 * exact
