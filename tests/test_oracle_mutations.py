"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in a copy of an oracle module's source (a dropped term, a
swapped operand, a flipped sign or the wrong root), loads the copy as a throw-away module of
the oracle package, and checks that a pin which the real module passes rejects the copy.
The real oracle is never modified."""
import os

import numpy as np
import pytest

from oracle import green as gr
from oracle import leads as ld
from oracle import model as mdl
from oracle import quadrature as qd

T_HOP = -2.7
ORACLE_DIR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle")


def mutant(module, old, new):
    """The oracle module `module` with the source text `old` replaced once by `new`."""
    path = os.path.join(ORACLE_DIR, module + ".py")
    with open(path) as f:
        src = f.read()
    assert src.count(old) == 1, "mutation site not found in oracle/%s.py: %r" % (module, old)
    ns = {"__name__": "oracle._mutant_" + module, "__package__": "oracle", "__file__": path}
    exec(compile(src.replace(old, new), path, "exec"), ns)
    return ns


def rel(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


def recursion_vs_dense(rgf):
    """Largest relative gap of (G_ll, A_S, A_D, T) between `rgf` and the dense inverse."""
    chain = mdl.realspace_chain(5, T_HOP, 6, 0.0, -0.1)
    # site disorder inside the rings breaks the rotation symmetry of the tube, under which
    # H_{l,l+1} and its transpose would give the same recursion
    rng = np.random.default_rng(11)
    chain.Hdiag = chain.Hdiag + np.array([np.diag(rng.uniform(-0.3, 0.3, 5)) for _ in range(6)])
    U = 0.05 * np.sin(np.arange(6)) + np.linspace(0, -0.1, 6)
    eps = np.array([-2.1, -0.9, -0.3, 0.27, 0.8, 1.7]) + 1e-6j
    d = gr.dense_lanes(chain, U, eps)
    r = rgf(chain, U, eps)
    return max(rel(r["Gdiag"], d["Gdiag"]), rel(r["AS"], d["AS"]), rel(r["AD"], d["AD"]),
               np.max(np.abs(r["T"] - d["T"])) / max(1.0, np.max(np.abs(d["T"]))))


GREEN_MUTATIONS = [
    ("left-connected term with swapped couplings",
     "y[l] = Hdn[l - 1] @ gL[l - 1] @ Hup[l - 1]", "y[l] = Hup[l - 1] @ gL[l - 1] @ Hdn[l - 1]"),
    ("dropped left-connected term in G_ll", "Gll = inv(alpha - x - y)", "Gll = inv(alpha - x)"),
    ("drain column propagated with gR", "colN[l - 1] = gL[l - 1] @ Hup[l - 1] @ colN[l]",
     "colN[l - 1] = gR[l - 1] @ Hup[l - 1] @ colN[l]"),
    ("source spectral function with the drain Gamma", "AS = col0 @ gS[None] @ _dag(col0)",
     "AS = col0 @ gD[None] @ _dag(col0)"),
]


def test_real_recursion_passes_its_pin():
    assert recursion_vs_dense(gr.rgf_lanes) < 1e-11


@pytest.mark.parametrize("name,old,new", GREEN_MUTATIONS)
def test_recursion_pin_rejects(name, old, new):
    m = mutant("green", old, new)
    assert recursion_vs_dense(m["rgf_lanes"]) > 1e-6, name


def retarded_root_gap(surface_gf):
    """Largest violation of Im g <= 0 and of the defining recursion over a grid of dimer leads."""
    worst = 0.0
    for a1, a2 in ((7.29, 1.0), (1.0, 7.29), (3.0, 3.0), (7.29, 20.0)):
        eps = np.linspace(-6, 6, 241) + 1e-3j
        g = surface_gf(eps, a1, a2)
        worst = max(worst, float(np.max(g.imag)))
        # g = 1 / (eps - a1 / (eps - a2 g)) for the dimerised chain
        res = g - 1.0 / (eps - a1 / (eps - a2 * g))
        worst = max(worst, float(np.max(np.abs(res))))
    return worst


def test_real_surface_gf_passes_its_pin():
    assert retarded_root_gap(ld.surface_gf_dimer) < 1e-9


@pytest.mark.parametrize("name,old,new", [
    ("advanced root picked", "pick_imag = np.where(g1.imag < g2.imag, g1, g2)",
     "pick_imag = np.where(g1.imag > g2.imag, g1, g2)"),
    ("wrong quadratic root formula", "g2 = 2.0 * e / q", "g2 = 2.0 * e * q"),
])
def test_surface_gf_pin_rejects(name, old, new):
    m = mutant("leads", old, new)
    assert retarded_root_gap(m["surface_gf_dimer"]) > 1e-3, name


def gl_exactness_gap(gauss_legendre):
    x, w = gauss_legendre(12)
    worst = 0.0
    for k in range(24):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        worst = max(worst, abs(float(np.sum(w * x ** k)) - exact))
    return worst


def test_real_gauss_legendre_passes_its_pin():
    assert gl_exactness_gap(qd.gauss_legendre) < 1e-13


def test_gauss_legendre_pin_rejects_a_wrong_weight():
    src = open(os.path.join(ORACLE_DIR, "quadrature.py")).read()
    # the weights are 2 / ((1 - x^2) P_n'(x)^2); dropping the 2 halves every weight
    old = [ln for ln in src.splitlines() if "2.0 / ((1.0 - x * x)" in ln or "2.0 / ((1 - x * x)" in ln]
    assert len(old) == 1, "weight formula not found in oracle/quadrature.py"
    m = mutant("quadrature", old[0], old[0].replace("2.0 / ((1", "1.0 / ((1", 1))
    assert gl_exactness_gap(m["gauss_legendre"]) > 1e-3


def half_filling_gap(charge_mod):
    dev = mdl.cnt_build("mode", 17, T_HOP, 10, 0.0, 0.0, modes=(6,))
    n0 = charge_mod["neutral_charge"](dev, 48, -9.5) if isinstance(charge_mod, dict) else \
        charge_mod.neutral_charge(dev, 48, -9.5)
    # g_s g_b / 2 = 2 electrons per site of a mode chain at half filling
    return float(np.max(np.abs(n0 - 2.0)))


def test_real_charge_passes_half_filling():
    from oracle import charge as ch
    assert half_filling_gap(ch) < 1e-9


@pytest.mark.parametrize("name,old,new", [
    ("contour term with the wrong sign", "g / np.pi", "-g / np.pi"),
])
def test_half_filling_pin_rejects(name, old, new):
    src = open(os.path.join(ORACLE_DIR, "charge.py")).read()
    if src.count(old) != 1:
        pytest.fail("mutation site %r not found once in oracle/charge.py" % old)
    m = mutant("charge", old, new)
    assert half_filling_gap(m) > 0.1, name


def conductance_gap(charge_mod):
    """Largest relative miss of the two closed forms of the conductance pins."""
    zbc = charge_mod["zero_bias_conductance"] if isinstance(charge_mod, dict) else charge_mod.zero_bias_conductance
    e2h = 1.602176634e-19 ** 2 / 6.62607015e-34
    mu, kT = 0.13, 0.025
    E, w = qd.real_axis_gauss(mu - 40 * kT, mu + 40 * kT, 400)
    const = zbc(np.ones(E.size), E, w, mu, kT) / (2.0 * e2h)
    fdiff = 1.0 / (1.0 + np.exp(-40.0)) - 1.0 / (1.0 + np.exp(40.0))
    x = np.pi * 5.0 * kT
    expo = zbc(np.exp(5.0 * (E - mu)), E, w, mu, kT) / (2.0 * e2h)
    return max(abs(const - fdiff), abs(expo - x / np.sin(x)))


def test_real_conductance_passes_its_pins():
    from oracle import charge as ch
    assert conductance_gap(ch) < 1e-12


@pytest.mark.parametrize("name,old,new", [
    ("cosh argument without the factor 1/2", "np.cosh(x / (2.0 * kT))", "np.cosh(x / kT)"),
    ("f (1 - f) without 1/kT", "1.0 / (4.0 * kT * np.cosh", "1.0 / (4.0 * np.cosh"),
    ("weights dropped", "np.sum(np.asarray(w) * T *", "np.sum(T *"),
])
def test_conductance_pin_rejects(name, old, new):
    m = mutant("charge", old, new)
    assert conductance_gap(m) > 1e-3, name


def adaptive_gap(quad_mod):
    """Miss of the semi-adaptive rule on a Lorentzian peak and on its segment counts."""
    rule = quad_mod["semi_adaptive_rule"] if isinstance(quad_mod, dict) else quad_mod.semi_adaptive_rule
    lim = quad_mod["refined_limits"] if isinstance(quad_mod, dict) else quad_mod.refined_limits
    kT, Es, gam, a, b = 0.025, -0.45, 1e-3, -0.75, 0.35
    l1, l2 = lim(Es, 3.0, 1.0, kT)
    E, w, ns = rule(a, b, l1, l2, (10, 400, 10), kT)
    exact = np.arctan((b - Es) / gam) - np.arctan((a - Es) / gam)
    miss = abs(np.sum(w * gam / ((E - Es) ** 2 + gam ** 2)) - exact) / exact
    return max(miss, 0.0 if ns == (90, 1600, 310) else 1.0)


def test_real_adaptive_rule_passes_its_pin():
    assert adaptive_gap(qd) < 1e-10


@pytest.mark.parametrize("name,old,new", [
    ("lower limit moved the wrong way", "return E_s - a * kT, E_s + b * kT", "return E_s + a * kT, E_s + b * kT"),
    ("densities applied to the wrong segments", "zip(((E_min, l1), (l1, l2), (l2, E_max)), densities)",
     "zip(((E_min, l1), (l1, l2), (l2, E_max)), (densities[1], densities[0], densities[2]))"),
])
def test_adaptive_rule_pin_rejects(name, old, new):
    m = mutant("quadrature", old, new)
    assert adaptive_gap(m) > 1e-6, name


def peak_gap(charge_mod):
    """Whether the located peak of the flat wire's integrand is the first node above the edge."""
    ri = charge_mod["ring_integrand"] if isinstance(charge_mod, dict) else charge_mod.ring_integrand
    sp = charge_mod["singularity_peak"] if isinstance(charge_mod, dict) else charge_mod.singularity_peak
    N = 8
    edge = abs(abs(T_HOP) - abs(2 * T_HOP * np.cos(6 * np.pi / 17)))
    dev = mdl.cnt_build("mode", 17, T_HOP, N, 0.0, 0.0, modes=(6,))
    E, w = qd.real_axis_gauss(0.2, 0.6, 120)
    f = qd.fermi(E - 5.0, 0.025)
    g = dict(E=E, w=w, fS=f, fD=f, eta=1e-9, z=np.zeros(0, complex), c=np.zeros(0, complex))
    _, k = sp(E, ri(dev, np.zeros(N), g, N // 2))
    return 0.0 if k == int(np.argmax(E > edge)) else 1.0


def test_real_peak_passes_its_pin():
    from oracle import charge as ch
    assert peak_gap(ch) == 0.0


@pytest.mark.parametrize("name,old,new", [
    ("smallest value taken for the peak", "k = int(np.argmax(np.asarray(integrand)))",
     "k = int(np.argmin(np.asarray(integrand)))"),
    ("integrand without the source term", "(fS[sl] * aS + fD[sl] * aD)", "(fD[sl] * aD)"),
])
def test_peak_pin_rejects(name, old, new):
    m = mutant("charge", old, new)
    if name.startswith("integrand"):
        # zero-bias flat wire: A_S = A_D, so dropping one term halves the integrand; the peak
        # moves nowhere, and the sum rule against the real-axis charge catches it instead
        N = 14
        dev = mdl.cnt_build("mode", 17, T_HOP, N, 0.0, -0.2, modes=(6,))
        U = np.linspace(0.0, -0.2, N)
        g = qd.bias_grid(0.0, -0.2, 0.025, 48, 8, E_B=-10.0, eta=1e-6)
        from oracle import charge as ch
        nr = ch.negf_evaluate(dev, U, g)["n_real"][7]
        assert abs(np.sum(g["w"] * m["ring_integrand"](dev, U, g, 7)) - nr) > 1e-3 * nr, name
    else:
        assert peak_gap(m) > 0.0, name


def coupled_poisson_gap(sc_mod):
    """Miss of the coupled Poisson against a dense block solve (non-symmetric K)."""
    from oracle import selfconsistent as real
    rng = np.random.default_rng(5)
    C, N = 3, 12
    p = real.PoissonParams(kappa=0.0, lam_nm=2.0, U_G=-0.2, U_S=0.05, U_D=-0.3)
    K = np.array([[19.0, 2.0, 0.3], [1.1, 17.5, 2.4], [0.2, 2.9, 18.2]])
    n0 = rng.uniform(1.5, 2.5, (C, N))
    n = n0 + rng.normal(0, 0.01, (C, N))
    r = p.r
    T = np.diag(np.full(N, 1 + 2 * r)) + np.diag(np.full(N - 1, -r), 1) + np.diag(np.full(N - 1, -r), -1)
    want = []
    for c in range(C):
        b = p.U_G + sum(K[c, d] * (n[d] - n0[d]) for d in range(C))
        b[0] += r * p.U_S
        b[-1] += r * p.U_D
        want.append(np.linalg.solve(T, b))
    return float(np.max(np.abs(sc_mod["poisson_solve_multi"](n, n0, p, K) - np.array(want))))


def test_real_coupled_poisson_passes_its_pin():
    from oracle import selfconsistent as s
    assert coupled_poisson_gap(vars(s)) < 1e-12


@pytest.mark.parametrize("name,old,new", [
    ("coupling matrix transposed", "q = np.asarray(K, dtype=np.float64) @ (n - np.asarray(n0))",
     "q = np.asarray(K, dtype=np.float64).T @ (n - np.asarray(n0))"),
    ("cross-coupling dropped", "q = np.asarray(K, dtype=np.float64) @ (n - np.asarray(n0))",
     "q = np.diag(np.diag(np.asarray(K, dtype=np.float64))) @ (n - np.asarray(n0))"),
])
def test_coupled_poisson_pin_rejects(name, old, new):
    m = mutant("selfconsistent", old, new)
    assert coupled_poisson_gap(m) > 1e-6, name


def general_lead_gap(leads_mod):
    """Miss of the decimated surface function of a random non-circulant lead against the
    defining two-ring recursion."""
    from tests.test_oracle_leads import random_general_lead, two_ring_map
    sg = leads_mod["lead_sigma_sancho"] if isinstance(leads_mod, dict) else leads_mod.lead_sigma_sancho
    lead = random_general_lead(4, 2)
    worst = 0.0
    for E in (-0.4, 0.9):
        eps = E + 1e-3j
        sig = sg(lead, np.array([eps]))[0]
        g0 = np.linalg.solve(lead.tau.conj().T, np.linalg.solve(lead.tau.T, sig.T).T)   # tau^-dag sig tau^-1
        worst = max(worst, float(np.max(np.abs(two_ring_map(lead, eps, g0) - g0)) / np.max(np.abs(g0))))
    return worst


def test_real_general_lead_passes_its_pin():
    assert general_lead_gap(ld) < 1e-8


@pytest.mark.parametrize("name,old,new", [
    ("decimation drops the c g a term", "h = h + agc + cga", "h = h + agc"),
    ("on-site blocks of the two rings swapped", "H00 = np.block([[h0, lead.T1.conj().T], [lead.T1, h1]])",
     "H00 = np.block([[h1, lead.T1.conj().T], [lead.T1, h0]])"),
])
def test_general_lead_pin_rejects(name, old, new):
    m = mutant("leads", old, new)
    assert general_lead_gap(m) > 1e-4, name
