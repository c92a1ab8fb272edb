"""Pins of the oracle's surface Green's functions and self-energies (Eq. GR, Sec. 2.2.2)."""
import numpy as np
import pytest

from oracle import leads as ld
from oracle import model as mdl


def textbook_chain(eps, t):
    # uniform chain: g = (eps - sqrt(eps - 2|t|) sqrt(eps + 2|t|)) / (2 t^2); the product of
    # two principal roots is the branch that is analytic in the upper half plane
    a = abs(t)
    return (eps - np.sqrt(eps - 2 * a) * np.sqrt(eps + 2 * a)) / (2 * a * a)


def test_uniform_chain_reduces_to_textbook():
    t = -2.7
    E = np.linspace(-7, 7, 301)
    for eps in (E + 1e-6j, E + 0.3j, -3 + 2.0 * np.exp(1j * np.linspace(0.01, 3.1, 50))):
        g = ld.surface_gf_dimer(eps, t * t, t * t)
        assert np.max(np.abs(g - textbook_chain(eps, t))) < 1e-10


@pytest.mark.parametrize("a1,a2", [(2.7 ** 2, (2 * 2.7 * np.cos(np.pi / 17)) ** 2),
                                   (2.7 ** 2, (2 * 2.7 * np.cos(6 * np.pi / 17)) ** 2),
                                   ((2 * 2.7 * np.cos(6 * np.pi / 17)) ** 2, 2.7 ** 2),
                                   (1.0, 0.0), (0.0, 4.0)])
def test_dimer_root_is_retarded_and_solves_recursion(a1, a2):
    E = np.linspace(-9, 9, 2001)
    for eps in (E + 1e-6j, E + 1e-3j):
        g = ld.surface_gf_dimer(eps, a1, a2)
        assert np.all(g.imag <= 0.0)
        # the defining recursion g = 1/(eps - a1/(eps - a2 g))
        rhs = 1.0 / (eps - a1 / (eps - a2 * g))
        assert np.max(np.abs(g - rhs) / np.abs(g)) < 1e-9
    z = -4 + 5 * np.exp(1j * np.linspace(0.001, np.pi - 0.001, 300))
    g = ld.surface_gf_dimer(z, a1, a2)
    assert np.all(g.imag < 0)


def _away_from_edges(E, edges, margin):
    return np.array([e for e in E if np.min(np.abs(e - np.asarray(edges))) > margin])


def test_analytic_matches_decimation_mode_chain():
    n, t = 17, -2.7
    for j in (1, 6):
        ch = mdl.mode_chain(n, j, t, 8, 0.05, -0.1)
        bj = abs(mdl.mode_hopping(n, j, t))
        edges = [s * e for s in (1, -1) for e in (abs(abs(t) - bj), abs(t) + bj)]
        for lead in (ch.lead_S, ch.lead_D):
            # band edges and the zero-energy surface state of zigzag-terminated leads
            E = _away_from_edges(np.linspace(-6, 6, 241), np.array(edges + [0.0]) + lead.U, 0.02)
            for eps in (E + 1e-6j, -3 + 4 * np.exp(1j * np.linspace(0.05, 3.0, 20))):
                sa = ld.lead_sigma_analytic(lead, eps)
                ss = ld.lead_sigma_sancho(lead, eps)
                assert np.max(np.abs(sa - ss)) < 1e-9 * max(1.0, np.max(np.abs(ss)))


def test_analytic_matches_decimation_realspace_lead():
    n, t = 7, -2.7
    ch = mdl.realspace_chain(n, t, 8, 0.0, -0.2)
    c = np.abs(np.cos(np.pi * np.arange(n) / n))
    edges = np.concatenate([np.abs(1 - 2 * c), 1 + 2 * c]) * abs(t)
    edges = np.concatenate([edges, -edges])
    for lead in (ch.lead_S, ch.lead_D):
        E = _away_from_edges(np.linspace(-8, 8, 97), np.append(edges, 0.0) + lead.U, 0.02)
        eps = E + 1e-6j
        sa = ld.lead_sigma_analytic(lead, eps)
        ss = ld.lead_sigma_sancho(lead, eps)
        assert np.max(np.abs(sa - ss)) < 1e-9 * max(1.0, np.max(np.abs(ss)))
        gam = ld.broadening(sa)
        ev = np.linalg.eigvalsh(0.5 * (gam + np.conj(np.swapaxes(gam, 1, 2))))
        assert ev.min() > -1e-12


def test_non_circulant_lead_rejected_by_analytic():
    lead = mdl.Lead(0.0, np.diag([1.0, 2.0]).astype(complex), np.eye(2, dtype=complex),
                    np.eye(2, dtype=complex), np.arange(2))
    with pytest.raises(ValueError):
        ld.lead_sigma_analytic(lead, np.array([0.1 + 1e-6j]))


def test_zigzag_surface_state_pole():
    # a lead whose surface bond is the weaker one (|t| < |b_j|) has a bound surface state at
    # eps = 0: g ~ (1 - a1/a2)/eps, so Sigma grows like 1/eta at E = U_lead
    t, b = 2.7, 2 * 2.7 * np.cos(np.pi / 17)
    for eta in (1e-3, 1e-6):
        g = ld.surface_gf_dimer(np.array([1j * eta]), t * t, b * b)[0]
        assert abs(g * 1j * eta - (1 - t * t / (b * b))) < 10 * eta
    # the other termination has no surface state: g -> 0 like eps/(a2 - a1)
    g = ld.surface_gf_dimer(np.array([1e-6j]), b * b, t * t)[0]
    assert abs(g) < 1e-5


def test_mode_basis_gamma_is_the_definition():
    # Gamma = i (Sigma - Sigma^dagger); for a circulant lead both evaluations agree to
    # rounding of |Sigma|, and the mode-basis one keeps relative accuracy when Gamma ~ eta
    ch = mdl.realspace_chain(5, -2.7, 6, 0.0, -0.4)
    eps = np.array([-0.3 + 1e-6j, 0.1 + 1e-6j, -3.0 + 1e-6j, -2 + 0.5j])
    for lead in (ch.lead_S, ch.lead_D):
        s, gm = ld.lead_sigma_gamma_analytic(lead, eps)
        assert np.max(np.abs(gm - ld.broadening(s))) < 1e-14 * max(1.0, np.abs(s).max())
        ev = np.linalg.eigvalsh(gm)
        assert ev.min() >= -1e-300
    # its eigenvalues are -2 Im sigma_j of the per-mode closed form
    lead = ch.lead_S
    s, gm = ld.lead_sigma_gamma_analytic(lead, np.array([0.1 + 1e-6j]))
    a1 = np.abs(ld.circulant_eigenvalues(lead.T1)) ** 2
    a2 = np.abs(ld.circulant_eigenvalues(lead.T2)) ** 2
    at = np.abs(ld.circulant_eigenvalues(lead.tau)) ** 2
    sig = at * ld.surface_gf_dimer(np.full(5, 0.1 + 1e-6j - lead.U), a1, a2)
    assert np.allclose(np.sort(np.linalg.eigvalsh(gm[0])), np.sort(-2 * sig.imag), rtol=1e-12, atol=1e-18)


# ---- general (non-circulant) leads by decimation

def random_general_lead(m, seed, onsite=True):
    """A lead with random couplings and on-site blocks: no circulant structure, no closed form."""
    rng = np.random.default_rng(seed)
    T1 = -2.7 * np.eye(m) + 0.4 * (rng.normal(size=(m, m)) + 1j * rng.normal(size=(m, m)))
    T2 = -2.2 * np.eye(m) + 0.4 * (rng.normal(size=(m, m)) + 1j * rng.normal(size=(m, m)))
    tau = -2.5 * np.eye(m) + 0.3 * rng.normal(size=(m, m))
    def herm():
        X = rng.normal(size=(m, m)) + 1j * rng.normal(size=(m, m))
        return 0.3 * (X + X.conj().T)
    return mdl.Lead(0.1, T1, T2, tau, np.arange(m), H0=herm() if onsite else None, H1=herm() if onsite else None)


def two_ring_map(lead, eps, g0):
    """One step of the defining recursion of the two-ring lead: the surface function of ring
    s0 from that of ring s2 (= s0 by periodicity):
    g1 = (eps - U - H1 - T2^dag g0 T2)^{-1}, new g0 = (eps - U - H0 - T1^dag g1 T1)^{-1}."""
    m = lead.m
    I = np.eye(m)
    h0 = lead.U * I + (0 if lead.H0 is None else lead.H0)
    h1 = lead.U * I + (0 if lead.H1 is None else lead.H1)
    g1 = np.linalg.inv(eps * I - h1 - lead.T2.conj().T @ g0 @ lead.T2)
    return np.linalg.inv(eps * I - h0 - lead.T1.conj().T @ g1 @ lead.T1)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_general_lead_decimation_solves_the_defining_recursion(seed):
    lead = random_general_lead(4, seed)
    m = lead.m
    I = np.eye(m)
    h0 = lead.U * I + lead.H0
    H00 = np.block([[h0, lead.T1.conj().T], [lead.T1, lead.U * I + lead.H1]])
    H01 = np.block([[np.zeros((m, m)), np.zeros((m, m))], [lead.T2.conj().T, np.zeros((m, m))]])
    for E in (-3.1, -0.4, 0.9, 4.2):
        eps = E + 1e-4j
        g0 = ld.surface_gf_sancho(np.array([eps]), H00, H01)[0, :m, :m]
        assert np.max(np.abs(two_ring_map(lead, eps, g0) - g0)) < 1e-9 * np.max(np.abs(g0))
        # retarded: the surface spectral function i (g - g^dagger) is positive semidefinite
        assert np.min(np.linalg.eigvalsh(1j * (g0 - g0.conj().T))) > -1e-10 * np.max(np.abs(g0))
        sig = ld.lead_sigma_sancho(lead, np.array([eps]))[0]
        assert np.max(np.abs(sig - lead.tau.conj().T @ g0 @ lead.tau)) < 1e-12 * np.max(np.abs(sig))


@pytest.mark.parametrize("seed", [4, 5])
def test_general_lead_decimation_equals_plain_iteration(seed):
    # with a broadening of 0.05 eV the plain fixed-point iteration of the recursion contracts to
    # the retarded solution (an independent route to the same surface function)
    lead = random_general_lead(3, seed)
    for E in (-2.0, 0.3, 3.5):
        eps = E + 0.05j
        g = np.zeros((3, 3), complex)
        for _ in range(20000):
            g = two_ring_map(lead, eps, g)
        sig_iter = lead.tau.conj().T @ g @ lead.tau
        sig = ld.lead_sigma_sancho(lead, np.array([eps]))[0]
        assert np.max(np.abs(sig - sig_iter)) < 1e-10 * np.max(np.abs(sig))


def test_lead_with_onsite_blocks_has_no_closed_form_here():
    with pytest.raises(ValueError):
        ld.lead_sigma_analytic(random_general_lead(3, 7), np.array([0.3 + 1e-3j]))
