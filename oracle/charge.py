"""Fermi-weighted quadrature to per-ring electron count, T(E) and current
(Eq. Rho, Eq. deviceCharacteristics, Sec. 2.2.1).

Oracle (test infrastructure only).

Electron count of ring r (the paper's rho is minus this, Eq. Rho; readings: electron
counts are reported, and the net charge is -(n - n0)):

  n_r = (g_s g_b / pi) Im sum_k c_k Tr_r G(z_k)                       (contour part)
      + (g_s g_b / 2 pi) sum_k w_k [f_S(E_k) Tr_r A_S(E_k) + f_D(E_k) Tr_r A_D(E_k)]

where Tr_r sums the diagonal over the sites of ring r, and c_k are the complex contour
weights of ``quadrature.bias_grid`` (integral_{E_B}^{E_min} G f dE = -sum_k c_k G(z_k), so
-(1/pi) Im of that integral is +(1/pi) Im sum c_k G).  Both terms are summed over chains.

Transmission reported per energy: T(E) = sum_chains g_b T_chain(E) (spin excluded).
Current (reading: the Landauer form of Eq. deviceCharacteristics, which the literal
Tr[F Gamma A + i Gamma G^<] equals as eta -> 0 without the spurious 2 eta Gamma G G^dagger f
term):  I = g_s (e^2/h) sum_k w_k T(E_k) [f_S(E_k) - f_D(E_k)]  in ampere, energies in eV.

Zero-bias conductance (Eq. zeroBiasG): G = g_s (e^2/h) sum_k w_k T(E_k) (-df/dE)(E_k - mu).

Parity: pinned (neutrality n0 = g_s g_b / 2 per site, zero bias => I = 0, contour ==
real-axis integral at equilibrium, real space == sum of modes).
"""
import numpy as np
from .model import G_SPIN
from .green import rgf_lanes, dense_lanes
from .quadrature import neutral_grid

E_CHARGE = 1.602176634e-19      # C (exact, SI 2019)
H_PLANCK = 6.62607015e-34       # J s (exact, SI 2019)
E2_OVER_H = E_CHARGE * E_CHARGE / H_PLANCK   # A / V; with E in eV, I = g_s e^2/h sum w T df


def ring_sum(chain, n_rings, site_vals):
    """(E, L, b) site values -> (E, n_rings) sums over the sites of each ring."""
    E = site_vals.shape[0]
    out = np.zeros((E, n_rings), dtype=site_vals.dtype)
    flat_ring = chain.site_ring.reshape(-1)
    vals = site_vals.reshape(E, -1)
    for s, r in enumerate(flat_ring):
        out[:, r] += vals[:, s]
    return out


def negf_evaluate(device, U, grid, method="analytic", chunk=64, lanes="rgf"):
    """One NEGF evaluation of a device on a bias grid.

    Returns dict n (n_rings,), n_cont, n_real, T (n_real energies,), I (A),
    and per-energy ring traces for sampled checks: AS_ring, AD_ring (E_real, n_rings) and
    G_ring (E_cont, n_rings) complex (summed over chains, without g factors).
    """
    NR = device.n_rings
    E, w, fS, fD, eta = grid["E"], grid["w"], grid["fS"], grid["fD"], grid["eta"]
    z, c = grid["z"], grid["c"]
    n_real = np.zeros(NR)
    n_cont = np.zeros(NR)
    T = np.zeros(E.size)
    AS_ring = np.zeros((E.size, NR))
    AD_ring = np.zeros((E.size, NR))
    G_ring = np.zeros((z.size, NR), complex)
    for ch in device.chains:
        g = G_SPIN * ch.g_b
        for k0 in range(0, E.size, chunk):
            sl = slice(k0, min(E.size, k0 + chunk))
            eps = E[sl] + 1j * eta
            if lanes == "rgf":
                r = rgf_lanes(ch, U, eps, method, spectral=True)
            else:
                r = dense_lanes(ch, U, eps, method)
            aS = ring_sum(ch, NR, r["AS"])
            aD = ring_sum(ch, NR, r["AD"])
            AS_ring[sl] += aS
            AD_ring[sl] += aD
            n_real += g / (2 * np.pi) * np.einsum("k,kr->r", w[sl], fS[sl, None] * aS + fD[sl, None] * aD)
            T[sl] += ch.g_b * r["T"]
        for k0 in range(0, z.size, chunk):
            sl = slice(k0, min(z.size, k0 + chunk))
            if lanes == "rgf":
                r = rgf_lanes(ch, U, z[sl], method, spectral=False)
            else:
                r = dense_lanes(ch, U, z[sl], method)
            gr = ring_sum(ch, NR, r["Gdiag"])
            G_ring[sl] += gr
            n_cont += g / np.pi * np.einsum("k,kr->r", c[sl], gr).imag
    I = G_SPIN * E2_OVER_H * np.sum(w * T * (fS - fD))
    return dict(n=n_real + n_cont, n_real=n_real, n_cont=n_cont, T=T, I=I,
                AS_ring=AS_ring, AD_ring=AD_ring, G_ring=G_ring)


def neutral_charge(device, n_cont, E_B, method="analytic", chunk=64):
    """Neutral reference electron count n0 per ring (Sec. 2.2.1: rho_0 with E_l = E_u = 0).

    Reading: the same contour closed at E = 0, occupation 1 below it, zero potential in the
    device and in both leads.
    """
    grid = neutral_grid(n_cont, E_B)
    zero = np.zeros(device.n_rings)
    from .model import Device, Chain, Lead
    chains = []
    for ch in device.chains:
        lS = Lead(0.0, ch.lead_S.T1, ch.lead_S.T2, ch.lead_S.tau, ch.lead_S.sites, ch.lead_S.H0, ch.lead_S.H1)
        lD = Lead(0.0, ch.lead_D.T1, ch.lead_D.T2, ch.lead_D.tau, ch.lead_D.sites, ch.lead_D.H0, ch.lead_D.H1)
        chains.append(Chain(ch.Hdiag, ch.Hup, ch.site_ring, lS, lD, ch.g_b))
    r = negf_evaluate(Device(device.n_rings, chains), zero, grid, method, chunk)
    return r["n_cont"]


def minus_dfermi(x, kT):
    """-df/dE of the Fermi function at x = E - mu: (1/kT) f (1 - f) = 1 / (4 kT cosh^2(x / 2kT))."""
    x = np.asarray(x, dtype=np.float64)
    return 1.0 / (4.0 * kT * np.cosh(x / (2.0 * kT)) ** 2)


def zero_bias_conductance(T, E, w, mu, kT):
    """Zero-bias conductance (Eq. zeroBiasG, Sec. 2.2.1): G = G_0 integral T(E) (-df/dE) dE with
    G_0 = g_s e^2/h, discretised on the real-axis rule (E_k, w_k) that T was evaluated on:

      G = g_s (e^2/h) sum_k w_k T(E_k) (-df/dE)(E_k - mu)     [siemens]

    T is the transmission per energy summed over chains with their band degeneracy (the
    quantity ``negf_evaluate`` reports), so one open spin-degenerate mode-space subband
    (g_b = 2) inside a band contributes 2 G_0 = 4 e^2/h.

    Parity: pinned (closed forms for constant and exponential T, ballistic plateau).
    """
    T = np.asarray(T, dtype=np.float64)
    return G_SPIN * E2_OVER_H * float(np.sum(np.asarray(w) * T * minus_dfermi(np.asarray(E) - mu, kT)))


def ring_integrand(device, U, grid, ring, method="analytic", chunk=64):
    """Charge integrand of one ring on the real axis (Sec. 3.3, the A_1 F_1 + A_2 F_2 curve the
    paper plots at the centre of the channel), per unit energy:

      I_r(E_k) = sum_chains (g_s g_b / 2 pi) [f_S(E_k) Tr_r A_S(E_k) + f_D(E_k) Tr_r A_D(E_k)],

    so that sum_k w_k I_r(E_k) is the real-axis part of n_r.  Parity: pinned (the
    closed-form local density of states of the infinite dimerised chain; sum rule against
    ``negf_evaluate``).
    """
    E, fS, fD, eta = grid["E"], grid["fS"], grid["fD"], grid["eta"]
    out = np.zeros(E.size)
    for ch in device.chains:
        g = G_SPIN * ch.g_b
        for k0 in range(0, E.size, chunk):
            sl = slice(k0, min(E.size, k0 + chunk))
            r = rgf_lanes(ch, U, E[sl] + 1j * eta, method, spectral=True)
            aS = ring_sum(ch, device.n_rings, r["AS"])[:, ring]
            aD = ring_sum(ch, device.n_rings, r["AD"])[:, ring]
            out[sl] += g / (2 * np.pi) * (fS[sl] * aS + fD[sl] * aD)
    return out


def singularity_peak(E, integrand):
    """Location E_s of the integrand's peak (Sec. 3.3): the node of largest value, the first
    such node when several are equal.  Returns (E_s, index)."""
    k = int(np.argmax(np.asarray(integrand)))
    return float(E[k]), k
