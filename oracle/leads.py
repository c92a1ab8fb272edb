"""Surface Green's functions and contact self-energies (Eq. GR, Sec. 2.2.2).

Oracle (test infrastructure only).

Sigma_l = tau_l^dagger g_l tau_l with g_l the retarded surface Green's function of lead l
(Eq. GR).  The paper computes g either by decimation (Lopez Sancho et al. 1985) or, for
nanotubes, by a closed form (Sec. 2.2.2).  Both are written here:

* ``surface_gf_dimer``: semi-infinite chain s0 - s1 - s2 - ... whose bonds alternate with
  |H_{s1,s0}|^2 = a1 and |H_{s2,s1}|^2 = a2.  From g_0 = 1/(eps - a1 g_1) and
  g_1 = 1/(eps - a2 g_0):   a2 eps g^2 - (eps^2 - a1 + a2) g + eps = 0.
  Root selection (reading, the paper does not state it): the retarded root is the one
  with Im g < 0 (for Im eps > 0 the two roots satisfy g_+ g_- = 1/a2, so exactly one of
  them has negative imaginary part).  If the two imaginary parts agree to 1e-12 of the
  scale of g (never met for Im eps > 0 in double precision), the root with
  sqrt(a2)|g| < 1 (decaying into the lead) is taken.  The larger-modulus combination
  q = B +/- sqrt(B^2 - 4 a2 eps^2) is formed first and the roots are q/(2 a2 eps) and
  2 eps/q, which avoids cancellation.
* ``lead_sigma_analytic``: leads whose couplings T1, T2, tau are circulant m x m
  matrices (every (n,0) tube) are diagonal in the ring Fourier basis
  F[s, j] = w^{js}/sqrt(m), w = exp(2 pi i/m), with eigenvalues lambda_j(C) =
  sum_d C[0, d] w^{jd}.  Each angular mode is then a dimerised chain with
  a1 = |lambda_j(T1)|^2, a2 = |lambda_j(T2)|^2 and Sigma = F diag(|lambda_j(tau)|^2 g_j) F^dagger.
* ``lead_sigma_sancho``: decimation of the lead written as a uniform chain of two-ring
  principal layers, fully general (no circulant assumption; the rings may carry on-site
  blocks H0, H1 besides U, as a lead of another material or with a non-uniform potential
  would).

Gamma_l = i (Sigma_l - Sigma_l^dagger) (Sec. 2.2.1).

Parity: pinned (textbook uniform chain, analytic vs decimation, Im g <= 0 on the real
axis, the defining recursion).
"""
import numpy as np


def surface_gf_dimer(eps, a1, a2):
    """Retarded surface Green's function of the dimerised chain (see module docstring)."""
    eps = np.asarray(eps, dtype=complex)
    a1 = np.broadcast_to(np.asarray(a1, dtype=np.float64), eps.shape)
    a2 = np.broadcast_to(np.asarray(a2, dtype=np.float64), eps.shape)
    out = np.empty(eps.shape, complex)
    dimer = a2 == 0.0
    if np.any(dimer):
        e = eps[dimer]
        out[dimer] = e / (e * e - a1[dimer])
    m = ~dimer
    if np.any(m):
        e, p, q2 = eps[m], a1[m], a2[m]
        B = e * e - p + q2
        s = np.sqrt(B * B - 4.0 * q2 * e * e)
        qp, qm = B + s, B - s
        q = np.where(np.abs(qp) >= np.abs(qm), qp, qm)
        g1 = q / (2.0 * q2 * e)
        g2 = 2.0 * e / q
        scale = np.abs(g1) + np.abs(g2)
        tie = np.abs(g1.imag - g2.imag) <= 1e-12 * scale
        pick_imag = np.where(g1.imag < g2.imag, g1, g2)
        pick_decay = np.where(np.sqrt(q2) * np.abs(g1) < 1.0, g1, g2)
        out[m] = np.where(tie, pick_decay, pick_imag)
    return out


def circulant_eigenvalues(C):
    """lambda_j = sum_d C[0, d] w^{j d}, w = exp(2 pi i / m), of a circulant matrix C.

    Raises if C is not circulant (C[r, s] must depend on (s - r) mod m only)."""
    C = np.asarray(C, complex)
    m = C.shape[0]
    row = C[0]
    for r in range(m):
        if not np.allclose(C[r], np.roll(row, r), atol=1e-14, rtol=0):
            raise ValueError("lead coupling is not circulant")
    j = np.arange(m)
    w = np.exp(2j * np.pi * np.outer(j, j) / m)   # w[j, d] = w^{jd}
    return w @ row


def fourier_matrix(m):
    """F[s, j] = exp(2 pi i j s / m) / sqrt(m)."""
    s = np.arange(m)
    return np.exp(2j * np.pi * np.outer(s, s) / m) / np.sqrt(m)


def lead_sigma_analytic(lead, eps):
    """Sigma (E, m, m) of a lead with circulant couplings, closed form per angular mode."""
    return lead_sigma_gamma_analytic(lead, eps)[0]


def lead_sigma_gamma_analytic(lead, eps):
    """Sigma and Gamma (E, m, m) of a circulant lead.

    Gamma = i (Sigma - Sigma^dagger) is evaluated in the ring Fourier basis, where Sigma is
    diagonal: Gamma = F diag(i (sigma_j - conj sigma_j)) F^dagger = F diag(-2 Im sigma_j) F^dagger.
    This is the same matrix as the site-basis difference, without its cancellation when
    every mode is closed (Gamma ~ eta, far below |Sigma|)."""
    eps = np.atleast_1d(np.asarray(eps, complex))
    if lead.H0 is not None or lead.H1 is not None:
        raise ValueError("leads with on-site blocks have no closed form here: use decimation")
    a1 = np.abs(circulant_eigenvalues(lead.T1)) ** 2
    a2 = np.abs(circulant_eigenvalues(lead.T2)) ** 2
    at = np.abs(circulant_eigenvalues(lead.tau)) ** 2
    e = (eps - lead.U)[:, None]
    g = surface_gf_dimer(np.broadcast_to(e, (eps.size, a1.size)),
                         np.broadcast_to(a1, (eps.size, a1.size)),
                         np.broadcast_to(a2, (eps.size, a1.size)))
    sig = at[None, :] * g                       # (E, m) per-mode self-energies
    F = fourier_matrix(lead.m)
    Sigma = np.einsum("sj,ej,tj->est", F, sig, F.conj())
    Gamma = np.einsum("sj,ej,tj->est", F, (-2.0 * sig.imag).astype(complex), F.conj())
    return Sigma, Gamma


def surface_gf_sancho(eps, H00, H01, tol=1e-14, max_iter=400):
    """Surface Green's function of a uniform semi-infinite chain of principal layers by
    decimation (Lopez Sancho, Lopez Sancho and Rubio 1985).

    Layers 0, 1, 2, ... with H_{k,k} = H00 and H_{k,k+1} = H01 (H_{k+1,k} = H01^dagger).
    Eliminating every odd layer renormalises (a = H01, c = H01^dagger, g = (E - h)^{-1}):
        h_s <- h_s + a g c,   h <- h + a g c + c g a,   a <- a g a,   c <- c g c,
    until the couplings vanish; then g_surface = (E - h_s)^{-1}.
    eps: (E,) complex energies.  Returns (E, p, p).
    """
    eps = np.atleast_1d(np.asarray(eps, complex))
    p = H00.shape[0]
    I = np.eye(p)
    hs = np.broadcast_to(H00, (eps.size, p, p)).astype(complex).copy()
    h = hs.copy()
    a = np.broadcast_to(H01, (eps.size, p, p)).astype(complex).copy()
    c = np.broadcast_to(H01.conj().T, (eps.size, p, p)).astype(complex).copy()
    Ez = eps[:, None, None] * I
    scale = max(np.abs(H00).max(), np.abs(H01).max(), 1.0)
    for _ in range(max_iter):
        g = np.linalg.inv(Ez - h)
        agc = a @ g @ c
        cga = c @ g @ a
        hs = hs + agc
        h = h + agc + cga
        a = a @ g @ a
        c = c @ g @ c
        if max(np.abs(a).max(), np.abs(c).max()) < tol * scale:
            break
    else:
        raise RuntimeError("decimation did not converge")
    return np.linalg.inv(Ez - hs)


def lead_sigma_sancho(lead, eps):
    """Sigma (E, m, m) of a lead by decimation over two-ring principal layers (s0, s1).

    H00 = [[U + H0, T1^dag], [T1, U + H1]], H_{k,k+1} = [[0, 0], [T2^dag, 0]] (ring s1 of
    layer k to ring s2 of layer k+1), g_{s0} = upper-left block of the layer surface
    function, and Sigma = tau^dagger g_{s0} tau.
    """
    eps = np.atleast_1d(np.asarray(eps, complex))
    m = lead.m
    I = np.eye(m)
    h0 = lead.U * I + (0.0 if lead.H0 is None else np.asarray(lead.H0))
    h1 = lead.U * I + (0.0 if lead.H1 is None else np.asarray(lead.H1))
    H00 = np.block([[h0, lead.T1.conj().T], [lead.T1, h1]])
    Z = np.zeros((m, m))
    H01 = np.block([[Z, Z], [lead.T2.conj().T, Z]])
    gs = surface_gf_sancho(eps, H00, H01)[:, :m, :m]
    return lead.tau.conj().T[None] @ gs @ lead.tau[None]


def lead_sigma(lead, eps, method="analytic"):
    if method == "analytic":
        return lead_sigma_analytic(lead, eps)
    if method == "sancho":
        return lead_sigma_sancho(lead, eps)
    raise ValueError(method)


def broadening(sigma):
    """Gamma = i (Sigma - Sigma^dagger) for stacks (..., m, m)."""
    return 1j * (sigma - np.conj(np.swapaxes(sigma, -1, -2)))
