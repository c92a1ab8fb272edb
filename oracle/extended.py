"""Extended-precision ground truth for general (non-circulant) leads (Eq. GR, Sec. 2.2.2;
Alg. 1 / Alg. 2 as read; Eq. Rho, Eq. deviceCharacteristics).

Oracle (test infrastructure only; needs mpmath).  The FP64 oracle decimates a general lead
and runs the block recursion in double precision; near a lead band edge both steps are
ill-conditioned, and two FP64 implementations (the oracle and the GPU) can then differ by more
than 1e-10 without either being wrong.  This module runs the same mathematics with mpmath at
``DPS`` significant digits, so that its results serve as a ground truth for both:

* ``surface_gf``: the decimation of a uniform semi-infinite chain of principal layers
  (renormalised couplings a = H01, c = H01^dagger, g = (E - h)^{-1};
  h_s <- h_s + a g c, h <- h + a g c + c g a, a <- a g a, c <- c g c until the couplings fall
  below 1e-(DPS - 4) of the layer blocks; g_surface = (E - h_s)^{-1});
* ``lead_sigma``: the two-ring principal layer of a lead (rings s0, s1 with on-site blocks
  U + H0, U + H1, coupling T1, next coupling T2) and Sigma = tau^dagger g_s0 tau;
* ``lanes``: per energy the left- and right-connected recursions, G_ll = (alpha_l - x_l -
  y_l)^{-1}, the lead columns G_{l,0} and G_{l,L-1}, the spectral diagonals
  A_l = G Gamma_l G^dagger and T = Tr[Gamma_S G_{0,L-1} Gamma_D G_{0,L-1}^dagger];
* ``evaluate``: the ring electron counts, T(E) and the Landauer current on a given grid (the
  same quadrature sums as ``oracle.charge.negf_evaluate``);
* ``condition``: the relative sensitivity of T(E) and of the ring counts to relative
  perturbations of every Hamiltonian and lead block (a condition estimate kappa, so that an
  FP64 result is expected within a modest multiple of kappa u, u = 2^-53).

Parity: pinned by ``tests/test_oracle_extended.py`` (the FP64 oracle against this module on
circulant leads, where the FP64 closed form is well conditioned; decimation of a circulant
lead against the closed-form surface function; the textbook uniform chain).
"""
import mpmath as mp
import numpy as np

DPS = 30
mp.mp.dps = DPS
G_SPIN = 2.0
E_CHARGE = mp.mpf("1.602176634e-19")   # C (exact, SI 2019)
H_PLANCK = mp.mpf("6.62607015e-34")    # J s (exact, SI 2019)
E2_OVER_H = E_CHARGE * E_CHARGE / H_PLANCK   # A / V (current with energies in eV)


def _c(v):
    """A double (or an mpmath number of a perturbed block) as an mpmath complex, exactly."""
    if isinstance(v, (mp.mpc, mp.mpf)):
        return mp.mpc(v)
    return mp.mpc(float(np.real(v)), float(np.imag(v)))


def _m(a):
    """(p, q) array of doubles or mpmath numbers -> mpmath matrix (exact)."""
    a = np.asarray(a)
    out = mp.matrix(a.shape[0], a.shape[1])
    for i in range(a.shape[0]):
        for j in range(a.shape[1]):
            out[i, j] = _c(a[i, j])
    return out


def _eye(p):
    return mp.eye(p)


def _dag(a):
    return a.transpose_conj()


def _maxabs(a):
    return max(abs(a[i, j]) for i in range(a.rows) for j in range(a.cols))


def _block(rows):
    """Assemble a block matrix from a list of rows of mpmath matrices."""
    nr = sum(r[0].rows for r in rows)
    nc = sum(b.cols for b in rows[0])
    out = mp.matrix(nr, nc)
    i0 = 0
    for r in rows:
        j0 = 0
        for b in r:
            for i in range(b.rows):
                for j in range(b.cols):
                    out[i0 + i, j0 + j] = b[i, j]
            j0 += b.cols
        i0 += r[0].rows
    return out


def _sub(a, i0, i1, j0, j1):
    out = mp.matrix(i1 - i0, j1 - j0)
    for i in range(i0, i1):
        for j in range(j0, j1):
            out[i - i0, j - j0] = a[i, j]
    return out


def surface_gf(eps, H00, H01, max_iter=400):
    """Surface Green's function of the semi-infinite chain H00, H01 at one complex energy."""
    p = H00.rows
    Ez = eps * _eye(p)
    hs = H00.copy()
    h = H00.copy()
    a = H01.copy()
    c = _dag(H01)
    scale = max(_maxabs(H00), _maxabs(H01), mp.mpf(1))
    tol = mp.mpf(10) ** (-(DPS - 4)) * scale
    for _ in range(max_iter):
        g = mp.inverse(Ez - h)
        ga = g * a
        gc = g * c
        agc = a * gc
        cga = c * ga
        hs = hs + agc
        h = h + agc + cga
        a = a * ga
        c = c * gc
        if max(_maxabs(a), _maxabs(c)) < tol:
            return mp.inverse(Ez - hs)
    raise RuntimeError("extended-precision decimation did not converge")


def lead_sigma(lead, eps):
    """Sigma (m x m) of a lead at one complex energy, by decimation of two-ring layers."""
    m = lead.m
    I = _eye(m)
    h0 = mp.mpf(float(lead.U)) * I + (_m(lead.H0) if lead.H0 is not None else mp.zeros(m, m))
    h1 = mp.mpf(float(lead.U)) * I + (_m(lead.H1) if lead.H1 is not None else mp.zeros(m, m))
    # (T1, T2, tau may be object arrays of a perturbed lead; _m keeps them exact)
    T1 = _m(lead.T1)
    T2 = _m(lead.T2)
    Z = mp.zeros(m, m)
    H00 = _block([[h0, _dag(T1)], [T1, h1]])
    H01 = _block([[Z, Z], [_dag(T2), Z]])
    gs = _sub(surface_gf(eps, H00, H01), 0, m, 0, m)
    tau = _m(lead.tau)
    return _dag(tau) * gs * tau


def _embed(blk, sites, b):
    out = mp.zeros(b, b)
    for s, i in enumerate(sites):
        for t, j in enumerate(sites):
            out[int(i), int(j)] = blk[s, t]
    return out


def lanes(chain, U, eps, spectral=True, sig=None):
    """One energy: ring-resolved diagonals of one chain.  Returns dict with Gdiag (L, b) and,
    if spectral, AS, AD (L, b) and T.  sig = (Sigma_S, Sigma_D) may be passed in (they depend
    on the energy only)."""
    L, b = chain.L, chain.b
    if sig is None:
        sig = (lead_sigma(chain.lead_S, eps), lead_sigma(chain.lead_D, eps))
    sS = _embed(sig[0], chain.lead_S.sites, b)
    sD = _embed(sig[1], chain.lead_D.sites, b)
    alpha = []
    for l in range(L):
        Dl = _m(chain.Hdiag[l])   # H_ll + U of the site's ring on the diagonal
        for i in range(b):
            Dl[i, i] = Dl[i, i] + mp.mpf(float(U[int(chain.site_ring[l, i])]))
        a = eps * _eye(b) - Dl
        if l == 0:
            a = a - sS
        if l == L - 1:
            a = a - sD
        alpha.append(a)
    Hup = [_m(chain.Hup[l]) for l in range(L - 1)]
    Hdn = [_dag(x) for x in Hup]
    gL = [None] * L
    y = [mp.zeros(b, b) for _ in range(L)]
    gL[0] = mp.inverse(alpha[0])
    for l in range(1, L):
        y[l] = Hdn[l - 1] * gL[l - 1] * Hup[l - 1]
        gL[l] = mp.inverse(alpha[l] - y[l])
    gR = [None] * L
    x = [mp.zeros(b, b) for _ in range(L)]
    gR[L - 1] = mp.inverse(alpha[L - 1])
    for l in range(L - 2, -1, -1):
        x[l] = Hup[l] * gR[l + 1] * Hdn[l]
        gR[l] = mp.inverse(alpha[l] - x[l])
    G = [mp.inverse(alpha[l] - x[l] - y[l]) for l in range(L)]
    out = {"Gdiag": [[G[l][i, i] for i in range(b)] for l in range(L)]}
    if not spectral:
        return out
    gamS = 1j * (sS - _dag(sS))
    gamD = 1j * (sD - _dag(sD))
    col0 = [None] * L
    colN = [None] * L
    col0[0] = G[0]
    for l in range(L - 1):
        col0[l + 1] = gR[l + 1] * Hdn[l] * col0[l]
    colN[L - 1] = G[L - 1]
    for l in range(L - 1, 0, -1):
        colN[l - 1] = gL[l - 1] * Hup[l - 1] * colN[l]
    AS, AD = [], []
    for l in range(L):
        a_s = col0[l] * gamS * _dag(col0[l])
        a_d = colN[l] * gamD * _dag(colN[l])
        AS.append([a_s[i, i].real for i in range(b)])
        AD.append([a_d[i, i].real for i in range(b)])
    G0N = colN[0]
    M = gamS * G0N * gamD * _dag(G0N)
    out["AS"] = AS
    out["AD"] = AD
    out["T"] = sum(M[i, i] for i in range(b)).real
    return out


def _ring_sum(chain, n_rings, vals):
    out = [mp.mpf(0)] * n_rings
    for l in range(chain.L):
        for i in range(chain.b):
            r = int(chain.site_ring[l, i])
            out[r] = out[r] + vals[l][i]
    return out


def evaluate(device, U, grid):
    """Ring electron counts, T(E) and the current on a grid (the quadrature sums of
    oracle.charge.negf_evaluate).  Returns mpmath values: n, n_real, n_cont (lists), T (list),
    I."""
    NR = device.n_rings
    E, w, fS, fD, eta = grid["E"], grid["w"], grid["fS"], grid["fD"], grid["eta"]
    z, c = grid["z"], grid["c"]
    n_real = [mp.mpf(0)] * NR
    n_cont = [mp.mpf(0)] * NR
    T = [mp.mpf(0)] * len(E)
    for ch in device.chains:
        g = mp.mpf(G_SPIN * ch.g_b)
        for k in range(len(E)):
            eps = mp.mpc(float(E[k]), float(eta))
            r = lanes(ch, U, eps)
            aS = _ring_sum(ch, NR, r["AS"])
            aD = _ring_sum(ch, NR, r["AD"])
            wk, fs, fd = mp.mpf(float(w[k])), mp.mpf(float(fS[k])), mp.mpf(float(fD[k]))
            for i in range(NR):
                n_real[i] += g / (2 * mp.pi) * wk * (fs * aS[i] + fd * aD[i])
            T[k] += mp.mpf(ch.g_b) * r["T"]
        for k in range(len(z)):
            zk = mp.mpc(float(z[k].real), float(z[k].imag))
            ck = mp.mpc(float(c[k].real), float(c[k].imag))
            r = lanes(ch, U, zk, spectral=False)
            gr = _ring_sum(ch, NR, r["Gdiag"])
            for i in range(NR):
                n_cont[i] += g / mp.pi * (ck * gr[i]).imag
    I = G_SPIN * E2_OVER_H * sum(mp.mpf(float(w[k])) * T[k] * (mp.mpf(float(fS[k])) - mp.mpf(float(fD[k])))
                                         for k in range(len(E)))
    return {"n": [a + b for a, b in zip(n_real, n_cont)], "n_real": n_real, "n_cont": n_cont, "T": T, "I": I}


def condition(device, U, grid, delta=1e-20, samples=2, seed=0):
    """Condition estimate: the largest relative change of T(E) (per energy, relative to
    max_k |T|) and of the ring counts (relative to max_i |n_i|) under relative perturbations
    of size delta of every Hamiltonian and lead block (independent random signs per
    element), divided by delta; the largest over a few samples."""
    import copy
    base = evaluate(device, U, grid)
    Tmax = max(abs(t) for t in base["T"]) if base["T"] else mp.mpf(1)
    nmax = max(abs(x) for x in base["n"])
    rng = np.random.default_rng(seed)
    kT = [mp.mpf(0)] * len(base["T"])
    kn = mp.mpf(0)
    old = mp.mp.dps
    mp.mp.dps = DPS + 15
    try:
        for _ in range(samples):
            dev = copy.deepcopy(device)
            for ch in dev.chains:
                ch.Hdiag = _perturb(ch.Hdiag, rng, delta)
                ch.Hup = _perturb(ch.Hup, rng, delta)
                for ld in (ch.lead_S, ch.lead_D):
                    for f in ("T1", "T2", "tau", "H0", "H1"):
                        if getattr(ld, f) is not None:
                            setattr(ld, f, _perturb(getattr(ld, f), rng, delta))
            pert = evaluate(dev, U, grid)
            for k in range(len(kT)):
                kT[k] = max(kT[k], abs(pert["T"][k] - base["T"][k]) / (Tmax * delta))
            kn = max(kn, max(abs(a - b) for a, b in zip(pert["n"], base["n"])) / (nmax * delta))
    finally:
        mp.mp.dps = old
    return {"kappa_T": [float(x) for x in kT], "kappa_n": float(kn)}


def _perturb(a, rng, delta):
    """Relative perturbation of every element, kept in extended precision as an object array
    of mpmath complex numbers (so that a perturbation of 1e-20 survives)."""
    a = np.asarray(a)
    s = rng.choice([-1.0, 1.0], size=a.shape)
    out = np.empty(a.shape, dtype=object)
    for idx in np.ndindex(a.shape):
        out[idx] = _c(a[idx]) * (1 + mp.mpf(s[idx]) * mp.mpf(delta))
    return out
