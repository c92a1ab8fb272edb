"""Retarded Green's function, lead spectral functions and transmission per energy
(Eq. GR, Eq. RhoGeneral, Eq. deviceCharacteristics, Alg. 1, Alg. 2).

Oracle (test infrastructure only).  All functions take a stack of complex energies
``eps`` (E + i eta on the real axis, z on the contour, no eta added there) and work on
every energy at once; nothing else is batched, fused or reordered.

For one chain with layers l = 0..L-1:
  alpha_l = eps I - H_{l,l} - U_l - delta_{l,0} Sigma_S - delta_{l,L-1} Sigma_D
(Eq. GR; the sign of H in the paper's alpha is read as minus), and with the
off-diagonal blocks of G^{-1} equal to -H_{l,l+1}, -H_{l+1,l}:

``dense_lanes``  -- the plain definition: invert the whole (L b) x (L b) matrix.
``rgf_lanes``    -- Alg. 2 read as the textbook left/right-connected recursion:
    y_l = H_{l,l-1} gL_{l-1} H_{l-1,l},  gL_l = (alpha_l - y_l)^{-1}        (forward)
    x_l = H_{l,l+1} gR_{l+1} H_{l+1,l},  gR_l = (alpha_l - x_l)^{-1}        (backward)
    G_{l,l} = (alpha_l - x_l - y_l)^{-1}                                   (Alg. 1, diag)
    G_{l+1,0} = gR_{l+1} H_{l+1,l} G_{l,0}       (first column, below the diagonal)
    G_{l-1,L-1} = gL_{l-1} H_{l-1,l} G_{l,L-1}   (last column, above the diagonal)
  (Alg. 2 as printed uses y before it is defined and swaps beta/gamma; this is the
  reading.)  Then
    A_S,ll = G_{l,0} Gamma_S G_{l,0}^dagger,  A_D,ll = G_{l,L-1} Gamma_D G_{l,L-1}^dagger,
    T(E) = Tr[Gamma_S G_{0,L-1} Gamma_D G_{0,L-1}^dagger].
  Only the two columns the two leads need are formed (the diagonal-only mode of Sec.
  2.2.4 still needs G_{T,k} for the lead blocks k).

Parity: pinned (dense == recursion, sum rule i(G - G^dagger) = G (Gamma_S + Gamma_D +
2 eta I) G^dagger, reciprocity, Hermiticity and positivity of A_l, integer transmission
plateaus, real space == sum of mode chains).
"""
import numpy as np
from .leads import lead_sigma, broadening, lead_sigma_gamma_analytic


def _embed(blocks, sites, b):
    """Place (E, m, m) lead blocks at rows/cols ``sites`` of (E, b, b) zero blocks."""
    out = np.zeros((blocks.shape[0], b, b), complex)
    out[:, sites[:, None], sites[None, :]] = blocks
    return out


def contact_blocks(chain, eps, method="analytic"):
    """Sigma_S on layer 0 and Sigma_D on layer L-1, as (E, b, b) stacks, and their Gammas
    (Gamma = i (Sigma - Sigma^dagger); analytic leads evaluate it in the mode basis)."""
    if method == "analytic":
        out = []
        for lead in (chain.lead_S, chain.lead_D):
            s, gm = lead_sigma_gamma_analytic(lead, eps)
            out.append((_embed(s, lead.sites, chain.b), _embed(gm, lead.sites, chain.b)))
        return out[0][0], out[1][0], out[0][1], out[1][1]
    sS = _embed(lead_sigma(chain.lead_S, eps, method), chain.lead_S.sites, chain.b)
    sD = _embed(lead_sigma(chain.lead_D, eps, method), chain.lead_D.sites, chain.b)
    return sS, sD, broadening(sS), broadening(sD)


def _alphas(chain, U, eps, sS, sD):
    E = eps.size
    b, L = chain.b, chain.L
    D = chain.diag_blocks(U)                                   # (L, b, b)
    alpha = eps[None, :, None, None] * np.eye(b) - D[:, None]  # (L, E, b, b)
    alpha = alpha.copy()
    alpha[0] -= sS
    alpha[L - 1] -= sD
    return alpha


def _dag(x):
    return np.conj(np.swapaxes(x, -1, -2))


def dense_lanes(chain, U, eps, method="analytic", eta=0.0):
    """Dense inverse of eps I - H - Sigma (tiny systems only).

    Returns dict: G (E, Lb, Lb), Gdiag (E, L, b), AS, AD (E, L, b) real diagonals of the lead
    spectral functions, T (E,), GammaS_full / GammaD_full (E, Lb, Lb) embedded Gammas.
    """
    eps = np.atleast_1d(np.asarray(eps, complex))
    L, b = chain.L, chain.b
    n = L * b
    sS, sD, gS, gD = contact_blocks(chain, eps, method)
    from .model import dense_hamiltonian
    H = dense_hamiltonian(chain, U)
    M = eps[:, None, None] * np.eye(n) - H[None]
    M[:, :b, :b] -= sS
    M[:, n - b:, n - b:] -= sD
    G = np.linalg.inv(M)
    GamS = np.zeros_like(M)
    GamD = np.zeros_like(M)
    GamS[:, :b, :b] = gS
    GamD[:, n - b:, n - b:] = gD
    AS = G @ GamS @ _dag(G)
    AD = G @ GamD @ _dag(G)
    idx = np.arange(n)
    G0N = G[:, :b, n - b:]
    T = np.einsum("eij,ejk,ekl,eli->e", gS, G0N, gD, _dag(G0N)).real
    return dict(G=G, Gdiag=G[:, idx, idx].reshape(-1, L, b),
                AS=AS[:, idx, idx].real.reshape(-1, L, b),
                AD=AD[:, idx, idx].real.reshape(-1, L, b),
                T=T, AS_full=AS, AD_full=AD, GammaS_full=GamS, GammaD_full=GamD)


def rgf_lanes(chain, U, eps, method="analytic", spectral=True, blocks=False):
    """Block recursion of Alg. 1 / Alg. 2 (reading in the module docstring).

    spectral=False (contour lanes): only G_ll is formed.
    Returns dict with Gdiag (E, L, b) complex and, if spectral, AS, AD (E, L, b) real
    diagonals, T (E,), T_DS (E,) = Tr[Gamma_D G_{L-1,0} Gamma_S G_{L-1,0}^dagger]; with
    blocks=True also the full (L, E, b, b) blocks G_ll, A_S,ll, A_D,ll.
    """
    eps = np.atleast_1d(np.asarray(eps, complex))
    L, b = chain.L, chain.b
    E = eps.size
    sS, sD, gS, gD = contact_blocks(chain, eps, method)
    alpha = _alphas(chain, U, eps, sS, sD)
    Hup = chain.Hup.astype(complex)                 # H_{l,l+1}
    Hdn = _dag(Hup)                                 # H_{l+1,l}
    inv = np.linalg.inv

    gL = np.empty((L, E, b, b), complex)
    y = np.zeros((L, E, b, b), complex)
    gL[0] = inv(alpha[0])
    for l in range(1, L):
        y[l] = Hdn[l - 1] @ gL[l - 1] @ Hup[l - 1]
        gL[l] = inv(alpha[l] - y[l])

    gR = np.empty((L, E, b, b), complex)
    x = np.zeros((L, E, b, b), complex)
    gR[L - 1] = inv(alpha[L - 1])
    for l in range(L - 2, -1, -1):
        x[l] = Hup[l] @ gR[l + 1] @ Hdn[l]
        gR[l] = inv(alpha[l] - x[l])

    Gll = inv(alpha - x - y)                        # (L, E, b, b)
    idx = np.arange(b)
    out = dict(Gdiag=np.moveaxis(Gll[:, :, idx, idx], 0, 1))
    if blocks:
        out["G_blocks"] = Gll
    if not spectral:
        return out

    col0 = np.empty((L, E, b, b), complex)          # G_{l,0}
    colN = np.empty((L, E, b, b), complex)          # G_{l,L-1}
    col0[0] = Gll[0]
    for l in range(0, L - 1):
        col0[l + 1] = gR[l + 1] @ Hdn[l] @ col0[l]
    colN[L - 1] = Gll[L - 1]
    for l in range(L - 1, 0, -1):
        colN[l - 1] = gL[l - 1] @ Hup[l - 1] @ colN[l]

    AS = col0 @ gS[None] @ _dag(col0)
    AD = colN @ gD[None] @ _dag(colN)
    out["AS"] = np.moveaxis(AS[:, :, idx, idx].real, 0, 1)
    out["AD"] = np.moveaxis(AD[:, :, idx, idx].real, 0, 1)
    G0N = colN[0]
    GN0 = col0[L - 1]
    out["T"] = np.einsum("eij,ejk,ekl,eli->e", gS, G0N, gD, _dag(G0N)).real
    out["T_DS"] = np.einsum("eij,ejk,ekl,eli->e", gD, GN0, gS, _dag(GN0)).real
    if blocks:
        out["AS_blocks"] = AS
        out["AD_blocks"] = AD
    return out
