"""Block-tridiagonal tight-binding chains of (n,0) zigzag nanotubes (Sec. 2.2.1-2.2.2, Sec. 3.1).

Oracle (test infrastructure only).

A *chain* is one block-tridiagonal Hamiltonian with L layers of width b:
  Hdiag[l]  = H_{l,l}   without the electrostatic potential,
  Hup[l]    = H_{l,l+1} (the lower blocks are Hup[l]^dagger, H is Hermitian),
  site_ring[l, a] = ring index of site a of layer l (the potential U is per ring and the
                    charge is reported per ring),
  g_b       = band degeneracy of the chain (spin degeneracy g_s = 2 is global),
plus a semi-infinite lead at each end.  A *device* is a ring count and a list of chains
sharing one potential: several mode-space subbands are independent chains, as the paper
stores multi-mode blocks as arrays of diagonal entries (Sec. 2.2.2, Sec. 3.2).

Leads.  A lead is a semi-infinite sequence of rings s0, s1, s2, ... moving away from the
device, each of m sites with on-site energy U_lead, couplings H_{s1,s0} = T1,
H_{s2,s1} = T2, H_{s3,s2} = T1, ... and device coupling tau = H_{s0, boundary ring}.  The
boundary ring occupies ``sites`` of the first (source) or last (drain) layer.

Nanotube readings (Sec. 3.1 gives a (17,0) tube with nearest-neighbour coupling between
rings; the mode-space chain follows the cited Guo et al. construction):
* Bond k joins ring k and ring k+1.  Mode j of an (n,0) tube: bond k is t for even k and
  b_j = 2 t cos(pi j / n) for odd k ("t first"); the leads continue the same
  alternation outwards.  Each mode is doubly degenerate (j and n - j), g_b = 2.
* Real space: ring blocks are n x n with no intra-ring bonds; bond k is t I for even k
  (axial bonds), t (I + S) for k = 1 mod 4 and t (I + S^T) for k = 3 mod 4 (the two
  orientations of the zigzag bonds), with S the cyclic shift S[r, r-1] = 1.  All n
  angular modes are explicit, g_b = 1.
* 2 x 2 unit-cell blocks regroup rings (2l, 2l+1) of a mode chain into one layer.

Parity: pinned by the Bloch dispersion of the infinite chain (closed form), the band gap
the paper prints for (17,0), and the block/mode equivalences in the tests.
"""
from dataclasses import dataclass
import numpy as np

G_SPIN = 2.0


@dataclass
class Lead:
    U: float            # on-site potential energy of the lead rings (eV)
    T1: np.ndarray      # (m, m) H_{s1,s0}
    T2: np.ndarray      # (m, m) H_{s2,s1}
    tau: np.ndarray     # (m, m) H_{s0, boundary ring of the device}
    sites: np.ndarray   # (m,) site indices of the boundary ring inside its layer
    H0: np.ndarray = None   # (m, m) on-site block of rings s0, s2, ... besides U (None: zero)
    H1: np.ndarray = None   # (m, m) on-site block of rings s1, s3, ... besides U (None: zero)

    @property
    def m(self):
        return self.T1.shape[0]


@dataclass
class Chain:
    Hdiag: np.ndarray       # (L, b, b) complex
    Hup: np.ndarray         # (L-1, b, b) complex
    site_ring: np.ndarray   # (L, b) int
    lead_S: Lead
    lead_D: Lead
    g_b: float = 1.0

    @property
    def L(self):
        return self.Hdiag.shape[0]

    @property
    def b(self):
        return self.Hdiag.shape[1]

    def diag_blocks(self, U):
        """H_{l,l} + U at every site (U indexed by ring)."""
        U = np.asarray(U, dtype=np.float64)
        D = self.Hdiag.astype(complex).copy()
        idx = np.arange(self.b)
        D[:, idx, idx] += U[self.site_ring]
        return D


@dataclass
class Device:
    n_rings: int
    chains: list


def mode_bond(k, t, bj):
    """Bond k of a mode-space chain: t for even k, b_j for odd k (any integer k)."""
    return t if k % 2 == 0 else bj


def mode_hopping(n_tube, j, t):
    """b_j = 2 t cos(pi j / n) of mode j of an (n,0) zigzag tube."""
    return 2.0 * t * np.cos(np.pi * j / n_tube)


def _scalar_lead(U, T1, T2, tau, site):
    one = lambda v: np.array([[v]], dtype=complex)
    return Lead(U=float(U), T1=one(T1), T2=one(T2), tau=one(tau), sites=np.array([site]))


def mode_chain(n_tube, j, t, N, U_S, U_D, g_b=2.0):
    """1 x 1 mode-space chain of N rings for mode j (bond k = t if k even else b_j)."""
    bj = mode_hopping(n_tube, j, t)
    Hdiag = np.zeros((N, 1, 1), complex)
    Hup = np.array([[[mode_bond(k, t, bj)]] for k in range(N - 1)], complex).reshape(N - 1, 1, 1)
    site_ring = np.arange(N).reshape(N, 1)
    # source: s0 = ring -1, tau = H_{-1,0} = bond(-1); T1 = H_{-2,-1} = bond(-2); T2 = bond(-3)
    lS = _scalar_lead(U_S, mode_bond(-2, t, bj), mode_bond(-3, t, bj), mode_bond(-1, t, bj), 0)
    # drain: s0 = ring N, tau = H_{N,N-1} = bond(N-1); T1 = bond(N); T2 = bond(N+1)
    lD = _scalar_lead(U_D, mode_bond(N, t, bj), mode_bond(N + 1, t, bj), mode_bond(N - 1, t, bj), 0)
    return Chain(Hdiag, Hup, site_ring, lS, lD, g_b)


def mode_chain_cells(n_tube, j, t, N, U_S, U_D, g_b=2.0):
    """The same mode chain regrouped into N/2 layers of 2 x 2 blocks (rings 2l, 2l+1)."""
    if N % 2:
        raise ValueError("2x2 unit cells need an even ring count")
    bj = mode_hopping(n_tube, j, t)
    L = N // 2
    Hdiag = np.zeros((L, 2, 2), complex)
    Hup = np.zeros((L - 1, 2, 2), complex)
    for l in range(L):
        h = mode_bond(2 * l, t, bj)
        Hdiag[l, 0, 1] = h
        Hdiag[l, 1, 0] = h
    for l in range(L - 1):
        Hup[l, 1, 0] = mode_bond(2 * l + 1, t, bj)   # ring 2l+1 -> ring 2l+2
    site_ring = np.arange(N).reshape(L, 2)
    lS = _scalar_lead(U_S, mode_bond(-2, t, bj), mode_bond(-3, t, bj), mode_bond(-1, t, bj), 0)
    lD = _scalar_lead(U_D, mode_bond(N, t, bj), mode_bond(N + 1, t, bj), mode_bond(N - 1, t, bj), 1)
    return Chain(Hdiag, Hup, site_ring, lS, lD, g_b)


def shift_matrix(m):
    """Cyclic shift S with S[r, r-1 mod m] = 1."""
    S = np.zeros((m, m))
    for r in range(m):
        S[r, (r - 1) % m] = 1.0
    return S


def realspace_bond(k, t, n_tube):
    """H_{k,k+1} of the real-space (n,0) tube: t I (k even), t(I+S) (k=1 mod 4), t(I+S^T) (k=3 mod 4)."""
    I = np.eye(n_tube)
    S = shift_matrix(n_tube)
    if k % 2 == 0:
        return t * I
    if k % 4 == 1:
        return t * (I + S)
    return t * (I + S.T)


def realspace_chain(n_tube, t, N, U_S, U_D, g_b=1.0):
    """Real-space (n,0) chain of N rings, n x n ring blocks, leads continuing the tube."""
    n = n_tube
    Hdiag = np.zeros((N, n, n), complex)
    Hup = np.array([realspace_bond(k, t, n) for k in range(N - 1)], complex)
    site_ring = np.repeat(np.arange(N), n).reshape(N, n)
    sites = np.arange(n)
    cplx = lambda M: np.asarray(M, complex)
    lS = Lead(U=float(U_S), T1=cplx(realspace_bond(-2, t, n)), T2=cplx(realspace_bond(-3, t, n)),
              tau=cplx(realspace_bond(-1, t, n)), sites=sites)
    lD = Lead(U=float(U_D), T1=cplx(realspace_bond(N, t, n).conj().T),
              T2=cplx(realspace_bond(N + 1, t, n).conj().T),
              tau=cplx(realspace_bond(N - 1, t, n).conj().T), sites=sites)
    return Chain(Hdiag, Hup, site_ring, lS, lD, g_b)


def dense_hamiltonian(chain, U):
    """The full (L b) x (L b) Hermitian matrix of a chain with potential U."""
    L, b = chain.L, chain.b
    H = np.zeros((L * b, L * b), complex)
    D = chain.diag_blocks(U)
    for l in range(L):
        H[l * b:(l + 1) * b, l * b:(l + 1) * b] = D[l]
    for l in range(L - 1):
        H[l * b:(l + 1) * b, (l + 1) * b:(l + 2) * b] = chain.Hup[l]
        H[(l + 1) * b:(l + 2) * b, l * b:(l + 1) * b] = chain.Hup[l].conj().T
    return H


def bloch_hamiltonian(bond, cell, k):
    """Bloch matrix of an infinite chain of blocks with H_{r,r+1} = bond(r), cell rings per period.

    H(k) = sum over bonds inside one period plus the bond leaving it times exp(i k),
    on the basis of the `cell` rings of one period.
    """
    B0 = np.atleast_2d(bond(0))
    m = B0.shape[0]
    H = np.zeros((cell * m, cell * m), complex)
    for r in range(cell - 1):
        Br = np.atleast_2d(bond(r))
        H[r * m:(r + 1) * m, (r + 1) * m:(r + 2) * m] += Br
        H[(r + 1) * m:(r + 2) * m, r * m:(r + 1) * m] += Br.conj().T
    Bx = np.atleast_2d(bond(cell - 1))     # ring cell-1 -> ring cell (= ring 0 of next period)
    H[(cell - 1) * m:cell * m, 0:m] += Bx * np.exp(1j * k)
    H[0:m, (cell - 1) * m:cell * m] += Bx.conj().T * np.exp(-1j * k)
    return H


def cnt_build(kind, n_tube, t, N, U_S, U_D, modes=(1,), cells=False):
    """Device of one nanotube: mode space (one chain per listed mode) or real space."""
    if kind == "mode":
        mk = mode_chain_cells if cells else mode_chain
        return Device(N, [mk(n_tube, j, t, N, U_S, U_D) for j in modes])
    if kind == "real":
        return Device(N, [realspace_chain(n_tube, t, N, U_S, U_D)])
    raise ValueError(kind)
