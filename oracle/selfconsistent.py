"""Self-consistent NEGF-electrostatics loop (Sec. 2.3, Alg. 3) with a 1D Poisson stand-in.

Oracle (test infrastructure only).

Broyden's modified second method (Alg. 3), clean reading:
  * the loop runs while eps_max > tol and m < M (the printed test is inverted);
  * the mixing fraction in the W update is zeta (printed as eta);
  * f_old is saved every iteration (not printed);
  * the variable is the electron count n (the printed denominator rho_in + rho_out can
    vanish for net charges; electron counts are positive);
  * if ||Delta f||^2 = 0 the new V column is zero (the printed step divides by it).
With columns j = 1..m of V^T (M x N) and W (N x M):
  f = n_in - n_out,  Delta f = f - f_old,  eps_max = max_i |f_i| / (n_in,i + n_out,i),
  d = ||Delta f||^2;  if m > 0:
     s = sum_{j<m} W_j (V_j . Delta f);  V_m = Delta f / d;
     W_m = -zeta Delta f + (n_in - n_in_old) - s;   s = sum_{j<=m} W_j (V_j . f)
  else s = 0;   n_in_old <- n_in;  n_in <- n_in_old - zeta f - s;  f_old <- f;  m <- m+1.
This is the rank-one inverse-Jacobian update B_m = B_{m-1} + (Delta n - B_{m-1} Delta f)
Delta f^T / ||Delta f||^2 with B_0 = zeta I and n <- n - B_m f, which ``BroydenDense``
implements literally (the pin).

Poisson stand-in (not in the paper, which solves 3D Poisson with multigrid, Sec. 2.1):
one node per ring, potential energy U in eV,
  U_i - U_G - (lambda/dx)^2 (U_{i+1} - 2 U_i + U_{i-1}) = kappa (n_i - n0_i),
Dirichlet U_{-1} = U_S, U_N = U_D, gate term U_G = Phi_G - V_GS, kappa = e / (C_g dx) with
the coaxial gate capacitance per length C_g = 2 pi eps0 eps_r / ln((2 t_ox + d)/d).
dx = 3 a_cc / 4 = 0.1065 nm (512 rings span 54.53 nm in Table 1), eps_r = 3.9, d = 1.3 nm
(Sec. 3.1), t_ox = 10 nm (Sec. 3.4).  Solved with the Thomas algorithm.

Semi-adaptive real-axis grid inside the loop (Sec. 3.3): the limits E_l1, E_l2 are set from
the singularity peak of the centre-ring integrand at the first iteration of a solve and again
every `period` iterations (the paper uses 50); at such an iteration the peak is located with
the iteration's own potential on the grid in use, then the grid is rebuilt before the NEGF
evaluation.

Several channels (Sec. 2.3): their charge vectors are concatenated into one Broyden
variable; a C x C coupling matrix K in the Poisson stand-in's source term couples the tubes.

Parity: pinned (Thomas vs dense solve, closed-form solution for n = n0, Broyden vs the
dense rank-one form, convergence on a linear map; the refining loop with a period beyond its
iteration count against the plain loop on the refined grid; the coupled Poisson against a dense
block solve, two identical coupled tubes against one tube with kappa + kappa_x).
"""
from dataclasses import dataclass
import numpy as np

EPS0 = 8.8541878128e-12      # F/m
E_CHARGE = 1.602176634e-19   # C


def kappa_from_geometry(eps_r=3.9, d_nm=1.3, t_ox_nm=10.0, dx_nm=0.1065):
    """Potential-energy shift (eV) per electron per ring of the coaxial gate capacitance."""
    Cg = 2.0 * np.pi * EPS0 * eps_r / np.log((2.0 * t_ox_nm + d_nm) / d_nm)   # F/m
    return E_CHARGE / (Cg * dx_nm * 1e-9)                                    # V == eV/e


@dataclass
class PoissonParams:
    kappa: float
    dx_nm: float = 0.1065
    lam_nm: float = 3.0
    U_G: float = 0.0
    U_S: float = 0.0
    U_D: float = 0.0

    @property
    def r(self):
        return (self.lam_nm / self.dx_nm) ** 2


def thomas(sub, diag, sup, rhs):
    """Solve a tridiagonal system (sub[i] = A[i, i-1], sup[i] = A[i, i+1]) by the Thomas
    algorithm (forward elimination, back substitution), no pivoting."""
    n = diag.size
    cp = np.zeros(n)
    dp = np.zeros(n)
    cp[0] = sup[0] / diag[0]
    dp[0] = rhs[0] / diag[0]
    for i in range(1, n):
        den = diag[i] - sub[i] * cp[i - 1]
        cp[i] = sup[i] / den if i < n - 1 else 0.0
        dp[i] = (rhs[i] - sub[i] * dp[i - 1]) / den
    x = np.zeros(n)
    x[n - 1] = dp[n - 1]
    for i in range(n - 2, -1, -1):
        x[i] = dp[i] - cp[i] * x[i + 1]
    return x


def poisson_system(N, p):
    """Bands of the Poisson matrix: diag 1 + 2r, off-diagonals -r."""
    r = p.r
    return np.full(N, -r), np.full(N, 1.0 + 2.0 * r), np.full(N, -r)


def poisson_rhs(n, n0, p):
    r = p.r
    rhs = p.U_G + p.kappa * (np.asarray(n) - np.asarray(n0))
    rhs = rhs.astype(np.float64).copy()
    rhs[0] += r * p.U_S
    rhs[-1] += r * p.U_D
    return rhs


def poisson_solve(n, n0, p):
    sub, dia, sup = poisson_system(len(n), p)
    return thomas(sub, dia, sup, poisson_rhs(n, n0, p))


def poisson_charge(U, n0, p):
    """The electron count whose Poisson solution is exactly U (used to start the loop from
    a given potential)."""
    U = np.asarray(U, dtype=np.float64)
    r = p.r
    left = np.concatenate([[p.U_S], U[:-1]])
    right = np.concatenate([U[1:], [p.U_D]])
    return np.asarray(n0) + ((1.0 + 2.0 * r) * U - r * (left + right) - p.U_G) / p.kappa


def residual(n_in, n_out):
    """eps_max = max_i |n_in - n_out| / (n_in + n_out) (Alg. 3, step 4-7)."""
    return float(np.max(np.abs(n_in - n_out) / (n_in + n_out)))


class Broyden:
    """Broyden's modified second method in the V/W form of Alg. 3 (reading above)."""

    def __init__(self, n_in, zeta, M):
        n_in = np.asarray(n_in, dtype=np.float64)
        N = n_in.size
        self.zeta, self.M = zeta, M
        self.n_in = n_in.copy()
        self.n_in_old = np.zeros(N)
        self.f_old = np.zeros(N)
        self.V = np.zeros((M, N))
        self.W = np.zeros((N, M))
        self.m = 0

    def step(self, n_out):
        if self.m >= self.M:
            raise RuntimeError("Broyden history full")
        f = self.n_in - np.asarray(n_out, dtype=np.float64)
        m = self.m
        if m > 0:
            df = f - self.f_old
            d = float(df @ df)
            k = self.V[:m - 1] @ df
            s = self.W[:, :m - 1] @ k
            self.V[m - 1] = df / d if d > 0.0 else 0.0
            self.W[:, m - 1] = -self.zeta * df + (self.n_in - self.n_in_old) - s
            k = self.V[:m] @ f
            s = self.W[:, :m] @ k
        else:
            s = np.zeros_like(f)
        self.n_in_old = self.n_in.copy()
        self.n_in = self.n_in_old - self.zeta * f - s
        self.f_old = f
        self.m = m + 1
        return self.n_in


class BroydenDense:
    """The same update with the inverse Jacobian stored densely (N x N)."""

    def __init__(self, n_in, zeta):
        n_in = np.asarray(n_in, dtype=np.float64)
        self.n_in = n_in.copy()
        self.n_in_old = None
        self.f_old = None
        self.B = zeta * np.eye(n_in.size)

    def step(self, n_out):
        f = self.n_in - np.asarray(n_out, dtype=np.float64)
        if self.f_old is not None:
            df = f - self.f_old
            dn = self.n_in - self.n_in_old
            d = float(df @ df)
            if d > 0.0:
                self.B = self.B + np.outer(dn - self.B @ df, df) / d
        self.n_in_old = self.n_in.copy()
        self.n_in = self.n_in - self.B @ f
        self.f_old = f
        return self.n_in


def sc_solve(evaluate, U0, n0, p, zeta=0.1, M=64, tol=1e-8):
    """Self-consistent loop: n_in -> Poisson -> U -> NEGF -> n_out -> Broyden (Alg. 3).

    evaluate(U) must return the NEGF dict (``charge.negf_evaluate``) for potential U.
    The loop starts from the potential U0: n_in = poisson_charge(U0), so the first Poisson
    solve returns U0.  Stops when eps_max < tol (converged) or after M NEGF evaluations.
    Returns dict converged, iterations, history, n (n_out of the last evaluation), n_in,
    U, T, I.
    """
    br = Broyden(poisson_charge(U0, n0, p), zeta, M)
    history = []
    r = None
    U = None
    for it in range(M):
        U = poisson_solve(br.n_in, n0, p)
        r = evaluate(U)
        eps = residual(br.n_in, r["n"])
        history.append(eps)
        if eps < tol:
            return dict(converged=True, iterations=it + 1, history=history, n=r["n"],
                        n_in=br.n_in.copy(), U=U, T=r["T"], I=r["I"])
        br.step(r["n"])
    return dict(converged=False, iterations=M, history=history, n=r["n"],
                n_in=br.n_in.copy(), U=U, T=r["T"], I=r["I"])


def sc_solve_adaptive(evaluate, integrand, make_grid, U0, n0, p, limits, a, b, kT, period,
                      zeta=0.1, M=64, tol=1e-8):
    """``sc_solve`` with the semi-adaptive real-axis grid (Sec. 3.3).

    evaluate(U, grid) -> NEGF dict; integrand(U, grid) -> the refinement ring's integrand at
    the grid's real-axis nodes; make_grid(E_l1, E_l2) -> grid.  limits: the initial (E_l1,
    E_l2).  At iteration 0 and at every iteration that is a multiple of `period` (period 0:
    the first only): E_s = peak of integrand(U, grid), limits = (E_s - a kT, E_s + b kT),
    grid = make_grid(limits).  Returns the ``sc_solve`` dict plus grid, limits and the list
    of located peaks.
    """
    from .quadrature import refined_limits
    from .charge import singularity_peak
    grid = make_grid(*limits)
    br = Broyden(poisson_charge(U0, n0, p), zeta, M)
    history, peaks = [], []
    r = None
    U = None
    for it in range(M):
        U = poisson_solve(br.n_in, n0, p)
        if it == 0 or (period > 0 and it % period == 0):
            E_s, _ = singularity_peak(grid["E"], integrand(U, grid))
            peaks.append(E_s)
            limits = refined_limits(E_s, a, b, kT)
            grid = make_grid(*limits)
        r = evaluate(U, grid)
        eps = residual(br.n_in, r["n"])
        history.append(eps)
        if eps < tol:
            return dict(converged=True, iterations=it + 1, history=history, n=r["n"], n_in=br.n_in.copy(),
                        U=U, T=r["T"], I=r["I"], grid=grid, limits=limits, peaks=peaks)
        br.step(r["n"])
    return dict(converged=False, iterations=M, history=history, n=r["n"], n_in=br.n_in.copy(), U=U,
                T=r["T"], I=r["I"], grid=grid, limits=limits, peaks=peaks)


# ---- several channels sharing one Broyden vector (Sec. 2.3, the multi-channel extension)

def poisson_solve_multi(n, n0, p, K):
    """Poisson stand-in of C channels of equal length N, coupled through their charges:

      U_c,i - U_G - r (U_c,i+1 - 2 U_c,i + U_c,i-1) = sum_c' K[c, c'] (n_c',i - n0_c',i),

    Dirichlet U_c,-1 = U_S, U_c,N = U_D for every channel (shared contacts and gate).  K (C x C,
    eV per electron per ring) replaces kappa: K[c, c] is a tube's own gate-screened coupling,
    K[c, c'] the capacitive cross-coupling of two tubes at the same axial position (not in the
    paper, whose 3D electrostatics couples the tubes; a builder-defined stand-in).  n, n0: (C, N).
    """
    n = np.asarray(n, dtype=np.float64)
    q = np.asarray(K, dtype=np.float64) @ (n - np.asarray(n0))
    U = np.zeros_like(n)
    for c in range(n.shape[0]):
        sub, dia, sup = poisson_system(n.shape[1], p)
        rhs = p.U_G + q[c]
        rhs[0] += p.r * p.U_S
        rhs[-1] += p.r * p.U_D
        U[c] = thomas(sub, dia, sup, rhs)
    return U


def poisson_charge_multi(U, n0, p, K):
    """The charges (C, N) whose coupled Poisson solution is exactly U: per ring, K q = L with
    L_c = (1 + 2r) U_c,i - r (U_c,i-1 + U_c,i+1) - U_G."""
    U = np.asarray(U, dtype=np.float64)
    r = p.r
    L = np.zeros_like(U)
    for c in range(U.shape[0]):
        left = np.concatenate([[p.U_S], U[c, :-1]])
        right = np.concatenate([U[c, 1:], [p.U_D]])
        L[c] = (1.0 + 2.0 * r) * U[c] - r * (left + right) - p.U_G
    return np.asarray(n0) + np.linalg.solve(np.asarray(K, dtype=np.float64), L)


def sc_solve_multi(evaluates, U0, n0, p, K, zeta=0.1, M=64, tol=1e-8):
    """Self-consistent loop of C channels with one Broyden vector n = (n^1, ..., n^C) (the
    paper's multi-channel form of Alg. 3: the channel vectors are concatenated before the
    Broyden step and split after it; eps_max and every dot product run over the whole vector).

    evaluates[c](U_c) -> NEGF dict of channel c.  U0, n0: (C, N).  Returns converged,
    iterations, history and per-channel n, U, T, I (lists).
    """
    C, N = np.asarray(U0).shape
    br = Broyden(poisson_charge_multi(U0, n0, p, K).reshape(-1), zeta, M)
    history = []
    for it in range(M):
        U = poisson_solve_multi(br.n_in.reshape(C, N), n0, p, K)
        rs = [evaluates[c](U[c]) for c in range(C)]
        n_out = np.concatenate([r["n"] for r in rs])
        eps = residual(br.n_in, n_out)
        history.append(eps)
        done = eps < tol
        if done or it == M - 1:
            return dict(converged=bool(done), iterations=it + 1, history=history,
                        n=[r["n"] for r in rs], U=list(U), T=[r["T"] for r in rs], I=[r["I"] for r in rs])
        br.step(n_out)
