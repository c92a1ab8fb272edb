"""Quadrature rules and energy grids of the charge integral (Sec. 2.2.1, Eq. Rho).

Oracle (test infrastructure only). The paper splits the electron density into an
equilibrium part integrated on a complex contour below E_min and a non-equilibrium part
integrated on the real axis between E_min = mu_min - f1 kT and E_max = mu_max + f2 kT,
with f1 = f2 = 14 by default, using Gauss-Legendre rules (Sec. 2.2.1 and Sec. 3.3).

Readings (the paper gives neither the contour shape nor every grid rule):

* Contour: a semicircle in the upper half plane over [E_B, E_min], centre
  c = (E_B + E_min)/2, radius R = (E_min - E_B)/2, z(theta) = c + R exp(i theta) with a
  Gauss-Legendre rule in theta on [0, pi].  Because G^R is analytic in the upper half
  plane and the Fermi poles mu + i pi kT (2k+1) lie to the right of E_min, Cauchy's
  theorem turns the real-axis integral from E_B to E_min into minus the integral along
  the arc taken from theta = 0 to theta = pi.  No residue terms are needed.
* E_B lies below every band of the device and of the leads, so nothing below E_B
  contributes (apart from O(eta) tails).
* The uniform real-axis grid of the small mode-space workload is read as the midpoint
  rule, which never places a node on the end shared with the contour.

Parity: pinned (GL exactness on polynomials, agreement with numpy's leggauss, closed-form
contour integrals of rational functions, Fermi symmetry).
"""
import numpy as np

F1_DEFAULT = 14.0
F2_DEFAULT = 14.0


def gauss_legendre(n):
    """Nodes and weights of the n-point Gauss-Legendre rule on [-1, 1].

    Method: Newton's iteration on the Legendre polynomial P_n, evaluated with the
    three-term (Bonnet) recurrence (j+1) P_{j+1} = (2j+1) x P_j - j P_{j-1}, started from
    the Tricomi-type guess cos(pi (k - 1/4)/(n + 1/2)).  Weights w_k = 2 / ((1 - x_k^2)
    P_n'(x_k)^2).  Returned in ascending order of the nodes.
    """
    if n < 1:
        raise ValueError("n must be >= 1")
    k = np.arange(1, n + 1, dtype=np.float64)
    x = np.cos(np.pi * (k - 0.25) / (n + 0.5))
    for _ in range(100):
        p_prev = np.ones_like(x)
        p = x.copy()
        for j in range(1, n):
            p_prev, p = p, ((2 * j + 1) * x * p - j * p_prev) / (j + 1)
        dp = n * (x * p - p_prev) / (x * x - 1.0)
        dx = p / dp
        x = x - dx
        if np.max(np.abs(dx)) < 1e-16:
            break
    # final derivative at the converged nodes
    p_prev = np.ones_like(x)
    p = x.copy()
    for j in range(1, n):
        p_prev, p = p, ((2 * j + 1) * x * p - j * p_prev) / (j + 1)
    dp = n * (x * p - p_prev) / (x * x - 1.0)
    w = 2.0 / ((1.0 - x * x) * dp * dp)
    order = np.argsort(x)
    return x[order], w[order]


def fermi(x, kT):
    """Fermi-Dirac occupation f(x) = 1 / (1 + exp(x / kT)) of an energy x = E - mu.

    Real x uses the overflow-free branch; complex x (contour nodes, Re x << 0 there) uses
    the definition directly, which is the analytic continuation used in Eq. Rho.
    """
    x = np.asarray(x)
    if np.iscomplexobj(x):
        return 1.0 / (1.0 + np.exp(x / kT))
    y = x / kT
    out = np.empty_like(y, dtype=np.float64)
    pos = y > 0
    e = np.exp(-y[pos])
    out[pos] = e / (1.0 + e)
    out[~pos] = 1.0 / (1.0 + np.exp(y[~pos]))
    return out


def real_axis_midpoint(a, b, n):
    """Midpoint rule on [a, b]: E_k = a + (k + 1/2) h, w_k = h, h = (b - a)/n."""
    h = (b - a) / n
    E = a + (np.arange(n, dtype=np.float64) + 0.5) * h
    return E, np.full(n, h)


def real_axis_gauss(a, b, n):
    """n-point Gauss-Legendre rule mapped affinely onto [a, b]."""
    x, w = gauss_legendre(n)
    half = 0.5 * (b - a)
    return 0.5 * (a + b) + half * x, half * w


def contour_semicircle(E_B, E_min, n):
    """Nodes z_k and Jacobian-weighted weights W_k z'(theta_k) of the arc over [E_B, E_min].

    theta_k = (pi/2)(1 + x_k), W_k = (pi/2) w_k with (x_k, w_k) the n-point GL rule, and
    z'(theta) = i R exp(i theta).  For F analytic in the closed upper half disc,
    integral_{E_B}^{E_min} F(E) dE = - sum_k W_k z'_k F(z_k) (up to the GL error).
    """
    if not E_min > E_B:
        raise ValueError("need E_min > E_B")
    x, w = gauss_legendre(n)
    theta = 0.5 * np.pi * (1.0 + x)
    W = 0.5 * np.pi * w
    c = 0.5 * (E_B + E_min)
    R = 0.5 * (E_min - E_B)
    z = c + R * np.exp(1j * theta)
    dz = 1j * R * np.exp(1j * theta)
    return z, W * dz


def bias_grid(mu_S, mu_D, kT, n_real, n_cont, E_B, eta, rule="gauss",
              E_min=None, E_max=None, f1=F1_DEFAULT, f2=F2_DEFAULT):
    """Energy grid of one bias point (Sec. 2.2.1, Eq. Rho).

    Returns a dict with
      E, w        real-axis nodes and weights on [E_min, E_max]
      fS, fD      source / drain occupations f(E - mu_S), f(E - mu_D)
      eta         broadening added to real-axis energies
      z           contour nodes (complex, Im z > 0)
      c           complex contour weights c_k = W_k z'_k f(z_k - mu_min), so that
                  integral_{E_B}^{E_min} G f_min dE ~= - sum_k c_k G(z_k)
      E_min, E_max, mu_min, kT
    E_min / E_max default to mu_min - f1 kT / mu_max + f2 kT.
    """
    mu_min = min(mu_S, mu_D)
    mu_max = max(mu_S, mu_D)
    if E_min is None:
        E_min = mu_min - f1 * kT
    if E_max is None:
        E_max = mu_max + f2 * kT
    if rule == "gauss":
        E, w = real_axis_gauss(E_min, E_max, n_real)
    elif rule == "midpoint":
        E, w = real_axis_midpoint(E_min, E_max, n_real)
    else:
        raise ValueError(rule)
    if n_cont > 0:
        z, zw = contour_semicircle(E_B, E_min, n_cont)
        c = zw * fermi(z - mu_min, kT)
    else:
        z = np.zeros(0, complex)
        c = np.zeros(0, complex)
    return dict(E=E, w=w, fS=fermi(E - mu_S, kT), fD=fermi(E - mu_D, kT), eta=float(eta),
                z=z, c=c, E_min=E_min, E_max=E_max, mu_min=mu_min, kT=kT,
                mu_S=mu_S, mu_D=mu_D)


def neutral_grid(n_cont, E_B):
    """Contour of the neutral reference charge rho_0: the same arc with E_l = E_u = 0
    (Sec. 2.2.1) and occupation 1 below the end point (reading: f == 1, no real-axis part)."""
    z, zw = contour_semicircle(E_B, 0.0, n_cont)
    return dict(E=np.zeros(0), w=np.zeros(0), fS=np.zeros(0), fD=np.zeros(0), eta=0.0,
                z=z, c=zw.astype(complex), E_min=0.0, E_max=0.0, mu_min=0.0, kT=0.0,
                mu_S=0.0, mu_D=0.0)


def segment_points(a, b, density, kT):
    """Number of Gauss-Legendre points of one sub-interval [a, b] at `density` points per kT
    (Sec. 3.3): ceil(density * ((b - a) / kT) - 1e-6), at least one, none for an empty
    interval (reading: the slack of a millionth of a point keeps a width that is a whole
    number of kT, up to rounding, from gaining a point)."""
    if not b > a:
        return 0
    return max(1, int(np.ceil(density * ((b - a) / kT) - 1e-6)))


def semi_adaptive_rule(E_min, E_max, E_l1, E_l2, densities, kT):
    """Real-axis rule of the semi-adaptive scheme (Sec. 3.3): the path E_min -> E_max split
    at E_l1 <= E_l2 into three sub-intervals, each integrated with its own Gauss-Legendre
    rule whose point count follows the user's density (points per kT) of that sub-interval.

    Readings: E_l1 and E_l2 are clipped into [E_min, E_max] (E_l2 no lower than E_l1); a
    sub-interval of zero width gets no points.  Returns (E, w, (n1, n2, n3)).
    """
    l1 = min(max(E_l1, E_min), E_max)
    l2 = min(max(E_l2, l1), E_max)
    Es, ws, ns = [], [], []
    for (a, b), d in zip(((E_min, l1), (l1, l2), (l2, E_max)), densities):
        n = segment_points(a, b, d, kT)
        ns.append(n)
        if n:
            e, w = real_axis_gauss(a, b, n)
            Es.append(e)
            ws.append(w)
    return np.concatenate(Es), np.concatenate(ws), tuple(ns)


def refined_limits(E_s, a, b, kT):
    """Limits after locating the singularity peak E_s (Sec. 3.3): E_l1 = E_s - a kT,
    E_l2 = E_s + b kT (reading: the printed "E_l1 = E_l1 - a kT" takes E_s as its base, as
    E_l2 does; a = 3, b = 1 are the paper's typical values)."""
    return E_s - a * kT, E_s + b * kT


def adaptive_grid(mu_S, mu_D, kT, E_l1, E_l2, densities, n_cont, E_B, eta, E_min=None, E_max=None,
                  f1=F1_DEFAULT, f2=F2_DEFAULT):
    """``bias_grid`` with the semi-adaptive real-axis rule in place of the single rule; the
    contour part is unchanged.  Also returns the clipped limits and segment sizes."""
    g = bias_grid(mu_S, mu_D, kT, 1, n_cont, E_B, eta, E_min=E_min, E_max=E_max, f1=f1, f2=f2)
    E, w, ns = semi_adaptive_rule(g["E_min"], g["E_max"], E_l1, E_l2, densities, kT)
    l1 = min(max(E_l1, g["E_min"]), g["E_max"])
    g.update(E=E, w=w, fS=fermi(E - mu_S, kT), fD=fermi(E - mu_D, kT), E_l1=l1,
             E_l2=min(max(E_l2, l1), g["E_max"]), segments=ns, densities=tuple(densities))
    return g
