"""Seeded synthetic inputs for the nanotube NEGF workloads.

This module holds no part of the NEGF method: only potential profiles, device shapes,
bias points and arrival times drawn from fixed seeds.  The CUDA path and the CPU oracle
both take their inputs from here and from nowhere else.

Workloads (the paper measures on no public dataset; these stand in for its (17,0)
nanotube transistors, Sec. 3.1-3.3):

* ``modespace_small``   (17,0) mode space, N = 64 rings, linear drain ramp 0 -> -0.1 eV plus
  a Gaussian barrier (0.2 eV, width 8 rings), 256 midpoint energies on [-1, 1] eV and a
  64-node contour, eta = 1e-6 eV, kT = 0.025 eV, mu_S = 0, mu_D = -0.1 eV.
* ``realspace_17``      (17,0) real space, 17 x 17 ring blocks, N = 512 rings, sum of eight
  seeded sinusoids scaled to 0.15 eV amplitude, 2048 Gauss-Legendre real-axis energies
  plus 128 contour nodes, V_DS = 0.4 V, V_GS = 0.2 V, self-consistent to 1e-8.
* ``batched_uneven``    64 mode-space devices, N in [100, 2000], 1-4 modes, 1 x 1 or
  2 x 2 blocks, energy grids of 1024-8192 points.
* ``mixed_precision``   real-space (17,0), (26,0), (34,0), N = 1024, 4096 energies, a quarter
  of them within 20 meV of a lead subband edge.
* ``serving_sweep``     256 self-consistent requests with Poisson arrivals.
* ``gate_sweep``        zero-bias conductance against the gate voltage of a 10 nm (96-ring)
  (17,0) mode-space channel, subbands j = 6, 5, V_GS from -1 to 2 V in 31 steps, each solve
  started from the previous one's potential (the paper's sweep, Sec. 3.3-3.4).  The contact
  Fermi level sits 1 eV below midgap (the paper's Pd contacts, Sec. 3.1): mu = -1 eV with
  the leads at zero potential, so the contacts are metallic (p-type).
* ``adaptive_lengths``  (17,0) mode-space channels of 224, 736 and 1760 rings (23.9, 78.4 and
  187.4 nm, the lengths of Sec. 3.3), subband j = 6, drain ramp 0 -> -0.4 eV plus a 0.1 eV
  barrier, V_DS = 0.4 V: quadrature error of the real-axis charge against the point count.
* ``paper_scaling``     the shapes of the paper's timing tables, for context: one doubly
  degenerate (17,0) subband (j = 6) at N = 512 ... 4096 rings with 11,904 + 96 energies
  (Table 1), and N = 524,288 rings with 90 contour nodes and 1, 2, 4, 8 subbands (Table 2).
* ``planar_array``      tubes side by side sharing contacts and gate (Sec. 3.4): five 96-ring
  (10 nm) tubes at zero bias, and twenty 940-ring (100 nm) tubes at V_DS = 0.1 V, subbands
  j = 6, 5, 2048 + 64 energies, contacts 1 eV below midgap; neighbouring tubes coupled with
  a tenth of a tube's own gate coupling.
"""
import numpy as np

T_HOP = -2.7          # eV, nearest-neighbour coupling of the workloads
KT = 0.025            # eV
ETA = 1e-6            # eV
N_TUBE = 17
GAP_MODES = (6, 5, 7, 4)   # (17,0) subbands in ascending gap order


def ramp_barrier(N, drop=0.1, height=0.2, width=8.0, center=None):
    """Linear ramp 0 -> -drop over the rings plus a Gaussian barrier (height, width in rings)."""
    i = np.arange(N, dtype=np.float64)
    c = 0.5 * (N - 1) if center is None else center
    return -drop * i / (N - 1) + height * np.exp(-((i - c) ** 2) / (2.0 * width * width))


def sinusoid_profile(N, seed, amplitude=0.15, terms=8):
    """Sum of `terms` sinusoids with seeded amplitudes and phases, scaled to max |U| = amplitude."""
    rng = np.random.default_rng(seed)
    a = rng.uniform(0.5, 1.0, terms)
    phi = rng.uniform(0.0, 2.0 * np.pi, terms)
    i = np.arange(N, dtype=np.float64)
    U = np.zeros(N)
    for k in range(terms):
        U += a[k] * np.sin(2.0 * np.pi * (k + 1) * i / (N - 1) + phi[k])
    return amplitude * U / np.max(np.abs(U))


def modespace_small(mode=1):
    N = 64
    U = ramp_barrier(N)
    return dict(name="modespace_small", N=N, n_tube=N_TUBE, t=T_HOP, modes=(mode,), block=1,
                U=U, U_S=float(U[0]), U_D=float(U[-1]), mu_S=0.0, mu_D=-0.1, kT=KT, eta=ETA,
                n_real=256, n_cont=64, rule="midpoint", E_min=-1.0, E_max=1.0,
                E_B=float(min(U.min(), U[0], U[-1]) - 3.0 * abs(T_HOP) - 1.0))


def realspace_17(N=512, n_real=2048, n_cont=128, seed=2):
    U = sinusoid_profile(N, seed)
    V_DS, V_GS = 0.4, 0.2
    return dict(name="realspace_17", N=N, n_tube=N_TUBE, t=T_HOP, block=N_TUBE, U=U,
                U_S=0.0, U_D=-V_DS, mu_S=0.0, mu_D=-V_DS, kT=KT, eta=ETA,
                n_real=n_real, n_cont=n_cont, rule="gauss", V_DS=V_DS, V_GS=V_GS,
                E_B=float(min(U.min(), -V_DS) - 3.0 * abs(T_HOP) - 2.0),
                zeta=0.1, M=64, tol=1e-8, lam_nm=3.0)


def batched_uneven(n_devices=64, seed=3):
    rng = np.random.default_rng(seed)
    devs = []
    for d in range(n_devices):
        N = int(rng.integers(100, 2001))
        nm = int(rng.integers(1, 5))
        block = int(rng.choice([1, 2]))
        if block == 2 and N % 2:
            N += 1
        n_E = int(rng.integers(1024, 8193))
        V_DS = float(rng.uniform(0.0, 0.6))
        height = float(rng.uniform(0.05, 0.3))
        center = float(rng.uniform(0.25, 0.75)) * (N - 1)
        U = ramp_barrier(N, drop=V_DS, height=height, width=8.0, center=center)
        devs.append(dict(N=N, modes=GAP_MODES[:nm], block=block, U=U, U_S=0.0, U_D=-V_DS,
                         mu_S=0.0, mu_D=-V_DS, n_real=n_E - 64, n_cont=64, V_DS=V_DS,
                         E_B=float(min(U.min(), -V_DS) - 3.0 * abs(T_HOP) - 1.0)))
    return dict(name="batched_uneven", n_tube=N_TUBE, t=T_HOP, kT=KT, eta=ETA, devices=devs)


def band_edge_energies(n_tube, t, n_near, half_width, U_lead, seed):
    """n_near energies spread uniformly within +-half_width of the conduction and valence
    edges of the two lowest subbands of an (n,0) tube (edges +-|t| |1 - 2|cos(pi j/n)||)."""
    c = np.abs(np.cos(np.pi * np.arange(n_tube) / n_tube))
    gaps = np.abs(1.0 - 2.0 * c) * abs(t)
    edges_half = np.sort(np.unique(np.round(gaps, 12)))[:2]
    edges = np.concatenate([edges_half, -edges_half]) + U_lead
    rng = np.random.default_rng(seed)
    which = rng.integers(0, edges.size, n_near)
    return np.sort(edges[which] + rng.uniform(-half_width, half_width, n_near))


def mixed_precision(n_tube=17, N=1024, n_energies=4096, seed=4):
    U = sinusoid_profile(N, seed)
    n_near = n_energies // 4
    E_uniform = -1.0 + (np.arange(n_energies - n_near) + 0.5) * (2.0 / (n_energies - n_near))
    E_near = band_edge_energies(n_tube, T_HOP, n_near, 0.020, 0.0, seed)
    return dict(name=f"mixed_precision_{n_tube}", N=N, n_tube=n_tube, t=T_HOP, block=n_tube,
                U=U, U_S=0.0, U_D=0.0, E=np.sort(np.concatenate([E_uniform, E_near])),
                kT=KT, eta=ETA, mu_S=0.0, mu_D=-0.1)


def serving_sweep(n_requests=256, seed=5, rate=None):
    """Requests: (V_DS, V_GS) from a shuffled 16 x 16 grid, N in [200, 3000], two modes."""
    rng = np.random.default_rng(seed)
    vds = np.linspace(0.0, 0.6, 16)
    vgs = np.linspace(-0.5, 0.5, 16)
    grid = np.array([(a, b) for a in vds for b in vgs])
    rng.shuffle(grid)
    reqs = []
    for i in range(n_requests):
        V_DS, V_GS = grid[i % grid.shape[0]]
        N = int(rng.integers(200, 3001))
        reqs.append(dict(N=N, modes=(6, 5), V_DS=float(V_DS), V_GS=float(V_GS),
                         n_real=2048, n_cont=64))
    gaps = rng.exponential(1.0, n_requests)
    return dict(name="serving_sweep", n_tube=N_TUBE, t=T_HOP, kT=KT, eta=ETA, requests=reqs,
                unit_gaps=gaps)


def gate_sweep(N=96, n_points=31, v_lo=-1.0, v_hi=2.0, n_real=256, n_cont=64, mu=-1.0):
    """Gate-voltage sweep at zero drain bias: a 96-ring (10.2 nm) channel, two subbands,
    Gauss-Legendre real-axis energies on mu -+ 14 kT and a contour from E_B."""
    return dict(name="gate_sweep", N=N, n_tube=N_TUBE, t=T_HOP, modes=(6, 5), kT=KT, eta=ETA,
                mu=mu, V_DS=0.0, V_GS=np.linspace(v_lo, v_hi, n_points), n_real=n_real, n_cont=n_cont,
                E_B=-3.0 * abs(T_HOP) - 1.0 - 0.5)


def adaptive_lengths(lengths=(224, 736, 1760), V_DS=0.4):
    """Channels for the semi-adaptive grid study (fixed potential, no self-consistency)."""
    cases = []
    for N in lengths:
        U = ramp_barrier(N, drop=V_DS, height=0.1, width=N / 8.0)
        cases.append(dict(N=N, U=U, U_S=0.0, U_D=-V_DS))
    return dict(name="adaptive_lengths", n_tube=N_TUBE, t=T_HOP, modes=(6,), kT=KT, eta=ETA, mu_S=0.0,
                mu_D=-V_DS, n_cont=64, E_B=-3.0 * abs(T_HOP) - 1.0 - V_DS, cases=cases)


def planar_array(n_tubes=5, N=96, V_DS=0.0, V_GS=0.5, n_real=2048, n_cont=64, neighbour=0.1, mu=-1.0):
    """Tubes of one planar array: coupling matrix K = kappa (I + neighbour * (nearest-neighbour
    adjacency)), in units of kappa (the caller multiplies by the gate coupling), and the
    seeded starting potentials (the linear drop between the contacts)."""
    A = np.zeros((n_tubes, n_tubes))
    for c in range(n_tubes - 1):
        A[c, c + 1] = A[c + 1, c] = neighbour
    U0 = np.tile(np.linspace(0.0, -V_DS, N), (n_tubes, 1))
    return dict(name="planar_array", n_tubes=n_tubes, N=N, n_tube=N_TUBE, t=T_HOP, modes=(6, 5), kT=KT,
                eta=ETA, mu_S=mu, mu_D=mu - V_DS, V_DS=V_DS, V_GS=V_GS, n_real=n_real, n_cont=n_cont,
                E_B=-3.0 * abs(T_HOP) - 1.0 - V_DS + min(mu, 0.0), K_over_kappa=np.eye(n_tubes) + A, U0=U0)


def general_lead(m, seed, t=T_HOP, onsite=0.3, disorder=0.4):
    """A lead without circulant structure: couplings T1, T2, tau near t I with seeded complex
    (T1, T2) or real (tau) perturbations, and seeded Hermitian on-site blocks H0, H1 (interleaved
    m x m complex arrays, as the C ABI takes them)."""
    rng = np.random.default_rng(seed)
    def pert(cplx):
        X = rng.normal(size=(m, m)) + (1j * rng.normal(size=(m, m)) if cplx else 0.0)
        return disorder * X
    def herm():
        X = rng.normal(size=(m, m)) + 1j * rng.normal(size=(m, m))
        return onsite * 0.5 * (X + X.conj().T)
    T1 = t * np.eye(m) + pert(True)
    T2 = 0.8 * t * np.eye(m) + pert(True)
    tau = 0.9 * t * np.eye(m) + pert(False)
    return dict(T1=T1, T2=T2, tau=tau.astype(complex), H0=herm(), H1=herm())


def paper_scaling():
    """Workload shapes of the paper's timing tables (Sec. 3.2), for context timings."""
    return dict(name="paper_scaling", n_tube=N_TUBE, t=T_HOP, kT=KT, eta=ETA,
                table1=dict(N=(512, 1024, 2048, 4096), modes=(6,), n_real=11904, n_cont=96, V_DS=0.1,
                            paper_s=(2.04, 3.12, 5.28, 8.76), paper_gpus=(64, 128, 256, 512)),
                table2=dict(N=524288, modes=((6,), (6, 5), (6, 5, 7, 4), (6, 5, 7, 4, 8, 3, 9, 2)), n_cont=90,
                            paper_s=(1.98, 2.75, 3.24, 5.63)))
