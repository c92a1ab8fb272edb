"""GPU parity of general (non-circulant) leads, decimated per energy on the device (Eq. GR,
Sec. 2.2.2): against the oracle's FP64 decimation (ring counts at 1e-10; T and I per energy at
1e-10 or a condition bound), against a 30-digit ground truth on small tubes, and a circulant
lead given as full matrices against its closed form."""
import numpy as np
import pytest

from paper_2407_14633_gb300 import synth
from tests.cases import rel_inf, current_err
from oracle import charge as ochg
from oracle import model as omdl
from oracle import quadrature as oq
from oracle import selfconsistent as osc

pytestmark = pytest.mark.gpu

KT, ETA, E_B = 0.025, 1e-6, -12.0


@pytest.fixture(scope="module")
def ctx():
    from paper_2407_14633_gb300 import negf
    c = negf.Context()
    yield c
    c.close()


def circulant(row):
    row = np.asarray(row)
    m = row.size
    return np.array([[row[(s - r) % m] for s in range(m)] for r in range(m)])


def lib_tube(ctx, n_tube, N, U, U_S, U_D, leads, sites):
    dev = ctx.device_create(N, block=n_tube, rings_per_block=1, n_chains=1)
    ctx.build_cnt_realspace(dev, n_tube, -2.7, U_S, U_D)
    for side, (lead, U_l) in enumerate(zip(leads, (U_S, U_D))):
        ctx.set_lead_general(dev, 0, side, U_l, lead["T1"], lead["T2"], lead["tau"], sites,
                             H0=lead.get("H0"), H1=lead.get("H1"))
    ctx.set_potential(dev, U)
    return dev


def oracle_tube(n_tube, N, U_S, U_D, leads, sites):
    dev = omdl.cnt_build("real", n_tube, -2.7, N, U_S, U_D)
    ch = dev.chains[0]
    ch.lead_S = omdl.Lead(U_S, leads[0]["T1"], leads[0]["T2"], leads[0]["tau"], np.asarray(sites),
                          H0=leads[0].get("H0"), H1=leads[0].get("H1"))
    ch.lead_D = omdl.Lead(U_D, leads[1]["T1"], leads[1]["T2"], leads[1]["tau"], np.asarray(sites),
                          H0=leads[1].get("H0"), H1=leads[1].get("H1"))
    return dev


def fp64_condition(od, U, g, leads, sites, delta=1e-7, seed=0):
    """Condition estimate of T(E) per energy (relative to max |T|) and of the current, from the
    FP64 oracle: relative perturbations of size delta (random signs) of every lead block and of
    the device's coupling blocks, divided by delta."""
    import copy
    rng = np.random.default_rng(seed)
    base = ochg.negf_evaluate(od, U, g, method="sancho")
    dev = copy.deepcopy(od)
    ch = dev.chains[0]
    ch.Hup = ch.Hup * (1.0 + delta * rng.choice([-1.0, 1.0], ch.Hup.shape))
    for ld in (ch.lead_S, ch.lead_D):
        for f in ("T1", "T2", "tau", "H0", "H1"):
            x = getattr(ld, f)
            if x is not None:
                setattr(ld, f, x * (1.0 + delta * rng.choice([-1.0, 1.0], x.shape)))
    pert = ochg.negf_evaluate(dev, U, g, method="sancho")
    kT = np.abs(pert["T"] - base["T"]) / (delta * np.max(np.abs(base["T"])))
    kI = abs(pert["I"] - base["I"]) / (delta * abs(base["I"]))
    return kT, kI


@pytest.mark.parametrize("n_tube,N,m", [(5, 12, 5), (7, 9, 4), (17, 6, 17)])
def test_general_leads_match_oracle(ctx, n_tube, N, m):
    mu_S, mu_D, n_real, n_cont = 0.0, -0.3, 40, 12
    U = synth.sinusoid_profile(N, 9, amplitude=0.2)
    sites = list(range(m)) if m == n_tube else [0, 2, 3, 6][:m]
    leads = [synth.general_lead(m, 100 + n_tube), synth.general_lead(m, 200 + n_tube)]
    dev = lib_tube(ctx, n_tube, N, U, 0.05, -0.3, leads, sites)
    ctx.set_grid_spec(dev, mu_S, mu_D, KT, ETA, E_B, n_real, n_cont)
    r = ctx.compute([dev])[0]
    od = oracle_tube(n_tube, N, 0.05, -0.3, leads, sites)
    g = oq.bias_grid(mu_S, mu_D, KT, n_real, n_cont, E_B, ETA)
    o = ochg.negf_evaluate(od, U, g, method="sancho")
    assert rel_inf(r["n"], o["n"]) < 1e-10
    # T and I: two FP64 computations (the oracle's and the GPU's) each carry the decimation's
    # rounding, up to 4 (s / eta) u at real energies (s the scale of the lead blocks, eta the
    # broadening; see tests/test_oracle_extended.py), and errors of order kappa u where the
    # inputs are ill-conditioned; per energy the bound is 1e-10, or twice the larger of those
    # where it says more.  The extended-precision test below checks the GPU against the exact
    # values directly.
    from tests.test_oracle_extended import decimation_scale
    kT, kI = fp64_condition(od, U, g, leads, sites)
    dec = 4.0 * decimation_scale(leads, (0.05, -0.3)) / ETA * 2.0 ** -53
    eT = np.abs(r["T"] - o["T"]) / np.max(np.abs(o["T"]))
    tol_T = np.maximum(1e-10, 2.0 * np.maximum(1e3 * kT * 2.0 ** -53, dec))
    print("(%d,0) vs FP64 oracle: T %.1e (bound %.1e), I %.1e" % (n_tube, eT.max(), tol_T.max(),
                                                                 current_err(r["I"], o["I"], 2.0, mu_S - mu_D)))
    assert np.all(eT < tol_T), (eT.max(), tol_T[np.argmax(eT / tol_T)])
    assert current_err(r["I"], o["I"], 2.0, mu_S - mu_D) < max(1e-10, 2.0 * max(1e3 * kI * 2.0 ** -53, dec))


@pytest.mark.parametrize("i", range(3))
def test_general_leads_against_extended_precision(ctx, i):
    """The GPU against the 30-digit ground truth of tests/golden/general_leads_mp.json (three
    small tubes with non-circulant leads; energies include two at 2e-4 eV from a band edge of
    the source lead): T per energy, ring counts and current within 1e-10 of the exact values,
    or the condition and decimation bounds where those say more."""
    from paper_2407_14633_gb300 import negf
    from tests.test_oracle_extended import golden, bounds, errors
    case = golden()["cases"][i]
    sites = case["sites"]
    leads = [synth.general_lead(len(sites), s) for s in case["lead_seeds"]]
    N = case["N"]
    dev = lib_tube(ctx, case["n_tube"], N, np.array(case["U"]), case["U_S"], case["U_D"], leads, sites)
    z = np.array([complex(*x) for x in case["z"]])
    c = np.array([complex(*x) for x in case["c"]])
    ctx.set_grid(dev, np.array(case["E"]), np.array(case["w"]), np.array(case["fS"]), np.array(case["fD"]),
                 case["eta"], z, c)
    r = ctx.compute([dev])[0]
    eT, en, eI = errors(case, r["n"], r["T"], r["I"])
    tol_T, tol_n, tol_I = bounds(case)
    print("(%d,0) vs 30 digits: T %.1e n %.1e I %.1e" % (case["n_tube"], eT.max(), en, eI))
    assert np.all(eT < tol_T), (eT, tol_T)
    assert en < tol_n and eI < tol_I, (en, tol_n, eI, tol_I)


def test_circulant_lead_as_matrices_equals_closed_form(ctx):
    # the (17,0) lead rows of the builder, given as full matrices, decimated on the GPU
    from paper_2407_14633_gb300 import negf
    n, N = 17, 8
    U = synth.sinusoid_profile(N, 2)
    a = ctx.device_create(N, block=n, rings_per_block=1, n_chains=1)
    ctx.build_cnt_realspace(a, n, -2.7, 0.0, -0.2)
    b = ctx.device_create(N, block=n, rings_per_block=1, n_chains=1)
    ctx.build_cnt_realspace(b, n, -2.7, 0.0, -0.2)
    # the builder's alternation continued into the leads: bond k is t I for even k, and for odd
    # k t I plus the shift with entries (r, r-1) (k = 1 mod 4) or (r, r+1) (k = 3 mod 4); the
    # drain side takes the Hermitian conjugates of the bonds beyond ring N - 1
    t = -2.7

    def bond(k):
        B = t * np.eye(n)
        if k % 2 == 1:
            B = B + t * (np.roll(np.eye(n), -1, axis=1) if k % 4 == 1 else np.roll(np.eye(n), 1, axis=1))
        return B.astype(complex)
    src = (bond(-2 % 4), bond(-3 % 4), bond(-1 % 4))
    drn = (bond(N % 4).conj().T, bond((N + 1) % 4).conj().T, bond((N - 1) % 4).conj().T)
    for side, (T1, T2, tau) in enumerate((src, drn)):
        ctx.set_lead_general(b, 0, side, 0.0 if side == 0 else -0.2, T1, T2, tau, list(range(n)))
    for d in (a, b):
        ctx.set_potential(d, U)
        ctx.set_grid_spec(d, 0.0, -0.2, KT, ETA, E_B, 48, 12)
    ra, rb = ctx.compute([a])[0], ctx.compute([b])[0]
    assert rel_inf(rb["n"], ra["n"]) < 1e-9
    assert rel_inf(rb["T"], ra["T"]) < 1e-9


def test_general_leads_self_consistent_solve_matches_oracle(ctx):
    from paper_2407_14633_gb300 import negf
    n, N, V_DS, V_GS = 5, 10, 0.2, 0.1
    sites = list(range(n))
    leads = [synth.general_lead(n, 31), synth.general_lead(n, 32)]
    dev = lib_tube(ctx, n, N, np.zeros(N), 0.0, -V_DS, leads, sites)
    ctx.set_grid_spec(dev, 0.0, -V_DS, KT, ETA, E_B, 40, 12)
    U0 = np.linspace(0.0, -V_DS, N)
    r = ctx.sc_solve(dev, V_DS, V_GS, U0, negf.poisson_kappa(), M=64, tol=1e-9, check=False)
    od = oracle_tube(n, N, 0.0, -V_DS, leads, sites)
    g = oq.bias_grid(0.0, -V_DS, KT, 40, 12, E_B, ETA)
    n0 = ochg.neutral_charge(od, 12, E_B, method="sancho")
    p = osc.PoissonParams(kappa=osc.kappa_from_geometry(), U_G=-V_GS, U_S=0.0, U_D=-V_DS)
    o = osc.sc_solve(lambda U: ochg.negf_evaluate(od, U, g, method="sancho"), U0, n0, p, M=64, tol=1e-9)
    assert r["converged"] == o["converged"] and r["iterations"] == o["iterations"]
    assert rel_inf(r["n"], o["n"]) < 1e-9 and rel_inf(r["U"], o["U"]) < 1e-9


def test_general_lead_arguments_and_limits(ctx):
    from paper_2407_14633_gb300 import negf
    lead = synth.general_lead(5, 3)
    one = ctx.device_create(8, block=1, rings_per_block=1, n_chains=1)
    with pytest.raises(negf.NegfError) as e:   # single-site leads have a closed form
        ctx.set_lead_general(one, 0, 0, 0.0, lead["T1"][:1, :1], lead["T2"][:1, :1], lead["tau"][:1, :1], [0])
    assert e.value.status == negf.EINVAL
    dev = ctx.device_create(6, block=5, rings_per_block=1, n_chains=1)
    ctx.build_cnt_realspace(dev, 5, -2.7, 0.0, 0.0)
    bad = dict(lead, H0=lead["H0"] + 0.5j * np.eye(5))   # not Hermitian
    with pytest.raises(negf.NegfError) as e:
        ctx.set_lead_general(dev, 0, 0, 0.0, bad["T1"], bad["T2"], bad["tau"], list(range(5)), H0=bad["H0"])
    assert e.value.status == negf.EINVAL
    with pytest.raises(negf.NegfError) as e:
        ctx.set_lead_general(dev, 0, 0, 0.0, lead["T1"], lead["T2"], lead["tau"], [0, 1, 2, 3, 3])
    assert e.value.status == negf.EINVAL
    # a decimation cut off after one step is reported, not used
    ctx.set_lead_general(dev, 0, 0, 0.0, lead["T1"], lead["T2"], lead["tau"], list(range(5)), max_iter=1)
    ctx.set_potential(dev, np.zeros(6))
    ctx.set_grid_spec(dev, 0.0, 0.0, KT, ETA, E_B, 16, 4)
    with pytest.raises(negf.NegfError) as e:
        ctx.compute([dev])
    assert e.value.status == negf.ENOTCONVERGED


@pytest.mark.parametrize("n_tube,N,m", [(7, 9, 4), (17, 6, 17)])
def test_general_leads_in_complex64_and_mixed_precision(n_tube, N, m):
    """General leads in the complex64 sweeps (the per-energy Sigma blocks and Gamma factors of
    the decimation, rounded once to complex64 in the sweep): the plain complex64 sweep within
    1e-3 of the oracle, the mixed path within its stated bound (n 5e-5, T 1e-4, I 2e-5)."""
    from paper_2407_14633_gb300 import negf
    mu_S, mu_D, n_real, n_cont = 0.0, -0.3, 40, 12
    U = synth.sinusoid_profile(N, 9, amplitude=0.2)
    sites = list(range(m)) if m == n_tube else [0, 2, 3, 6][:m]
    leads = [synth.general_lead(m, 100 + n_tube), synth.general_lead(m, 200 + n_tube)]
    od = oracle_tube(n_tube, N, 0.05, -0.3, leads, sites)
    o = ochg.negf_evaluate(od, U, oq.bias_grid(mu_S, mu_D, KT, n_real, n_cont, E_B, ETA), method="sancho")
    for prec, bound in ((negf.PREC_FP32, (1e-3, 1e-3, 1e-3)), (negf.PREC_MIXED, (5e-5, 1e-4, 2e-5))):
        with negf.Context(precision=prec) as c2:
            dev = lib_tube(c2, n_tube, N, U, 0.05, -0.3, leads, sites)
            c2.set_grid_spec(dev, mu_S, mu_D, KT, ETA, E_B, n_real, n_cont)
            r = c2.compute([dev])[0]
        errs = (rel_inf(r["n"], o["n"]), rel_inf(r["T"], o["T"]),
                current_err(r["I"], o["I"], 2.0, mu_S - mu_D))
        print("(%d,0) m = %d precision %d: n %.2e T %.2e I %.2e" % ((n_tube, m, prec) + errs))
        assert all(e < b for e, b in zip(errs, bound)), (errs, bound)
