"""GPU parity: the CUDA path through the C ABI against the FP64 oracle, element by element
on the same seeded inputs.  Tolerance: 1e-10 norm-wise relative on ring electron counts and
T(E), and on the current relative to max(|I|, 1e-6 of the one-channel current scale)."""
import numpy as np
import pytest

from paper_2407_14633_gb300 import synth
from tests.cases import case_params, current_err, rel_inf, run_lib, run_oracle, lib_device, lib_grid
from oracle import charge as ochg
from oracle import green as ogr
from oracle import model as omdl

pytestmark = pytest.mark.gpu
TOL = 1e-10


@pytest.fixture(scope="module")
def ctx():
    from paper_2407_14633_gb300 import negf
    c = negf.Context()
    yield c
    c.close()


def check(p, r, o, tol=TOL):
    assert rel_inf(r["n"], o["n"]) < tol, rel_inf(r["n"], o["n"])
    if p["n_real"]:
        assert rel_inf(r["T"], o["T"]) < tol, rel_inf(r["T"], o["T"])
        g = 2.0 * 2.0 * len(p["modes"]) if p["kind"] == "mode" else 2.0
        assert current_err(r["I"], o["I"], g, p["mu_S"] - p["mu_D"]) < tol
    assert rel_inf(r["n_cont"], o["n_cont"]) < tol


@pytest.mark.parametrize("mode", [1, 6])
def test_modespace_small_workload(ctx, mode):
    # (17,0) mode space, N = 64, 256 midpoint energies on [-1, 1] + 64-node contour
    w = synth.modespace_small(mode)
    p = case_params("mode", w["N"], w["n_real"], w["n_cont"], w["U"], mu_S=w["mu_S"], mu_D=w["mu_D"],
                    kT=w["kT"], eta=w["eta"], rule="midpoint", E_min=-1.0, E_max=1.0, modes=(mode,))
    p["E_B"] = w["E_B"]
    _, r = run_lib(ctx, p)
    check(p, r, run_oracle(p))


@pytest.mark.parametrize("N,n_real,n_cont", [(1, 33, 5), (2, 31, 1), (37, 45, 7), (100, 64, 32), (130, 97, 0)])
def test_modespace_ragged_sizes(ctx, N, n_real, n_cont):
    U = synth.ramp_barrier(N) if N > 1 else np.array([0.05])
    p = case_params("mode", N, n_real, n_cont, U, modes=(6,))
    if n_cont == 0:
        p["n_cont"] = 0
    _, r = run_lib(ctx, p)
    check(p, r, run_oracle(p))


def test_modespace_multimode_and_cells(ctx):
    N = 48
    U = synth.ramp_barrier(N, drop=0.3, height=0.15)
    p1 = case_params("mode", N, 70, 20, U, mu_D=-0.3, modes=(6, 5, 7))
    _, r1 = run_lib(ctx, p1)
    o = run_oracle(p1)
    check(p1, r1, o)
    p2 = dict(p1, cells=True)
    _, r2 = run_lib(ctx, p2)
    check(p2, r2, o, tol=1e-10)


@pytest.mark.parametrize("n_tube,N", [(5, 12), (17, 9), (7, 40)])
def test_realspace_blocks(ctx, n_tube, N):
    U = synth.sinusoid_profile(N, 2)
    p = case_params("real", N, 37, 9, U, mu_D=-0.4, n_tube=n_tube, U_S=0.0, U_D=-0.4)
    _, r = run_lib(ctx, p)
    check(p, r, run_oracle(p, chunk=16))


@pytest.mark.parametrize("n_tube,N,blk_warps", [(7, 16, 1), (17, 9, 1), (17, 9, 4), (26, 5, 2)])
def test_flux_threaded_tube_general_blocks(n_tube, N, blk_warps):
    """A flux through the tube (H_ll += i d (S - S^T), a Peierls phase on the ring bonds)
    makes every block complex and the Green's functions non-symmetric: the general update
    path, for the compact and the wider shared-memory layouts."""
    from paper_2407_14633_gb300 import negf
    U = synth.sinusoid_profile(N, 6)
    p = case_params("real", N, 41, 9, U, mu_D=-0.3, n_tube=n_tube, U_S=0.0, U_D=-0.3)
    dev_o = omdl.cnt_build("real", n_tube, p["t"], N, p["U_S"], p["U_D"])
    ch = dev_o.chains[0]
    S = omdl.shift_matrix(n_tube)
    ch.Hdiag = ch.Hdiag + 1j * 0.15 * (S - S.T)[None, :, :]
    ch.Hup = ch.Hup * np.exp(1j * 0.3)
    o = ochg.negf_evaluate(dev_o, U, ogr_grid(p), chunk=16)
    with negf.Context(blk_warps=blk_warps) as c2:
        dev = lib_device(c2, "real", n_tube, p["t"], N, p["U_S"], p["U_D"])
        c2.set_hamiltonian(dev, 0, ch.Hdiag.reshape(-1), ch.Hup.reshape(-1), 1.0)
        c2.set_potential(dev, U)
        lib_grid(c2, dev, p)
        r = c2.compute([dev])[0]
    check(p, r, o)


@pytest.mark.parametrize("n_tube,N,blk_warps,prec,tol", [(17, 9, 1, "fp64", TOL), (26, 5, 2, "fp64", TOL),
                                                         (17, 9, 1, "fp32", 1e-3), (26, 5, 2, "fp32", 1e-3)])
def test_layer_dependent_blocks(n_tube, N, blk_warps, prec, tol):
    """Every layer its own blocks: on-site disorder per ring, coupling strengths per layer and
    one missing ring-to-ring bond, so that no two layers share H_ll or H_{l,l+1} and the
    sparse forms' counts differ between layers.  A uniform tube's sweeps read layer 0's blocks
    for every layer; this one must index each layer (FP64 to 1e-10, the complex64 sweep to
    its plain-precision bound)."""
    from paper_2407_14633_gb300 import negf
    rng = np.random.default_rng(11)
    U = synth.sinusoid_profile(N, 6)
    p = case_params("real", N, 41, 9, U, mu_D=-0.3, n_tube=n_tube, U_S=0.0, U_D=-0.3)
    dev_o = omdl.cnt_build("real", n_tube, p["t"], N, p["U_S"], p["U_D"])
    ch = dev_o.chains[0]
    ch.Hdiag = ch.Hdiag + np.einsum("lr,rs->lrs", rng.uniform(-0.2, 0.2, (N, n_tube)), np.eye(n_tube))
    ch.Hup = ch.Hup * rng.uniform(0.9, 1.1, (N - 1, 1, 1))
    r0, c0 = np.argwhere(ch.Hup[N // 2] != 0)[0]
    ch.Hup[N // 2, r0, c0] = 0.0
    o = ochg.negf_evaluate(dev_o, U, ogr_grid(p), chunk=16)
    precision = negf.PREC_FP64 if prec == "fp64" else negf.PREC_FP32
    with negf.Context(blk_warps=blk_warps, precision=precision) as c2:
        dev = lib_device(c2, "real", n_tube, p["t"], N, p["U_S"], p["U_D"])
        c2.set_hamiltonian(dev, 0, ch.Hdiag.reshape(-1).astype(complex), ch.Hup.reshape(-1).astype(complex), 1.0)
        c2.set_potential(dev, U)
        lib_grid(c2, dev, p)
        r = c2.compute([dev])[0]
    check(p, r, o, tol=tol)


@pytest.mark.parametrize("N,n_real", [(64, 96), (192, 512)])
def test_symmetric_update_with_bound_states(N, n_real):
    """A potential well deep enough to hold states in the gap: lanes near those states have a
    nearly singular half-chain gL_l and must take the general update.  The default run (the
    symmetric update where it is safe) must match the general update and, for the shorter
    channel, the oracle."""
    from paper_2407_14633_gb300 import negf
    i = np.arange(N)
    U = -0.1 * i / (N - 1) - 0.35 * np.exp(-((i - 0.5 * N) / (0.08 * N)) ** 2)
    p = case_params("real", N, n_real, 16, U, mu_D=-0.1, n_tube=17, U_S=0.0, U_D=-0.1)
    out = []
    for gen in (0, 1):
        with negf.Context(general_update=gen) as c2:
            _, r = run_lib(c2, p)
            out.append(r)
    check(p, out[0], out[1])
    if N <= 64:
        check(p, out[0], run_oracle(p, chunk=16))


def ogr_grid(p):
    from tests.cases import oracle_grid
    return oracle_grid(p)


def test_zero_bias_current_is_zero(ctx):
    N = 30
    U = 0.05 * np.sin(np.arange(N))
    p = case_params("mode", N, 40, 8, U, mu_S=0.05, mu_D=0.05, modes=(6, 5))
    _, r = run_lib(ctx, p)
    assert r["I"] == 0.0


def test_batch_is_bitwise_alone(ctx):
    cases = [case_params("mode", 70, 50, 9, synth.ramp_barrier(70), modes=(6,)),
             case_params("mode", 33, 41, 3, synth.ramp_barrier(33, drop=0.2), mu_D=-0.2, modes=(5, 4)),
             case_params("real", 10, 13, 4, synth.sinusoid_profile(10, 1), n_tube=5, U_S=0.0, U_D=-0.1)]
    alone = []
    devs = []
    for p in cases:
        d, r = run_lib(ctx, p)
        alone.append(r)
        devs.append(d)
    batch = ctx.compute(devs)
    for a, b in zip(alone, batch):
        assert np.array_equal(a["n"], b["n"])
        assert np.array_equal(a["T"], b["T"])
        assert a["I"] == b["I"]


def test_neutral_charge_matches_oracle(ctx):
    for kind, n_tube, modes in (("mode", 17, (6, 1)), ("real", 7, (1,))):
        N = 12
        dev = lib_device(ctx, kind, n_tube, -2.7, N, 0.1, -0.1, modes)
        n0 = ctx.neutral_charge(dev, 64, -10.0)
        od = omdl.cnt_build(kind, n_tube, -2.7, N, 0.1, -0.1, modes=modes)
        ref = ochg.neutral_charge(od, 64, -10.0)
        assert rel_inf(n0, ref) < TOL


def test_sampled_lanes_match_oracle(ctx):
    N = 20
    U = synth.sinusoid_profile(N, 3)
    p = case_params("real", N, 50, 10, U, mu_D=-0.2, n_tube=7, U_S=0.0, U_D=-0.2)
    dev, _ = run_lib(ctx, p)
    ir, ic = [0, 7, 49], [0, 9]
    AS, AD, G = ctx.sample_lanes(dev, ir, ic)
    from tests.cases import oracle_device, oracle_grid
    od = oracle_device("real", 7, -2.7, N, 0.0, -0.2)
    g = oracle_grid(p)
    ch = od.chains[0]
    r = ogr.rgf_lanes(ch, U, g["E"][ir] + 1j * g["eta"])
    c = ogr.rgf_lanes(ch, U, g["z"][ic], spectral=False)
    assert rel_inf(AS, ochg.ring_sum(ch, N, r["AS"])) < TOL
    assert rel_inf(AD, ochg.ring_sum(ch, N, r["AD"])) < TOL
    assert rel_inf(G, ochg.ring_sum(ch, N, c["Gdiag"])) < TOL


def test_full_size_realspace_sampled(ctx):
    # the benchmark's workload in its launch configuration: (17,0) real space, N = 512,
    # 2048 + 128 energies; sampled energies checked against the oracle one by one
    w = synth.realspace_17()
    p = case_params("real", w["N"], w["n_real"], w["n_cont"], w["U"], mu_S=w["mu_S"], mu_D=w["mu_D"],
                    n_tube=17, U_S=w["U_S"], U_D=w["U_D"])
    p["E_B"] = w["E_B"]
    dev, r = run_lib(ctx, p)
    from tests.cases import oracle_device, oracle_grid
    od = oracle_device("real", 17, -2.7, w["N"], w["U_S"], w["U_D"])
    g = oracle_grid(p)
    ir = [0, 517, 1023, 1500, 2047]
    ic = [0, 64, 127]
    AS, AD, G = ctx.sample_lanes(dev, ir, ic)
    ch = od.chains[0]
    o = ogr.rgf_lanes(ch, w["U"], g["E"][ir] + 1j * g["eta"])
    oc = ogr.rgf_lanes(ch, w["U"], g["z"][ic], spectral=False)
    assert rel_inf(AS, ochg.ring_sum(ch, w["N"], o["AS"])) < TOL
    assert rel_inf(AD, ochg.ring_sum(ch, w["N"], o["AD"])) < TOL
    assert rel_inf(G, ochg.ring_sum(ch, w["N"], oc["Gdiag"])) < TOL
    assert rel_inf(r["T"][ir], o["T"]) < TOL
    # properties that hold at any size: T >= 0, electron counts positive and finite
    assert np.all(r["T"] >= -1e-12) and np.all(np.isfinite(r["n"])) and np.all(r["n"] > 0)


def test_invalid_arguments_rejected(ctx):
    from paper_2407_14633_gb300 import negf
    with pytest.raises(negf.NegfError):
        ctx.device_create(0)
    with pytest.raises(negf.NegfError):
        ctx.device_create(10, block=3, rings_per_block=2)
    d = ctx.device_create(8)
    with pytest.raises(negf.NegfError):
        ctx.compute([d])          # nothing set yet
    with pytest.raises(negf.NegfError):
        ctx.set_potential(d, np.full(8, np.nan))
