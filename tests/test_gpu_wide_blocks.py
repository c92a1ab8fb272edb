"""(26,0) and (34,0) real-space tubes against the FP64 oracle (Sec. 3.1's (n,0) construction
at the widths of the mixed-precision workload; Eq. GR, Alg. 1 / Alg. 2 as read).

Ring blocks of 26 and 34 sites exercise both shared-memory layouts of the wide-block sweep:
at 4 warps every b x b product fits the register tiles (the compact layout: three b x b
buffers and one b x m buffer), at 1 and 2 warps it does not (four b x b and three b x m
buffers).  A potential well with states in the gap makes some lanes' half-chain gL_l nearly
singular, so the sweep runs the complex-symmetric G_ll update on some lanes and the general
one on others; the lane counters confirm both forms ran.  The mixed-precision path is held
to its stated bound on a grid with a quarter of the energies within 20 meV of a lead subband
edge.  Tolerances: 1e-10 norm-wise relative (FP64), the documented mixed bound otherwise."""
import functools

import numpy as np
import pytest

from oracle import charge as ochg
from oracle import quadrature as oq
from paper_2407_14633_gb300 import synth
from tests.cases import case_params, current_err, lib_device, lib_grid, oracle_device, rel_inf, run_oracle

pytestmark = pytest.mark.gpu
TOL = 1e-10
MIXED_DEFAULT_BOUND = 5e-5
SIZES = {26: 10, 34: 7}


def _check(p, r, o, tol=TOL, g=2.0):
    errs = dict(n=rel_inf(r["n"], o["n"]), n_cont=rel_inf(r["n_cont"], o["n_cont"]))
    if p["n_real"]:
        errs["T"] = rel_inf(r["T"], o["T"])
        errs["I"] = current_err(r["I"], o["I"], g, p["mu_S"] - p["mu_D"])
    bad = {k: v for k, v in errs.items() if not v < tol}
    assert not bad, (bad, errs)
    return errs


def _run(p, **kw):
    from paper_2407_14633_gb300 import negf
    with negf.Context(**kw) as ctx:
        dev = lib_device(ctx, p["kind"], p["n_tube"], p["t"], p["N"], p["U_S"], p["U_D"])
        ctx.set_potential(dev, p["U"])
        lib_grid(ctx, dev, p)
        ctx.profile(True)
        ctx.sweep_lanes()
        r = ctx.compute([dev])[0]
        return r, ctx.sweep_lanes()


def _sinusoid_case(n_tube):
    N = SIZES[n_tube]
    return case_params("real", N, 44, 9, synth.sinusoid_profile(N, 7), mu_D=-0.3, n_tube=n_tube, U_S=0.0,
                       U_D=-0.3)


@functools.lru_cache(maxsize=None)
def _sinusoid_oracle(n_tube):
    return run_oracle(_sinusoid_case(n_tube), chunk=16)


@pytest.mark.parametrize("warps", [1, 2, 4])
@pytest.mark.parametrize("n_tube", [26, 34])
def test_wide_tube_matches_oracle(n_tube, warps):
    p = _sinusoid_case(n_tube)
    r, lanes = _run(p, blk_warps=warps)
    print("(%d,0) %d warps: errors %s, lanes %s" % (n_tube, warps, _check(p, r, _sinusoid_oracle(n_tube)), lanes))
    assert sum(lanes) == p["n_real"] + p["n_cont"]


def _well_case(n_tube):
    # 24 rings, a 0.35 eV deep well over about 2 rings in the middle of a 0.1 eV drain ramp:
    # bound states of the half chains put |gL_l| above the symmetric update's gate on a few
    # real-axis lanes of each tube (and none of the contour lanes)
    N = 24
    i = np.arange(N)
    U = -0.1 * i / (N - 1) - 0.35 * np.exp(-((i - 0.5 * N) / (0.08 * N)) ** 2)
    return case_params("real", N, 96, 16, U, mu_D=-0.1, n_tube=n_tube, U_S=0.0, U_D=-0.1)


@pytest.mark.parametrize("warps", [1, 4])
@pytest.mark.parametrize("n_tube", [26, 34])
def test_wide_tube_bound_states_switch_update_form(n_tube, warps):
    p = _well_case(n_tube)
    o = run_oracle(p, chunk=32)
    r, lanes = _run(p, blk_warps=warps)
    real_sym, real_gen, cont_sym, cont_gen = lanes
    print("(%d,0) %d warps: lanes %s errors %s" % (n_tube, warps, lanes, _check(p, r, o)))
    assert real_sym > 0 and real_gen > 0, lanes
    assert real_sym + real_gen == p["n_real"] and cont_sym + cont_gen == p["n_cont"]
    # the general update everywhere gives the same result within the tolerance
    rg, lanes_g = _run(p, blk_warps=warps, general_update=1)
    assert lanes_g[0] == 0 and lanes_g[2] == 0
    _check(p, r, rg)


def _edge_grids(n_tube, N, n_energies, seed):
    """The mixed-precision workload's grid at reduced size: 3/4 midpoint energies on [-1, 1],
    1/4 within 20 meV of the conduction and valence edges of the leads' two lowest subbands,
    equal weights 2 / n_energies, and a 16-node contour; built once for the oracle (oracle
    quadrature) and once for the library (its grid helper for the contour)."""
    from paper_2407_14633_gb300 import negf
    from paper_2407_14633_gb300 import workloads
    w = synth.mixed_precision(n_tube=n_tube, N=N, n_energies=n_energies, seed=seed)
    E = w["E"]
    wts = np.full(E.size, 2.0 / E.size)
    E_B = float(np.min(w["U"]) - 3.0 * abs(w["t"]) - 1.0)
    z, c = oq.contour_semicircle(E_B, -1.0, 16)
    og = dict(E=E, w=wts, fS=oq.fermi(E - w["mu_S"], w["kT"]), fD=oq.fermi(E - w["mu_D"], w["kT"]),
              eta=w["eta"], z=z, c=c)
    cg = negf.make_grid(w["mu_S"], w["mu_D"], w["kT"], w["eta"], E_B, 1, 16, E_min=-1.0, E_max=1.0)
    lg = dict(E=E, w=wts, fS=workloads._fermi(E - w["mu_S"], w["kT"]),
              fD=workloads._fermi(E - w["mu_D"], w["kT"]), eta=w["eta"], z=cg["z"], c=cg["c"])
    return w, og, lg


@functools.lru_cache(maxsize=None)
def _edge_oracle(n_tube):
    w, og, _ = _edge_grids(n_tube, SIZES[n_tube], 96, 4)
    dev = oracle_device("real", n_tube, w["t"], w["N"], w["U_S"], w["U_D"])
    return ochg.negf_evaluate(dev, w["U"], og, chunk=16)


def _run_edge(n_tube, **kw):
    from paper_2407_14633_gb300 import negf
    w, _, lg = _edge_grids(n_tube, SIZES[n_tube], 96, 4)
    with negf.Context(**kw) as ctx:
        dev = ctx.device_create(w["N"], block=n_tube, rings_per_block=1, n_chains=1)
        ctx.build_cnt_realspace(dev, n_tube, w["t"], w["U_S"], w["U_D"])
        ctx.set_potential(dev, w["U"])
        ctx.set_grid(dev, lg["E"], lg["w"], lg["fS"], lg["fD"], lg["eta"], lg["z"], lg["c"])
        r = ctx.compute_diag(dev)
    p = dict(n_real=w["E"].size, mu_S=w["mu_S"], mu_D=w["mu_D"])
    return p, r


@pytest.mark.parametrize("n_tube", [26, 34])
def test_wide_tube_band_edge_grid_fp64(n_tube):
    p, r = _run_edge(n_tube)
    print("(%d,0) band-edge grid FP64: %s" % (n_tube, _check(p, r, _edge_oracle(n_tube))))


@pytest.mark.parametrize("n_tube", [26, 34])
def test_wide_tube_mixed_precision_bound(n_tube):
    from paper_2407_14633_gb300 import negf
    o = _edge_oracle(n_tube)
    p, r = _run_edge(n_tube, precision=negf.PREC_MIXED)
    errs = dict(n=rel_inf(r["n"], o["n"]), T=rel_inf(r["T"], o["T"]),
                I=current_err(r["I"], o["I"], 2.0, p["mu_S"] - p["mu_D"]))
    print("(%d,0) mixed: errors %s, recomputed %.3f" % (n_tube, errs, float(np.mean(r["flags"]))))
    assert max(errs.values()) < MIXED_DEFAULT_BOUND, errs
    # contour lanes stay FP64
    assert rel_inf(r["n_cont"], o["n_cont"]) < TOL


@pytest.mark.parametrize("n_tube", [37, 40])
def test_blocks_wider_than_the_register_tiles(n_tube):
    """Ring blocks wider than 36 (past the widest register-tile class): the shared-memory
    kernels in FP64 (the wider layout: four b x b and three b x m buffers) and in complex64, and
    the mixed path on top of them, against the oracle on a short tube."""
    from paper_2407_14633_gb300 import negf
    N = 4
    p = case_params("real", N, 24, 8, synth.sinusoid_profile(N, 3), mu_D=-0.3, n_tube=n_tube, U_S=0.0,
                    U_D=-0.3)
    o = run_oracle(p, chunk=8)
    r, _ = _run(p)
    print("(%d,0) FP64: %s" % (n_tube, _check(p, r, o)))
    r, _ = _run(p, precision=negf.PREC_FP32)
    print("(%d,0) complex64: %s" % (n_tube, _check(p, r, o, tol=1e-3)))
    r, _ = _run(p, precision=negf.PREC_MIXED)
    print("(%d,0) mixed: %s" % (n_tube, _check(p, r, o, tol=MIXED_DEFAULT_BOUND)))
