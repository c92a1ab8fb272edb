"""CTA width of the wide-block sweep: forced widths, the size policy and the autotuner give
bitwise the same outputs (every output element and reduction of that kernel has a fixed
evaluation order), and the autotuner records its choice; the tuned result still matches the
FP64 oracle."""
import numpy as np
import pytest

from paper_2407_14633_gb300 import synth
from tests.cases import case_params, lib_device, lib_grid, rel_inf, run_oracle

pytestmark = pytest.mark.gpu


def _run(p, **kw):
    from paper_2407_14633_gb300 import negf
    with negf.Context(**kw) as ctx:
        dev = lib_device(ctx, p["kind"], p["n_tube"], p["t"], p["N"], p["U_S"], p["U_D"], p["modes"], p["cells"])
        ctx.set_potential(dev, p["U"])
        lib_grid(ctx, dev, p)
        r = ctx.compute([dev])[0]
        return r, ctx.blk_width(p["n_tube"], p["n_tube"], fp32=kw.get("precision", 0) == negf.PREC_FP32)


@pytest.mark.parametrize("n_tube,N", [(17, 12), (26, 6), (34, 5)])
@pytest.mark.parametrize("fp32", [False, True])
def test_width_does_not_change_results(n_tube, N, fp32):
    from paper_2407_14633_gb300 import negf
    p = case_params("real", N, 40, 8, synth.sinusoid_profile(N, 3), mu_D=-0.1, n_tube=n_tube, U_S=0.0, U_D=0.0)
    prec = negf.PREC_FP32 if fp32 else negf.PREC_FP64
    ref, _ = _run(p, precision=prec, blk_warps=-1)
    for w in (1, 2, 4):
        r, _ = _run(p, precision=prec, blk_warps=w)
        for k in ("n", "T", "n_cont", "n_real"):
            assert np.array_equal(r[k], ref[k]), (w, k)
        assert r["I"] == ref["I"]


def test_autotuner_records_width_and_matches_oracle():
    from paper_2407_14633_gb300 import negf
    # 160 + 32 energies: more lanes than SMs, so the first compute tunes the width
    N = 10
    p = case_params("real", N, 160, 32, synth.sinusoid_profile(N, 5), mu_D=-0.1, n_tube=17, U_S=0.0, U_D=0.0)
    r, w = _run(p, blk_warps=0)
    assert w in (1, 2, 4)
    fixed, _ = _run(p, blk_warps=-1)
    assert np.array_equal(r["n"], fixed["n"]) and np.array_equal(r["T"], fixed["T"])
    o = run_oracle(p, chunk=32)
    assert rel_inf(r["n"], o["n"]) < 1e-10
    assert rel_inf(r["T"], o["T"]) < 1e-10


def _run_mode(**kw):
    from paper_2407_14633_gb300 import negf
    # two mode-space devices, two subbands each, 4096 + 64 energies: 260 thread-per-lane items
    # per kernel class (more than one per SM, so the autotuner tunes), 1 x 1 and 2 x 2 blocks
    with negf.Context(**kw) as ctx:
        devs = []
        for N, cells in ((60, False), (48, True)):
            U = synth.ramp_barrier(N, drop=0.2, height=0.1, width=N / 6.0)
            d = lib_device(ctx, "mode", 17, -2.7, N, 0.0, -0.2, (6, 5), cells)
            ctx.set_potential(d, U)
            ctx.set_grid_spec(d, 0.0, -0.2, 0.025, 1e-6, -10.0, 4096, 64)
            devs.append(d)
        r = ctx.compute(devs)
        # under the FP32 policy every lane (contour too) runs in complex64
        fp32 = kw.get("precision", negf.PREC_FP64) == negf.PREC_FP32
        return r, ctx.chain_width(1, fp32), ctx.chain_width(2, fp32)


@pytest.mark.parametrize("fp32", [False, True])
def test_chain_width_does_not_change_results(fp32):
    from paper_2407_14633_gb300 import negf
    prec = negf.PREC_FP32 if fp32 else negf.PREC_FP64
    ref, _, _ = _run_mode(precision=prec, chain_warps=2)
    for w in (1, 4, 8):
        r, _, _ = _run_mode(precision=prec, chain_warps=w)
        for a, b in zip(r, ref):
            for k in ("n", "T", "n_cont", "n_real"):
                assert np.array_equal(a[k], b[k]), (w, k)
            assert a["I"] == b["I"]
    tuned, w1, w2 = _run_mode(precision=prec)
    assert w1 in (1, 2, 4, 8) and w2 in (1, 2, 4, 8)
    for a, b in zip(tuned, ref):
        assert np.array_equal(a["n"], b["n"]) and np.array_equal(a["T"], b["T"])
