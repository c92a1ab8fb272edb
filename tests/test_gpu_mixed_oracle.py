"""The mixed-precision workload at full size against the FP64 oracle: the (17,0) real-space
tube of 1024 rings on 4096 real-axis energies (a quarter within 20 meV of a lead subband
edge) and 64 contour nodes, with the oracle's outputs stored by
tests/golden/make_mixed_cnt17_N1024.py (Sec. 3.1's (n,0) construction, Eq. GR leads, Alg. 1 /
Alg. 2 as read).

Bounds, norm-wise relative (current: relative to |I|):
- complex128 sweep: 1e-10 for n, T and I;
- mixed path with its defaults (residual 1e-3, 2 meV band-edge window, growth criterion off),
  and with a residual threshold of 1e-4: n 5e-5, T 1e-4, I 2e-5, the stated bound of the mixed
  path;
- plain complex64 sweep (contour lanes in complex64 too): T 1e-4 and I 1e-4; its n is
  reported, not bounded (8.7e-3 on this grid: a few lanes in the lead gap and the contour
  nodes near the real axis, which is what the mixed path's flags and FP64 contour are for)."""
import functools
import json
import os

import numpy as np
import pytest

from oracle import quadrature as oq
from paper_2407_14633_gb300 import synth
from tests.cases import current_err, rel_inf

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


@functools.lru_cache(maxsize=None)
def golden():
    with open(os.path.join(HERE, "golden", "mixed_cnt17_N1024.json")) as fh:
        g = json.load(fh)
    g["n"] = np.array([float(x) for x in g["n"]])
    g["T"] = np.array([float(x) for x in g["T"]])
    g["I"] = float(g["I"])
    return g


def run(precision, **kw):
    from paper_2407_14633_gb300 import negf
    g = golden()
    w = synth.mixed_precision(n_tube=g["n_tube"], N=g["N"], n_energies=g["n_energies"])
    E = np.asarray(w["E"], dtype=np.float64)
    z = np.array([complex(*x) for x in g["z"]])
    c = np.array([complex(*x) for x in g["c"]])
    with negf.Context(precision=precision, **kw) as ctx:
        dev = ctx.device_create(g["N"], block=g["n_tube"], rings_per_block=1, n_chains=1)
        ctx.build_cnt_realspace(dev, g["n_tube"], g["t"], g["U_S"], g["U_D"])
        ctx.set_potential(dev, w["U"])
        ctx.set_grid(dev, E, np.full(E.size, 2.0 / E.size), oq.fermi(E - g["mu_S"], g["kT"]),
                     oq.fermi(E - g["mu_D"], g["kT"]), g["eta"], z, c)
        return ctx.compute_diag(dev)


def errors(r):
    g = golden()
    return dict(n=rel_inf(r["n"], g["n"]), T=rel_inf(r["T"], g["T"]),
                I=current_err(r["I"], g["I"], 2.0, g["mu_S"] - g["mu_D"]))


@pytest.mark.parametrize("name,bounds", [("c128", dict(n=1e-10, T=1e-10, I=1e-10)),
                                         ("mixed", dict(n=5e-5, T=1e-4, I=2e-5)),
                                         ("mixed_r1e-4", dict(n=5e-5, T=1e-4, I=2e-5)),
                                         ("c64", dict(T=1e-4, I=1e-4))])
def test_mixed_workload_against_oracle(name, bounds):
    from paper_2407_14633_gb300 import negf
    if name == "c128":
        r = run(negf.PREC_FP64)
    elif name.startswith("mixed"):
        kw = dict(flag_threshold=1e-4) if name == "mixed_r1e-4" else {}
        r = run(negf.PREC_MIXED, **kw)
        assert 0 < np.mean(r["flags"]) < 0.5
    else:
        r = run(negf.PREC_FP32)
    e = errors(r)
    print(name, e)
    assert all(e[k] < bounds[k] for k in bounds), (e, bounds)



def test_in_kernel_re_sweep_is_bitwise_the_second_pass():
    """At full size (4096 lanes, several per resident CTA) the complex64 kernel re-sweeping its
    flagged lanes in FP64 itself gives bitwise the outputs and flags of the second pass."""
    from paper_2407_14633_gb300 import negf
    a = run(negf.PREC_MIXED, mixed_two_pass=-1)
    b = run(negf.PREC_MIXED, mixed_two_pass=1)
    assert np.array_equal(a["flags"], b["flags"]) and a["flags"].sum() > 0
    for k in ("n", "T", "n_cont", "n_real"):
        assert np.array_equal(a[k], b[k]), k
    assert a["I"] == b["I"]
