"""The C-ABI library builds, loads and exports every symbol include/negf.h declares; host
logic that needs no GPU (grid helper, Poisson constant, status strings) is checked against
the oracle here."""
import os
import re

import numpy as np
import pytest

from oracle import quadrature as oq
from oracle import selfconsistent as osc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2407_14633_gb300 import build
    build.build()
    from paper_2407_14633_gb300 import negf
    return negf.load()


def declared_symbols():
    h = open(os.path.join(ROOT, "include", "negf.h")).read()
    h = re.sub(r"/\*.*?\*/", "", h, flags=re.S)
    return sorted(set(re.findall(r"\b(negf_[a-z0-9_]+)\s*\(", h)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_symbols()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_header():
    from paper_2407_14633_gb300 import negf
    assert set(negf.exported_symbols()) == set(declared_symbols())


def test_status_strings(lib):
    from paper_2407_14633_gb300 import negf
    assert lib.negf_strerror(negf.OK) == b"ok"
    assert b"converge" in lib.negf_strerror(negf.ENOTCONVERGED)


@pytest.mark.parametrize("rule", ["gauss", "midpoint"])
def test_library_grid_matches_oracle_grid(lib, rule):
    from paper_2407_14633_gb300 import negf
    r = negf.make_grid(0.0, -0.4, 0.025, 1e-6, -11.0, 2048, 128,
                       rule=negf.RULE_GAUSS if rule == "gauss" else negf.RULE_MIDPOINT)
    o = oq.bias_grid(0.0, -0.4, 0.025, 2048, 128, -11.0, 1e-6, rule=rule)
    for k in ("E", "w", "fS", "fD"):
        assert np.max(np.abs(r[k] - o[k])) < 1e-13 * max(1.0, np.max(np.abs(o[k])))
    assert np.max(np.abs(r["z"] - o["z"])) < 1e-13 * np.max(np.abs(o["z"]))
    assert np.max(np.abs(r["c"] - o["c"])) < 1e-13 * np.max(np.abs(o["c"]))


def test_poisson_kappa_matches_oracle(lib):
    from paper_2407_14633_gb300 import negf
    assert abs(negf.poisson_kappa() - osc.kappa_from_geometry()) < 1e-12 * osc.kappa_from_geometry()


def test_make_grid_rejects_bad_spec(lib):
    from paper_2407_14633_gb300 import negf
    with pytest.raises(negf.NegfError):
        negf.make_grid(0.0, 0.0, 0.025, 1e-6, 5.0, 16, 8)   # E_B above E_min


def test_product_path_never_imports_oracle():
    # the package and the C sources must not reference the oracle
    pkg = os.path.join(ROOT, "paper_2407_14633_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f


@pytest.mark.parametrize("limits,dens", [((-0.5, -0.4), (20.0, 80.0, 5.0)), ((-2.0, -0.7), (3.0, 7.5, 2.25)),
                                         ((-0.2, 9.0), (1.0, 33.3, 0.7)), ((0.1, -0.3), (5.0, 5.0, 5.0))])
def test_library_adaptive_grid_matches_oracle(lib, limits, dens):
    from paper_2407_14633_gb300 import negf
    r = negf.make_grid_adaptive(0.0, -0.4, 0.025, 1e-6, -11.0, 32, limits[0], limits[1], dens)
    o = oq.adaptive_grid(0.0, -0.4, 0.025, limits[0], limits[1], dens, 32, -11.0, 1e-6)
    assert r["E"].size == o["E"].size == sum(o["segments"])
    for k in ("E", "w", "fS", "fD"):
        assert np.max(np.abs(r[k] - o[k])) < 1e-13 * max(1.0, np.max(np.abs(o[k])))
    assert np.max(np.abs(r["c"] - o["c"])) < 1e-13 * np.max(np.abs(o["c"]))


def test_struct_layouts_match_header(tmp_path):
    # the ctypes structures of the binding must lay out exactly as the C structs of the header
    import shutil
    import subprocess
    import ctypes as C
    from paper_2407_14633_gb300 import negf
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"negf_opts": negf.Opts, "negf_lead": negf.Lead, "negf_lead_general": negf.LeadGeneral,
               "negf_grid": negf.Grid, "negf_grid_spec": negf.GridSpec, "negf_adaptive": negf.Adaptive,
               "negf_out": negf.Out, "negf_poisson": negf.Poisson, "negf_bias": negf.Bias,
               "negf_broyden": negf.Broyden, "negf_request": negf.Request, "negf_sc_result": negf.ScResult}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "negf.h"', 'int main(void) {']
    for cname, py in structs.items():
        lines.append('printf("%s size %%zu\\n", sizeof(%s));' % (cname, cname))
        for fname, _ in py._fields_:
            lines.append('printf("%s %s %%zu\\n", offsetof(%s, %s));' % (cname, fname, cname, fname))
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for ln in out:
        if ln:
            a, b, v = ln.split()
            got[(a, b)] = int(v)
    for cname, py in structs.items():
        assert got[(cname, "size")] == C.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)
