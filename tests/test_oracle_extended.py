"""Pins of the extended-precision oracle (oracle/extended.py), and the FP64 oracle's general-lead
results against it.

The extended-precision module is pinned by things it does not share with itself: the textbook
surface function of a uniform chain, the closed-form surface functions of a circulant lead
(decimation of the same lead as a two-ring layer must reproduce them), and the FP64 oracle on a
well-conditioned circulant case.  The stored ground truth (tests/golden/general_leads_mp.json,
written by tests/golden/make_general_leads_mp.py from oracle/ only) then bounds the FP64
oracle: T(E) per energy, ring counts and current within 1e-10, or where the stored condition
estimate kappa or the decimation's rounding (s / eta) u says more, within 1e3 kappa u and
4 (s / eta) u (u = 2^-53, s the scale of the lead blocks, eta the broadening)."""
import json
import os

import numpy as np
import pytest

from oracle import charge as ochg
from oracle import leads as oleads
from oracle import model as omdl
from paper_2407_14633_gb300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))
U64 = 2.0 ** -53


def golden():
    with open(os.path.join(HERE, "golden", "general_leads_mp.json")) as fh:
        return json.load(fh)


def golden_device(case):
    """The oracle device and grid of a stored case (inputs exactly as stored)."""
    sites = case["sites"]
    m = len(sites)
    leads = [synth.general_lead(m, s) for s in case["lead_seeds"]]
    dev = omdl.cnt_build("real", case["n_tube"], -2.7, case["N"], case["U_S"], case["U_D"])
    ch = dev.chains[0]
    for side, (ld, U_l) in enumerate(zip(leads, (case["U_S"], case["U_D"]))):
        L = omdl.Lead(U_l, ld["T1"], ld["T2"], ld["tau"], np.asarray(sites), H0=ld.get("H0"), H1=ld.get("H1"))
        if side == 0:
            ch.lead_S = L
        else:
            ch.lead_D = L
    g = dict(E=np.array(case["E"]), w=np.array(case["w"]), fS=np.array(case["fS"]), fD=np.array(case["fD"]),
             eta=case["eta"], z=np.array([complex(*x) for x in case["z"]]),
             c=np.array([complex(*x) for x in case["c"]]))
    return dev, np.array(case["U"]), g


def decimation_scale(leads, U_leads):
    """Largest entry of the two-ring layer blocks of the leads (U on the diagonal): the scale s
    of the decimation's rounding, which grows like (s / eta) u at real energies E + i eta."""
    s = 0.0
    for ld, U in zip(leads, U_leads):
        m = ld["T1"].shape[0]
        for blk in (ld.get("H0"), ld.get("H1")):
            s = max(s, float(np.max(np.abs((0.0 if blk is None else blk) + U * np.eye(m)))))
        for f in ("T1", "T2"):
            s = max(s, float(np.max(np.abs(ld[f]))))
    return s


def decimation_bound(case):
    """Relative error an FP64 decimation may leave in T(E) at a real energy: 4 (s / eta) u.  At
    small eta the decimation's intermediate chains of 2^k layers carry resonances of width eta,
    and rounding inside it is amplified by about s / eta, whatever the condition of the result
    with respect to the inputs (measured: the FP64 oracle 7.2e-10 from the exact value at one
    energy of a 17-site lead, where perturbing the inputs moves T by only 47 u)."""
    leads = [synth.general_lead(len(case["sites"]), sd) for sd in case["lead_seeds"]]
    return 4.0 * decimation_scale(leads, (case["U_S"], case["U_D"])) / case["eta"] * U64


def bounds(case):
    """Tolerances of an FP64 result against the stored ground truth: T per energy (relative to
    max |T|), ring counts (relative to max |n|), current (relative to |I|): 1e-10, or where the
    condition estimate of the inputs (kappa, stored) or the decimation's rounding says more,
    1e3 kappa u and 4 (s / eta) u."""
    kT = np.array(case["kappa_T"])
    dec = decimation_bound(case)
    tol_T = np.maximum(np.maximum(1e-10, 1e3 * kT * U64), dec)
    tol_n = max(1e-10, 1e3 * case["kappa_n"] * U64, dec)
    tol_I = max(1e-10, 1e3 * float(kT.max()) * U64, dec)
    return tol_T, tol_n, tol_I


def errors(case, n, T, I):
    n_ref = np.array([float(x) for x in case["n"]])
    T_ref = np.array([float(x) for x in case["T"]])
    I_ref = float(case["I"])
    eT = np.abs(np.asarray(T) - T_ref) / np.max(np.abs(T_ref))
    en = float(np.max(np.abs(np.asarray(n) - n_ref)) / np.max(np.abs(n_ref)))
    eI = abs(I - I_ref) / abs(I_ref)
    return eT, en, eI


def test_uniform_chain_textbook():
    mp = pytest.importorskip("mpmath")
    from oracle import extended as ex
    t = mp.mpf(-2.7)   # the reference is formed in extended precision too
    for E in (0.7, -3.1, 6.0):
        e = mp.mpc(E, 1e-6)
        g = ex.surface_gf(e, mp.matrix([[0]]), mp.matrix([[t]]))[0, 0]
        s = mp.sqrt(e * e - 4 * t * t)
        roots = [(e - s) / (2 * t * t), (e + s) / (2 * t * t)]
        ref = min(roots, key=lambda r: r.imag)   # the retarded root (Im g < 0)
        assert abs(g - ref) < mp.mpf(10) ** -25 * abs(ref)


def test_decimation_of_circulant_lead_equals_closed_form():
    mp = pytest.importorskip("mpmath")
    from oracle import extended as ex
    dev = omdl.cnt_build("real", 5, -2.7, 2, 0.05, -0.3)
    lead = dev.chains[0].lead_S
    for E in (0.3, -0.9, 1.7):
        eps = np.array([E + 1e-3j])
        S_fp64, _ = oleads.lead_sigma_gamma_analytic(lead, eps)
        S_mp = ex.lead_sigma(lead, mp.mpc(E, 1e-3))
        S_mp = np.array([[complex(S_mp[i, j]) for j in range(lead.m)] for i in range(lead.m)])
        assert np.max(np.abs(S_mp - S_fp64[0])) < 1e-12 * np.max(np.abs(S_fp64[0]))


def test_extended_equals_fp64_oracle_on_circulant_leads():
    pytest.importorskip("mpmath")
    from oracle import extended as ex
    from oracle import quadrature as oq
    N = 3
    dev = omdl.cnt_build("real", 5, -2.7, N, 0.05, -0.3)
    U = synth.sinusoid_profile(N, 9, amplitude=0.2)
    g = oq.bias_grid(0.0, -0.3, 0.025, 4, 2, -12.0, 1e-6)
    r = ex.evaluate(dev, U, g)
    o = ochg.negf_evaluate(dev, U, g)
    n = np.array([float(x) for x in r["n"]])
    T = np.array([float(x) for x in r["T"]])
    assert np.max(np.abs(o["n"] - n)) < 1e-12 * np.max(np.abs(n))
    assert np.max(np.abs(o["T"] - T)) < 1e-11 * np.max(np.abs(T))
    assert abs(o["I"] - float(r["I"])) < 1e-11 * abs(float(r["I"]))


@pytest.mark.parametrize("i", range(3))
def test_fp64_oracle_within_condition_bound_of_ground_truth(i):
    case = golden()["cases"][i]
    dev, U, g = golden_device(case)
    o = ochg.negf_evaluate(dev, U, g, method="sancho")
    eT, en, eI = errors(case, o["n"], o["T"], o["I"])
    tol_T, tol_n, tol_I = bounds(case)
    assert np.all(eT < tol_T), (eT, tol_T)
    assert en < tol_n and eI < tol_I, (en, tol_n, eI, tol_I)
