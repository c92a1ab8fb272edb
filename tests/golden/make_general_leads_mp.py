"""Writes tests/golden/general_leads_mp.json: ring electron counts, T(E) and current of three
small tubes with general (non-circulant) leads, computed by the extended-precision oracle
(oracle/extended.py, mpmath at 30 digits), with a condition estimate per energy.

The grids take Gauss-Legendre nodes of the bias window and two energies 2e-4 eV on either
side of a band edge of the source lead (where decimation is ill-conditioned), plus contour
nodes.  Every input is stored beside the expected values, so that the FP64 oracle and the GPU
are evaluated on exactly these energies, weights and Fermi factors.

Usage: python tests/golden/make_general_leads_mp.py   (calls only oracle/ and the seeded
input generators; runs for tens of minutes in pure-Python multiprecision)
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import extended as ex            # noqa: E402
from oracle import model as omdl             # noqa: E402
from oracle import quadrature as oq          # noqa: E402
from paper_2407_14633_gb300 import synth     # noqa: E402

KT, ETA, E_B, MU_S, MU_D, U_S, U_D = 0.025, 1e-6, -12.0, 0.0, -0.3, 0.05, -0.3
CASES = [  # (n_tube, rings, lead sites, Gauss-Legendre nodes taken, contour nodes)
    (5, 4, [0, 1, 2, 3, 4], 6, 2),
    (7, 4, [0, 2, 3, 6], 6, 2),
    (17, 2, list(range(17)), 4, 1),
]


def band_edges(lead):
    """Energies of the lead's bands at k = 0 and k = pi (two-ring principal layer), where a
    band of a chain of layers starts or ends."""
    m = lead.m
    h0 = lead.U * np.eye(m) + (0.0 if lead.H0 is None else lead.H0)
    h1 = lead.U * np.eye(m) + (0.0 if lead.H1 is None else lead.H1)
    H00 = np.block([[h0, lead.T1.conj().T], [lead.T1, h1]])
    Z = np.zeros((m, m))
    H01 = np.block([[Z, Z], [lead.T2.conj().T, Z]])
    out = []
    for k in (0.0, np.pi):
        Hk = H00 + H01 * np.exp(1j * k) + H01.conj().T * np.exp(-1j * k)
        out.extend(np.linalg.eigvalsh(0.5 * (Hk + Hk.conj().T)))
    return np.array(sorted(out))


def build(n_tube, N, sites):
    m = len(sites)
    leads = [synth.general_lead(m, 100 + n_tube), synth.general_lead(m, 200 + n_tube)]
    dev = omdl.cnt_build("real", n_tube, -2.7, N, U_S, U_D)
    ch = dev.chains[0]
    ch.lead_S = omdl.Lead(U_S, leads[0]["T1"], leads[0]["T2"], leads[0]["tau"], np.asarray(sites),
                          H0=leads[0].get("H0"), H1=leads[0].get("H1"))
    ch.lead_D = omdl.Lead(U_D, leads[1]["T1"], leads[1]["T2"], leads[1]["tau"], np.asarray(sites),
                          H0=leads[1].get("H0"), H1=leads[1].get("H1"))
    U = synth.sinusoid_profile(N, 9, amplitude=0.2)
    return dev, U


def grid(dev, n_gl, n_cont):
    lo, hi = MU_D - 14 * KT, MU_S + 14 * KT
    E_gl, w_gl = oq.real_axis_gauss(lo, hi, 40)
    pick = np.linspace(0, 39, n_gl).round().astype(int)
    edges = band_edges(dev.chains[0].lead_S)
    e = edges[np.argmin(np.abs(edges - 0.5 * (lo + hi)))]   # the edge nearest the window
    E = np.concatenate([E_gl[pick], [e - 2e-4, e + 2e-4]])
    w = np.concatenate([w_gl[pick], [1e-3, 1e-3]])
    z, c = oq.contour_semicircle(E_B, lo, n_cont)
    return dict(E=E, w=w, fS=oq.fermi(E - MU_S, KT), fD=oq.fermi(E - MU_D, KT), eta=ETA, z=z, c=c,
                edge=float(e))


def main():
    out = {"source": "oracle/extended.py at %d digits; inputs as stored" % ex.DPS, "cases": []}
    for n_tube, N, sites, n_gl, n_cont in CASES:
        dev, U = build(n_tube, N, sites)
        g = grid(dev, n_gl, n_cont)
        r = ex.evaluate(dev, U, g)
        k = ex.condition(dev, U, g, samples=1)
        out["cases"].append({
            "n_tube": n_tube, "N": N, "sites": sites, "U_S": U_S, "U_D": U_D, "mu_S": MU_S, "mu_D": MU_D,
            "lead_seeds": [100 + n_tube, 200 + n_tube], "U": [float(x) for x in U],
            "E": [float(x) for x in g["E"]], "w": [float(x) for x in g["w"]],
            "fS": [float(x) for x in g["fS"]], "fD": [float(x) for x in g["fD"]], "eta": ETA,
            "z": [[float(x.real), float(x.imag)] for x in g["z"]],
            "c": [[float(x.real), float(x.imag)] for x in g["c"]], "lead_band_edge": g["edge"],
            "n": [str(x) for x in r["n"]], "n_cont": [str(x) for x in r["n_cont"]],
            "T": [str(x) for x in r["T"]], "I": str(r["I"]),
            "kappa_T": k["kappa_T"], "kappa_n": k["kappa_n"]})
        print("case", n_tube, N, "kappa_T", ["%.2g" % x for x in k["kappa_T"]], "kappa_n %.2g" % k["kappa_n"],
              flush=True)
    with open(os.path.join(HERE, "general_leads_mp.json"), "w") as fh:
        json.dump(out, fh, indent=1)


if __name__ == "__main__":
    main()
