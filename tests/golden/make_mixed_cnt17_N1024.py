"""Writes tests/golden/mixed_cnt17_N1024.json: ring electron counts n, T(E) at every real-axis
energy and the current I of the (17,0) real-space tube of the mixed-precision workload (1024
rings, 4096 energies, a quarter of them within 20 meV of a lead subband edge; Sec. 3.1's
(n,0) construction, Eq. GR leads, Alg. 1 / Alg. 2 as read), computed by the FP64 oracle.

The grid is built here from oracle/quadrature.py and the seeded inputs of synth: uniform
weights 2 / 4096 over [-1, 1] eV, Fermi factors at mu_S = 0 and mu_D = -0.1 eV (kT = 25 meV),
and a 64-node semicircle from E_B = min U - 3|t| - 1 eV to -1 eV.  The contour nodes and
weights are stored beside the outputs, so that the GPU test evaluates exactly this grid.

Usage: python tests/golden/make_mixed_cnt17_N1024.py   (calls only oracle/ and the seeded
input generators; a few minutes on eight cores)
"""
import json
import multiprocessing as mp
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

N_TUBE, N, N_E, N_CONT = 17, 1024, 4096, 64


def grid():
    from oracle import quadrature as oq
    from paper_2407_14633_gb300 import synth
    w = synth.mixed_precision(n_tube=N_TUBE, N=N, n_energies=N_E)
    E = np.asarray(w["E"], dtype=np.float64)
    E_B = float(np.min(w["U"]) - 3.0 * abs(w["t"]) - 1.0)
    z, c = oq.contour_semicircle(E_B, -1.0, N_CONT)
    return w, dict(E=E, w=np.full(E.size, 2.0 / E.size), fS=oq.fermi(E - w["mu_S"], w["kT"]),
                   fD=oq.fermi(E - w["mu_D"], w["kT"]), eta=w["eta"], z=z, c=c)


def part(args):
    """The oracle on a slice of the real-axis energies and of the contour nodes."""
    sl_r, sl_c = args
    from oracle import charge as ochg
    from oracle import model as omdl
    w, g = grid()
    dev = omdl.cnt_build("real", N_TUBE, w["t"], N, w["U_S"], w["U_D"])
    sub = dict(E=g["E"][sl_r], w=g["w"][sl_r], fS=g["fS"][sl_r], fD=g["fD"][sl_r], eta=g["eta"],
               z=g["z"][sl_c], c=g["c"][sl_c])
    r = ochg.negf_evaluate(dev, w["U"], sub, chunk=32)
    return r["n_real"], r["n_cont"], r["T"], r["I"]


def main():
    w, g = grid()
    k = 64
    jobs = [(slice(i * N_E // k, (i + 1) * N_E // k), slice(i * N_CONT // k, (i + 1) * N_CONT // k)) for i in range(k)]
    with mp.get_context("spawn").Pool(os.cpu_count()) as pool:
        parts = pool.map(part, jobs)
    n_real = np.sum([p[0] for p in parts], axis=0)
    n_cont = np.sum([p[1] for p in parts], axis=0)
    T = np.concatenate([p[2] for p in parts])
    I = float(np.sum([p[3] for p in parts]))
    out = {"source": "oracle/charge.py negf_evaluate (FP64); inputs as stated in the module docstring",
           "n_tube": N_TUBE, "N": N, "n_energies": N_E, "n_cont": N_CONT,
           "mu_S": w["mu_S"], "mu_D": w["mu_D"], "kT": w["kT"], "eta": w["eta"], "U_S": w["U_S"], "U_D": w["U_D"],
           "t": w["t"], "z": [[float(x.real), float(x.imag)] for x in g["z"]],
           "c": [[float(x.real), float(x.imag)] for x in g["c"]],
           "n": ["%.17g" % x for x in n_real + n_cont], "n_cont": ["%.17g" % x for x in n_cont],
           "T": ["%.15e" % x for x in T], "I": "%.17g" % I}
    with open(os.path.join(HERE, "mixed_cnt17_N1024.json"), "w") as fh:
        json.dump(out, fh, separators=(",", ":"))


if __name__ == "__main__":
    main()
