"""Pins of the oracle's nanotube Hamiltonians (Sec. 3.1, Table 1; Guo et al. mode space)."""
import json
import os

import numpy as np
import pytest

from oracle import model as mdl

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def zigzag_bands(t, c, k):
    """Closed form of the dimerised chain: E = +-|t| sqrt(1 + 4c^2 + 4c cos k), c = cos(pi j/n)."""
    return abs(t) * np.sqrt(1 + 4 * c * c + 4 * c * np.cos(k))


@pytest.mark.parametrize("j", [1, 4, 6, 11])
def test_mode_chain_bloch_dispersion(j):
    n, t = 17, -2.7
    bj = mdl.mode_hopping(n, j, t)
    c = np.cos(np.pi * j / n)
    for k in np.linspace(-np.pi, np.pi, 13):
        H = mdl.bloch_hamiltonian(lambda r: mdl.mode_bond(r, t, bj), 2, k)
        ev = np.sort(np.linalg.eigvalsh(H))
        e = zigzag_bands(t, c, k)
        assert np.allclose(ev, [-e, e], atol=1e-13)


def test_realspace_bloch_is_union_of_modes():
    # 4-ring period (the zigzag bonds alternate I+S and I+S^T); the 2-ring-cell momentum
    # K of each mode folds onto k as K in {k/2, k/2 + pi}
    n, t = 7, -2.7
    for k in np.linspace(-np.pi, np.pi, 7):
        H = mdl.bloch_hamiltonian(lambda r: mdl.realspace_bond(r, t, n), 4, k)
        ev = np.sort(np.linalg.eigvalsh(H))
        ref = []
        for j in range(n):
            c = np.cos(np.pi * j / n)
            for K in (k / 2, k / 2 + np.pi):
                e = zigzag_bands(t, c, K)
                ref += [e, -e]
        assert np.allclose(ev, np.sort(ref), atol=1e-12)


def test_band_gap_matches_paper():
    gold = GOLD["band_gap_17_0"]
    n, t = gold["n_tube"], gold["t_eV"]
    gap = np.inf
    for j in range(1, n):
        bj = mdl.mode_hopping(n, j, t)
        for k in np.linspace(-np.pi, np.pi, 721):
            ev = np.linalg.eigvalsh(mdl.bloch_hamiltonian(lambda r: mdl.mode_bond(r, t, bj), 2, k))
            gap = min(gap, ev[1] - ev[0])
    assert abs(gap - gold["gap_eV"]) < gold["tolerance_eV"]
    assert abs(gap - 0.5426) < 1e-3


def test_ring_pitch_from_table1():
    gold = GOLD["ring_pitch"]
    dx = 0.75 * gold["a_cc_nm"]
    assert abs(512 * dx - gold["overall_nm_512"]) / gold["overall_nm_512"] < gold["tolerance_rel"]
    for N, Lc in zip(gold["rings"], gold["channel_nm"]):
        total = Lc + 2 * gold["contact_nm"]
        assert abs(N * dx - total) / total < gold["tolerance_rel"]


def test_realspace_spectrum_is_union_of_mode_chains():
    # finite tubes: the real-space matrix with a ring-uniform potential is unitarily
    # equivalent to the direct sum of the n mode chains (all j, the S phases gauge away)
    n, t, N = 5, -2.7, 6
    U = np.linspace(-0.2, 0.3, N)
    Hr = mdl.dense_hamiltonian(mdl.realspace_chain(n, t, N, 0, 0), U)
    ev = np.sort(np.linalg.eigvalsh(Hr))
    ref = []
    for j in range(n):
        ref += list(np.linalg.eigvalsh(mdl.dense_hamiltonian(mdl.mode_chain(n, j, t, N, 0, 0), U)))
    assert np.allclose(ev, np.sort(ref), atol=1e-12)


def test_unit_cell_regrouping_is_same_matrix():
    n, t, N = 17, -2.7, 10
    U = np.linspace(0, 0.1, N)
    a = mdl.dense_hamiltonian(mdl.mode_chain(n, 6, t, N, 0, 0), U)
    b = mdl.dense_hamiltonian(mdl.mode_chain_cells(n, 6, t, N, 0, 0), U)
    assert np.array_equal(a, b)
