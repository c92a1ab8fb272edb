"""CPU check of the algebra behind the sweep of 1 x 1 chains split along the channel.

A plain numpy model of its five steps (per-segment Moebius maps of the forward recursion,
their two-level scan, the re-run with per-segment affine maps of the backward update and the
drain/source products, their scan, the backward re-run) is compared with the oracle's block
recursion on a long 1 x 1 chain at band, band-edge, gap and contour energies.  The model is
test code: it shares nothing with the CUDA path or the oracle, and it pins the decomposition
(which the GPU tests then check kernel by kernel against the oracle) to the plain recursion.
"""
import numpy as np
import pytest

from oracle import green as ogr
from oracle import model as omdl
from paper_2407_14633_gb300 import synth


def _rescale(maps):
    """Scale a 2 x 2 projective map by a power of two so that its largest component is in [1, 2)."""
    parts = np.stack([np.abs(m.real) for m in maps] + [np.abs(m.imag) for m in maps])
    big = np.max(parts, axis=0)
    ok = (big > 0) & np.isfinite(big)
    e = np.where(ok, -np.floor(np.log2(np.where(ok, big, 1.0))), 0).astype(int)
    return tuple(np.ldexp(m.real, e) + 1j * np.ldexp(m.imag, e) for m in maps)


def split_model(x, hsq, gam_s, gam_d, seg=512, chunks=16):
    """x: (L, E) layer terms eps - H_ll - U_l - Sigma; hsq: (L-1,) |h|^2; gam_*: (E,).
    Returns G_ll (L, E), A_S and A_D diagonals (L, E), T (E,)."""
    L, E = x.shape
    ns = (L + seg - 1) // seg
    bounds = [(s * seg, min(L, s * seg + seg)) for s in range(ns)]
    # 1. forward maps per segment: [[0, 1], [-|h_{l-1}|^2, x_l]] applied in order
    fmap = []
    for l0, l1 in bounds:
        a, b, c, d = np.ones(E, complex), np.zeros(E, complex), np.zeros(E, complex), np.ones(E, complex)
        for l in range(l0, l1):
            h = hsq[l - 1] if l > 0 else 0.0
            a, b, c, d = c, d, x[l] * c - h * a, x[l] * d - h * b
            if (l - l0) % 8 == 7:
                a, b, c, d = _rescale((a, b, c, d))
        fmap.append(_rescale((a, b, c, d)))
    # 2. two-level scan: chunk products, chain over chunks, walk inside each chunk
    per = (ns + chunks - 1) // chunks
    cr = [(min(ns, k * per), min(ns, k * per + per)) for k in range(chunks)]
    prod = []
    for s0, s1 in cr:
        A, B, C, D = np.ones(E, complex), np.zeros(E, complex), np.zeros(E, complex), np.ones(E, complex)
        for s in range(s0, s1):
            a, b, c, d = fmap[s]
            A, B, C, D = _rescale((a * A + b * C, a * B + b * D, c * A + d * C, c * B + d * D))
        prod.append((A, B, C, D))
    g = np.zeros(E, complex)
    entry = []
    for A, B, C, D in prod:
        entry.append(g)
        g = (A * g + B) / (C * g + D)
    g_out = [None] * ns
    for k, (s0, s1) in enumerate(cr):
        g = entry[k]
        for s in range(s0, s1):
            a, b, c, d = fmap[s]
            g = (a * g + b) / (c * g + d)
            g_out[s] = g
    # 3. re-run per segment from its entry value; backward affine map and products
    gl = np.zeros((L, E), complex)
    qrel = np.zeros((L, E))
    amap = []
    for s, (l0, l1) in enumerate(bounds):
        gp = g_out[s - 1] if s > 0 else np.zeros(E, complex)
        q, cp = np.ones(E), np.ones(E)
        A, B = np.zeros(E, complex), np.ones(E, complex)
        for l in range(l0, l1):
            xl = x[l].copy()
            if l > 0:
                xl = xl - hsq[l - 1] * gp
                q = hsq[l - 1] * np.abs(gp) ** 2 * q
            g = 1.0 / xl
            gl[l], qrel[l] = g, q
            A = A + B * g
            if l < L - 1:
                B = B * hsq[l] * g * g
                cp = hsq[l] * np.abs(g) ** 2 * cp
            else:
                B = np.zeros(E, complex)
                cp = np.abs(g) ** 2 * cp
            gp = g
        amap.append((A, B, q, cp))
    # 4. entry values of the backward re-run, two-level like the forward scan
    comp = []
    for s0, s1 in cr:
        A, B, cp, qp = np.zeros(E, complex), np.ones(E, complex), np.ones(E), np.ones(E)
        for s in range(s0, s1):
            A, B = A + B * amap[s][0], B * amap[s][1]
            qp, cp = amap[s][2] * qp, cp * amap[s][3]
        comp.append((A, B, qp, cp))
    G, c, q = np.zeros(E, complex), np.ones(E), np.ones(E)
    eg, ec, eq = [None] * chunks, [None] * chunks, [None] * chunks
    for k in range(chunks - 1, -1, -1):
        eg[k], ec[k] = G, c
        G, c = comp[k][0] + comp[k][1] * G, comp[k][3] * c
    for k in range(chunks):
        eq[k] = q
        q = comp[k][2] * q
    g_in, c_in, q_in = [None] * ns, [None] * ns, [None] * ns
    for k, (s0, s1) in enumerate(cr):
        G, c = eg[k], ec[k]
        for s in range(s1 - 1, s0 - 1, -1):
            g_in[s], c_in[s] = G, c
            G, c = amap[s][0] + amap[s][1] * G, amap[s][3] * c
        q = eq[k]
        for s in range(s0, s1):
            q_in[s] = q
            q = amap[s][2] * q
    # 5. backward re-run
    Gd, AS, AD = np.zeros((L, E), complex), np.zeros((L, E)), np.zeros((L, E))
    T = None
    for s, (l0, l1) in enumerate(bounds):
        G, c = g_in[s], c_in[s]
        for l in range(l1 - 1, l0 - 1, -1):
            g = gl[l]
            if l < L - 1:
                G = g + g * (hsq[l] * g * G)
                c = hsq[l] * np.abs(g) ** 2 * c
            else:
                G, c = g, np.abs(g) ** 2 * c
            Gd[l], AD[l] = G, gam_d * c
            AS[l] = gam_s * q_in[s] * qrel[l] * np.abs(G) ** 2
        if l0 == 0:
            T = gam_s * gam_d * c
    return Gd, AS, AD, T


def _rel(x, ref):
    return float(np.max(np.abs(x - ref)) / np.max(np.abs(ref)))


def _chain(L):
    dev = omdl.cnt_build("mode", 17, -2.7, L, 0.0, -0.1, modes=(6,))
    return dev.chains[0], (synth.ramp_barrier(L) if L > 1 else np.array([0.05]))


@pytest.mark.parametrize("L", [1, 700, 3000])
def test_split_model_matches_oracle_recursion(L):
    # L = 700: a full and a ragged segment; 3000: six segments, ten empty scan chunks
    ch, U = _chain(L)
    E = np.array([-2.0, -0.45, -0.3, 0.0, 0.33, 2.5]) + 1e-6j     # band, edge, gap, band
    sS, sD, gS, gD = ogr.contact_blocks(ch, E)
    x = ogr._alphas(ch, U, E, sS, sD)[:, :, 0, 0]
    hsq = np.abs(ch.Hup[:, 0, 0]) ** 2 if L > 1 else np.zeros(0)
    Gd, AS, AD, T = split_model(x, hsq, gS[:, 0, 0].real, gD[:, 0, 0].real)
    o = ogr.rgf_lanes(ch, U, E)
    assert _rel(Gd.T, o["Gdiag"][:, :, 0]) < 1e-10
    assert _rel(AS.T, o["AS"][:, :, 0]) < 1e-10
    assert _rel(AD.T, o["AD"][:, :, 0]) < 1e-10
    for k in range(E.size):   # each T on its own scale (gap values are ~1e-70)
        assert abs(T[k] - o["T"][k]) <= 1e-10 * abs(o["T"][k])


def test_split_model_contour_energies():
    ch, U = _chain(3000)
    z = np.array([-9.0 + 0.3j, -5.0 + 3.9j, -1.0 + 1.0j, -0.2 + 0.01j])
    sS, sD, gS, gD = ogr.contact_blocks(ch, z)
    x = ogr._alphas(ch, U, z, sS, sD)[:, :, 0, 0]
    Gd, _, _, _ = split_model(x, np.abs(ch.Hup[:, 0, 0]) ** 2, np.zeros(z.size), np.zeros(z.size))
    o = ogr.rgf_lanes(ch, U, z, spectral=False)
    assert _rel(Gd.T, o["Gdiag"][:, :, 0]) < 1e-12


def test_split_model_catches_a_wrong_join():
    # a plausible mistake at a join (the bond across the first segment boundary dropped, so the
    # two halves decouple) must fail the same comparison
    ch, U = _chain(1100)
    E = np.array([-1.2, 0.9]) + 1e-6j
    sS, sD, gS, gD = ogr.contact_blocks(ch, E)
    x = ogr._alphas(ch, U, E, sS, sD)[:, :, 0, 0]
    hsq = np.abs(ch.Hup[:, 0, 0]) ** 2
    o = ogr.rgf_lanes(ch, U, E)
    Gd, _, _, _ = split_model(x, hsq, gS[:, 0, 0].real, gD[:, 0, 0].real)
    assert _rel(Gd.T, o["Gdiag"][:, :, 0]) < 1e-10
    cut = hsq.copy()
    cut[511] = 0.0
    Gc, _, _, _ = split_model(x, cut, gS[:, 0, 0].real, gD[:, 0, 0].real)
    assert _rel(Gc.T, o["Gdiag"][:, :, 0]) > 1e-3
