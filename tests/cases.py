"""Test cases built twice from the same seeded inputs: once with the oracle's own builders
and grids, once through the C ABI's builders and grid helper.  Nothing computed by one side
is fed to the other."""
import numpy as np

from oracle import charge as ochg
from oracle import model as omdl
from oracle import quadrature as oq

RULES = {"gauss": 0, "midpoint": 1}


def rel_inf(x, ref):
    """||x - ref||_inf / ||ref||_inf (norm-wise relative error of a vector output)."""
    x = np.asarray(x)
    ref = np.asarray(ref)
    den = np.max(np.abs(ref)) if ref.size else 0.0
    return float(np.max(np.abs(x - ref)) / den) if den > 0 else float(np.max(np.abs(x - ref), initial=0.0))


def current_err(I, Iref, g, dmu):
    """|I - I_ref| / max(|I_ref|, 1e-6 * g e^2/h |mu_S - mu_D|) (net currents can be ~0)."""
    scale = max(abs(Iref), 1e-6 * g * ochg.E2_OVER_H * max(abs(dmu), 1e-3))
    return abs(I - Iref) / scale


def oracle_device(kind, n_tube, t, N, U_S, U_D, modes=(1,), cells=False):
    return omdl.cnt_build(kind, n_tube, t, N, U_S, U_D, modes=modes, cells=cells)


def oracle_grid(p):
    return oq.bias_grid(p["mu_S"], p["mu_D"], p["kT"], p["n_real"], p["n_cont"], p["E_B"], p["eta"],
                        rule=p.get("rule", "gauss"), E_min=p.get("E_min"), E_max=p.get("E_max"))


def lib_device(ctx, kind, n_tube, t, N, U_S, U_D, modes=(1,), cells=False):
    if kind == "mode":
        if cells:
            dev = ctx.device_create(N, block=2, rings_per_block=2, n_chains=len(modes))
        else:
            dev = ctx.device_create(N, block=1, rings_per_block=1, n_chains=len(modes))
        ctx.build_cnt_modespace(dev, n_tube, t, list(modes), U_S, U_D)
    else:
        dev = ctx.device_create(N, block=n_tube, rings_per_block=1, n_chains=1)
        ctx.build_cnt_realspace(dev, n_tube, t, U_S, U_D)
    return dev


def lib_grid(ctx, dev, p):
    nan = float("nan")
    E_min = p.get("E_min")
    E_max = p.get("E_max")
    ctx.set_grid_spec(dev, p["mu_S"], p["mu_D"], p["kT"], p["eta"], p["E_B"], p["n_real"], p["n_cont"],
                      rule=RULES[p.get("rule", "gauss")], E_min=nan if E_min is None else E_min,
                      E_max=nan if E_max is None else E_max)


def case_params(kind, N, n_real, n_cont, U, mu_S=0.0, mu_D=-0.1, kT=0.025, eta=1e-6, rule="gauss",
                E_min=None, E_max=None, t=-2.7, n_tube=17, modes=(1,), cells=False, U_S=None, U_D=None):
    U = np.asarray(U, dtype=np.float64)
    return dict(kind=kind, N=N, n_real=n_real, n_cont=n_cont, U=U, mu_S=mu_S, mu_D=mu_D, kT=kT, eta=eta,
                rule=rule, E_min=E_min, E_max=E_max, t=t, n_tube=n_tube, modes=tuple(modes), cells=cells,
                U_S=float(U[0]) if U_S is None else U_S, U_D=float(U[-1]) if U_D is None else U_D,
                E_B=float(min(U.min(), -abs(mu_D - mu_S)) - 3.0 * abs(t) - 1.0))


def run_oracle(p, chunk=64):
    dev = oracle_device(p["kind"], p["n_tube"], p["t"], p["N"], p["U_S"], p["U_D"], p["modes"], p["cells"])
    return ochg.negf_evaluate(dev, p["U"], oracle_grid(p), chunk=chunk)


def run_lib(ctx, p):
    dev = lib_device(ctx, p["kind"], p["n_tube"], p["t"], p["N"], p["U_S"], p["U_D"], p["modes"], p["cells"])
    ctx.set_potential(dev, p["U"])
    lib_grid(ctx, dev, p)
    return dev, ctx.compute([dev])[0]
