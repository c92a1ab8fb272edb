"""Runners for the batched, mixed-precision, serving and gate-sweep workloads through the C ABI
(used by bench.py --extras).  Timing uses the library's event-bracketed sweep time and host
wall clock; inputs come from synth.py."""
import time

import numpy as np

from . import negf, synth


def _rel(x, ref):
    den = np.max(np.abs(ref))
    return float(np.max(np.abs(np.asarray(x) - ref)) / den) if den > 0 else 0.0


def build_uneven(ctx, w, n_devices=None):
    """The uneven batch: mode-space (17,0) devices, 1x1 or 2x2 blocks, 1-4 modes."""
    devs = []
    for d in w["devices"][:n_devices]:
        N = d["N"]
        cells = d["block"] == 2
        dev = ctx.device_create(N, block=2 if cells else 1, rings_per_block=2 if cells else 1,
                                n_chains=len(d["modes"]))
        ctx.build_cnt_modespace(dev, w["n_tube"], w["t"], list(d["modes"]), 0.0, -d["V_DS"])
        ctx.set_potential(dev, d["U"])
        ctx.set_grid_spec(dev, 0.0, -d["V_DS"], w["kT"], w["eta"], d["E_B"], d["n_real"], d["n_cont"])
        devs.append(dev)
    return devs


def modespace_small(reps=20):
    """The small plain-FP64 case: (17,0) mode space, N = 64, 256 midpoint + 64 contour
    energies, modes j = 1 (literal) and j = 6; one negf_compute per call (latency-bound)."""
    out = {}
    for j in (1, 6):
        w = synth.modespace_small(j)
        with negf.Context() as ctx:
            dev = ctx.device_create(w["N"], block=1, rings_per_block=1, n_chains=1)
            ctx.build_cnt_modespace(dev, w["n_tube"], w["t"], [j], w["U_S"], w["U_D"])
            ctx.set_potential(dev, w["U"])
            ctx.set_grid_spec(dev, w["mu_S"], w["mu_D"], w["kT"], w["eta"], w["E_B"], w["n_real"], w["n_cont"],
                              rule=negf.RULE_MIDPOINT, E_min=-1.0, E_max=1.0)
            ctx.compute([dev])
            ctx.profile(True)
            ctx.kernel_time()
            t0 = time.perf_counter()
            for _ in range(reps):
                ctx.compute([dev])
            wall = (time.perf_counter() - t0) / reps
            ms, k = ctx.kernel_time()
        units = w["N"] * (w["n_real"] + w["n_cont"])
        out["j=%d" % j] = {"sweep_ms": ms / max(k, 1), "updates_per_s_sweep": units / (ms / max(k, 1) * 1e-3),
                           "call_ms": wall * 1e3, "updates_per_s_call": units / wall}
    return out


def batched_uneven(reps=3):
    """All 64 uneven devices in one negf_compute (one launch per kernel class and element
    type), complex128 and complex64; updates counted per (ring, energy, mode)."""
    w = synth.batched_uneven()
    units = sum(d["N"] * len(d["modes"]) * (d["n_real"] + d["n_cont"]) for d in w["devices"])
    out = {"devices": len(w["devices"]), "ring_energy_mode_updates": units}
    ref = None
    for name, prec in (("c128", negf.PREC_FP64), ("c64", negf.PREC_FP32)):
        with negf.Context(precision=prec) as ctx:
            t0 = time.perf_counter()
            devs = build_uneven(ctx, w)
            t_setup = time.perf_counter() - t0
            res = ctx.compute(devs)
            ctx.profile(True)
            ctx.kernel_time()
            t0 = time.perf_counter()
            for _ in range(reps):
                res = ctx.compute(devs)
            wall = (time.perf_counter() - t0) / reps
            ms, k = ctx.kernel_time()
            fp32 = prec == negf.PREC_FP32
            widths = {"1x1": ctx.chain_width(1, fp32), "2x2": ctx.chain_width(2, fp32)}
        sweep_s = ms / max(k, 1) * 1e-3
        entry = {"updates_per_s_sweep": units / sweep_s, "sweep_ms": sweep_s * 1e3,
                 "updates_per_s_e2e": units / wall, "e2e_ms": wall * 1e3, "setup_s": t_setup,
                 "cta_warps": widths}
        if ref is None:
            ref = res
        else:
            entry["max_rel_err_n_vs_c128"] = max(_rel(a["n"], b["n"]) for a, b in zip(res, ref))
            entry["max_rel_err_T_vs_c128"] = max(_rel(a["T"], b["T"]) for a, b in zip(res, ref))
        out[name] = entry
    return out


def _fermi(x, kT):
    return 0.5 * (1.0 - np.tanh(0.5 * np.asarray(x) / kT))


def _edge_near(n_tube, t, E, U_lead, window):
    """Energies within window of a subband edge of the (n,0) lead, edges
    U_lead +- |t| |1 -+ 2 cos(pi j / n)| (the zone-centre and zone-boundary energies)."""
    j = np.arange(n_tube)
    b = 2.0 * abs(t) * np.abs(np.cos(np.pi * j / n_tube))
    edges = np.concatenate([abs(t) - b, b - abs(t), abs(t) + b, -abs(t) - b])
    d = np.min(np.abs(np.asarray(E)[:, None] - U_lead - edges[None, :]), axis=1)
    return d < window


def mixed_precision(tubes=(17, 26, 34), N=1024, n_energies=4096,
                    variants=((0.02, 20.0, 1e-4), (0.002, 20.0, 1e-4), (0.002, 0.0, 1e-4), (0.002, 0.0, 1e-3))):
    """Real-space (n,0) tubes, a quarter of the energies within 20 meV of a lead subband edge:
    complex128 sweep vs the mixed path (complex64 sweep, FP64 recompute of flagged energies;
    one run per (band-edge window, growth threshold, residual threshold); a growth threshold
    of 0 switches that criterion off) vs the plain complex64 sweep; errors per output against
    the complex128 result, and which criterion flagged how many energies."""
    out = {}
    thr, gthr = 1e-3, 20.0
    for n_tube in tubes:
        w = synth.mixed_precision(n_tube=n_tube, N=N, n_energies=n_energies)
        E = w["E"]
        wts = np.full(E.size, 2.0 / E.size)
        fS, fD = _fermi(E - w["mu_S"], w["kT"]), _fermi(E - w["mu_D"], w["kT"])
        E_B = float(np.min(w["U"]) - 3.0 * abs(w["t"]) - 1.0)
        cg = negf.make_grid(w["mu_S"], w["mu_D"], w["kT"], w["eta"], E_B, 1, 64, E_min=-1.0, E_max=1.0)
        runs = [("c128", negf.PREC_FP64, {})] + \
            [("mixed_w%g_g%g_r%g" % (win, gro, rth), negf.PREC_MIXED,
              dict(flag_threshold=rth, growth_threshold=gro if gro > 0 else 1e300, edge_window=win))
             for win, gro, rth in variants] + [("c64", negf.PREC_FP32, {})]
        res = {}
        for name, prec, kw in runs:
            with negf.Context(precision=prec, **kw) as ctx:
                dev = ctx.device_create(N, block=n_tube, rings_per_block=1, n_chains=1)
                ctx.build_cnt_realspace(dev, n_tube, w["t"], w["U_S"], w["U_D"])
                ctx.set_potential(dev, w["U"])
                ctx.set_grid(dev, E, wts, fS, fD, w["eta"], cg["z"], cg["c"])
                ctx.profile(True)
                ctx.kernel_time()
                t0 = time.perf_counter()
                r = ctx.compute_diag(dev)
                wall = time.perf_counter() - t0
                ms, _ = ctx.kernel_time()
            r["sweep_ms"], r["wall_s"] = ms, wall
            res[name] = r
        ref = res["c128"]
        Tmax = float(np.max(np.abs(ref["T"])))
        entry = {"c128_sweep_ms": ref["sweep_ms"]}
        c64 = res["c64"]
        by_resid = ~(c64["resid"] <= thr)
        by_growth = ~(c64["growth"] <= gthr)
        entry["c64_residual_quantiles"] = {q: float(np.nanpercentile(c64["resid"], float(q)))
                                           for q in ("50", "90", "99")}
        entry["flagged_by_residual"] = float(np.mean(by_resid))
        entry["flagged_by_growth"] = float(np.mean(by_growth))
        entry["c64_T_err_unflagged_by_residual_growth"] = float(
            np.max(np.abs(c64["T"] - ref["T"])[~(by_resid | by_growth)], initial=0.0) / Tmax)
        for name, _, kw in runs[1:]:
            r = res[name]
            dI = abs(r["I"] - ref["I"]) / max(abs(ref["I"]), 1e-30)
            e = {"sweep_ms": r["sweep_ms"], "speedup_vs_c128": ref["sweep_ms"] / r["sweep_ms"],
                 "rel_err_n": _rel(r["n"], ref["n"]), "rel_err_T": _rel(r["T"], ref["T"]), "rel_err_I": dI}
            if name.startswith("mixed"):
                near = _edge_near(n_tube, w["t"], E, w["U_S"], kw["edge_window"])
                e["edge_window_eV"] = kw["edge_window"]
                e["growth_threshold"] = kw["growth_threshold"] if kw["growth_threshold"] < 1e300 else None
                e["residual_threshold"] = kw["flag_threshold"]
                e["recomputed_fraction"] = float(np.mean(r["flags"]))
                e["flagged_by_edge_window"] = float(np.mean(near))
            entry[name] = e
        out["(%d,0)" % n_tube] = entry
    return out


def serving_sweep(n_requests=256, rate_factor=2.0, tol=1e-5, M=64):
    """Self-consistent I-V requests (the first n_requests of the seeded 256-request stream): a
    sequential loop of negf_sc_solve calls, then the continuous-batching server with Poisson
    arrivals at rate_factor x the sequential rate, the sequential loop again under the same
    arrivals, and the server with every request queued at once (its capacity).  tol is the
    convergence threshold of Alg. 3 (1e-5).  Rates are given over all requests and over the
    converged ones alone; latencies run from a request's arrival to its result."""
    w = synth.serving_sweep(n_requests=256)
    w["requests"] = w["requests"][:n_requests]
    w["unit_gaps"] = w["unit_gaps"][:n_requests]
    reqs = w["requests"]
    kappa = negf.poisson_kappa()
    # sequential baseline: one solve at a time on the GPU
    seq_lat = []
    seq_res = []
    with negf.Context() as ctx:
        t_all = time.perf_counter()
        for q in reqs:
            t0 = time.perf_counter()
            dev = ctx.device_create(q["N"], n_chains=len(q["modes"]))
            ctx.build_cnt_modespace(dev, w["n_tube"], w["t"], list(q["modes"]), 0.0, -q["V_DS"])
            E_B = -q["V_DS"] - 3.0 * abs(w["t"]) - 1.0
            ctx.set_grid_spec(dev, 0.0, -q["V_DS"], w["kT"], w["eta"], E_B, q["n_real"], q["n_cont"])
            U0 = np.linspace(0.0, -q["V_DS"], q["N"])
            r = ctx.sc_solve(dev, q["V_DS"], q["V_GS"], U0, kappa, M=M, tol=tol, check=False)
            ctx.device_destroy(dev)
            seq_lat.append(time.perf_counter() - t0)
            seq_res.append(r)
        seq_total = time.perf_counter() - t_all
    seq_rate = n_requests / seq_total
    # served: Poisson arrivals
    arrivals = np.cumsum(w["unit_gaps"]) / (rate_factor * seq_rate)
    lat = []
    served = []
    with negf.Context() as ctx:
        t0 = time.perf_counter()
        tickets = [None] * n_requests
        nxt = 0
        done = 0
        while done < n_requests:
            now = time.perf_counter() - t0
            while nxt < n_requests and arrivals[nxt] <= now:
                q = reqs[nxt]
                tickets[nxt] = ctx.submit(q["N"], list(q["modes"]), q["V_DS"], q["V_GS"], n_real=q["n_real"],
                                          n_cont=q["n_cont"], tol=tol, M=M,
                                          U0=np.linspace(0.0, -q["V_DS"], q["N"]))
                nxt += 1
            active = ctx.serve_step()
            done = sum(1 for t in tickets[:nxt] if t is not None and ctx.poll(t) is not None)
            if active == 0 and done < nxt:
                continue
            if active == 0 and nxt < n_requests and done == nxt:
                time.sleep(max(0.0, arrivals[nxt] - (time.perf_counter() - t0)))
        total = time.perf_counter() - t0
        for i, tk in enumerate(tickets):
            ts, tst, td = ctx.request_times(tk)
            lat.append(td - ts)
            served.append(ctx.poll(tk))
    # the sequential loop under the same arrivals, run: each request is solved once it has
    # arrived and the one before it is done; its latency runs from its arrival
    seq_q = []
    with negf.Context() as ctx:
        t0 = time.perf_counter()
        for arr, q in zip(arrivals, reqs):
            idle = arr - (time.perf_counter() - t0)
            if idle > 0:
                time.sleep(idle)
            dev = ctx.device_create(q["N"], n_chains=len(q["modes"]))
            ctx.build_cnt_modespace(dev, w["n_tube"], w["t"], list(q["modes"]), 0.0, -q["V_DS"])
            E_B = -q["V_DS"] - 3.0 * abs(w["t"]) - 1.0
            ctx.set_grid_spec(dev, 0.0, -q["V_DS"], w["kT"], w["eta"], E_B, q["n_real"], q["n_cont"])
            ctx.sc_solve(dev, q["V_DS"], q["V_GS"], np.linspace(0.0, -q["V_DS"], q["N"]), kappa, M=M, tol=tol,
                         check=False)
            ctx.device_destroy(dev)
            seq_q.append(time.perf_counter() - t0 - arr)
    # capacity: all requests queued at t = 0
    with negf.Context() as ctx:
        t0 = time.perf_counter()
        tks = [ctx.submit(q["N"], list(q["modes"]), q["V_DS"], q["V_GS"], n_real=q["n_real"],
                          n_cont=q["n_cont"], tol=tol, M=M, U0=np.linspace(0.0, -q["V_DS"], q["N"]))
               for q in reqs]
        steps = 0
        while any(ctx.poll(t) is None for t in tks):
            ctx.serve_step()
            steps += 1
        sat_total = time.perf_counter() - t0
        sat = [ctx.poll(t) for t in tks]
    same = sum(1 for a, b, c in zip(seq_res, served, sat) if a["iterations"] == b["iterations"] == c["iterations"]
               and np.array_equal(a["n"], b["n"]) and np.array_equal(a["n"], c["n"]))
    # equal accuracy: a bias point counts once it reached the tolerance (the same requests
    # converge in every loop, the results being bitwise the same)
    conv = np.array([bool(r["converged"]) for r in served])
    n_conv = int(conv.sum())
    lat_c = np.asarray(lat)[conv] if n_conv else np.zeros(1)
    seqq_c = np.asarray(seq_q)[conv] if n_conv else np.zeros(1)
    return {"requests": n_requests, "converged_requests": n_conv,
            "converged_bias_points_per_s": {"sequential": n_conv / seq_total, "served": n_conv / total,
                                            "saturated": n_conv / sat_total},
            "converged_served_p50_s": float(np.percentile(lat_c, 50)),
            "converged_served_p99_s": float(np.percentile(lat_c, 99)),
            "converged_sequential_queued_p50_s": float(np.percentile(seqq_c, 50)),
            "converged_sequential_queued_p99_s": float(np.percentile(seqq_c, 99)),
            "sequential_bias_points_per_s": seq_rate,
            "sequential_p50_s": float(np.percentile(seq_lat, 50)), "sequential_p99_s": float(np.percentile(seq_lat, 99)),
            "sequential_queued_p50_s": float(np.percentile(seq_q, 50)),
            "sequential_queued_p99_s": float(np.percentile(seq_q, 99)),
            "served_bias_points_per_s": n_requests / total, "served_p50_s": float(np.percentile(lat, 50)),
            "served_p99_s": float(np.percentile(lat, 99)), "arrival_rate_per_s": rate_factor * seq_rate,
            "converged": int(sum(r["converged"] for r in served)),
            "saturated_bias_points_per_s": n_requests / sat_total, "saturated_steps": steps,
            "bitwise_same_as_sequential": same, "tol": tol,
            "mean_iterations": float(np.mean([r["iterations"] for r in served]))}


def gate_sweep(w=None, tol=1e-8, M=64, warm=True):
    """Zero-bias conductance against V_GS (Eq. zeroBiasG): per gate voltage one
    self-consistent solve at V_DS = 0 (negf_sc_solve), started from the previous point's
    potential when `warm` (the paper's sweep), then negf_conductance on the converged state.
    Returns the conductances (S), iterations, and the points per second of the whole sweep."""
    w = w or synth.gate_sweep()
    N = w["N"]
    with negf.Context() as ctx:
        dev = ctx.device_create(N, block=1, rings_per_block=1, n_chains=len(w["modes"]))
        ctx.build_cnt_modespace(dev, w["n_tube"], w["t"], list(w["modes"]), 0.0, 0.0)
        ctx.set_grid_spec(dev, w["mu"], w["mu"], w["kT"], w["eta"], w["E_B"], w["n_real"], w["n_cont"])
        kappa = negf.poisson_kappa()
        U0 = np.zeros(N)
        G, iters, conv = [], [], []
        t0 = time.perf_counter()
        for v in w["V_GS"]:
            r = ctx.sc_solve(dev, w["V_DS"], float(v), U0, kappa, M=M, tol=tol, check=False)
            G.append(float(ctx.conductance([dev], w["mu"], w["kT"])[0]))
            iters.append(r["iterations"])
            conv.append(r["converged"])
            if warm:
                U0 = r["U"]
        wall = time.perf_counter() - t0
    lanes = len(w["modes"]) * (w["n_real"] + w["n_cont"])
    # one NEGF evaluation per iteration plus the real-axis lanes of each conductance call
    updates = N * (lanes * sum(iters) + len(w["modes"]) * w["n_real"] * len(G))
    return {"V_GS": [float(v) for v in w["V_GS"]], "G_S": G, "iterations": iters, "converged": conv,
            "points_per_s": len(G) / wall, "seconds": wall,
            "ring_energy_mode_updates_per_s_wall": updates / wall}


def adaptive_grid(budgets=(256, 512, 1024, 2048, 4096, 8192), ref_points=131072, ratios=(500.0, 1600.0, 50.0)):
    """Semi-adaptive real-axis grid (Sec. 3.3) against one Gauss-Legendre rule at equal point
    counts.  Per channel length: the real-axis charge of a 131072-point rule is the reference
    (its own error estimated against half as many points); each budget is met by the plain rule
    and by the semi-adaptive rule with densities in the paper's 500 : 1600 : 50 ratio and limits
    E_s - 3 kT, E_s + kT around the peak E_s of the centre ring's integrand (located by two
    refinements from a guess).  Reports the
    norm-wise relative error of the real-axis charge, and the refinement cost next to one
    evaluation of the same grid."""
    w = synth.adaptive_lengths()
    kT = w["kT"]
    out = {}
    for case in w["cases"]:
        N = case["N"]
        res = {"nm": round(N * 0.1065, 1), "plain": {}, "adaptive": {}}
        with negf.Context() as ctx:
            dev = ctx.device_create(N, block=1, rings_per_block=1, n_chains=1)
            ctx.build_cnt_modespace(dev, w["n_tube"], w["t"], list(w["modes"]), case["U_S"], case["U_D"])
            ctx.set_potential(dev, case["U"])

            def real_part(n_real):
                ctx.set_grid_spec(dev, w["mu_S"], w["mu_D"], kT, w["eta"], w["E_B"], n_real, w["n_cont"])
                return ctx.compute([dev])[0]["n_real"]
            ref = real_part(ref_points)
            res["reference_self_error"] = _rel(real_part(ref_points // 2), ref)
            for nb in budgets:
                res["plain"][nb] = _rel(real_part(nb), ref)
            E_min = min(w["mu_S"], w["mu_D"]) - 14 * kT

            def densities_for(nb, l1, l2):
                # scale the 500 : 1600 : 50 densities so that the grid holds about nb points
                lo, hi = 1e-6, 1e3
                for _ in range(60):
                    s = (lo * hi) ** 0.5
                    g = negf.make_grid_adaptive(w["mu_S"], w["mu_D"], kT, w["eta"], w["E_B"], 0, l1, l2,
                                                tuple(s * r for r in ratios))
                    lo, hi = (s, hi) if g["E"].size < nb else (lo, s)
                return tuple(hi * r for r in ratios)

            # locate the peak: the first limits are a guess, two refinements move them onto it
            l1, l2 = E_min + 0.3, E_min + 0.3 + 4 * kT
            ctx.set_grid_adaptive(dev, w["mu_S"], w["mu_D"], kT, w["eta"], w["E_B"], w["n_cont"], l1, l2,
                                  densities_for(4096, l1, l2))
            ctx.refine_grid(dev)
            t0 = time.perf_counter()
            E_s = ctx.refine_grid(dev)
            res["refine_ms"] = (time.perf_counter() - t0) * 1e3
            t0 = time.perf_counter()
            ctx.compute([dev])
            res["evaluate_ms"] = (time.perf_counter() - t0) * 1e3
            res["refine_points"] = ctx.grid_info(dev)["n_real"]
            res["E_s"] = E_s
            l1, l2 = E_s - 3 * kT, E_s + kT
            for nb in budgets:
                ctx.set_grid_adaptive(dev, w["mu_S"], w["mu_D"], kT, w["eta"], w["E_B"], w["n_cont"], l1, l2,
                                      densities_for(nb, l1, l2))
                nr = ctx.compute([dev])[0]["n_real"]
                res["adaptive"][nb] = {"points": ctx.grid_info(dev)["n_real"], "error": _rel(nr, ref)}
        out["N=%d" % N] = res
    return out


def multichannel(M=40, tol=1e-6):
    """Planar arrays solved with one Broyden vector (negf_sc_solve_multi, Sec. 2.3).
    Five 10 nm tubes at zero bias: iterations and the zero-bias conductance of each tube (the
    outer tubes have one neighbour, the inner ones two).  Twenty 100 nm tubes at V_DS = 0.1 V:
    time per self-consistent iteration of the coupled solve (all tubes in one launch) against
    one tube solved alone, in ring-energy-mode updates per second."""
    out = {}
    kappa = negf.poisson_kappa()
    w = synth.planar_array()
    with negf.Context() as ctx:
        devs = []
        for _ in range(w["n_tubes"]):
            d = ctx.device_create(w["N"], block=1, rings_per_block=1, n_chains=len(w["modes"]))
            ctx.build_cnt_modespace(d, w["n_tube"], w["t"], list(w["modes"]), 0.0, -w["V_DS"])
            ctx.set_grid_spec(d, w["mu_S"], w["mu_D"], w["kT"], w["eta"], w["E_B"], w["n_real"], w["n_cont"])
            devs.append(d)
        t0 = time.perf_counter()
        r = ctx.sc_solve_multi(devs, w["V_DS"], w["V_GS"], w["U0"], kappa * w["K_over_kappa"], M=M, tol=tol,
                               check=False)
        wall = time.perf_counter() - t0
        G = ctx.conductance(devs, w["mu_S"], w["kT"])
        out["five_10nm"] = {"converged": r["converged"], "iterations": r["iterations"], "seconds": wall,
                            "G_S": [float(x) for x in G], "U_mid": [float(u[w["N"] // 2]) for u in r["U"]]}
    w = synth.planar_array(n_tubes=20, N=940, V_DS=0.1, V_GS=0.3)
    lanes = len(w["modes"]) * (w["n_real"] + w["n_cont"])
    with negf.Context() as ctx:
        devs = []
        for _ in range(w["n_tubes"]):
            d = ctx.device_create(w["N"], block=1, rings_per_block=1, n_chains=len(w["modes"]))
            ctx.build_cnt_modespace(d, w["n_tube"], w["t"], list(w["modes"]), 0.0, -w["V_DS"])
            ctx.set_grid_spec(d, w["mu_S"], w["mu_D"], w["kT"], w["eta"], w["E_B"], w["n_real"], w["n_cont"])
            devs.append(d)
        ctx.sc_solve_multi(devs[:2], w["V_DS"], w["V_GS"], w["U0"][:2], kappa * w["K_over_kappa"][:2, :2], M=2,
                           tol=tol, check=False)   # load the kernels
        t0 = time.perf_counter()
        r = ctx.sc_solve_multi(devs, w["V_DS"], w["V_GS"], w["U0"], kappa * w["K_over_kappa"], M=M, tol=tol,
                               check=False)
        wall = time.perf_counter() - t0
        t0 = time.perf_counter()
        one = ctx.sc_solve(devs[0], w["V_DS"], w["V_GS"], w["U0"][0], kappa, M=M, tol=tol, check=False)
        wall1 = time.perf_counter() - t0
        out["twenty_100nm"] = {
            "cta_warps": ctx.chain_width(1),
            "converged": r["converged"], "iterations": r["iterations"], "seconds": wall,
            "ms_per_iteration": wall / r["iterations"] * 1e3,
            "updates_per_s": w["n_tubes"] * w["N"] * lanes * r["iterations"] / wall,
            "one_tube": {"iterations": one["iterations"], "ms_per_iteration": wall1 / one["iterations"] * 1e3,
                         "updates_per_s": w["N"] * lanes * one["iterations"] / wall1}}
    return out


def general_leads(reps=3):
    """General (non-circulant) leads on the 17 x 17 real-space workload (N = 512, 2048 + 128
    energies): one evaluation with seeded non-circulant leads (synth.general_lead), decimated
    per energy when the plan is built, against the same tube with its circulant leads (closed
    form per angular mode).  Wall time per negf_compute (plan, decimation, sweep, second stage)
    and the event-timed sweep alone."""
    w = synth.realspace_17()
    out = {}
    for kind in ("circulant", "general"):
        with negf.Context() as ctx:
            dev = ctx.device_create(w["N"], block=17, rings_per_block=1, n_chains=1)
            ctx.build_cnt_realspace(dev, 17, w["t"], w["U_S"], w["U_D"])
            if kind == "general":
                for side, (seed, U_l) in enumerate(((41, w["U_S"]), (42, w["U_D"]))):
                    ld = synth.general_lead(17, seed)
                    ctx.set_lead_general(dev, 0, side, U_l, ld["T1"], ld["T2"], ld["tau"], list(range(17)),
                                         H0=ld["H0"], H1=ld["H1"])
            ctx.set_potential(dev, w["U"])
            ctx.set_grid_spec(dev, w["mu_S"], w["mu_D"], w["kT"], w["eta"], w["E_B"], w["n_real"], w["n_cont"])
            ctx.compute([dev])   # tuning and kernel loads
            ctx.profile(True)
            ctx.kernel_time()
            t0 = time.perf_counter()
            for _ in range(reps):
                r = ctx.compute([dev])[0]
            wall = (time.perf_counter() - t0) / reps
            ms, k = ctx.kernel_time()
        out[kind] = {"compute_ms": wall * 1e3, "sweep_ms": ms / max(k, 1), "I": r["I"],
                     "updates_per_s": w["N"] * (w["n_real"] + w["n_cont"]) / wall}
    out["decimation_ms_per_plan"] = (out["general"]["compute_ms"] - out["general"]["sweep_ms"]) - \
        (out["circulant"]["compute_ms"] - out["circulant"]["sweep_ms"])
    out["energies_x_leads"] = 2 * (w["n_real"] + w["n_cont"])
    return out


def paper_scaling(reps=2):
    """Context against the paper's timing tables (A100, NERSC Perlmutter; the paper's NEGF puts
    one thread per Green's-function column with a host recursion, Sec. 2.2.4).  Table 1: one
    NEGF evaluation (negf_compute, sweeps + second stage) of a (17,0) tube with one doubly
    degenerate subband, drain ramp 0 -> -0.1 eV, 11,904 Gauss-Legendre real-axis energies plus
    96 contour nodes, N = 512 ... 4096.  Table 2: equilibrium-style evaluation of N = 524,288
    rings on 90 contour nodes with 1, 2, 4, 8 subbands (no real-axis lanes)."""
    w = synth.paper_scaling()
    out = {"table1": [], "table2": []}
    t1 = w["table1"]
    for N, ps, ng in zip(t1["N"], t1["paper_s"], t1["paper_gpus"]):
        with negf.Context() as ctx:
            dev = ctx.device_create(N, block=1, rings_per_block=1, n_chains=len(t1["modes"]))
            ctx.build_cnt_modespace(dev, w["n_tube"], w["t"], list(t1["modes"]), 0.0, -t1["V_DS"])
            ctx.set_potential(dev, synth.ramp_barrier(N, drop=t1["V_DS"], height=0.0))
            ctx.set_grid_spec(dev, 0.0, -t1["V_DS"], w["kT"], w["eta"], -3.0 * abs(w["t"]) - 1.5, t1["n_real"],
                              t1["n_cont"])
            ctx.compute([dev])
            ctx.profile(True)
            ctx.kernel_time()
            t0 = time.perf_counter()
            for _ in range(reps):
                ctx.compute([dev])
            wall = (time.perf_counter() - t0) / reps
            ms, k = ctx.kernel_time()
        out["table1"].append({"N": N, "negf_ms": wall * 1e3, "sweep_ms": ms / max(k, 1),
                              "paper_s": ps, "paper_a100s": ng})
    # Table 2 twice: the sweep split along the channel (the default for these shapes) and the
    # thread-per-lane sweep of whole chains
    t2 = w["table2"]
    N = t2["N"]
    for modes, ps in zip(t2["modes"], t2["paper_s"]):
        row = {"modes": len(modes), "paper_s": ps}
        n_ref = None
        for key, split in (("negf_ms", 0), ("unsplit_ms", -1)):
            with negf.Context(long_chain_split=split) as ctx:
                dev = ctx.device_create(N, block=1, rings_per_block=1, n_chains=len(modes))
                ctx.build_cnt_modespace(dev, w["n_tube"], w["t"], list(modes), 0.0, 0.0)
                ctx.set_potential(dev, np.zeros(N))
                ctx.set_grid_spec(dev, 0.0, 0.0, w["kT"], w["eta"], -3.0 * abs(w["t"]) - 1.0, 0, t2["n_cont"])
                ctx.compute([dev])
                ctx.profile(True)
                ctx.kernel_time()
                t0 = time.perf_counter()
                r = ctx.compute([dev])[0]
                row[key] = (time.perf_counter() - t0) * 1e3
                ms, k = ctx.kernel_time()
                row[key.replace("negf", "sweep").replace("unsplit", "unsplit_sweep")] = ms / max(k, 1)
                if n_ref is None:
                    n_ref = r["n"]
                else:
                    row["max_rel_diff_n"] = float(np.max(np.abs(r["n"] - n_ref)) / np.max(np.abs(n_ref)))
        out["table2"].append(row)
    return out
