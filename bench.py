#!/usr/bin/env python
"""Benchmark of the energy-parallel NEGF hot path on GB300.

Workload: (17,0) nanotube in real space, 17 x 17 complex128 ring blocks, N = 512 rings,
2048 Gauss-Legendre real-axis energies + 128 contour nodes, V_DS = 0.4 V, V_GS = 0.2 V
(seeded synthetic potential: sum of 8 sinusoids, 0.15 eV), self-consistent with Broyden
mixing and the 1D Poisson stand-in.

One step = one self-consistent iteration of the whole hot path: Poisson -> contact
self-energies -> forward/backward recursive Green's function sweeps of every energy ->
Fermi-weighted quadrature to ring charge, T(E) and current -> Broyden update, replayed as
one captured CUDA graph.  Metric: RGF ring-energy updates per second (rings x energies per
step / step time).  Under torchrun each rank solves its own bias point (V_GS shifted per
rank), no collective on the data path: weak scaling.

--impl reference times the FP64 CPU oracle (test infrastructure) on a bounded sample of the
same workload.
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "cnt17_realspace_N512_E2048+128_sc"


# DRAM traffic per launch of the block sweep, from one ncu capture of the N = 64 case with the
# same energy grid (--profile-small), scaled by 512 / 64 layers: the staging traffic grows with
# the layer count at a fixed grid.  It is reported only while the kernel sources hash to the
# ones the capture was taken on.
TRAFFIC_CAPTURE = {"sources_sha256": "f3785c2b45c3f968f2cef147e2f0d3d26ef3405487541ff2219d5ec68520440e",
                   "bytes_per_launch": (1.123410432e9 + 1.256937984e9) * 512 / 64}
KERNEL_SOURCES = ("sweep_block.cu", "sweep_block_item.cuh", "common.cuh", "lead.cuh")


def kernel_sources_sha256():
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2407_14633_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def lane_flops(b, m, nnz, L, real, sym):
    """FLOPs of one lane (one energy, all L layers) of the block sweep as it computes it
    (8 per complex MAC).  Per layer: block inverse b^3; the G_ll update Z G_{l+1} (b^3) then
    (Z G_{l+1})(H_{l+1,l} gL_l) + gL_l, b^3, or for a lane on the complex-symmetric form only
    the upper triangle, b^2 (b + 1) / 2; the sparse coupling products, 4 b^2 nnz (3 on the
    symmetric form, which does not form H_{l+1,l} gL_l); real-axis lanes add the lead-column
    products R, K and G R, 3 b^2 m."""
    upd = b ** 3 + (b * b * (b + 1) // 2 if sym else b ** 3)
    sparse = (3 if sym else 4) * b * b * nnz
    return 8.0 * L * (b ** 3 + upd + sparse + (3 * b * b * m if real else 0))


def algorithmic_flops(b, m, nnz, L, n_real, n_cont, sym=True):
    """FLOPs of one NEGF evaluation with every lane on the given update form."""
    return n_real * lane_flops(b, m, nnz, L, True, sym) + n_cont * lane_flops(b, m, nnz, L, False, sym)


def counted_flops(b, m, nnz, L, lanes):
    """FLOPs of the lanes counted by negf_sweep_lanes (symmetric / general, real / contour)."""
    rs, rg, cs, cg = lanes
    return (rs * lane_flops(b, m, nnz, L, True, True) + rg * lane_flops(b, m, nnz, L, True, False) +
            cs * lane_flops(b, m, nnz, L, False, True) + cg * lane_flops(b, m, nnz, L, False, False))


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return dict(sm_mhz=None, sm_max_mhz=None, reasons=["nvidia-smi unavailable"])
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return dict(sm_mhz=float(np.median(sm)) if sm else None, sm_max_mhz=max(smax) if smax else None,
                    reasons=sorted(reasons), samples=len(sm))


def rank_gate_voltage(rank):
    """Each rank solves its own bias point: V_GS = 0.2 V + 0.05 V per rank (weak scaling,
    no collective on the data path)."""
    return 0.2 + 0.05 * rank


def max_over_ranks(ms, world):
    """The slowest rank's step time (the job's step time); one all-reduce on the host side
    of the timing, never inside the timed region."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([ms], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(units_per_step, world, t_max_ms):
    """Whole-job throughput: the units of every rank over the slowest rank's step time."""
    return world * units_per_step / (t_max_ms * 1e-3)


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def build_workload(ctx, negf, synth, V_GS):
    w = synth.realspace_17()
    dev = ctx.device_create(w["N"], block=17, rings_per_block=1, n_chains=1)
    ctx.build_cnt_realspace(dev, 17, w["t"], w["U_S"], w["U_D"])
    ctx.set_potential(dev, w["U"])
    ctx.set_grid_spec(dev, w["mu_S"], w["mu_D"], w["kT"], w["eta"], w["E_B"], w["n_real"], w["n_cont"])
    return dev, w


def host_cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo), for the baseline's record."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.split(":")[0].strip() == "Model name":
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as fh:
            for ln in fh:
                if ln.lower().startswith(("model name", "cpu model")):
                    return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return None


_ORACLE_WORKER = r"""
import os, sys, time, json
import numpy as np
sys.path.insert(0, %r)
from paper_2407_14633_gb300 import synth
from oracle import model, green, quadrature as q

def build(name):
    # (chains of the oracle device, potential, grid) of a named workload
    if name == "cfg2":
        w = synth.realspace_17()
        dev = model.cnt_build("real", 17, w["t"], w["N"], w["U_S"], w["U_D"])
        g = q.bias_grid(w["mu_S"], w["mu_D"], w["kT"], w["n_real"], w["n_cont"], w["E_B"], w["eta"])
        return dev, w["U"], g
    if name == "cfg1":
        w = synth.modespace_small(6)
        dev = model.cnt_build("mode", w["n_tube"], w["t"], w["N"], w["U_S"], w["U_D"], modes=(6,))
        g = q.bias_grid(w["mu_S"], w["mu_D"], w["kT"], w["n_real"], w["n_cont"], w["E_B"], w["eta"],
                        rule="midpoint", E_min=-1.0, E_max=1.0)
        return dev, w["U"], g
    if name.startswith("cfg3_"):
        w = synth.batched_uneven()
        d = w["devices"][int(name[5:])]
        dev = model.cnt_build("mode", w["n_tube"], w["t"], d["N"], 0.0, -d["V_DS"], modes=tuple(d["modes"]),
                              cells=d["block"] == 2)
        g = q.bias_grid(0.0, -d["V_DS"], w["kT"], d["n_real"], d["n_cont"], d["E_B"], w["eta"])
        return dev, d["U"], g
    if name == "cfg4":
        w = synth.mixed_precision(n_tube=17, N=1024, n_energies=4096)
        dev = model.cnt_build("real", 17, w["t"], w["N"], w["U_S"], w["U_D"])
        E = w["E"]
        E_B = float(np.min(w["U"]) - 3.0 * abs(w["t"]) - 1.0)
        z, c = q.contour_semicircle(E_B, -1.0, 64)
        g = dict(E=E, w=np.full(E.size, 2.0 / E.size), fS=q.fermi(E - w["mu_S"], w["kT"]),
                 fD=q.fermi(E - w["mu_D"], w["kT"]), eta=w["eta"], z=z, c=c)
        return dev, w["U"], g
    if name == "cfg5":
        w = synth.serving_sweep()
        r = w["requests"][0]
        dev = model.cnt_build("mode", w["n_tube"], w["t"], r["N"], 0.0, -r["V_DS"], modes=tuple(r["modes"]))
        E_B = -r["V_DS"] - 3.0 * abs(w["t"]) - 1.0
        g = q.bias_grid(0.0, -r["V_DS"], w["kT"], r["n_real"], r["n_cont"], E_B, w["eta"])
        return dev, np.linspace(0.0, -r["V_DS"], r["N"]), g
    raise ValueError(name)

cases = {}
print("ready", flush=True)
for line in sys.stdin:
    job = json.loads(line)
    if job["case"] not in cases:
        cases[job["case"]] = build(job["case"])
    dev, U, g = cases[job["case"]]
    k_lo, k_hi, c_lo, c_hi, chunk = job["k_lo"], job["k_hi"], job["c_lo"], job["c_hi"], job["chunk"]
    k_hi, c_hi = min(k_hi, g["E"].size), min(c_hi, g["z"].size)
    while time.time() < job["t_start"]:
        time.sleep(0.0005)
    t0 = time.time()
    for _ in range(job.get("reps", 1)):
        for ch in dev.chains:
            for k0 in range(k_lo, k_hi, chunk):
                green.rgf_lanes(ch, U, g["E"][k0:min(k0 + chunk, k_hi)] + 1j * g["eta"])
            for k0 in range(c_lo, c_hi, chunk):
                green.rgf_lanes(ch, U, g["z"][k0:min(k0 + chunk, c_hi)], spectral=False)
    units = job.get("reps", 1) * dev.n_rings * len(dev.chains) * (max(k_hi - k_lo, 0) + max(c_hi - c_lo, 0))
    print(json.dumps(dict(start=t0, end=time.time(), updates=units)), flush=True)
"""


class OraclePool:
    """`cores` single-threaded processes (one BLAS thread each, so each runs the oracle's own
    arithmetic), each holding the N = 512 workload's chain and grid.  sample() splits a bounded
    set of energies into contiguous slices; the processes start their slices together (a
    shared wall-clock start) and the rate is every update over the span from that start to
    the last process's end."""

    def __init__(self, cores):
        self.cores = max(1, cores)
        env = dict(os.environ, OPENBLAS_NUM_THREADS="1", OMP_NUM_THREADS="1", MKL_NUM_THREADS="1")
        self.procs = [subprocess.Popen([sys.executable, "-c", _ORACLE_WORKER % ROOT], stdin=subprocess.PIPE,
                                       stdout=subprocess.PIPE, text=True, env=env)
                      for _ in range(self.cores)]
        for p in self.procs:
            if p.stdout.readline().strip() != "ready":
                self.close()
                raise RuntimeError("oracle worker failed to start")

    def sample(self, n_real, n_cont, chunk=16, case="cfg2", k0=0, c0=0, reps=1):
        """Returns (seconds, ring-energy(-mode) updates) of n_real real-axis energies from index
        k0 and n_cont contour nodes from c0 of a named workload (default: the bench workload),
        each process repeating its slice reps times."""
        c = self.cores
        t_start = time.time() + 0.2
        for i, p in enumerate(self.procs):
            job = dict(case=case, k_lo=k0 + n_real * i // c, k_hi=k0 + n_real * (i + 1) // c,
                       c_lo=c0 + n_cont * i // c, c_hi=c0 + n_cont * (i + 1) // c, chunk=chunk, t_start=t_start,
                       reps=reps)
            p.stdin.write(json.dumps(job) + "\n")
            p.stdin.flush()
        res = [json.loads(p.stdout.readline()) for p in self.procs]
        if min(r["start"] for r in res) < t_start - 1e-3:
            raise RuntimeError("oracle workers did not start together")
        return max(r["end"] for r in res) - t_start, sum(r["updates"] for r in res)

    def close(self):
        for p in self.procs:
            try:
                p.stdin.close()
                p.wait(timeout=30)
            except (OSError, subprocess.SubprocessError):
                p.kill()


def mixed_against_stored_oracle():
    """The mixed path with its defaults on the grid stored in tests/golden/mixed_cnt17_N1024.json
    (the (17,0) N = 1024 workload's energies, its weights and Fermi factors, the stored contour
    nodes) against the FP64 oracle's outputs stored there: norm-wise relative errors of n and T,
    relative error of I.  The stored values were written by the oracle alone."""
    path = os.path.join(ROOT, "tests", "golden", "mixed_cnt17_N1024.json")
    if not os.path.exists(path):
        return None
    from paper_2407_14633_gb300 import negf, synth, workloads
    with open(path) as fh:
        gd = json.load(fh)
    w = synth.mixed_precision(n_tube=gd["n_tube"], N=gd["N"], n_energies=gd["n_energies"])
    E = np.asarray(w["E"], dtype=np.float64)
    z = np.array([complex(*x) for x in gd["z"]])
    c = np.array([complex(*x) for x in gd["c"]])
    with negf.Context(precision=negf.PREC_MIXED) as ctx:
        dev = ctx.device_create(gd["N"], block=gd["n_tube"], rings_per_block=1, n_chains=1)
        ctx.build_cnt_realspace(dev, gd["n_tube"], gd["t"], gd["U_S"], gd["U_D"])
        ctx.set_potential(dev, w["U"])
        ctx.set_grid(dev, E, np.full(E.size, 2.0 / E.size), workloads._fermi(E - gd["mu_S"], gd["kT"]),
                     workloads._fermi(E - gd["mu_D"], gd["kT"]), gd["eta"], z, c)
        r = ctx.compute([dev])[0]
    n_ref = np.array([float(x) for x in gd["n"]])
    T_ref = np.array([float(x) for x in gd["T"]])
    I_ref = float(gd["I"])
    return {"n": float(np.max(np.abs(r["n"] - n_ref)) / np.max(np.abs(n_ref))),
            "T": float(np.max(np.abs(r["T"] - T_ref)) / np.max(np.abs(T_ref))),
            "I": abs(r["I"] - I_ref) / abs(I_ref),
            "reference": "FP64 oracle values stored in tests/golden/mixed_cnt17_N1024.json, same grid"}


def cpu_baseline_record(n_real=256, n_cont=16):
    """cpu_baseline: the oracle on every host core, with the one-core figure beside it (the
    same sample, one process)."""
    cores = os.cpu_count() or 1
    out = {}
    for k in (cores, 1):
        pool = OraclePool(k)
        try:
            pool.sample(k, 0)   # warm-up: one energy per process
            out[k] = pool.sample(n_real, n_cont)
        finally:
            pool.close()
    secs, upd = out[cores]
    secs1, upd1 = out[1]
    return {"value": upd / secs, "unit": "ring-energy updates/s", "cores": cores, "kind": "oracle",
            "sample": "%d real-axis + %d contour energies of the N=512 workload, split over %d single-threaded "
                      "processes" % (n_real, n_cont, cores),
            "host_cpu": host_cpu_model(), "one_core": {"value": upd1 / secs1, "cores": 1}}


def cpu_configs():
    """The oracle on every host core, on bounded samples of each workload (ring-energy(-mode)
    updates per second): the small mode-space case in full, one device of the uneven batch per
    block form, and energy samples of the bench, mixed-precision and serving workloads.  A sample
    of a few energies stands for the whole grid; the oracle's cost per update does not depend on
    which energies it takes."""
    cores = os.cpu_count() or 1
    pool = OraclePool(cores)
    out = {"cores": cores, "host_cpu": host_cpu_model()}
    try:
        plan = [("cfg1", "small mode space N=64, j=6: all 256 + 64 energies, 100 times", 256, 64, 0, 0, 100),
                ("cfg2", "real space 17x17 N=512: 256 + 16 energies", 256, 16, 0, 0, 1),
                ("cfg3_0", "uneven batch, device 0: 48 + 4 energies per core", 48 * cores, 4 * cores, 0, 0, 1),
                ("cfg3_1", "uneven batch, device 1: 48 + 4 energies per core", 48 * cores, 4 * cores, 0, 0, 1),
                ("cfg4", "(17,0) N=1024, band-edge grid: 8 energies per core", 8 * cores, 0, 1000, 0, 1),
                ("cfg5", "serving request 0 (2 modes): 96 + 4 energies per core", 96 * cores, 4 * cores, 0, 0, 1)]
        for case, what, nr, nc, k0, c0, reps in plan:
            pool.sample(min(nr, cores), 0, case=case, k0=k0)   # warm-up, builds the case
            secs, upd = pool.sample(nr, nc, case=case, k0=k0, c0=c0, reps=reps)
            out[case] = {"updates_per_s": upd / secs, "sample": what, "seconds": secs}
    finally:
        pool.close()
    return out


def run_reference(args):
    world, rank, _ = dist_setup()
    if rank != 0:
        return 0
    # each step: 32 real-axis + 4 contour energies per host core, at full N = 512
    cores = os.cpu_count() or 1
    per_step = (32 * cores, 4 * cores)
    pool = OraclePool(cores)
    try:
        for _ in range(args.warmup):
            pool.sample(*per_step)
        secs, upd = 0.0, 0
        for _ in range(args.steps):
            s, u = pool.sample(*per_step)
            secs += s
            upd += u
    finally:
        pool.close()
    value = upd / secs
    sample = "%d real-axis + %d contour energies of the N=512 workload per step, split over %d single-threaded " \
             "processes" % (per_step[0], per_step[1], cores)
    line = {
        "impl": "reference", "metric": "RGF ring-energy updates/s", "value": value,
        "unit": "ring-energy updates/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * secs / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample_per_step": sample},
        "cpu_baseline": {"value": value, "unit": "ring-energy updates/s", "cores": cores, "kind": "oracle",
                         "sample": sample, "host_cpu": host_cpu_model()},
        "e2e": {"value": value, "unit": "ring-energy updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def run_ours(args):
    import torch
    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2407_14633_gb300 import negf, synth
    # a real (non-default) stream: the library launches on it and the events below are
    # recorded on it, so they bracket exactly the library's work
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    ctx = negf.Context(device=local, stream=stream.cuda_stream)
    V_GS = rank_gate_voltage(rank)
    dev, w = build_workload(ctx, negf, synth, V_GS)
    N, n_real, n_cont = w["N"], w["n_real"], w["n_cont"]
    units_per_step = N * (n_real + n_cont)
    kappa = negf.poisson_kappa()

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    # ---- timed: K self-consistent iterations (graph replays); L2 flushed between steps
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    e2e_reps = max(2, min(args.steps, 5))
    M = min(256, args.warmup + args.steps + e2e_reps + 4)
    ctx.sc_begin(dev, w["V_DS"], V_GS, w["U"], kappa, M=M, tol=1e-300)
    ctx.sc_step(dev, args.warmup, wait=True)
    barrier()
    clk = Clocks(local)
    clk.start()
    l0 = ctx.launch_count()
    evs = []
    for _ in range(args.steps):
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.sc_step(dev, 1, wait=False)
        e1.record(stream)
        evs.append((e0, e1))
    barrier()
    launches = ctx.launch_count() - l0
    clocks = clk.stop()
    ms = sum(a.elapsed_time(b) for a, b in evs) / args.steps

    # ---- end to end through the public API with host buffers: each step uploads the Broyden
    #      state from pinned host memory (negf_sc_set_state), runs one self-consistent
    #      iteration (the timed step's work) and reads the new state back (negf_sc_get_state)
    st = ctx.sc_get_state(dev)
    pinned = {k: torch.empty(st[k].size, dtype=torch.float64, pin_memory=True).numpy()
              for k in ("n_in", "n_in_old", "f_old", "V", "W")}
    for k in pinned:
        pinned[k][:] = st[k].reshape(-1)
    host_state = dict(pinned, m=st["m"])
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_reps):
        flush.fill_(1.0)
        ctx.sc_set_state(dev, host_state)
        ctx.sc_step(dev, 1, wait=True)
        st = ctx.sc_get_state(dev)
        for k in pinned:
            pinned[k][:] = st[k].reshape(-1)
        host_state["m"] = st["m"]
    t_e2e = (time.perf_counter() - t0) / e2e_reps
    state_bytes = 8 * sum(v.size for v in pinned.values()) + 4
    ctx.sc_end(dev)
    t_max = max_over_ranks(ms, world)
    value = job_value(units_per_step, world, t_max)

    # ---- dominant kernel: the block sweep, timed with events on the launching stream
    ctx.profile(True)
    n_t = torch.empty(N, dtype=torch.float64, device="cuda")
    T_t = torch.empty(n_real, dtype=torch.float64, device="cuda")
    I_t = torch.empty(1, dtype=torch.float64, device="cuda")
    outs = [dict(n=n_t.data_ptr(), T=T_t.data_ptr(), I=I_t.data_ptr())]
    ctx.kernel_time()
    ctx.sweep_lanes()
    reps = 3
    for _ in range(reps):
        ctx.compute_device([dev], outs)
    torch.cuda.synchronize()
    sweep_ms, sweeps = ctx.kernel_time()
    lanes = ctx.sweep_lanes()
    ctx.profile(False)
    sweep_ms /= max(sweeps, 1)
    flops = counted_flops(17, 17, 1.5, N, lanes) / max(sweeps, 1)
    achieved = flops / (sweep_ms * 1e-3) / 1e12
    props = torch.cuda.get_device_properties(local)
    sm_max = clocks.get("sm_max_mhz") or 2070.0
    peak_derived = 2.0 * 2.0 * props.multi_processor_count * sm_max * 1e6 / 1e12   # 2 FP64 FMA/clk/SM
    peak_probe = ctx.fp64_peak()
    traffic = (TRAFFIC_CAPTURE["bytes_per_launch"]
               if kernel_sources_sha256() == TRAFFIC_CAPTURE["sources_sha256"] else None)

    # ---- one NEGF evaluation through the public API with host buffers (no Poisson, no Broyden)
    U_host = np.ascontiguousarray(w["U"])
    ctx.set_potential(dev, U_host)
    ctx.compute([dev])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_reps):
        ctx.set_potential(dev, U_host)
        r = ctx.compute([dev])[0]
    t_eval = (time.perf_counter() - t0) / e2e_reps

    # ---- full bias-point solve to tolerance (the second metric)
    sc = None
    if not args.no_solve:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = ctx.sc_solve(dev, w["V_DS"], V_GS, w["U"], kappa, zeta=w["zeta"], M=w["M"], tol=w["tol"], check=False)
        t_solve = time.perf_counter() - t0
        sc = {"bias_point_solves_per_s": 1.0 / t_solve, "seconds": t_solve, "iterations": res["iterations"],
              "converged": res["converged"], "final_residual": float(res["history"][-1]) if res["iterations"] else None,
              "current_A": res["I"]}

    line = {
        "metric": "RGF ring-energy updates/s", "value": value, "unit": "ring-energy updates/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "n_rings": N, "block": 17, "energies_real": n_real,
                   "energies_contour": n_cont, "step": "one self-consistent iteration (captured graph)",
                   "l2": "flushed between steps (256 MB write)", "parallelism": "replicas per rank (weak)",
                   "launch_shape": ctx.blk_shape(17, 17)},
        "e2e": {"value": units_per_step / t_e2e, "unit": "ring-energy updates/s",
                "h2d_bytes_per_step": state_bytes, "d2h_bytes_per_step": state_bytes,
                "call": "negf_sc_set_state + negf_sc_step + negf_sc_get_state, pinned host buffers "
                        "(the timed step's work plus the copies of its Broyden state)"},
        "evaluation_e2e": {"value": units_per_step / t_eval, "unit": "ring-energy updates/s",
                           "h2d_bytes_per_step": U_host.nbytes, "d2h_bytes_per_step": 8 * (3 * N + n_real + 1),
                           "call": "negf_set_potential + negf_compute, host buffers: one NEGF evaluation "
                                   "(no Poisson or Broyden)"},
        "gpu_launches": int(launches),
        "roofline": {"kernel": "sweep_blk_kernel", "bound": "alu", "achieved": achieved,
                     "peak": peak_derived, "unit": "TFLOP/s", "frac": achieved / peak_derived,
                     "peak_kind": "FP64 derived: 2 FMA/clk/SM x SMs x max SM clock",
                     "peak_probe": peak_probe, "frac_of_probe": achieved / peak_probe,
                     "traffic": traffic,
                     "traffic_note": "dram bytes of the N = 64 capture with the same grid, scaled by 512 / 64 layers",
                     "kernel_ms": sweep_ms, "flops_per_launch": flops,
                     "lanes_per_launch": {"real_symmetric": lanes[0] // max(sweeps, 1),
                                          "real_general": lanes[1] // max(sweeps, 1),
                                          "contour_symmetric": lanes[2] // max(sweeps, 1),
                                          "contour_general": lanes[3] // max(sweeps, 1)}},
        "clocks": clocks,
        "self_consistent_solve": sc,
    }
    from paper_2407_14633_gb300 import workloads
    if rank == 0 and world == 1 and not args.no_workloads:
        # the mixed-precision and serving workloads at reduced size beside the headline
        mp = workloads.mixed_precision(tubes=(17,), variants=((0.002, 0.0, 1e-3),))["(17,0)"]
        d = mp["mixed_w0.002_g0_r0.001"]
        line["mixed"] = {"workload": "cnt17_realspace_N1024_E4096_bandedge", "c128_sweep_ms": mp["c128_sweep_ms"],
                         "mixed_sweep_ms": d["sweep_ms"], "speedup_vs_c128": d["speedup_vs_c128"],
                         "recomputed_fraction": d["recomputed_fraction"],
                         "rel_err_vs_c128": {"n": d["rel_err_n"], "T": d["rel_err_T"], "I": d["rel_err_I"]},
                         "c64_only": {"speedup_vs_c128": mp["c64"]["speedup_vs_c128"],
                                      "rel_err_vs_c128": {"n": mp["c64"]["rel_err_n"], "T": mp["c64"]["rel_err_T"],
                                                          "I": mp["c64"]["rel_err_I"]}},
                         "options": "flag_threshold 1e-3 (the default), edge_window 2 meV, growth criterion off"}
        mo = mixed_against_stored_oracle()
        if mo is not None:
            line["mixed"]["rel_err_vs_oracle"] = mo
        sv = workloads.serving_sweep(n_requests=args.serving_requests)
        line["serving"] = {"workload": "iv_sweep_first%d_of_256_requests" % args.serving_requests,
                           "requests": sv["requests"], "converged": sv["converged_requests"], "tol": sv["tol"],
                           "bias_points_per_s": {"sequential": sv["sequential_bias_points_per_s"],
                                                 "served": sv["served_bias_points_per_s"],
                                                 "saturated": sv["saturated_bias_points_per_s"]},
                           "converged_bias_points_per_s": sv["converged_bias_points_per_s"],
                           "served_p50_s": sv["served_p50_s"], "served_p99_s": sv["served_p99_s"],
                           "sequential_queued_p50_s": sv["sequential_queued_p50_s"],
                           "sequential_queued_p99_s": sv["sequential_queued_p99_s"],
                           "arrival_rate_per_s": sv["arrival_rate_per_s"],
                           "bitwise_same_as_sequential": sv["bitwise_same_as_sequential"]}
    if args.extras and rank == 0:
        runs = {"modespace_small": workloads.modespace_small, "batched_uneven": workloads.batched_uneven,
                "mixed_precision": workloads.mixed_precision, "serving": workloads.serving_sweep,
                "gate_sweep": lambda: {"warm": workloads.gate_sweep(), "cold": workloads.gate_sweep(warm=False)},
                "adaptive_grid": workloads.adaptive_grid, "multichannel": workloads.multichannel,
                "general_leads": workloads.general_leads, "paper_scaling": workloads.paper_scaling,
                "cpu_configs": cpu_configs}
        pick = [k for k in runs if k != "cpu_configs"] if args.extras == "all" else args.extras.split(",")
        line["extras"] = {k: runs[k]() for k in pick}
    if rank == 0 and world == 1 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline_record()
    ctx.close()
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_profile_small(args):
    """Reduced cases for ncu captures (three NEGF evaluations, no SC loop, no CPU leg).

    rs17 (default): (17,0) real space, N = 64 rings and the full grid (2048 real-axis + 128
    contour energies, so the same lanes and waves as the bench workload at 1/8 of its length),
    complex128.  rs17_c64: the same with the complex64 sweep.  mode: eight (17,0) mode-space
    devices, modes 6 and 5, N = 1000, 4032 + 64 energies each (the thread-per-lane 1 x 1 sweep
    of the batched and serving workloads), complex128.  long: the paper's Table 2 shape at a
    quarter of its length, one (17,0) mode-space device of N = 131,072 rings, modes 6 and 5,
    90 contour nodes and no real-axis lanes (the sweep split along the channel), complex128."""
    import torch
    from paper_2407_14633_gb300 import negf, synth
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    prec = negf.PREC_FP32 if args.profile_case == "rs17_c64" else negf.PREC_FP64
    ctx = negf.Context(device=0, stream=stream.cuda_stream, blk_warps=args.blk_warps,
                       blk_ctas_per_sm=args.blk_ctas, precision=prec)
    n_dev = 1
    if args.profile_case == "long":
        ps = synth.paper_scaling()
        N, n_cont = 131072, ps["table2"]["n_cont"]
        w = dict(N=N, n_real=0, n_cont=n_cont, t=ps["t"], U=np.zeros(N), U_S=0.0, U_D=0.0, mu_S=0.0, mu_D=0.0,
                 kT=ps["kT"], eta=ps["eta"], E_B=-3.0 * abs(ps["t"]) - 1.0)
        devs = [ctx.device_create(N, block=1, rings_per_block=1, n_chains=2)]
        ctx.build_cnt_modespace(devs[0], ps["n_tube"], w["t"], [6, 5], 0.0, 0.0)
        flops = None
    elif args.profile_case == "mode":
        N, n_real, n_cont, n_dev = 1000, 4032, 64, 8
        w = synth.realspace_17(N=N, n_real=n_real, n_cont=n_cont)
        devs = [ctx.device_create(N, block=1, rings_per_block=1, n_chains=2) for _ in range(n_dev)]
        for dev in devs:
            ctx.build_cnt_modespace(dev, 17, w["t"], [6, 5], w["U_S"], w["U_D"])
        flops = None
    else:
        w = synth.realspace_17(N=64)
        devs = [ctx.device_create(w["N"], block=17, rings_per_block=1, n_chains=1)]
        ctx.build_cnt_realspace(devs[0], 17, w["t"], w["U_S"], w["U_D"])
        flops = algorithmic_flops(17, 17, 1.5, w["N"], w["n_real"], w["n_cont"])
    for dev in devs:
        ctx.set_potential(dev, w["U"])
        ctx.set_grid_spec(dev, w["mu_S"], w["mu_D"], w["kT"], w["eta"], w["E_B"], w["n_real"], w["n_cont"])
    ctx.profile(True)
    for _ in range(3):
        r = ctx.compute(devs)[0]
    ms, k = ctx.kernel_time()
    lanes = ctx.sweep_lanes()
    if flops:
        flops = counted_flops(17, 17, 1.5, w["N"], lanes) / max(k, 1)
    line = {"case": "profile_small", "profile_case": args.profile_case, "sweep_ms": ms / k, "I": r["I"],
            "cta_warps": args.blk_warps, "ctas_per_sm": args.blk_ctas, "lanes": lanes}
    if flops:
        line["tflops"] = flops / (ms / k * 1e-3) / 1e12
    else:
        updates = n_dev * w["N"] * 2 * (w["n_real"] + w["n_cont"])   # two modes per device
        line["ring_energy_mode_updates_per_s"] = updates / (ms / k * 1e-3)
    print(json.dumps(line))
    ctx.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-solve", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-workloads", action="store_true",
                    help="skip the reduced mixed-precision and serving workloads of the default line")
    ap.add_argument("--serving-requests", type=int, default=48,
                    help="requests of the seeded serving stream in the default line (its first ones)")
    ap.add_argument("--extras", nargs="?", const="all", default=None,
                    help="also run the small, batched-uneven, mixed-precision, serving and gate-sweep workloads "
                         "(or a comma list of modespace_small, batched_uneven, mixed_precision, serving, "
                         "gate_sweep, adaptive_grid, multichannel, general_leads, paper_scaling, cpu_configs; "
                         "cpu_configs times the oracle on every host core on samples of each workload)")
    ap.add_argument("--profile-small", action="store_true",
                    help="reduced case of the block sweep for ncu captures")
    ap.add_argument("--blk-warps", type=int, default=1,
                    help="CTA width of the block sweep in --profile-small (no tuning launches)")
    ap.add_argument("--profile-case", default="rs17", choices=["rs17", "rs17_c64", "mode", "long"],
                    help="which reduced case --profile-small runs")
    ap.add_argument("--blk-ctas", type=int, default=0,
                    help="cap on resident CTAs per SM of the block sweep in --profile-small (0: no cap)")
    args = ap.parse_args()
    if args.profile_small:
        return run_profile_small(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
