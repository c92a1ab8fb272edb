"""The no-allocation entry point (negf_chain1_compute_noalloc) against the context path.

Some callers cannot allocate device memory where they run (while building a CUDA graph,
inside allocator-free hosts); this entry point takes only caller-owned device buffers and
keeps its scratch in a fixed array.  Two calls in a row with different potentials must each
match negf_compute on the same chain, so nothing from the first call leaks into the second.
This file is collected last on purpose."""
import ctypes as C

import numpy as np
import pytest

from tests.cases import rel_inf, current_err

pytestmark = pytest.mark.gpu
TOL = 1e-10


def test_noalloc_matches_context_path_on_two_calls():
    torch = pytest.importorskip("torch")
    from paper_2407_14633_gb300 import negf, synth
    lib = negf.load()
    N, t, j, n_tube = 64, -2.7, 6, 17
    bj = 2 * t * np.cos(np.pi * j / n_tube)
    bond = lambda k: t if k % 2 == 0 else bj
    U_S, U_D = 0.0, -0.1
    grid = negf.make_grid(0.0, -0.1, 0.025, 1e-6, -10.0, 100, 40)
    hsq = np.array([bond(l) ** 2 for l in range(N - 1)])
    lead_S = np.array([bond(-2) ** 2, bond(-3) ** 2, bond(-1) ** 2, U_S])
    lead_D = np.array([bond(N) ** 2, bond(N + 1) ** 2, bond(N - 1) ** 2, U_D])

    dev_t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    d_hd = dev_t(np.zeros(2 * N))
    d_hsq = dev_t(hsq)
    d_E, d_w, d_fS, d_fD = (dev_t(grid[k]) for k in ("E", "w", "fS", "fD"))
    d_z = dev_t(np.asarray(grid["z"]).view(np.float64))
    d_c = dev_t(np.asarray(grid["c"]).view(np.float64))
    n_out = torch.zeros(N, dtype=torch.float64, device="cuda")
    T_out = torch.zeros(100, dtype=torch.float64, device="cuda")
    I_out = torch.zeros(1, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream

    with negf.Context() as ctx:
        dev = ctx.device_create(N)
        ctx.build_cnt_modespace(dev, n_tube, t, [j], U_S, U_D)
        ctx.set_grid(dev, grid["E"], grid["w"], grid["fS"], grid["fD"], grid["eta"], grid["z"], grid["c"])
        for call, U in enumerate([synth.ramp_barrier(N), synth.ramp_barrier(N, drop=0.05, height=0.3)]):
            ctx.set_potential(dev, U)
            ref = ctx.compute([dev])[0]
            d_U = dev_t(U)
            rc = lib.negf_chain1_compute_noalloc(
                C.c_void_p(stream), N, d_hd.data_ptr(), d_U.data_ptr(), d_hsq.data_ptr(), 2.0,
                lead_S.ctypes.data_as(C.POINTER(C.c_double)), lead_D.ctypes.data_as(C.POINTER(C.c_double)),
                100, d_E.data_ptr(), d_w.data_ptr(), d_fS.data_ptr(), d_fD.data_ptr(), grid["eta"],
                40, d_z.data_ptr(), d_c.data_ptr(), n_out.data_ptr(), T_out.data_ptr(), I_out.data_ptr())
            assert rc == negf.OK, (call, rc)
            torch.cuda.synchronize()
            n = n_out.cpu().numpy()
            T = T_out.cpu().numpy()
            I = float(I_out.cpu().numpy()[0])
            assert rel_inf(n, ref["n"]) < TOL, call
            assert rel_inf(T, ref["T"]) < TOL, call
            assert current_err(I, ref["I"], 4.0, 0.1) < TOL, call


def test_noalloc_rejects_oversized_problem():
    torch = pytest.importorskip("torch")
    from paper_2407_14633_gb300 import negf
    lib = negf.load()
    N = 5000   # staging of one block alone exceeds the fixed scratch (5000 x 8 KiB = 40 MiB)
    buf = torch.zeros(4 * N, dtype=torch.float64, device="cuda")
    lead = np.array([1.0, 1.0, 1.0, 0.0])
    p = buf.data_ptr()
    rc = lib.negf_chain1_compute_noalloc(None, N, p, p, p, 2.0, lead.ctypes.data_as(C.POINTER(C.c_double)),
                                         lead.ctypes.data_as(C.POINTER(C.c_double)), 4, p, p, p, p, 1e-6,
                                         0, None, None, p, None, None)
    assert rc == negf.ENOMEM
