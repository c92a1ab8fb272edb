"""ctypes binding of libnegf.so (include/negf.h): argument marshalling only.

Every call goes straight to the C ABI; arrays are numpy float64 / int32 host arrays, or
device pointers (ints, e.g. ``torch.Tensor.data_ptr()``) where the C call takes device
memory.  There is no fallback: ``load()`` raises if the library is missing.
"""
import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libnegf.so")

OK, EINVAL, ENOMEM, ECUDA, ETIMEDOUT, ENOTCONVERGED, EBUSY, ENOTFOUND = 0, -1, -2, -3, -4, -5, -6, -7
PREC_FP64, PREC_MIXED, PREC_FP32 = 0, 1, 2
SOURCE, DRAIN = 0, 1
RULE_GAUSS, RULE_MIDPOINT = 0, 1

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)


class Opts(C.Structure):
    _fields_ = [("device_ordinal", C.c_int), ("stream", C.c_void_p), ("hbm_budget_bytes", C.c_size_t),
                ("precision", C.c_int), ("flag_threshold", C.c_double), ("edge_window", C.c_double),
                ("fault_alloc_after", C.c_int), ("growth_threshold", C.c_double), ("blk_warps", C.c_int),
                ("blk_ctas_per_sm", C.c_int), ("general_update", C.c_int), ("chain_warps", C.c_int),
                ("long_chain_split", C.c_int), ("mixed_two_pass", C.c_int)]


class Lead(C.Structure):
    _fields_ = [("m", C.c_int), ("U_lead", C.c_double), ("T1", _dp), ("T2", _dp), ("tau", _dp),
                ("sites", _ip)]


class LeadGeneral(C.Structure):
    _fields_ = [("m", C.c_int), ("U_lead", C.c_double), ("H0", _dp), ("H1", _dp), ("T1", _dp), ("T2", _dp),
                ("tau", _dp), ("sites", _ip), ("max_iter", C.c_int), ("tol", C.c_double)]


class Grid(C.Structure):
    _fields_ = [("n_real", C.c_int), ("E", _dp), ("w", _dp), ("fS", _dp), ("fD", _dp), ("eta", C.c_double),
                ("n_cont", C.c_int), ("z", _dp), ("c", _dp)]


class GridSpec(C.Structure):
    _fields_ = [("mu_S", C.c_double), ("mu_D", C.c_double), ("kT", C.c_double), ("eta", C.c_double),
                ("E_B", C.c_double), ("E_min", C.c_double), ("E_max", C.c_double), ("f1", C.c_double),
                ("f2", C.c_double), ("n_real", C.c_int), ("n_cont", C.c_int), ("rule", C.c_int)]


class Adaptive(C.Structure):
    _fields_ = [("E_l1", C.c_double), ("E_l2", C.c_double), ("density", C.c_double * 3), ("a", C.c_double),
                ("b", C.c_double), ("period", C.c_int), ("ring", C.c_int)]


class Out(C.Structure):
    _fields_ = [("n", C.c_void_p), ("T", C.c_void_p), ("I", C.c_void_p), ("n_cont", C.c_void_p),
                ("n_real_part", C.c_void_p), ("flags", C.c_void_p), ("resid", C.c_void_p),
                ("growth", C.c_void_p), ("on_device", C.c_int)]


class Poisson(C.Structure):
    _fields_ = [("kappa", C.c_double), ("dx_nm", C.c_double), ("lam_nm", C.c_double), ("phi_gate", C.c_double)]


class Bias(C.Structure):
    _fields_ = [("V_DS", C.c_double), ("V_GS", C.c_double)]


class Broyden(C.Structure):
    _fields_ = [("zeta", C.c_double), ("M", C.c_int), ("tol", C.c_double)]


class Request(C.Structure):
    _fields_ = [("n_rings", C.c_int), ("n_tube", C.c_int), ("n_modes", C.c_int), ("modes", _ip),
                ("t", C.c_double), ("kT", C.c_double), ("eta", C.c_double), ("E_B", C.c_double),
                ("n_real", C.c_int), ("n_cont", C.c_int), ("bias", Bias), ("pois", Poisson),
                ("broyden", Broyden), ("U0", _dp)]


class ScResult(C.Structure):
    _fields_ = [("n", _dp), ("U", _dp), ("T", _dp), ("history", _dp), ("I", C.c_double),
                ("converged", C.c_int), ("iterations", C.c_int)]


_lib = None

# name -> (restype, argtypes)
_PROTOS = {
    "negf_create": (C.c_int, [C.POINTER(C.c_void_p), C.POINTER(Opts)]),
    "negf_destroy": (C.c_int, [C.c_void_p]),
    "negf_strerror": (C.c_char_p, [C.c_int]),
    "negf_last_error": (C.c_char_p, [C.c_void_p]),
    "negf_device_create": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, _ip]),
    "negf_device_destroy": (C.c_int, [C.c_void_p, C.c_int]),
    "negf_set_hamiltonian": (C.c_int, [C.c_void_p, C.c_int, C.c_int, _dp, _dp, C.c_double]),
    "negf_set_lead": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.POINTER(Lead)]),
    "negf_set_lead_potentials": (C.c_int, [C.c_void_p, C.c_int, C.c_double, C.c_double]),
    "negf_set_lead_general": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.POINTER(LeadGeneral)]),
    "negf_build_cnt_modespace": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_double, _ip, C.c_double, C.c_double]),
    "negf_build_cnt_realspace": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_double, C.c_double, C.c_double]),
    "negf_set_potential": (C.c_int, [C.c_void_p, C.c_int, _dp]),
    "negf_set_grid": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(Grid)]),
    "negf_make_grid": (C.c_int, [C.POINTER(GridSpec), _dp, _dp, _dp, _dp, _dp, _dp]),
    "negf_set_grid_spec": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(GridSpec)]),
    "negf_compute": (C.c_int, [C.c_void_p, _ip, C.c_int, C.POINTER(Out)]),
    "negf_sample_lanes": (C.c_int, [C.c_void_p, C.c_int, C.c_int, _ip, _dp, _dp, C.c_int, _ip, _dp]),
    "negf_neutral_charge": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_double, _dp]),
    "negf_conductance": (C.c_int, [C.c_void_p, _ip, C.c_int, C.c_double, C.c_double, _dp, _dp]),
    "negf_make_grid_adaptive": (C.c_int, [C.POINTER(GridSpec), C.POINTER(Adaptive), _ip, _dp, _dp, _dp, _dp, _dp,
                                          _dp]),
    "negf_set_grid_adaptive": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(GridSpec), C.POINTER(Adaptive)]),
    "negf_ring_integrand": (C.c_int, [C.c_void_p, C.c_int, C.c_int, _dp]),
    "negf_refine_grid": (C.c_int, [C.c_void_p, C.c_int, _dp]),
    "negf_grid_info": (C.c_int, [C.c_void_p, C.c_int, _ip, _ip, _dp, _dp]),
    "negf_poisson_kappa": (C.c_double, [C.c_double, C.c_double, C.c_double, C.c_double]),
    "negf_sc_solve": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(Bias), C.POINTER(Poisson), C.POINTER(Broyden),
                                _dp, C.POINTER(ScResult)]),
    "negf_launch_count": (C.c_int, [C.c_void_p, C.POINTER(C.c_uint64)]),
    "negf_sc_solve_multi": (C.c_int, [C.c_void_p, _ip, C.c_int, C.POINTER(Bias), C.POINTER(Poisson), _dp,
                                      C.POINTER(Broyden), _dp, C.c_void_p]),
    "negf_sc_begin": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(Bias), C.POINTER(Poisson), C.POINTER(Broyden), _dp]),
    "negf_sc_step": (C.c_int, [C.c_void_p, C.c_int, C.c_int, _ip]),
    "negf_sc_end": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(ScResult)]),
    "negf_sc_get_state": (C.c_int, [C.c_void_p, C.c_int, _dp, _dp, _dp, _dp, _dp, _ip]),
    "negf_sc_set_state": (C.c_int, [C.c_void_p, C.c_int, _dp, _dp, _dp, _dp, _dp, C.c_int]),
    "negf_profile": (C.c_int, [C.c_void_p, C.c_int]),
    "negf_kernel_time": (C.c_int, [C.c_void_p, _dp, C.POINTER(C.c_uint64)]),
    "negf_fp64_peak": (C.c_int, [C.c_void_p, _dp]),
    "negf_sweep_lanes": (C.c_int, [C.c_void_p, C.POINTER(C.c_uint64)]),
    "negf_blk_width": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, _ip, _ip]),
    "negf_chain_width": (C.c_int, [C.c_void_p, C.c_int, C.c_int, _ip]),
    "negf_plan_seg_waves": (C.c_int, [C.c_int, C.POINTER(C.c_longlong), _ip, C.c_longlong, _ip,
                                      C.POINTER(C.c_longlong), C.POINTER(C.c_longlong)]),
    "negf_submit": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(C.c_uint64)]),
    "negf_serve_step": (C.c_int, [C.c_void_p, _ip]),
    "negf_poll": (C.c_int, [C.c_void_p, C.c_uint64, C.POINTER(ScResult)]),
    "negf_wait": (C.c_int, [C.c_void_p, C.c_uint64, C.c_int, C.POINTER(ScResult)]),
    "negf_cancel": (C.c_int, [C.c_void_p, C.c_uint64]),
    "negf_request_times": (C.c_int, [C.c_void_p, C.c_uint64, _dp, _dp, _dp]),
    "negf_chain1_compute_noalloc": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_double,
                                              _dp, _dp, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                              C.c_double, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                                              C.c_void_p, C.c_void_p]),
}


def load(path=LIB_PATH):
    """Load libnegf.so and declare its prototypes.  Raises OSError if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise OSError("libnegf.so not built (run __graft_entry__.build()): %s" % path)
    lib = C.CDLL(path)
    for name, (res, args) in _PROTOS.items():
        if hasattr(lib, name):
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
    _lib = lib
    return lib


def exported_symbols():
    return sorted(_PROTOS)


class NegfError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("negf status %d: %s" % (status, msg))
        self.status = status


def _f64(a, n=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if n is not None and a.size != n:
        raise ValueError("expected %d doubles, got %d" % (n, a.size))
    return a


def _cplx(a, n=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.complex128)).view(np.float64)
    if n is not None and a.size != 2 * n:
        raise ValueError("expected %d complex values, got %d" % (n, a.size // 2))
    return a


def _p(a):
    return a.ctypes.data_as(_dp) if a is not None else None


def _pi(a):
    return a.ctypes.data_as(_ip) if a is not None else None


def make_grid(mu_S, mu_D, kT, eta, E_B, n_real, n_cont, rule=RULE_GAUSS, E_min=float("nan"),
              E_max=float("nan"), f1=float("nan"), f2=float("nan")):
    """negf_make_grid: the library's default grid of a bias point (host arrays)."""
    lib = load()
    s = GridSpec(mu_S, mu_D, kT, eta, E_B, E_min, E_max, f1, f2, n_real, n_cont, rule)
    E, w, fS, fD = (np.zeros(max(n_real, 1)) for _ in range(4))
    z = np.zeros(2 * max(n_cont, 1))
    c = np.zeros(2 * max(n_cont, 1))
    rc = lib.negf_make_grid(C.byref(s), _p(E), _p(w), _p(fS), _p(fD), _p(z), _p(c))
    if rc:
        raise NegfError(rc, "make_grid")
    zc = z.view(np.complex128)[:n_cont]
    cc = c.view(np.complex128)[:n_cont]
    return dict(E=E[:n_real], w=w[:n_real], fS=fS[:n_real], fD=fD[:n_real], z=zc, c=cc, eta=eta)


def _adaptive(E_l1, E_l2, densities, a, b, period, ring):
    return Adaptive(E_l1, E_l2, (C.c_double * 3)(*densities), a, b, period, ring)


def make_grid_adaptive(mu_S, mu_D, kT, eta, E_B, n_cont, E_l1, E_l2, densities, a=3.0, b=1.0,
                       E_min=float("nan"), E_max=float("nan"), f1=float("nan"), f2=float("nan")):
    """negf_make_grid_adaptive: the semi-adaptive grid of a bias point (host arrays)."""
    lib = load()
    s = GridSpec(mu_S, mu_D, kT, eta, E_B, E_min, E_max, f1, f2, 0, n_cont, RULE_GAUSS)
    ad = _adaptive(E_l1, E_l2, densities, a, b, 0, -1)
    n = C.c_int()
    rc = lib.negf_make_grid_adaptive(C.byref(s), C.byref(ad), C.byref(n), None, None, None, None, None, None)
    if rc:
        raise NegfError(rc, "make_grid_adaptive")
    nr = n.value
    E, w, fS, fD = (np.zeros(nr) for _ in range(4))
    z = np.zeros(2 * max(n_cont, 1))
    c = np.zeros(2 * max(n_cont, 1))
    rc = lib.negf_make_grid_adaptive(C.byref(s), C.byref(ad), C.byref(n), _p(E), _p(w), _p(fS), _p(fD), _p(z),
                                     _p(c))
    if rc:
        raise NegfError(rc, "make_grid_adaptive")
    return dict(E=E, w=w, fS=fS, fD=fD, z=z.view(np.complex128)[:n_cont], c=c.view(np.complex128)[:n_cont], eta=eta)


def plan_seg_waves(stage_bytes, n_seg, cap):
    """negf_plan_seg_waves (host only): wave of each split item, largest wave staging, most
    records of a wave."""
    lib = load()
    st = np.ascontiguousarray(stage_bytes, dtype=np.int64)
    ns = np.ascontiguousarray(n_seg, dtype=np.int32)
    wave = np.zeros(max(st.size, 1), dtype=np.int32)
    mst, mrec = C.c_longlong(), C.c_longlong()
    rc = lib.negf_plan_seg_waves(st.size, st.ctypes.data_as(C.POINTER(C.c_longlong)), _pi(ns), int(cap), _pi(wave),
                                 C.byref(mst), C.byref(mrec))
    if rc:
        raise NegfError(rc, lib.negf_strerror(rc).decode())
    return wave[:st.size], mst.value, mrec.value


def poisson_kappa(eps_r=3.9, d_nm=1.3, t_ox_nm=10.0, dx_nm=0.1065):
    return load().negf_poisson_kappa(eps_r, d_nm, t_ox_nm, dx_nm)


class Context:
    """One libnegf context (negf_create / negf_destroy)."""

    def __init__(self, device=0, stream=None, hbm_budget=0, precision=PREC_FP64, flag_threshold=0.0,
                 edge_window=0.0, fault_alloc_after=0, growth_threshold=0.0, blk_warps=0, blk_ctas_per_sm=0,
                 general_update=0, chain_warps=0, long_chain_split=0, mixed_two_pass=0):
        self.lib = load()
        o = Opts(device, stream or 0, hbm_budget, precision, flag_threshold, edge_window, fault_alloc_after,
                 growth_threshold, blk_warps, blk_ctas_per_sm, general_update, chain_warps, long_chain_split,
                 mixed_two_pass)
        h = C.c_void_p()
        rc = self.lib.negf_create(C.byref(h), C.byref(o))
        if rc:
            raise NegfError(rc, self.lib.negf_strerror(rc).decode())
        self.h = h
        self._dev = {}

    def close(self):
        if self.h:
            self.lib.negf_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _chk(self, rc):
        if rc:
            raise NegfError(rc, self.lib.negf_last_error(self.h).decode())
        return rc

    def last_error(self):
        return self.lib.negf_last_error(self.h).decode()

    # ---- devices
    def device_create(self, n_rings, block=1, rings_per_block=1, n_chains=1):
        d = C.c_int()
        self._chk(self.lib.negf_device_create(self.h, n_rings, block, rings_per_block, n_chains, C.byref(d)))
        self._dev[d.value] = dict(n_rings=n_rings, block=block, rpb=rings_per_block, n_chains=n_chains)
        return d.value

    def device_destroy(self, dev):
        self._chk(self.lib.negf_device_destroy(self.h, dev))
        self._dev.pop(dev, None)

    def set_hamiltonian(self, dev, chain, Hdiag, Hup, g_b):
        info = self._dev[dev]
        b = info["block"]
        L = info["n_rings"] // info["rpb"]
        hd = _cplx(Hdiag, L * b * b)
        hu = _cplx(Hup, (L - 1) * b * b) if L > 1 else _cplx(np.zeros(1))
        self._chk(self.lib.negf_set_hamiltonian(self.h, dev, chain, _p(hd), _p(hu), g_b))

    def set_lead(self, dev, chain, side, U_lead, T1_row, T2_row, tau_row, sites):
        m = len(sites)
        t1, t2, tau = _cplx(T1_row, m), _cplx(T2_row, m), _cplx(tau_row, m)
        st = np.ascontiguousarray(sites, dtype=np.int32)
        ld = Lead(m, U_lead, _p(t1), _p(t2), _p(tau), _pi(st))
        self._chk(self.lib.negf_set_lead(self.h, dev, chain, side, C.byref(ld)))

    def set_lead_general(self, dev, chain, side, U_lead, T1, T2, tau, sites, H0=None, H1=None, max_iter=0, tol=0.0):
        """negf_set_lead_general: a non-circulant lead (m x m complex blocks), decimated per energy."""
        m = len(sites)
        mats = [None if x is None else _cplx(np.asarray(x).reshape(-1), m * m) for x in (H0, H1, T1, T2, tau)]
        st = np.ascontiguousarray(sites, dtype=np.int32)
        ld = LeadGeneral(m, U_lead, *[_p(x) for x in mats], _pi(st), max_iter, tol)
        self._chk(self.lib.negf_set_lead_general(self.h, dev, chain, side, C.byref(ld)))

    def set_lead_potentials(self, dev, U_S, U_D):
        self._chk(self.lib.negf_set_lead_potentials(self.h, dev, U_S, U_D))

    def build_cnt_modespace(self, dev, n_tube, t, modes, U_S, U_D):
        m = np.ascontiguousarray(modes, dtype=np.int32)
        self._chk(self.lib.negf_build_cnt_modespace(self.h, dev, n_tube, t, _pi(m), U_S, U_D))

    def build_cnt_realspace(self, dev, n_tube, t, U_S, U_D):
        self._chk(self.lib.negf_build_cnt_realspace(self.h, dev, n_tube, t, U_S, U_D))

    def set_potential(self, dev, U):
        u = _f64(U, self._dev[dev]["n_rings"])
        self._chk(self.lib.negf_set_potential(self.h, dev, _p(u)))

    # ---- grids
    def set_grid(self, dev, E, w, fS, fD, eta, z, c):
        E, w, fS, fD = (_f64(x) for x in (E, w, fS, fD))
        zz = _cplx(z)
        cc = _cplx(c)
        g = Grid(E.size, _p(E), _p(w), _p(fS), _p(fD), eta, zz.size // 2, _p(zz), _p(cc))
        self._chk(self.lib.negf_set_grid(self.h, dev, C.byref(g)))
        self._dev[dev]["n_real"] = E.size
        self._dev[dev].pop("n_real_max", None)

    def set_grid_spec(self, dev, mu_S, mu_D, kT, eta, E_B, n_real, n_cont, rule=RULE_GAUSS,
                      E_min=float("nan"), E_max=float("nan"), f1=float("nan"), f2=float("nan")):
        s = GridSpec(mu_S, mu_D, kT, eta, E_B, E_min, E_max, f1, f2, n_real, n_cont, rule)
        self._chk(self.lib.negf_set_grid_spec(self.h, dev, C.byref(s)))
        self._dev[dev]["n_real"] = n_real
        self._dev[dev].pop("n_real_max", None)

    def set_grid_adaptive(self, dev, mu_S, mu_D, kT, eta, E_B, n_cont, E_l1, E_l2, densities, a=3.0, b=1.0,
                          period=50, ring=-1, E_min=float("nan"), E_max=float("nan")):
        """negf_set_grid_adaptive: the semi-adaptive real-axis grid (Sec. 3.3) on a device."""
        s = GridSpec(mu_S, mu_D, kT, eta, E_B, E_min, E_max, float("nan"), float("nan"), 0, n_cont, RULE_GAUSS)
        self._chk(self.lib.negf_set_grid_adaptive(self.h, dev, C.byref(s),
                                                  C.byref(_adaptive(E_l1, E_l2, densities, a, b, period, ring))))
        info = self.grid_info(dev)
        lo = min(mu_S, mu_D) - 14.0 * kT if E_min != E_min else E_min
        hi = max(mu_S, mu_D) + 14.0 * kT if E_max != E_max else E_max
        # room for any refined grid: each segment holds at most density * window / kT + 1 points
        self._dev[dev].update(n_real=info["n_real"],
                              n_real_max=int(sum(np.ceil(d * (hi - lo) / kT) + 1 for d in densities)))
        return info

    def grid_info(self, dev):
        nr, nc = C.c_int(), C.c_int()
        l1, l2 = C.c_double(), C.c_double()
        self._chk(self.lib.negf_grid_info(self.h, dev, C.byref(nr), C.byref(nc), C.byref(l1), C.byref(l2)))
        return dict(n_real=nr.value, n_cont=nc.value, E_l1=l1.value, E_l2=l2.value)

    def ring_integrand(self, dev, ring):
        out = np.zeros(max(self.grid_info(dev)["n_real"], 1))
        self._chk(self.lib.negf_ring_integrand(self.h, dev, ring, _p(out)))
        return out

    def refine_grid(self, dev):
        """negf_refine_grid: returns the located peak E_s; the device grid is rebuilt around it."""
        e = C.c_double()
        self._chk(self.lib.negf_refine_grid(self.h, dev, C.byref(e)))
        self._dev[dev]["n_real"] = self.grid_info(dev)["n_real"]
        return e.value

    # ---- evaluation
    def compute(self, devs):
        """negf_compute on host outputs; returns one dict per device."""
        devs = list(devs)
        outs = (Out * len(devs))()
        keep = []
        for i, d in enumerate(devs):
            info = self._dev[d]
            nr = info.get("n_real", 0)
            arr = dict(n=np.zeros(info["n_rings"]), T=np.zeros(max(nr, 1)), I=np.zeros(1),
                       n_cont=np.zeros(info["n_rings"]), n_real_part=np.zeros(info["n_rings"]))
            keep.append(arr)
            outs[i] = Out(arr["n"].ctypes.data, arr["T"].ctypes.data, arr["I"].ctypes.data,
                          arr["n_cont"].ctypes.data, arr["n_real_part"].ctypes.data, None, None, None, 0)
        ids = np.ascontiguousarray(devs, dtype=np.int32)
        self._chk(self.lib.negf_compute(self.h, _pi(ids), len(devs), outs))
        res = []
        for d, arr in zip(devs, keep):
            nr = self._dev[d].get("n_real", 0)
            res.append(dict(n=arr["n"], T=arr["T"][:nr], I=float(arr["I"][0]), n_cont=arr["n_cont"],
                            n_real=arr["n_real_part"]))
        return res

    def compute_device(self, devs, outs):
        """negf_compute with device outputs: outs is a list of dicts of device pointers
        (keys n, T, I, n_cont, n_real_part; missing keys are skipped)."""
        arr = (Out * len(devs))()
        for i, o in enumerate(outs):
            arr[i] = Out(o.get("n"), o.get("T"), o.get("I"), o.get("n_cont"), o.get("n_real_part"),
                         None, None, None, 1)
        ids = np.ascontiguousarray(devs, dtype=np.int32)
        return self._chk(self.lib.negf_compute(self.h, _pi(ids), len(devs), arr))

    def compute_diag(self, dev):
        """negf_compute of one device with the precision diagnostics (flags, resid, growth)."""
        info = self._dev[dev]
        N, nr = info["n_rings"], info.get("n_real", 0)
        a = dict(n=np.zeros(N), T=np.zeros(max(nr, 1)), I=np.zeros(1), n_cont=np.zeros(N), n_real=np.zeros(N),
                 flags=np.zeros(max(nr, 1), dtype=np.int32), resid=np.zeros(max(nr, 1)), growth=np.zeros(max(nr, 1)))
        out = (Out * 1)()
        out[0] = Out(a["n"].ctypes.data, a["T"].ctypes.data, a["I"].ctypes.data, a["n_cont"].ctypes.data,
                     a["n_real"].ctypes.data, a["flags"].ctypes.data, a["resid"].ctypes.data,
                     a["growth"].ctypes.data, 0)
        ids = np.array([dev], dtype=np.int32)
        self._chk(self.lib.negf_compute(self.h, _pi(ids), 1, out))
        a["I"] = float(a["I"][0])
        for k in ("T", "flags", "resid", "growth"):
            a[k] = a[k][:nr]
        return a

    def compute_raw(self, ids_arr, outs_arr):
        """negf_compute with pre-built ctypes arrays (no allocation in the call path)."""
        return self._chk(self.lib.negf_compute(self.h, ids_arr.ctypes.data_as(_ip), len(ids_arr), outs_arr))

    def sample_lanes(self, dev, idx_real, idx_cont):
        NR = self._dev[dev]["n_rings"]
        ir = np.ascontiguousarray(idx_real, dtype=np.int32)
        ic = np.ascontiguousarray(idx_cont, dtype=np.int32)
        AS = np.zeros((max(ir.size, 1), NR))
        AD = np.zeros((max(ir.size, 1), NR))
        G = np.zeros((max(ic.size, 1), NR), dtype=np.complex128)
        self._chk(self.lib.negf_sample_lanes(self.h, dev, ir.size, _pi(ir), _p(AS), _p(AD), ic.size, _pi(ic),
                                             G.view(np.float64).ctypes.data_as(_dp)))
        return AS[:ir.size], AD[:ir.size], G[:ic.size]

    def neutral_charge(self, dev, n_cont, E_B):
        n0 = np.zeros(self._dev[dev]["n_rings"])
        self._chk(self.lib.negf_neutral_charge(self.h, dev, n_cont, E_B, _p(n0)))
        return n0

    def conductance(self, devs, mu, kT, want_T=False):
        """negf_conductance: zero-bias conductance (S) per device, and optionally T(E) per device."""
        devs = list(devs)
        ids = np.ascontiguousarray(devs, dtype=np.int32)
        G = np.zeros(len(devs))
        nrs = [self._dev[d].get("n_real", 0) for d in devs]
        T = np.zeros(max(sum(nrs), 1)) if want_T else None
        self._chk(self.lib.negf_conductance(self.h, _pi(ids), len(devs), mu, kT, _p(G), _p(T)))
        if not want_T:
            return G
        return G, np.split(T[:sum(nrs)], np.cumsum(nrs)[:-1])

    def sc_solve(self, dev, V_DS, V_GS, U0, kappa, dx_nm=0.1065, lam_nm=3.0, phi_gate=0.0, zeta=0.1, M=64,
                 tol=1e-8, check=True):
        N = self._dev[dev]["n_rings"]
        nr = self._dev[dev].get("n_real_max", self._dev[dev].get("n_real", 0))
        n, U, T, hist = np.zeros(N), np.zeros(N), np.zeros(max(nr, 1)), np.zeros(M)
        r = ScResult(_p(n), _p(U), _p(T), _p(hist), 0.0, 0, 0)
        u0 = _f64(U0, N)
        rc = self.lib.negf_sc_solve(self.h, dev, C.byref(Bias(V_DS, V_GS)),
                                    C.byref(Poisson(kappa, dx_nm, lam_nm, phi_gate)),
                                    C.byref(Broyden(zeta, M, tol)), _p(u0), C.byref(r))
        if rc not in (OK, ENOTCONVERGED) or (check and rc):
            self._chk(rc)
        nr = self._dev[dev]["n_real"] = self.grid_info(dev)["n_real"]
        return dict(status=rc, n=n, U=U, T=T[:nr], history=hist[:r.iterations], I=r.I,
                    converged=bool(r.converged), iterations=r.iterations)

    def sc_solve_multi(self, devs, V_DS, V_GS, U0, K, dx_nm=0.1065, lam_nm=3.0, phi_gate=0.0, zeta=0.1, M=64,
                       tol=1e-8, check=True):
        """negf_sc_solve_multi: C coupled channels with one Broyden vector; U0 (C, N), K (C, C)."""
        devs = list(devs)
        Cn = len(devs)
        N = self._dev[devs[0]]["n_rings"]
        u0 = _f64(U0, Cn * N)
        k = _f64(K, Cn * Cn)
        arrs = []
        res = (ScResult * Cn)()
        for i, d in enumerate(devs):
            nr = self._dev[d].get("n_real", 0)
            a = dict(n=np.zeros(N), U=np.zeros(N), T=np.zeros(max(nr, 1)), history=np.zeros(M), nr=nr)
            arrs.append(a)
            res[i] = ScResult(_p(a["n"]), _p(a["U"]), _p(a["T"]), _p(a["history"]), 0.0, 0, 0)
        ids = np.ascontiguousarray(devs, dtype=np.int32)
        rc = self.lib.negf_sc_solve_multi(self.h, _pi(ids), Cn, C.byref(Bias(V_DS, V_GS)),
                                          C.byref(Poisson(0.0, dx_nm, lam_nm, phi_gate)), _p(k),
                                          C.byref(Broyden(zeta, M, tol)), _p(u0), res)
        if rc not in (OK, ENOTCONVERGED) or (check and rc):
            self._chk(rc)
        it = res[0].iterations
        return dict(status=rc, converged=bool(res[0].converged), iterations=it, history=arrs[0]["history"][:it],
                    n=[a["n"] for a in arrs], U=[a["U"] for a in arrs], T=[a["T"][:a["nr"]] for a in arrs],
                    I=[res[i].I for i in range(Cn)])

    def sc_begin(self, dev, V_DS, V_GS, U0, kappa, dx_nm=0.1065, lam_nm=3.0, phi_gate=0.0, zeta=0.1, M=64,
                 tol=1e-8):
        u0 = _f64(U0, self._dev[dev]["n_rings"])
        self._chk(self.lib.negf_sc_begin(self.h, dev, C.byref(Bias(V_DS, V_GS)),
                                         C.byref(Poisson(kappa, dx_nm, lam_nm, phi_gate)),
                                         C.byref(Broyden(zeta, M, tol)), _p(u0)))
        self._dev[dev]["M"] = M

    def sc_step(self, dev, k=1, wait=True):
        st = C.c_int(0)
        self._chk(self.lib.negf_sc_step(self.h, dev, k, C.byref(st) if wait else None))
        return st.value if wait else None

    def sc_end(self, dev, check=False):
        N = self._dev[dev]["n_rings"]
        nr = self._dev[dev].get("n_real_max", self._dev[dev].get("n_real", 0))
        M = self._dev[dev].get("M", 256)
        n, U, T, hist = np.zeros(N), np.zeros(N), np.zeros(max(nr, 1)), np.zeros(M)
        r = ScResult(_p(n), _p(U), _p(T), _p(hist), 0.0, 0, 0)
        rc = self.lib.negf_sc_end(self.h, dev, C.byref(r))
        if rc not in (OK, ENOTCONVERGED) or (check and rc):
            self._chk(rc)
        nr = self._dev[dev]["n_real"] = self.grid_info(dev)["n_real"]
        return dict(status=rc, n=n, U=U, T=T[:nr], history=hist[:min(r.iterations, M)], I=r.I,
                    converged=bool(r.converged), iterations=r.iterations)

    def sc_get_state(self, dev):
        N = self._dev[dev]["n_rings"]
        M = self._dev[dev]["M"]
        a = [np.zeros(N) for _ in range(3)] + [np.zeros(M * N), np.zeros(M * N)]
        m = C.c_int()
        self._chk(self.lib.negf_sc_get_state(self.h, dev, *[_p(x) for x in a], C.byref(m)))
        return dict(n_in=a[0], n_in_old=a[1], f_old=a[2], V=a[3].reshape(M, N), W=a[4].reshape(M, N), m=m.value)

    def sc_set_state(self, dev, st):
        a = [_f64(st[k]) for k in ("n_in", "n_in_old", "f_old", "V", "W")]
        self._chk(self.lib.negf_sc_set_state(self.h, dev, *[_p(x) for x in a], int(st["m"])))

    def profile(self, enable=True):
        self._chk(self.lib.negf_profile(self.h, 1 if enable else 0))

    def kernel_time(self):
        ms = C.c_double()
        n = C.c_uint64()
        self._chk(self.lib.negf_kernel_time(self.h, C.byref(ms), C.byref(n)))
        return ms.value, n.value

    def sweep_lanes(self):
        """Lanes of the wide-block sweep since the last call, by update form:
        (real symmetric, real general, contour symmetric, contour general)."""
        v = (C.c_uint64 * 4)()
        self._chk(self.lib.negf_sweep_lanes(self.h, v))
        return tuple(int(x) for x in v)

    def fp64_peak(self):
        t = C.c_double()
        self._chk(self.lib.negf_fp64_peak(self.h, C.byref(t)))
        return t.value

    def blk_width(self, b, m, fp32=False):
        """CTA width chosen by the autotuner for ring blocks of width b (None if not tuned)."""
        s = self.blk_shape(b, m, fp32)
        return s[0] if s else None

    def chain_width(self, block=1, fp32=False):
        """CTA width (warps) the autotuner chose for the thread-per-lane sweep (None if not tuned)."""
        w = C.c_int()
        rc = self.lib.negf_chain_width(self.h, 1 if fp32 else 0, block, C.byref(w))
        return w.value if rc == OK else None

    def blk_shape(self, b, m, fp32=False):
        """(CTA width, resident CTAs per SM) chosen by the autotuner (None if not tuned)."""
        w, k = C.c_int(), C.c_int()
        rc = self.lib.negf_blk_width(self.h, 1 if fp32 else 0, b, m, C.byref(w), C.byref(k))
        return (w.value, k.value) if rc == OK else None

    # ---- serving
    def submit(self, n_rings, modes, V_DS, V_GS, n_real=2048, n_cont=64, n_tube=17, t=-2.7, kT=0.025,
               eta=1e-6, E_B=None, kappa=None, dx_nm=0.1065, lam_nm=3.0, phi_gate=0.0, zeta=0.1, M=64,
               tol=1e-8, U0=None):
        m = np.ascontiguousarray(modes, dtype=np.int32)
        u0 = _f64(U0, n_rings) if U0 is not None else None
        if E_B is None:
            E_B = -V_DS - 3.0 * abs(t) - 1.0
        if kappa is None:
            kappa = poisson_kappa()
        q = Request(n_rings, n_tube, m.size, _pi(m), t, kT, eta, E_B, n_real, n_cont, Bias(V_DS, V_GS),
                    Poisson(kappa, dx_nm, lam_nm, phi_gate), Broyden(zeta, M, tol), _p(u0))
        tk = C.c_uint64()
        self._chk(self.lib.negf_submit(self.h, C.byref(q), C.byref(tk)))
        self._req = getattr(self, "_req", {})
        self._req[tk.value] = dict(n_rings=n_rings, n_real=n_real, M=M)
        return tk.value

    def serve_step(self):
        n = C.c_int()
        self._chk(self.lib.negf_serve_step(self.h, C.byref(n)))
        return n.value

    def _result(self, ticket, fn, *args):
        info = self._req[ticket]
        N, nr, M = info["n_rings"], info["n_real"], info["M"]
        n, U, T, hist = np.zeros(N), np.zeros(N), np.zeros(nr), np.zeros(M)
        r = ScResult(_p(n), _p(U), _p(T), _p(hist), 0.0, 0, 0)
        rc = fn(self.h, C.c_uint64(ticket), *args, C.byref(r))
        if rc == EBUSY:
            return None
        if rc not in (OK, ENOTCONVERGED):
            self._chk(rc)
        return dict(status=rc, n=n, U=U, T=T, history=hist[:min(r.iterations, M)], I=r.I,
                    converged=bool(r.converged), iterations=r.iterations)

    def poll(self, ticket):
        return self._result(ticket, self.lib.negf_poll)

    def wait(self, ticket, timeout_ms=600000):
        return self._result(ticket, self.lib.negf_wait, C.c_int(timeout_ms))

    def cancel(self, ticket):
        self._chk(self.lib.negf_cancel(self.h, C.c_uint64(ticket)))

    def request_times(self, ticket):
        a, b, c = C.c_double(), C.c_double(), C.c_double()
        self._chk(self.lib.negf_request_times(self.h, C.c_uint64(ticket), C.byref(a), C.byref(b), C.byref(c)))
        return a.value, b.value, c.value

    def launch_count(self):
        v = C.c_uint64()
        self._chk(self.lib.negf_launch_count(self.h, C.byref(v)))
        return v.value
