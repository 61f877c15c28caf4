"""Thin ctypes binding of libo2pic.so (C ABI in include/o2pic.h).

Argument marshalling only: every step of the simulation runs in the CUDA
library.  PyTorch provides the device workspace and the stream.  There is no
CPU fallback: if the library is missing or no GPU is present, the calls fail.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import inputs as _inputs

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libo2pic.so")

PIC_FP64, PIC_FP32_MIXED = 0, 1
STATUS = {0: "PIC_OK", 1: "PIC_EINVAL", 2: "PIC_ENOMEM", 3: "PIC_ECAPACITY",
          4: "PIC_ETIMEOUT", 5: "PIC_ECUDA", 6: "PIC_ENUMERIC"}


class PicError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class pic_xs_table(C.Structure):
    _fields_ = [("reaction", C.c_int), ("sub", C.c_int), ("n", C.c_int),
                ("E_eV", C.POINTER(C.c_double)), ("sigma_m2", C.POINTER(C.c_double)),
                ("threshold_eV", C.c_double)]


class pic_config(C.Structure):
    _fields_ = [
        ("L_m", C.c_double), ("p_Pa", C.c_double), ("T_gas_K", C.c_double),
        ("U_rf_V", C.c_double), ("f_rf_Hz", C.c_double), ("rf_phase", C.c_double),
        ("dt_s", C.c_double), ("weight_m2", C.c_double), ("C_delta", C.c_double),
        ("T0_eV", C.c_double * 3), ("ecap_eV", C.c_double * 3), ("numax_safety", C.c_double),
        ("eedf_emax_eV", C.c_double), ("iedf_emax_eV", C.c_double), ("fm_emax_eV", C.c_double),
        ("n_init", C.c_longlong * 3), ("capacity", C.c_longlong * 3), ("seed", C.c_ulonglong),
        ("n_cells", C.c_int), ("n1", C.c_int), ("sort_interval", C.c_int), ("diag_every", C.c_int),
        ("eedf_bins", C.c_int), ("iedf_bins", C.c_int), ("fm_bins", C.c_int), ("fm_xbins", C.c_int),
        ("cx_isotropic", C.c_int), ("numax_bins", C.c_int), ("n2", C.c_int), ("gas_scheme", C.c_int),
        ("ion_subcycle", C.c_int), ("coulomb_inter", C.c_int), ("precision", C.c_int),
        ("coulomb_log", C.c_double),
    ]


EXPORTS = ["pic_workspace_size", "pic_init", "pic_step", "pic_diagnostics", "pic_get_state",
           "pic_set_state", "pic_set_step", "pic_set_numeric_budget", "pic_fields", "pic_numax", "pic_set_timing",
           "pic_timing", "pic_kernel_timing", "pic_get_launch", "pic_set_launch", "pic_launch_shapes",
           "pic_get_launch_shape", "pic_set_launch_shape", "pic_destroy",
           "pic_last_error",
           "pic_field_solve_static"]
KERNELS = {"push": 0, "coulomb": 1, "sequential_gas": 2, "push_diag": 3}

_lib = None


def load(path: str = LIB_PATH):
    """Load libo2pic.so and declare the signatures (raises if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise FileNotFoundError(f"{path} is missing: build it with paper_0705_0495_gb300.build.build()")
    l = C.CDLL(path)
    dp, lp, ip, vp = (C.POINTER(C.c_double), C.POINTER(C.c_longlong), C.POINTER(C.c_int),
                      C.c_void_p)
    l.pic_workspace_size.restype = C.c_size_t
    l.pic_workspace_size.argtypes = [C.POINTER(pic_config), C.c_int, C.POINTER(pic_xs_table), C.c_int]
    l.pic_init.restype = C.c_int
    l.pic_init.argtypes = [C.POINTER(pic_config), C.c_int, C.POINTER(pic_xs_table), C.c_int, vp,
                           C.c_size_t, vp, C.POINTER(vp)]
    l.pic_step.restype = C.c_int
    l.pic_step.argtypes = [vp, C.c_longlong]
    l.pic_diagnostics.restype = C.c_int
    l.pic_diagnostics.argtypes = [vp, C.c_int, dp, dp, lp, lp, lp, lp, lp, C.c_int]
    l.pic_get_state.restype = C.c_int
    l.pic_get_state.argtypes = [vp, C.c_int, C.c_int, dp, dp, dp, dp, ip, C.c_longlong, lp]
    l.pic_set_state.restype = C.c_int
    l.pic_set_state.argtypes = [vp, C.c_int, C.c_int, C.c_longlong, dp, dp, dp, dp, ip]
    l.pic_set_step.restype = C.c_int
    l.pic_set_step.argtypes = [vp, C.c_longlong]
    l.pic_set_numeric_budget.restype = C.c_int
    l.pic_set_numeric_budget.argtypes = [vp, C.c_double]
    l.pic_fields.restype = C.c_int
    l.pic_fields.argtypes = [vp, C.c_int, dp, dp, dp]
    l.pic_numax.restype = C.c_double
    l.pic_numax.argtypes = [vp, C.c_int, C.c_int]
    l.pic_set_timing.restype = C.c_int
    l.pic_set_timing.argtypes = [vp, C.c_int]
    l.pic_timing.restype = C.c_int
    l.pic_timing.argtypes = [vp, dp, lp, lp, dp, C.c_int]
    l.pic_kernel_timing.restype = C.c_int
    l.pic_kernel_timing.argtypes = [vp, C.c_int, dp, lp, dp, C.c_int]
    l.pic_get_launch.restype = C.c_int
    l.pic_get_launch.argtypes = [vp, C.c_int, ip, ip]
    l.pic_set_launch.restype = C.c_int
    l.pic_set_launch.argtypes = [vp, C.c_int, C.c_int]
    l.pic_launch_shapes.restype = C.c_int
    l.pic_launch_shapes.argtypes = [vp, C.c_int, ip, ip, ip, C.c_int]
    l.pic_get_launch_shape.restype = C.c_int
    l.pic_get_launch_shape.argtypes = [vp, C.c_int, ip, ip]
    l.pic_set_launch_shape.restype = C.c_int
    l.pic_set_launch_shape.argtypes = [vp, C.c_int, C.c_int, C.c_int]
    l.pic_destroy.restype = None
    l.pic_destroy.argtypes = [vp]
    l.pic_last_error.restype = C.c_char_p
    l.pic_last_error.argtypes = [vp]
    l.pic_field_solve_static.restype = C.c_int
    l.pic_field_solve_static.argtypes = [C.POINTER(pic_config), C.c_longlong, C.POINTER(C.c_void_p),
                                         C.POINTER(C.c_void_p), lp, vp, vp, vp, vp]
    _lib = l
    return l


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _lp(a):
    return a.ctypes.data_as(C.POINTER(C.c_longlong))


def make_config(d: "_inputs.Discharge", fp64: bool | None = None) -> pic_config:
    """Marshal an inputs.Discharge into the C struct."""
    c = pic_config()
    c.L_m, c.p_Pa, c.T_gas_K = d.L, d.p_Pa, d.T_gas
    c.U_rf_V, c.f_rf_Hz, c.rf_phase, c.dt_s = d.U_rf, d.f_rf, d.rf_phase, d.dt
    c.weight_m2, c.C_delta = d.weight, d.C_delta
    for s in range(3):
        c.T0_eV[s] = d.T0_eV[s]
        c.ecap_eV[s] = d.ecap_eV[s]
        c.n_init[s] = int(d.n_init[s])
        c.capacity[s] = int(d.capacity[s])
    c.numax_safety = d.numax_safety
    c.eedf_emax_eV, c.iedf_emax_eV, c.fm_emax_eV = d.eedf_emax, d.iedf_emax, d.fm_emax
    c.seed = d.seed
    c.n_cells, c.n1, c.sort_interval, c.diag_every = d.n_cells, d.n1, d.sort_interval, d.diag_every
    c.eedf_bins, c.iedf_bins, c.fm_bins, c.fm_xbins = d.eedf_bins, d.iedf_bins, d.fm_bins, d.fm_xbins
    c.cx_isotropic = int(d.cx_isotropic)
    c.numax_bins = int(d.numax_bins)
    c.n2 = int(d.n2)
    c.coulomb_log = float(d.coulomb_log)
    c.gas_scheme = int(d.gas_scheme)
    c.ion_subcycle = int(d.ion_subcycle)
    c.coulomb_inter = int(d.coulomb_inter)
    use64 = d.fp64 if fp64 is None else fp64
    c.precision = PIC_FP64 if use64 else PIC_FP32_MIXED
    return c


def make_tables(tables):
    keep = []
    arr = (pic_xs_table * max(1, len(tables)))()
    for i, t in enumerate(tables):
        E = np.ascontiguousarray(t["E_eV"], dtype=np.float64)
        S = np.ascontiguousarray(t["sigma_m2"], dtype=np.float64)
        keep += [E, S]
        arr[i].reaction, arr[i].sub, arr[i].n = t["reaction"], t.get("sub", 0), len(E)
        arr[i].E_eV, arr[i].sigma_m2 = _dp(E), _dp(S)
        arr[i].threshold_eV = t.get("threshold_eV", 0.0)
    return arr, keep


def workspace_size(discharges, tables, fp64=None) -> int:
    lib = load()
    cfgs = (pic_config * len(discharges))(*[make_config(d, fp64) for d in discharges])
    arr, keep = make_tables(tables)
    n = lib.pic_workspace_size(cfgs, len(discharges), arr, len(tables))
    if n == 0:
        raise PicError(1, lib.pic_last_error(None).decode())
    return n


class Simulation:
    """Discharges advanced together on one GPU through libo2pic."""

    def __init__(self, discharges, tables, fp64=None, device="cuda", stream=None, numeric_budget=None):
        import torch
        self.lib = load()
        if not isinstance(discharges, (list, tuple)):
            discharges = [discharges]
        self.discharges = list(discharges)
        self.tables = tables
        cfgs = (pic_config * len(discharges))(*[make_config(d, fp64) for d in discharges])
        self._cfgs = cfgs
        arr, self._keep = make_tables(tables)
        n = self.lib.pic_workspace_size(cfgs, len(discharges), arr, len(tables))
        if n == 0:
            raise PicError(1, self.lib.pic_last_error(None).decode())
        self.ws_bytes = n
        self.device = torch.device(device)
        self.ws = torch.empty(n + 256, dtype=torch.uint8, device=self.device)
        ptr = self.ws.data_ptr()
        ptr = (ptr + 255) & ~255
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = C.c_void_p()
        rc = self.lib.pic_init(cfgs, len(discharges), arr, len(tables), C.c_void_p(ptr), n,
                               C.c_void_p(self.stream.cuda_stream), C.byref(h))
        if rc != 0:
            raise PicError(rc, self.lib.pic_last_error(None).decode())
        self.h = h
        if numeric_budget is not None:
            self.set_numeric_budget(numeric_budget)

    def _check(self, rc):
        if rc != 0:
            raise PicError(rc, self.lib.pic_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self.lib.pic_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n=1):
        self._check(self.lib.pic_step(self.h, int(n)))

    def set_step(self, k):
        self._check(self.lib.pic_set_step(self.h, int(k)))

    def set_numeric_budget(self, max_fraction):
        """largest accepted fraction of nu_max violations and of Eq. 1 P > 1
        clamps before pic_step reports PIC_ENUMERIC (default 1e-6)"""
        self._check(self.lib.pic_set_numeric_budget(self.h, float(max_fraction)))

    def count(self, d, s):
        n = C.c_longlong()
        self._check(self.lib.pic_get_state(self.h, d, s, None, None, None, None, None, 0, C.byref(n)))
        return n.value

    def get_state(self, d, s):
        n = self.count(d, s)
        x, vx, vy, vz = (np.zeros(max(n, 1)) for _ in range(4))
        alive = np.zeros(max(n, 1), dtype=np.int32)
        m = C.c_longlong()
        self._check(self.lib.pic_get_state(self.h, d, s, _dp(x), _dp(vx), _dp(vy), _dp(vz),
                                           alive.ctypes.data_as(C.POINTER(C.c_int)), len(x),
                                           C.byref(m)))
        n = m.value
        return {"x": x[:n], "vx": vx[:n], "vy": vy[:n], "vz": vz[:n], "alive": alive[:n].astype(bool)}

    def set_state(self, d, s, x, vx, vy, vz, alive=None):
        x, vx, vy, vz = (np.ascontiguousarray(a, dtype=np.float64) for a in (x, vx, vy, vz))
        al = None if alive is None else np.ascontiguousarray(alive, dtype=np.int32)
        ap = None if al is None else al.ctypes.data_as(C.POINTER(C.c_int))
        self._check(self.lib.pic_set_state(self.h, d, s, len(x), _dp(x), _dp(vx), _dp(vy),
                                           _dp(vz), ap))

    def fields(self, d=0):
        N = self.discharges[d].n_cells
        rho, phi, E = (np.zeros(N + 1) for _ in range(3))
        self._check(self.lib.pic_fields(self.h, d, _dp(rho), _dp(phi), _dp(E)))
        return rho, phi, E

    def numax(self, d, s):
        return self.lib.pic_numax(self.h, d, s)

    def diagnostics(self, d=0, reset=False):
        dd = self.discharges[d]
        N = dd.n_cells
        dens = np.zeros((3, N + 1))
        phi = np.zeros(N + 1)
        eedf = np.zeros(max(dd.eedf_bins, 1), dtype=np.int64)
        iedf = np.zeros((2, max(dd.iedf_bins, 1)), dtype=np.int64)
        fm = np.zeros((max(dd.fm_xbins, 1), max(dd.fm_bins, 1)), dtype=np.int64)
        cnt = np.zeros(40, dtype=np.int64)
        ns = C.c_longlong()
        self._check(self.lib.pic_diagnostics(self.h, d, _dp(dens), _dp(phi), _lp(eedf), _lp(iedf),
                                             _lp(fm), _lp(cnt), C.byref(ns), 1 if reset else 0))
        k = max(ns.value, 1)
        return {"n_samples": ns.value, "dens_sum": dens, "phi_sum": phi, "eedf": eedf,
                "dens_avg": dens / k, "phi_avg": phi / k,
                "iedf": iedf, "fm": fm, "absorbed": cnt[0:6].reshape(3, 2),
                "events": cnt[6:26].copy(), "violations": cnt[26:28].copy(),
                "slots": cnt[28:31].copy(), "steps": int(cnt[31]),
                "particle_steps": int(cnt[32]), "candidates": int(cnt[33]),
                "slots_visited": int(cnt[34]), "coulomb_particles": int(cnt[35]),
                "sequential_gas_slots": int(cnt[36]), "eq1_evaluations": int(cnt[37]),
                "graph_cycle_steps": int(cnt[38]), "graph_launch_calls": int(cnt[39])}

    def align_to_cycle(self):
        """step to the next whole RF cycle when one cycle runs as a captured
        CUDA graph, so that whole-cycle step() calls from here on replay that
        graph (a start off the schedule's period runs single steps); returns
        the number of time steps taken"""
        g = self.diagnostics(0)
        c = g["graph_cycle_steps"]
        n = (-g["steps"]) % c if c > 0 else 0
        if n:
            self.step(n)
        return n

    def set_timing(self, on=True):
        self._check(self.lib.pic_set_timing(self.h, 1 if on else 0))

    def timing(self, reset=False):
        ms, bts = C.c_double(), C.c_double()
        pl, la = C.c_longlong(), C.c_longlong()
        self._check(self.lib.pic_timing(self.h, C.byref(ms), C.byref(pl), C.byref(la), C.byref(bts),
                                        1 if reset else 0))
        return {"push_ms": ms.value, "push_launches": pl.value, "launches": la.value,
                "push_bytes": bts.value}

    def kernel_timing(self, kernel, reset=False):
        """device ms, launches and algorithmic bytes of one kernel kind
        ("push", "coulomb" or "sequential_gas") in timing mode"""
        ms, bts, n = C.c_double(), C.c_double(), C.c_longlong()
        self._check(self.lib.pic_kernel_timing(self.h, KERNELS[kernel], C.byref(ms), C.byref(n),
                                               C.byref(bts), 1 if reset else 0))
        return {"ms": ms.value, "launches": n.value, "bytes": bts.value}

    def launch(self, kernel="push"):
        """(blocks per SM, largest blocks per SM) of a kernel kind's grid"""
        cur, mx = C.c_int(), C.c_int()
        self._check(self.lib.pic_get_launch(self.h, KERNELS[kernel], C.byref(cur), C.byref(mx)))
        return cur.value, mx.value

    def launch_shapes(self, kernel="push"):
        """[(threads per block, slots per thread, largest blocks per SM)] of
        the shapes a kernel kind is compiled for"""
        cap = 16
        t, p, m = ((C.c_int * cap)() for _ in range(3))
        n = self.lib.pic_launch_shapes(self.h, KERNELS[kernel], t, p, m, cap)
        if n < 0:
            raise PicError(1, self.lib.pic_last_error(self.h).decode())
        return [(t[k], p[k], m[k]) for k in range(n)]

    def launch_shape(self, kernel="push"):
        """(shape index, blocks per SM) of a kernel kind's grid"""
        sh, b = C.c_int(), C.c_int()
        self._check(self.lib.pic_get_launch_shape(self.h, KERNELS[kernel], C.byref(sh), C.byref(b)))
        return sh.value, b.value

    def set_launch_shape(self, shape, blocks_per_sm, kernel="push"):
        """launch shape (index into launch_shapes()) and blocks per SM
        (results do not depend on them)"""
        self._check(self.lib.pic_set_launch_shape(self.h, KERNELS[kernel], int(shape), int(blocks_per_sm)))

    def set_launch(self, blocks_per_sm, kernel="push"):
        """blocks per SM of a kernel kind's grid (results do not depend on it)"""
        self._check(self.lib.pic_set_launch(self.h, KERNELS[kernel], int(blocks_per_sm)))


def field_solve_static(cfg: pic_config, step: int, cell_ptrs, off_ptrs, counts, rho_ptr, phi_ptr, E_ptr,
                       stream_ptr=0) -> None:
    """pic_field_solve_static: deposit and field solve from caller-owned device
    arrays (pointers as ints), with no allocation (see include/o2pic.h)."""
    lib = load()
    cells = (C.c_void_p * 3)(*[C.c_void_p(p) for p in cell_ptrs])
    offs = (C.c_void_p * 3)(*[C.c_void_p(p) for p in off_ptrs])
    n = (C.c_longlong * 3)(*[int(v) for v in counts])
    rc = lib.pic_field_solve_static(C.byref(cfg), int(step), cells, offs, n, C.c_void_p(rho_ptr),
                                    C.c_void_p(phi_ptr), C.c_void_p(E_ptr), C.c_void_p(stream_ptr))
    if rc != 0:
        raise PicError(rc, lib.pic_last_error(None).decode())
