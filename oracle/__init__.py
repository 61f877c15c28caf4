"""Python access to the FP64 CPU oracle (``o2pic_oracle.c``).

TEST INFRASTRUCTURE ONLY.  The oracle is the slow reference against which the
GPU library is checked; only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with ``paper_0705_0495_gb300``; both sides receive the same seeded inputs from
``paper_0705_0495_gb300.inputs``, which holds no arithmetic of the method.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "o2pic_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, so the rounding is the
    plain sequence of the source)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "o2pic_oracle.h"))
    ):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fPIC", "-shared",
             _SRC, "-o", tmp, "-lm"]
        )
        os.replace(tmp, _LIB)
    return _LIB


class _Cfg(C.Structure):
    _fields_ = [
        ("L", C.c_double), ("p_Pa", C.c_double), ("T_gas", C.c_double),
        ("U_rf", C.c_double), ("f_rf", C.c_double), ("rf_phase", C.c_double),
        ("dt", C.c_double),
        ("weight", C.c_double), ("C_delta", C.c_double),
        ("T0_eV", C.c_double * 3), ("ecap_eV", C.c_double * 3),
        ("numax_safety", C.c_double),
        ("eedf_emax", C.c_double), ("iedf_emax", C.c_double), ("fm_emax", C.c_double),
        ("n_init", C.c_longlong * 3), ("seed", C.c_ulonglong),
        ("n_cells", C.c_int), ("n1", C.c_int), ("sort_interval", C.c_int),
        ("diag_every", C.c_int), ("eedf_bins", C.c_int), ("iedf_bins", C.c_int),
        ("fm_bins", C.c_int), ("fm_xbins", C.c_int), ("discharge", C.c_int),
        ("cx_isotropic", C.c_int), ("numax_bins", C.c_int), ("n2", C.c_int),
        ("gas_scheme", C.c_int), ("ion_subcycle", C.c_int), ("coulomb_inter", C.c_int),
        ("coulomb_log", C.c_double),
    ]


class _Xs(C.Structure):
    _fields_ = [
        ("reaction", C.c_int), ("sub", C.c_int), ("n", C.c_int),
        ("E_eV", C.POINTER(C.c_double)), ("sigma_m2", C.POINTER(C.c_double)),
        ("threshold_eV", C.c_double),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        l = C.CDLL(build())
        dp = C.POINTER(C.c_double)
        lp = C.POINTER(C.c_longlong)
        ip = C.POINTER(C.c_int)
        u32p = C.POINTER(C.c_uint32)
        l.orc_create.restype = C.c_void_p
        l.orc_create.argtypes = [C.POINTER(_Cfg), C.POINTER(_Xs), C.c_int, C.c_int]
        l.orc_destroy.argtypes = [C.c_void_p]
        l.orc_step.argtypes = [C.c_void_p, C.c_longlong]
        l.orc_step_index.restype = C.c_longlong
        l.orc_step_index.argtypes = [C.c_void_p]
        l.orc_set_step.argtypes = [C.c_void_p, C.c_longlong]
        l.orc_particle_steps.restype = C.c_longlong
        l.orc_particle_steps.argtypes = [C.c_void_p]
        l.orc_count.restype = C.c_longlong
        l.orc_count.argtypes = [C.c_void_p, C.c_int]
        l.orc_get.argtypes = [C.c_void_p, C.c_int, dp, dp, dp, dp, ip]
        l.orc_set.restype = C.c_int
        l.orc_set.argtypes = [C.c_void_p, C.c_int, C.c_longlong, dp, dp, dp, dp, ip]
        l.orc_numax.restype = C.c_double
        l.orc_numax.argtypes = [C.c_void_p, C.c_int]
        l.orc_coulomb_pair.restype = None
        l.orc_coulomb_pair.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_double,
                                       C.c_double, C.c_double, C.c_double]
        l.orc_coulomb_pair2.restype = None
        l.orc_coulomb_pair2.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_double,
                                        C.c_double, C.c_double, C.c_double]
        l.orc_coulomb_inter_pairing.restype = None
        l.orc_coulomb_inter_pairing.argtypes = [C.c_void_p, C.c_int, C.c_longlong, C.c_longlong,
                                                C.c_longlong, C.c_uint32, C.c_void_p, C.c_void_p]
        l.orc_coulomb_pairing.restype = C.c_longlong
        l.orc_coulomb_pairing.argtypes = [C.c_void_p, C.c_int, C.c_longlong, C.c_longlong,
                                          C.c_uint32, C.c_void_p, C.c_void_p]
        l.orc_coulomb_cell.restype = None
        l.orc_coulomb_cell.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                                       C.c_longlong, C.c_double, C.c_double, C.c_longlong,
                                       C.c_uint32]
        l.orc_numax_bin.restype = C.c_double
        l.orc_numax_bin.argtypes = [C.c_void_p, C.c_int]
        l.orc_bin_of.restype = C.c_int
        l.orc_bin_of.argtypes = [C.c_void_p, C.c_double]
        l.orc_fields.argtypes = [C.c_void_p, dp, dp, dp]
        l.orc_counters.argtypes = [C.c_void_p, lp, lp, lp, lp]
        l.orc_eq1_evaluations.restype = C.c_longlong
        l.orc_eq1_evaluations.argtypes = [C.c_void_p]
        l.orc_reset_diag.restype = None
        l.orc_reset_diag.argtypes = [C.c_void_p]
        l.orc_diag.restype = C.c_longlong
        l.orc_diag.argtypes = [C.c_void_p, dp, dp, lp, lp, lp]
        l.orc_philox.argtypes = [u32p, u32p, u32p]
        l.orc_sigma.restype = C.c_double
        l.orc_sigma.argtypes = [C.c_void_p, C.c_int, C.c_double]
        l.orc_poisson.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double, dp, dp]
        l.orc_field.argtypes = [C.c_int, C.c_double, dp, dp, dp]
        l.orc_gas_event.restype = C.c_int
        l.orc_gas_event.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, dp, dp, dp, dp,
                                    dp, ip, ip, dp, dp]
        l.orc_pair19_event.argtypes = [C.c_void_p, C.c_int, dp, dp, dp, dp, dp, dp, dp]
        _lib = l
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def philox(ctr, key):
    c = (C.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (C.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (C.c_uint32 * 4)()
    lib().orc_philox(c, k, o)
    return [int(v) for v in o]


def poisson(n_cells, dx, phi0, phiN, rho):
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    phi = np.zeros(n_cells + 1)
    lib().orc_poisson(n_cells, dx, phi0, phiN, _dp(rho), _dp(phi))
    return phi


def field(n_cells, dx, rho, phi):
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    E = np.zeros(n_cells + 1)
    lib().orc_field(n_cells, dx, _dp(rho), _dp(phi), _dp(E))
    return E


class Oracle:
    """One discharge simulated by the oracle.  ``d`` is an
    ``inputs.Discharge``; ``tables`` the list of cross-section tables."""

    def __init__(self, d, tables, load=True, discharge=0):
        self.d = d
        cfg = _Cfg()
        cfg.L, cfg.p_Pa, cfg.T_gas = d.L, d.p_Pa, d.T_gas
        cfg.U_rf, cfg.f_rf, cfg.dt = d.U_rf, d.f_rf, d.dt
        cfg.rf_phase = d.rf_phase
        cfg.weight, cfg.C_delta = d.weight, d.C_delta
        for s in range(3):
            cfg.T0_eV[s] = d.T0_eV[s]
            cfg.ecap_eV[s] = d.ecap_eV[s]
            cfg.n_init[s] = int(d.n_init[s])
        cfg.numax_safety = d.numax_safety
        cfg.eedf_emax, cfg.iedf_emax, cfg.fm_emax = d.eedf_emax, d.iedf_emax, d.fm_emax
        cfg.seed = d.seed
        cfg.n_cells, cfg.n1, cfg.sort_interval = d.n_cells, d.n1, d.sort_interval
        cfg.diag_every = d.diag_every
        cfg.eedf_bins, cfg.iedf_bins, cfg.fm_bins = d.eedf_bins, d.iedf_bins, d.fm_bins
        cfg.fm_xbins = d.fm_xbins
        cfg.discharge = discharge
        cfg.cx_isotropic = int(d.cx_isotropic)
        cfg.numax_bins = int(d.numax_bins)
        cfg.n2 = int(d.n2)
        cfg.coulomb_log = float(d.coulomb_log)
        cfg.gas_scheme = int(d.gas_scheme)
        cfg.ion_subcycle = int(d.ion_subcycle)
        cfg.coulomb_inter = int(d.coulomb_inter)
        self._keep = []
        xs = (_Xs * len(tables))()
        for i, t in enumerate(tables):
            E = np.ascontiguousarray(t["E_eV"], dtype=np.float64)
            S = np.ascontiguousarray(t["sigma_m2"], dtype=np.float64)
            self._keep += [E, S]
            xs[i].reaction, xs[i].sub, xs[i].n = t["reaction"], t.get("sub", 0), len(E)
            xs[i].E_eV, xs[i].sigma_m2 = _dp(E), _dp(S)
            xs[i].threshold_eV = t.get("threshold_eV", 0.0)
        self.tables = tables
        self.h = lib().orc_create(C.byref(cfg), xs, len(tables), 1 if load else 0)
        self.N = d.n_cells

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            lib().orc_destroy(h)
            self.h = None

    def step(self, n=1):
        lib().orc_step(self.h, int(n))

    @property
    def step_index(self):
        return lib().orc_step_index(self.h)

    @property
    def particle_steps(self):
        return lib().orc_particle_steps(self.h)

    def set_step(self, k):
        lib().orc_set_step(self.h, int(k))

    def count(self, s):
        return lib().orc_count(self.h, s)

    def numax(self, s):
        return lib().orc_numax(self.h, s)

    def coulomb_pair(self, s, v1, v2, n, tau, xi, r):
        a = np.ascontiguousarray(v1, dtype=np.float64).copy()
        b = np.ascontiguousarray(v2, dtype=np.float64).copy()
        lib().orc_coulomb_pair(self.h, s, _dp(a), _dp(b), float(n), float(tau), float(xi), float(r))
        return a, b

    def coulomb_cell(self, s, vx, vy, vz, dens, tau, step, cell):
        """the Coulomb collisions of one cell's particles; returns new copies"""
        a = [np.ascontiguousarray(v, dtype=np.float64).copy() for v in (vx, vy, vz)]
        lib().orc_coulomb_cell(self.h, s, _dp(a[0]), _dp(a[1]), _dp(a[2]), len(a[0]),
                               float(dens), float(tau), int(step), int(cell))
        return a

    def coulomb_pair2(self, sa, sb, v1, v2, n, tau, xi, r):
        a = np.ascontiguousarray(v1, dtype=np.float64).copy()
        b = np.ascontiguousarray(v2, dtype=np.float64).copy()
        lib().orc_coulomb_pair2(self.h, sa, sb, _dp(a), _dp(b), float(n), float(tau), float(xi), float(r))
        return a, b

    def coulomb_inter_pairing(self, pair, nA, nB, step, cell):
        ia = np.zeros(nA, dtype=np.int64)
        ib = np.zeros(nA, dtype=np.int64)
        lib().orc_coulomb_inter_pairing(self.h, pair, int(nA), int(nB), int(step), int(cell),
                                        ia.ctypes.data_as(C.c_void_p), ib.ctypes.data_as(C.c_void_p))
        return ia, ib

    def coulomb_pairing(self, s, n, step, cell):
        """partners of each Coulomb collision of a cell of n particles"""
        pi = np.zeros(n // 2 + 2, dtype=np.int64)
        pj = np.zeros(n // 2 + 2, dtype=np.int64)
        k = lib().orc_coulomb_pairing(self.h, s, int(n), int(step), int(cell), _dp(pi), _dp(pj))
        return pi[:k], pj[:k]

    def numax_bin(self, b):
        return lib().orc_numax_bin(self.h, b)

    def bin_of(self, K_eV):
        return lib().orc_bin_of(self.h, float(K_eV))

    def get(self, s):
        n = self.count(s)
        x, vx, vy, vz = (np.zeros(n) for _ in range(4))
        alive = np.zeros(n, dtype=np.int32)
        lib().orc_get(self.h, s, _dp(x), _dp(vx), _dp(vy), _dp(vz),
                      alive.ctypes.data_as(C.POINTER(C.c_int)))
        return {"x": x, "vx": vx, "vy": vy, "vz": vz, "alive": alive.astype(bool)}

    def set(self, s, x, vx, vy, vz, alive=None):
        x, vx, vy, vz = (np.ascontiguousarray(a, dtype=np.float64) for a in (x, vx, vy, vz))
        al = np.ones(len(x), dtype=np.int32) if alive is None else \
            np.ascontiguousarray(alive, dtype=np.int32)
        lib().orc_set(self.h, s, len(x), _dp(x), _dp(vx), _dp(vy), _dp(vz),
                      al.ctypes.data_as(C.POINTER(C.c_int)))

    def fields(self):
        rho, phi, E = (np.zeros(self.N + 1) for _ in range(3))
        lib().orc_fields(self.h, _dp(rho), _dp(phi), _dp(E))
        return rho, phi, E

    def counters(self):
        ab = np.zeros(6, dtype=np.int64)
        ev = np.zeros(20, dtype=np.int64)
        vi = np.zeros(3, dtype=np.int64)
        bi = np.zeros(3, dtype=np.int64)
        lp = lambda a: a.ctypes.data_as(C.POINTER(C.c_longlong))
        lib().orc_counters(self.h, lp(ab), lp(ev), lp(vi), lp(bi))
        return {"absorbed": ab.reshape(3, 2), "events": ev, "violations": vi, "births": bi,
                "eq1_evaluations": int(lib().orc_eq1_evaluations(self.h))}

    def reset_diag(self):
        lib().orc_reset_diag(self.h)

    def diag(self):
        d, N = self.d, self.N
        dens = np.zeros((3, N + 1))
        phi = np.zeros(N + 1)
        eedf = np.zeros(max(d.eedf_bins, 1), dtype=np.int64)
        iedf = np.zeros((2, max(d.iedf_bins, 1)), dtype=np.int64)
        fm = np.zeros((max(d.fm_xbins, 1), max(d.fm_bins, 1)), dtype=np.int64)
        lp = lambda a: a.ctypes.data_as(C.POINTER(C.c_longlong))
        ns = lib().orc_diag(self.h, _dp(dens), _dp(phi), lp(eedf), lp(iedf), lp(fm))
        return {"n_samples": ns, "dens_sum": dens, "phi_sum": phi, "eedf": eedf,
                "iedf": iedf, "fm": fm}

    def sigma(self, table, E):
        return lib().orc_sigma(self.h, table, float(E))

    def gas_event(self, s, table, v, V, r4, r2=(0.5, 0.5)):
        reaction = self.tables[table]["reaction"]
        v = np.asarray(v, dtype=np.float64)
        V = np.asarray(V, dtype=np.float64)
        r4 = np.asarray(r4, dtype=np.float64)
        r2 = np.asarray(r2, dtype=np.float64)
        vo = np.zeros(3)
        Vo = np.zeros(3)
        pv = np.zeros(6)
        alive = C.c_int()
        psp = (C.c_int * 2)()
        n = lib().orc_gas_event(self.h, s, reaction, table, _dp(v), _dp(V), _dp(r4), _dp(r2),
                                _dp(vo), C.byref(alive), psp, _dp(pv), _dp(Vo))
        prods = [(psp[k], pv[3 * k:3 * k + 3].copy()) for k in range(n)]
        return vo, bool(alive.value), prods, Vo

    def pair19_event(self, table, v, vt, rc, r2):
        v, vt, rc, r2 = (np.asarray(a, dtype=np.float64) for a in (v, vt, rc, r2))
        v1, v2, Vo = np.zeros(3), np.zeros(3), np.zeros(3)
        lib().orc_pair19_event(self.h, table, _dp(v), _dp(vt), _dp(rc), _dp(r2),
                               _dp(v1), _dp(v2), _dp(Vo))
        return v1, v2, Vo
