"""Seeded synthetic inputs: discharge configurations and cross-section tables.

This module is the only thing the GPU library and the CPU oracle have in
common: both are fed from here.  It holds input specification only -- none of
the arithmetic of the time step.

Discharges mirror the operating range of Bronold et al. (Sec. II: planar gap,
13.56 MHz, 10-100 Pa, 75-800 V; Sec. IV: L = 2.5 cm).  Cross sections: the
paper's closed forms are used where it prints them -- Eq. 4 (O- + O2 elastic),
Eq. 8 (O- + O2+ neutralisation), Eq. 9 (associative detachment), Eq. 3 with
Eq. 6's B = 3 for the constructions of (6) and (13) -- and every other curve is
a smooth PLACEHOLDER chosen here, because the paper's measured curves are only
figures.  Placeholders keep the paper's stated thresholds (6.4 eV for (9),
8.6 eV for (10), about 1.3 eV for (16), zero below 4 eV for (15)); the other
thresholds are placeholders too.  Real tables can be passed through the same
interface.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List

import numpy as np

KB_EV = 8.617333262e-5  # Boltzmann constant in eV/K, for the 300 K ion load

# --------------------------------------------------------------- tables

E_GRID_E = (1e-3, 1e3, 241)    # electron-O2 and electron-ion pairs
E_GRID_ION = (1e-4, 1e3, 281)  # ion-O2 and ion-ion pairs


def geometric_grid(lo, hi, n):
    """Nodes E_k = lo (hi/lo)^(k/(n-1)), k = 0..n-1."""
    k = np.arange(n, dtype=np.float64)
    E = lo * (hi / lo) ** (k / (n - 1))
    E[0], E[-1] = lo, hi
    return E


def _ramp(E, th):
    return np.where(E >= th, 1.0 - th / np.maximum(E, th), 0.0)


def sigma_eq4(E):
    """Eq. 4, O- + O2 elastic (polarisation model, n = 3), in m^2."""
    n, C, s0 = 3.0, 3.77e-24, 1.2e-15
    return (n * math.pi / (n - 2.0) * ((n - 2.0) / 2.0 * C / E) ** (2.0 / n) + s0) * 1e-4


def sigma_eq8(E):
    """Eq. 8, O- + O2+ neutralisation, in m^2."""
    return 0.8 * (1.0 + 2.85 / E) * 1e-14 * 1e-4


def sigma_eq9(E):
    """Eq. 9, associative detachment on O2(a), in m^2."""
    return 5.96e-16 / np.sqrt(E) * 1e-4


def _sigma_m_placeholder(E):
    """Placeholder O2+ + O2 momentum-transfer cross section (m^2)."""
    return 1e-19 * (4.0 + 3.0 / np.sqrt(E))


def sigma_cx(E):
    """(6) built as in Sec. III A: sigma_cx = sigma_m / 2 (Eq. 3) below 0.251 eV
    and above 8.5 eV, linear in E in between (sigma_m is a placeholder)."""
    lo, hi = 0.251, 8.5
    base = 0.5 * _sigma_m_placeholder(E)
    s_lo = 0.5 * _sigma_m_placeholder(lo)
    s_hi = 0.5 * _sigma_m_placeholder(hi)
    mid = s_lo + (E - lo) / (hi - lo) * (s_hi - s_lo)
    return np.where((E > lo) & (E < hi), mid, base)


def sigma_dr(E, B=3.0):
    """(13) sigma_dr = B sigma_0 (Eq. 6) with B = 3; sigma_0 is a placeholder."""
    return B * 2e-21 / (E + 1e-3)


# placeholder electron-O2 channels: (reaction, sub, threshold eV, shape)
_E_O2 = [
    (4, 0, 0.0, lambda E: 1e-20 * (4.0 + 6.0 * E / (E + 5.0))),
    (7, 1, 0.19, None), (7, 2, 0.38, None), (7, 3, 0.57, None), (7, 4, 0.75, None),
    (8, 0, 8.0, lambda E: 4e-21 * _ramp(E, 8.0) / (1.0 + E / 150.0)),
    (9, 0, 6.4, lambda E: 9e-21 * _ramp(E, 6.4) / (1.0 + E / 100.0)),
    (10, 0, 8.6, lambda E: 1.2e-20 * _ramp(E, 8.6) / (1.0 + E / 100.0)),
    (11, 0, 0.98, lambda E: 1.5e-22 * _ramp(E, 0.98) / (1.0 + (E / 8.0) ** 2)),
    (12, 0, 1.63, lambda E: 4e-23 * _ramp(E, 1.63) / (1.0 + (E / 10.0) ** 2)),
    (15, 0, 4.0, lambda E: np.where(E >= 4.0, 1.4e-22 * np.exp(-((E - 6.5) / 1.5) ** 2), 0.0)),
    (18, 0, 12.06, lambda E: np.where(E > 12.06, 6e-20 * np.log(np.maximum(E, 12.06) / 12.06)
                                      / (np.maximum(E, 12.06) / 12.06), 0.0)),
]

_VIB_AMP = {1: 1.2e-21, 2: 6e-22, 3: 3e-22, 4: 1.5e-22}


def _vib(E, th, amp):
    x = np.maximum(E - th, 0.0) / 0.3
    return np.where(E >= th, amp * x * np.exp(1.0 - x), 0.0)


def xs_tables(B=3.0) -> List[dict]:
    """The synthetic cross-section set, in the channel order the walk uses.

    Gas channels of one projectile share one energy grid; each table is a
    dict(reaction, sub, E_eV, sigma_m2, threshold_eV, placeholder)."""
    Ee = geometric_grid(*E_GRID_E)
    Ei = geometric_grid(*E_GRID_ION)
    out = []
    for r, sub, th, f in _E_O2:
        s = _vib(Ee, th, _VIB_AMP[sub]) if r == 7 else f(Ee)
        s = np.where(Ee >= th, s, 0.0)
        out.append(dict(reaction=r, sub=sub, E_eV=Ee.copy(), sigma_m2=np.asarray(s, float),
                        threshold_eV=th, placeholder=True))
    out.append(dict(reaction=5, sub=0, E_eV=Ei.copy(), sigma_m2=sigma_eq4(Ei),
                    threshold_eV=0.0, placeholder=False))
    out.append(dict(reaction=16, sub=0, E_eV=Ei.copy(),
                    sigma_m2=4e-20 * _ramp(Ei, 1.3) / (1.0 + Ei / 200.0),
                    threshold_eV=1.3, placeholder=True))
    out.append(dict(reaction=17, sub=0, E_eV=Ei.copy(), sigma_m2=sigma_eq9(Ei),
                    threshold_eV=0.0, placeholder=False))
    out.append(dict(reaction=6, sub=0, E_eV=Ei.copy(), sigma_m2=sigma_cx(Ei),
                    threshold_eV=0.0, placeholder=True))
    out.append(dict(reaction=13, sub=0, E_eV=Ee.copy(), sigma_m2=sigma_dr(Ee, B),
                    threshold_eV=0.0, placeholder=True))
    out.append(dict(reaction=14, sub=0, E_eV=Ei.copy(), sigma_m2=sigma_eq8(Ei),
                    threshold_eV=0.0, placeholder=False))
    out.append(dict(reaction=19, sub=0, E_eV=Ee.copy(),
                    sigma_m2=1.5e-19 * _ramp(Ee, 1.46) / (1.0 + Ee / 50.0),
                    threshold_eV=1.46, placeholder=True))
    return out


# ------------------------------------------------------------ discharges

T_ION_EV = KB_EV * 300.0


@dataclasses.dataclass
class Discharge:
    """One capacitively coupled discharge: geometry, drive, gas, load."""
    L: float = 0.025
    n_cells: int = 128
    p_Pa: float = 20.0
    T_gas: float = 300.0
    U_rf: float = 100.0
    f_rf: float = 13.56e6
    rf_phase: float = 0.0           # U(t) = U_rf sin(2 pi f t + rf_phase)
    dt_override: float = 0.0        # > 0: time step in s instead of T_rf/steps_per_cycle
    steps_per_cycle: int = 1000
    n0_m3: float = 1e15             # O2+ density of the quasi-neutral load
    n_op: int = 20000               # O2+ superparticles; e and O- get half each
    T0_eV: tuple = (3.0, T_ION_EV, T_ION_EV)
    C_delta: float = 1.0 / 6.0      # Sec. IV fit value
    n1: int = 10
    sort_interval: int = 10
    seed: int = 1
    diag_every: int = 10
    eedf_bins: int = 200
    eedf_emax: float = 100.0
    iedf_bins: int = 200
    iedf_emax: float = 0.0          # 0 -> 2 U_rf
    fm_bins: int = 64
    fm_xbins: int = 64
    fm_emax: float = 4.0
    numax_safety: float = 1.0       # the bound is strict by construction (piecewise over the tables)
    numax_bins: int = 64            # electrons: bounds per quarter octave of lab energy
    n2: int = 0                     # intra-species Coulomb collisions every n2 steps (0: none)
    coulomb_log: float = 10.0       # ln Gamma of Eq. 2 (not given in the paper)
    gas_scheme: int = 0             # gas targets: 0 null collision, 1 sequential test every n1 steps
    ion_subcycle: int = 1           # k > 1: ions pushed every k steps with k dt
    coulomb_inter: bool = False     # inter-species Coulomb collisions as well (with n2 > 0)
    cx_isotropic: bool = False
    capacity_factor: float = 1.5
    capacity_extra: int = 4096
    fp64: bool = True
    weight_override: float = None
    ecap_override: float = 0.0
    rf_cycles: float = 2.0

    def __post_init__(self):
        if self.iedf_emax <= 0.0:
            self.iedf_emax = 2.0 * self.U_rf

    @property
    def dt(self):
        if self.dt_override > 0.0:
            return self.dt_override
        return 1.0 / (self.f_rf * self.steps_per_cycle)

    @property
    def n_init(self):
        ne = self.n_op // 2
        return (ne, self.n_op - ne, self.n_op)

    @property
    def weight(self):
        """Real particles per m^2 of electrode per superparticle (the paper's
        lateral area A enters only through this number, Sec. II)."""
        if self.weight_override is not None:
            return self.weight_override
        return self.n0_m3 * self.L / self.n_op if self.n_op > 0 else 0.0

    @property
    def ecap_eV(self):
        cap = self.ecap_override if self.ecap_override > 0.0 else 3.0 * self.U_rf + 50.0
        return (cap, cap, cap)

    @property
    def capacity(self):
        return tuple(int(self.capacity_factor * n) + self.capacity_extra for n in self.n_init)

    @property
    def total_steps(self):
        return int(round(self.rf_cycles * self.steps_per_cycle))


def cfg1(**kw) -> Discharge:
    """Plain FP64 single discharge: 2.5 cm, 128 cells, 20 Pa, 100 V, dt = T/1000,
    n0 = 1e15 m^-3, 10k e + 10k O- + 20k O2+, seed 1, 2 RF cycles."""
    d = dict(L=0.025, n_cells=128, p_Pa=20.0, U_rf=100.0, steps_per_cycle=1000,
             n0_m3=1e15, n_op=20000, seed=1, fp64=True, rf_cycles=2.0)
    d.update(kw)
    return Discharge(**d)


def cfg2(**kw) -> Discharge:
    """FP32 single discharge: 4 cm, 512 cells, 10 Pa, 300 V, dt = T/3000,
    n0 = 1e16 m^-3, 1e6 e + 1e6 O- + 2e6 O2+, 200 RF cycles."""
    d = dict(L=0.04, n_cells=512, p_Pa=10.0, U_rf=300.0, steps_per_cycle=3000,
             n0_m3=1e16, n_op=2_000_000, seed=1, fp64=False, rf_cycles=200.0)
    d.update(kw)
    return Discharge(**d)


def cfg4(**kw) -> Discharge:
    """Large FP32 discharge for the HBM roofline: 4 cm, 4096 cells, 20 Pa,
    400 V, dt = T/4000, 5e7 superparticles (1.25e7 e, 1.25e7 O-, 2.5e7 O2+),
    20 RF cycles."""
    d = dict(L=0.04, n_cells=4096, p_Pa=20.0, U_rf=400.0, steps_per_cycle=4000,
             n0_m3=1e16, n_op=25_000_000, seed=1, fp64=False, rf_cycles=20.0,
             capacity_factor=1.25)
    d.update(kw)
    return Discharge(**d)


def cfg5(seed=1, fp64=True, **kw) -> Discharge:
    """Long-horizon run: cfg1 for 1000 RF cycles, with room for the densities
    to grow sixteenfold."""
    kw.setdefault("capacity_factor", 16.0)
    return cfg1(seed=seed, fp64=fp64, rf_cycles=1000.0, **kw)


def cfg3_sweep(total=30_000_000, seed=1, **kw) -> List[Discharge]:
    """64 discharges on an 8x8 grid: V_i = 100 + 500 i/7 V, p_j = 5 + 45 j/7 Pa,
    L_ij = 2.5 + 1.5 (i+j)/14 cm, 256 cells below 3.25 cm else 512, dt = T/2000,
    n0 = 1e16 m^-3, O2+ populations log-uniform in [1e4, 2e6] from a seeded
    generator, rescaled so that all species add up to about ``total``."""
    rs = np.random.default_rng(seed)
    logs = rs.uniform(np.log(1e4), np.log(2e6), size=64)
    pops = np.exp(logs)
    pops *= (total / 2.0) / pops.sum()   # O2+ is half of each discharge's particles
    out = []
    for i in range(8):
        for j in range(8):
            L = (2.5 + 1.5 * (i + j) / 14.0) * 1e-2
            n_op = max(2, int(round(pops[8 * i + j])) & ~1)
            d = dict(L=L, n_cells=256 if L < 0.0325 else 512, p_Pa=5.0 + 45.0 * j / 7.0,
                     U_rf=100.0 + 500.0 * i / 7.0, steps_per_cycle=2000, n0_m3=1e16,
                     n_op=n_op, seed=seed, fp64=False, rf_cycles=50.0)
            d.update(kw)
            out.append(Discharge(**d))
    return out


SWEEP_13P8_VOLTS = (75.0, 100.0, 150.0, 200.0, 250.0, 300.0)


def sweep_13p8(n_op=20000, seed=1, fp64=False, rf_cycles=1000.0, **kw) -> List[Discharge]:
    """The voltage sweep of Sec. IV (Fig. Central): L = 2.5 cm, p = 13.8 Pa,
    f = 13.6 MHz, U = 75-300 V with C = 1/6, plus the discharge of Fig.
    Profiles at 150 V without associative detachment (C = 0); 128 cells,
    dt = T/1000, intra-species Coulomb collisions every 10 steps (kept in all
    of the paper's runs), load n0 = 1e15 m^-3 with n_op O2+ superparticles and
    room for the densities to grow sixteenfold."""
    base = dict(L=0.025, n_cells=128, p_Pa=13.8, f_rf=13.6e6, steps_per_cycle=1000, n0_m3=1e15,
                n_op=n_op, seed=seed, fp64=fp64, rf_cycles=rf_cycles, n2=10, capacity_factor=16.0)
    base.update(kw)
    out = [Discharge(U_rf=u, **base) for u in SWEEP_13P8_VOLTS]
    out.append(Discharge(U_rf=150.0, **dict(base, C_delta=0.0)))
    return out


WORKLOADS = {"cfg1": cfg1, "cfg2": cfg2, "cfg4": cfg4, "cfg5": cfg5}
