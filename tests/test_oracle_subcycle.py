"""Pins of the oracle's ion sub-cycling (not in the paper: a throughput
variant in which O- and O2+ are pushed, and tested for gas collisions, only
on steps n = 0 mod k, over k dt): the uniform-field leapfrog with step k dt
against its closed form, the ions resting in between, and the null-collision
real-event fraction 1 - exp(-n sigma v k dt) per ion push.  CPU only."""
import math

import numpy as np

import oracle
from paper_0705_0495_gb300 import inputs

QE = 1.602176634e-19
AMU = 1.66053906660e-27
ME = 9.1093837015e-31
KB = 1.380649e-23
M_O2 = 32 * AMU
MASS = (ME, 16 * AMU + ME, 32 * AMU - ME)


def _disch(**kw):
    base = dict(L=1.0, n_cells=128, p_Pa=20.0, U_rf=0.0, n_op=0, n0_m3=0.0,
                weight_override=0.0, n1=0, sort_interval=0, diag_every=0,
                T0_eV=(0.0, 0.0, 0.0), dt_override=1e-10)
    base.update(kw)
    return inputs.Discharge(**base)


def test_subcycled_ions_follow_the_leapfrog_of_step_k_dt():
    # E = U/L everywhere (no space charge, f = 0, phase pi/2); electrons every
    # step, O2+ every k = 4 steps over 4 dt: after 30 steps the ions have made
    # 8 pushes (steps 0, 4, ..., 28) of 4 dt each
    U, k = 30.0, 4
    d = _disch(L=0.05, U_rf=U, f_rf=0.0, rf_phase=math.pi / 2, dt_override=2e-11, ion_subcycle=k)
    o = oracle.Oracle(d, [])
    n = 200
    rs = np.random.default_rng(9)
    x0 = rs.uniform(0.02, 0.03, n)
    vh = rs.normal(0, 1e4, n)
    o.set(2, x0, vh, np.zeros(n), np.zeros(n))
    o.set(0, x0, vh * 10, np.zeros(n), np.zeros(n))
    o.set(1, [], [], [], [])
    seen = []
    for step in range(30):
        o.step(1)
        seen.append(o.get(2)["x"].copy())
    for q in range(1, 30):
        moved = not np.array_equal(seen[q], seen[q - 1])
        assert moved == (q % k == 0), q  # pushed in the step that starts at q
    for s, v, pushes, h in ((2, vh, 8, k * d.dt), (0, vh * 10, 30, d.dt)):
        a = (1.0 if s == 2 else -1.0) * QE * U / (d.L * MASS[s])
        st = o.get(s)
        xn = x0 + pushes * v * h + a * h**2 * pushes * (pushes + 1) / 2
        vn = v + pushes * a * h
        m = st["alive"]
        assert m.sum() > n // 2
        assert np.max(np.abs(st["x"][m] - xn[m])) < 1e-9 * d.L
        assert np.max(np.abs(st["vx"][m] - vn[m])) < 1e-9 * np.max(np.abs(vn))


def test_subcycled_ion_null_collision_fraction():
    # flat charge-exchange cross section for O2+ at rest: per push over k dt
    # the real-event fraction is (1 - exp(-nu_max k dt)) nu / nu_max
    sig, k, n = 1e-18, 5, 100000
    E = inputs.geometric_grid(*inputs.E_GRID_ION)
    tab = dict(reaction=6, sub=0, E_eV=E, sigma_m2=np.full_like(E, sig), threshold_eV=0.0)
    d = _disch(ion_subcycle=k, dt_override=2e-9, ecap_override=1.0)
    o = oracle.Oracle(d, [tab])
    rs = np.random.default_rng(4)
    o.set(2, np.full(n, 0.5), np.zeros(n), np.zeros(n), np.zeros(n))
    o.set(0, [], [], [], [])
    o.set(1, [], [], [], [])
    o.step(1)
    ev = o.counters()["events"][6]
    o.step(k - 1)
    assert o.counters()["events"][6] == ev  # no test between pushes
    # the relative speed is the gas molecule's: nu = n sigma <u> with <u> the
    # mean speed of the 300 K Maxwellian of O2 (the ion is at rest)
    ngas = d.p_Pa / (KB * d.T_gas)
    ubar = math.sqrt(8 * KB * d.T_gas / (math.pi * M_O2))
    numax = o.numax(2)
    pnull = 1 - math.exp(-numax * k * d.dt)
    p = pnull * ngas * sig * ubar / numax
    assert 0.01 < p < 0.5
    assert abs(ev - n * p) < 4 * math.sqrt(n * p * (1 - p)), (ev, n * p)
