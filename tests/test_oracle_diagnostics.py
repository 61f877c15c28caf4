"""Pins of the oracle's diagnostics (densities, potential, EEDF, IEDF and
f_-(E, x) of Sec. IV) against particles placed by hand.

Each case places a few superparticles whose bins, nodes and sample times
follow from the definitions alone: the EEDF counts electrons of the cell
holding L/2 by kinetic energy; the IEDF counts O2+ by kinetic energy at the
electrode they cross (row 0: x = 0, row 1: x = L); f_-(E, x) counts O- by
region of the gap and signed x energy sign(vx) M vx^2 / 2; the density sums
add the cloud-in-cell densities (boundary nodes with half a cell of volume)
and the potential sums add Phi at every sampled step, the steps n with
n mod diag_every = 0 (reading R15: after the free flight, before
collisions).  A wrong bin scale, energy, sign, region, wall, node volume or
sample step moves a count or a sum.  Runs on the CPU only.
"""
import math

import numpy as np
import pytest

import oracle
from paper_0705_0495_gb300 import inputs

QE = 1.602176634e-19
ME = 9.1093837015e-31
AMU = 1.66053906660e-27
M_OM = 16 * AMU + ME
M_OP = 32 * AMU - ME


def _disch(**kw):
    base = dict(L=0.064, n_cells=64, p_Pa=20.0, U_rf=0.0, n_op=0, n0_m3=0.0,
                weight_override=0.0, n1=0, sort_interval=0, diag_every=1,
                T0_eV=(0.0, 0.0, 0.0), dt_override=1e-12)
    base.update(kw)
    return inputs.Discharge(**base)


def _speed(E_eV, m):
    return math.sqrt(2.0 * E_eV * QE / m)


def _empty(o, keep):
    for s in range(3):
        if s not in keep:
            o.set(s, [], [], [], [])


def test_eedf_counts_electrons_of_the_middle_cell_by_energy():
    d = _disch(eedf_bins=50, eedf_emax=50.0)
    dx = d.L / d.n_cells
    o = oracle.Oracle(d, [])
    rs = np.random.default_rng(3)
    E_in = [0.5, 3.2, 3.7, 10.1, 49.6, 60.0]          # the last is beyond the range
    x, v = [], []
    for E in E_in:
        n = rs.normal(size=3)
        v.append(_speed(E, ME) * n / np.linalg.norm(n))
        x.append(32.5 * dx)                             # cell N/2 holds L/2
    for c in (31.5, 33.5):                              # neighbouring cells: not counted
        x.append(c * dx)
        v.append(np.array([_speed(7.5, ME), 0.0, 0.0]))
    v = np.array(v)
    o.set(0, x, v[:, 0], v[:, 1], v[:, 2])
    _empty(o, [0])
    o.step(1)
    g = o.diag()
    assert g["n_samples"] == 1
    expect = np.zeros(50, dtype=np.int64)
    for E in E_in:
        if E < 50.0:
            expect[int(E)] += 1
    assert np.array_equal(g["eedf"], expect)


def test_iedf_counts_ions_at_the_electrode_they_cross():
    d = _disch(iedf_bins=100, iedf_emax=100.0, dt_override=1e-9)
    L = d.L
    o = oracle.Oracle(d, [])
    hits = [(1, 5.3), (1, 12.7), (1, 12.2), (0, 40.2), (0, 99.5), (0, 150.0)]
    x, v = [], []
    for wall, E in hits:
        s = _speed(E, M_OP)
        # 0.8 of the speed across the gap, 0.6 along the electrode: the
        # histogram takes the whole kinetic energy
        if wall == 1:
            x.append(L - 1e-8)
            v.append([0.8 * s, 0.6 * s, 0.0])
        else:
            x.append(1e-8)
            v.append([-0.8 * s, 0.0, 0.6 * s])
    x.append(L / 2)                                     # stays inside: not counted
    v.append([_speed(3.0, M_OP), 0.0, 0.0])
    v = np.array(v)
    o.set(2, x, v[:, 0], v[:, 1], v[:, 2])
    _empty(o, [2])
    o.step(1)
    g = o.diag()
    expect = np.zeros((2, 100), dtype=np.int64)
    for wall, E in hits:
        if E < 100.0:
            expect[wall, int(E)] += 1
    assert np.array_equal(g["iedf"], expect)
    assert o.counters()["absorbed"][2].tolist() == [3, 3]


def test_f_minus_counts_o_minus_by_region_and_signed_x_energy():
    d = _disch(fm_bins=20, fm_xbins=4, fm_emax=10.0)
    dx = d.L / d.n_cells
    o = oracle.Oracle(d, [])
    # (cell, signed x energy [eV]); vy, vz large and ignored
    cases = [(3, -7.5), (3, -0.3), (17, 0.4), (40, 3.6), (63, 9.9), (63, -9.9), (20, 12.0)]
    x, v = [], []
    for c, Es in cases:
        x.append((c + 0.5) * dx)
        vx = math.copysign(_speed(abs(Es), M_OM), Es)
        v.append([vx, 3e3, -4e3])
    v = np.array(v)
    o.set(1, x, v[:, 0], v[:, 1], v[:, 2])
    _empty(o, [1])
    o.step(1)
    g = o.diag()
    expect = np.zeros((4, 20), dtype=np.int64)
    for c, Es in cases:
        if abs(Es) < 10.0:
            expect[c * 4 // 64, int(math.floor(Es + 10.0))] += 1
    assert np.array_equal(g["fm"], expect)


def test_density_sums_use_cloud_in_cell_weights_and_half_boundary_volumes():
    w = 1e3  # real particles per m^2 per superparticle: fields far too weak to move anyone
    d = _disch(weight_override=w, diag_every=1)
    N = d.n_cells
    dx = d.L / N
    o = oracle.Oracle(d, [])
    # O2+: three on node 5, two on node 0 (a boundary node); O-: one at a
    # quarter of cell 7; electrons: one at the middle of the last cell
    o.set(2, [5 * dx] * 3 + [0.0] * 2, [0.0] * 5, [0.0] * 5, [0.0] * 5)
    o.set(1, [7.25 * dx], [0.0], [0.0], [0.0])
    o.set(0, [(N - 0.5) * dx], [0.0], [0.0], [0.0])
    o.step(1)
    g = o.diag()
    dens = g["dens_sum"]
    exp = np.zeros((3, N + 1))
    exp[2, 5] = 3 * w / dx
    exp[2, 0] = 2 * w / (dx / 2)
    exp[1, 7] = 0.75 * w / dx
    exp[1, 8] = 0.25 * w / dx
    exp[0, N - 1] = 0.5 * w / dx
    exp[0, N] = 0.5 * w / (dx / 2)
    assert np.allclose(dens, exp, rtol=1e-12, atol=0.0)
    assert g["n_samples"] == 1


def test_potential_sums_sample_every_diag_every_steps():
    # no charge: Phi(x, t_n) = U sin(2 pi f t_n + phase) (1 - x/L); five steps
    # with diag_every = 2 sample steps 0, 2 and 4
    U, f, ph = 100.0, 13.56e6, 0.3
    dt = 1.0 / (f * 50)
    d = _disch(U_rf=U, f_rf=f, rf_phase=ph, dt_override=dt, diag_every=2)
    N = d.n_cells
    o = oracle.Oracle(d, [])
    _empty(o, [])
    o.step(5)
    g = o.diag()
    assert g["n_samples"] == 3
    xi = np.arange(N + 1) / N
    expect = sum(U * math.sin(2 * math.pi * f * n * dt + ph) for n in (0, 2, 4)) * (1 - xi)
    assert np.allclose(g["phi_sum"], expect, rtol=0.0, atol=1e-9 * U)
    assert np.all(g["dens_sum"] == 0.0)
