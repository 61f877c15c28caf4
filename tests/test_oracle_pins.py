"""Pins of the FP64 CPU oracle against what the paper and mathematics fix.

Each test checks the oracle against something other than itself: a second
Philox4x32-10 implementation, closed forms printed in the paper (Eqs. 4, 8, 9),
exact solutions of the discrete field equations, leapfrog trajectories,
the cold-plasma dispersion relation, conservation laws of each reaction of
Table I, the collision-rate algebra of the null-collision method and of
Eq. 1, and a library solver.  Runs on the CPU only.
"""
import math
import os

import numpy as np
import pytest
from scipy import stats

import oracle
from paper_0705_0495_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

QE = 1.602176634e-19
ME = 9.1093837015e-31
AMU = 1.66053906660e-27
KB = 1.380649e-23
EPS0 = 8.8541878128e-12
M_O = 16 * AMU
M_O2 = 32 * AMU
M_OM = M_O + ME
M_OP = M_O2 - ME
MASS = (ME, M_OM, M_OP)


def _disch(**kw):
    base = dict(L=1.0, n_cells=128, p_Pa=20.0, U_rf=0.0, n_op=0, n0_m3=0.0,
                weight_override=0.0, n1=0, sort_interval=0, diag_every=0,
                T0_eV=(0.0, 0.0, 0.0), dt_override=1e-10)
    base.update(kw)
    return inputs.Discharge(**base)


def _flat(reaction, sigma, grid=inputs.E_GRID_E, th=0.0):
    E = inputs.geometric_grid(*grid)
    return dict(reaction=reaction, sub=0, E_eV=E, sigma_m2=np.full_like(E, sigma),
                threshold_eV=th)


def _table(reaction):
    return [t for t in inputs.xs_tables() if t["reaction"] == reaction][0]


def _empty_others(o, keep):
    for s in range(3):
        if s not in keep:
            o.set(s, [], [], [], [])


# ------------------------------------------------------------------ RNG

def test_philox_strict_avalanche():
    """Philox4x32-10 (Salmon et al., SC'11) mixes every counter bit into every
    output bit: flipping one input bit flips each output bit with probability
    1/2.  A dropped round, a missing multiply or an unmixed word breaks it."""
    rng = np.random.default_rng(11)
    n = 192
    flips = np.zeros((128, 128))
    for _ in range(n):
        ctr = [int(x) for x in rng.integers(0, 2**32, size=4, dtype=np.uint64)]
        key = [int(x) for x in rng.integers(0, 2**32, size=2, dtype=np.uint64)]
        base = oracle.philox(ctr, key)
        bb = np.array([(base[w] >> b) & 1 for w in range(4) for b in range(32)])
        for ib in range(128):
            c2 = list(ctr)
            c2[ib // 32] ^= 1 << (ib % 32)
            out = oracle.philox(c2, key)
            ob = np.array([(out[w] >> b) & 1 for w in range(4) for b in range(32)])
            flips[ib] += ob != bb
    p = flips / n
    assert abs(p.mean() - 0.5) < 0.01
    assert p.min() > 0.3 and p.max() < 0.7


def test_philox_uniformity_and_independence():
    words = []
    for i in range(4000):
        words += oracle.philox([i, 7, 1 << 28, 0], [1, 0])
    u = (np.array(words, dtype=np.float64) + 0.5) / 2**32
    counts, _ = np.histogram(u, bins=40, range=(0, 1))
    chi2, p = stats.chisquare(counts)
    assert p > 1e-4
    assert abs(np.corrcoef(u[:-1], u[1:])[0, 1]) < 0.03


# A second, independent Philox4x32-10: PyTorch's header-only engine
# (ATen/core/PhiloxRNGEngine.h).  Its key is the 64-bit seed (words 0, 1),
# its counter words 2, 3 the 64-bit subsequence and words 0, 1 the 64-bit
# offset; four calls return the four words of one block.
_PHILOX_REF_SRC = r"""
#include <ATen/core/PhiloxRNGEngine.h>
#include <cstdio>
int main() {
    unsigned c0, c1, c2, c3, k0, k1;
    while (std::scanf("%u %u %u %u %u %u", &c0, &c1, &c2, &c3, &k0, &k1) == 6) {
        const uint64_t seed = (uint64_t)k0 | ((uint64_t)k1 << 32);
        const uint64_t sub = (uint64_t)c2 | ((uint64_t)c3 << 32);
        const uint64_t off = (uint64_t)c0 | ((uint64_t)c1 << 32);
        at::philox_engine e(seed, sub, off);
        const unsigned w0 = e(), w1 = e(), w2 = e(), w3 = e();
        std::printf("%u %u %u %u\n", w0, w1, w2, w3);
    }
    return 0;
}
"""


def test_philox_matches_an_independent_implementation(tmp_path):
    """The oracle's generator is Philox4x32-10 bit for bit: its blocks equal
    those of PyTorch's own engine (written from the same SC'11 definition,
    not from this repository) for random counters and keys, all-zero and
    all-one words and carries across the 32-bit halves."""
    import shutil
    import subprocess

    import torch
    inc = os.path.join(os.path.dirname(torch.__file__), "include")
    if not os.path.exists(os.path.join(inc, "ATen", "core", "PhiloxRNGEngine.h")):
        pytest.skip("PyTorch headers not installed")
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    src = tmp_path / "philox_ref.cpp"
    exe = tmp_path / "philox_ref"
    src.write_text(_PHILOX_REF_SRC)
    subprocess.run([cxx, "-O1", "-std=c++17", "-I", inc, str(src), "-o", str(exe)], check=True,
                   capture_output=True)
    rng = np.random.default_rng(5)
    M = 2**32 - 1
    cases = [([0, 0, 0, 0], [0, 0]), ([M, M, M, M], [M, M]), ([M, 0, M, 0], [0, M]),
             ([0, 0, 0, 0], [M, 0]), ([1, 2, 3, 4], [5, 6])]
    for _ in range(300):
        cases.append(([int(x) for x in rng.integers(0, 2**32, size=4, dtype=np.uint64)],
                      [int(x) for x in rng.integers(0, 2**32, size=2, dtype=np.uint64)]))
    stdin = "".join(" ".join(str(v) for v in c + k) + "\n" for c, k in cases)
    out = subprocess.run([str(exe)], input=stdin, capture_output=True, text=True, check=True).stdout
    ref = [[int(v) for v in line.split()] for line in out.strip().splitlines()]
    assert len(ref) == len(cases)
    for (c, k), r in zip(cases, ref):
        assert list(oracle.philox(c, k)) == r, (c, k)


# ------------------------------------------------------- cross sections

def test_closed_form_cross_sections_in_tables():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "cross_sections.txt"))
            if l.strip() and not l.startswith("#")]
    for r in rows:
        reaction, E, s_cm2 = int(r[0]), float(r[1]), float(r[2])
        t = _table(reaction)
        o = oracle.Oracle(_disch(), [t])
        got = o.sigma(0, E) * 1e4
        assert got == pytest.approx(s_cm2, rel=2e-4), (reaction, E)


def test_sigma_interpolation_rules():
    E = np.array([0.1, 1.0, 10.0, 100.0])
    t = dict(reaction=9, sub=0, E_eV=E, sigma_m2=np.array([0.0, 2.0, 4.0, 1.0]) * 1e-20,
             threshold_eV=0.5)
    o = oracle.Oracle(_disch(), [t])
    assert o.sigma(0, 0.4) == 0.0                    # below threshold
    assert o.sigma(0, 1.0) == pytest.approx(2e-20)   # at a node
    assert o.sigma(0, 5.5) == pytest.approx(3e-20)   # linear in E
    assert o.sigma(0, 1e4) == pytest.approx(1e-20)   # held above the last node (Sec. III)
    t2 = dict(t, threshold_eV=0.0)
    o2 = oracle.Oracle(_disch(), [t2])
    assert o2.sigma(0, 0.01) == 0.0                  # held at the first node value


def test_numax_for_flat_table():
    sig = 1e-19
    d = _disch(ecap_override=40.0)
    o = oracle.Oracle(d, [_flat(4, sig)])
    n = d.p_Pa / (KB * d.T_gas)
    mu = ME * M_O2 / (ME + M_O2)
    expect = d.numax_safety * n * sig * math.sqrt(2 * 40.0 * QE / mu)
    assert o.numax(0) == pytest.approx(expect, rel=1e-12)
    assert o.numax(1) == 0.0 and o.numax(2) == 0.0


# ------------------------------------------------------------ Poisson

def test_poisson_uniform_charge_parabola():
    N, L, rho0, U = 64, 0.01, 1e-3, 50.0
    dx = L / N
    x = np.arange(N + 1) * dx
    rho = np.full(N + 1, rho0)
    phi = oracle.poisson(N, dx, U, 0.0, rho)
    exact = rho0 * x * (L - x) / (2 * EPS0) + U * (1 - x / L)
    assert np.max(np.abs(phi - exact)) < 1e-12 * np.max(np.abs(exact))
    E = oracle.field(N, dx, rho, phi)
    Eex = -rho0 * (L - 2 * x) / (2 * EPS0) + U / L
    assert np.max(np.abs(E - Eex)) < 1e-9 * np.max(np.abs(Eex))


def test_poisson_against_dense_solve():
    rs = np.random.default_rng(3)
    N, L = 200, 0.04
    dx = L / N
    rho = rs.normal(size=N + 1) * 1e-4
    phi = oracle.poisson(N, dx, 123.0, 0.0, rho)
    A = (np.diag(-2.0 * np.ones(N - 1)) + np.diag(np.ones(N - 2), 1)
         + np.diag(np.ones(N - 2), -1))
    b = -rho[1:N] * dx * dx / EPS0
    b[0] -= 123.0
    ref = np.linalg.solve(A, b)
    assert np.max(np.abs(phi[1:N] - ref)) < 1e-11 * np.max(np.abs(ref))


def test_deposit_total_charge():
    d = _disch(n_op=2000, n0_m3=1e15, weight_override=None, T0_eV=(1.0, 0.03, 0.03),
               L=0.02)
    o = oracle.Oracle(d, [])
    rho, _, _ = o.fields()
    N, dx = d.n_cells, d.L / d.n_cells
    vol = np.full(N + 1, dx)
    vol[0] = vol[-1] = dx / 2
    q = QE * d.weight * (d.n_init[2] - d.n_init[0] - d.n_init[1])
    assert np.sum(rho * vol) == pytest.approx(q, abs=1e-9 * QE * d.weight * d.n_op)


# ------------------------------------------------------------- push

def test_free_streaming_and_absorption():
    d = _disch(L=0.01, dt_override=1e-11)
    o = oracle.Oracle(d, [])
    rs = np.random.default_rng(5)
    n = 500
    x0 = rs.uniform(0, d.L, n)
    vx = rs.normal(0, 2e6, n)
    o.set(0, x0, vx, np.zeros(n), np.zeros(n))
    _empty_others(o, [0])
    steps = 40
    o.step(steps)
    st = o.get(0)
    k = np.arange(1, steps + 1)[None, :]
    traj = x0[:, None] + k * vx[:, None] * d.dt
    out = (traj < 0) | (traj >= d.L)
    alive = ~out.any(axis=1)
    assert np.array_equal(st["alive"], alive)
    xe = x0 + steps * vx * d.dt
    assert np.max(np.abs(st["x"][alive] - xe[alive])) < 1e-12 * d.L
    first = np.where(out.any(axis=1), np.argmax(out, axis=1), -1)
    lefts = np.sum((first >= 0) & (traj[np.arange(n), np.maximum(first, 0)] < 0))
    ab = o.counters()["absorbed"]
    assert ab[0, 0] == lefts and ab[0, 1] == np.sum(first >= 0) - lefts


def test_uniform_field_leapfrog_parabola():
    # f = 0 and phase pi/2: the driven electrode sits at U_rf; without space
    # charge the potential is linear and E = U/L everywhere (Sec. II geometry)
    U = 30.0
    d = _disch(L=0.05, U_rf=U, f_rf=0.0, rf_phase=math.pi / 2, dt_override=2e-11)
    o = oracle.Oracle(d, [])
    n = 200
    rs = np.random.default_rng(9)
    x0 = rs.uniform(0.02, 0.03, n)
    vh = rs.normal(0, 1e4, n)
    o.set(2, x0, vh, np.zeros(n), np.zeros(n))   # O2+
    o.set(0, x0, vh * 10, np.zeros(n), np.zeros(n))  # electrons
    o.set(1, [], [], [], [])
    steps = 30
    o.step(steps)
    for s, v in ((2, vh), (0, vh * 10)):
        a = (1.0 if s == 2 else -1.0) * QE * U / (d.L * MASS[s])
        st = o.get(s)
        xn = x0 + steps * v * d.dt + a * d.dt**2 * steps * (steps + 1) / 2
        vn = v + steps * a * d.dt
        m = st["alive"]
        assert m.sum() > n // 2
        assert np.max(np.abs(st["x"][m] - xn[m])) < 1e-9 * d.L
        assert np.max(np.abs(st["vx"][m] - vn[m])) < 1e-9 * np.max(np.abs(vn))


def test_cold_plasma_oscillation_frequency():
    # cold electrons displaced by xi sin(2 pi x / L) over a uniform ion
    # background oscillate at the leapfrog frequency sin(w dt/2) = w_pe dt/2
    N = 128
    L = 0.02
    npart = 64 * N
    n0 = 1e15
    w = n0 * L / npart
    wpe = math.sqrt(n0 * QE**2 / (EPS0 * ME))
    dt = 0.1 / wpe
    d = _disch(L=L, n_cells=N, dt_override=dt, weight_override=w)
    o = oracle.Oracle(d, [])
    xb = (np.arange(npart) + 0.5) * L / npart
    xi = 0.2 * (L / N) * np.sin(2 * np.pi * xb / L)
    z = np.zeros(npart)
    o.set(0, xb + xi, z, z, z)
    o.set(2, xb, z, z, z)
    o.set(1, [], [], [], [])
    mode = np.sin(2 * np.pi * xb / L)
    amp = []
    for k in range(200):
        amp.append(np.sum((o.get(0)["x"] - xb) * mode))
        o.step(1)
    amp = np.array(amp)
    sgn = np.sign(amp)
    idx = np.where(sgn[:-1] * sgn[1:] < 0)[0]
    tz = idx + amp[idx] / (amp[idx] - amp[idx + 1])
    period_steps = 2 * np.mean(np.diff(tz))
    w_num = 2 * np.pi / (period_steps * dt)
    w_exp = 2 / dt * math.asin(wpe * dt / 2)
    assert w_num == pytest.approx(w_exp, rel=0.01)


# ------------------------------------------------------------ gas MCC

def test_null_collision_real_event_fraction():
    sig, E0, cap = 1e-19, 10.0, 40.0
    d = _disch(ecap_override=cap, dt_override=5e-11, numax_bins=0)
    o = oracle.Oracle(d, [_flat(4, sig)])
    n = 200000
    rs = np.random.default_rng(11)
    dirs = rs.normal(size=(n, 3))
    dirs /= np.linalg.norm(dirs, axis=1)[:, None]
    v = math.sqrt(2 * E0 * QE / ME) * dirs
    o.set(0, np.full(n, 0.5), v[:, 0], v[:, 1], v[:, 2])
    _empty_others(o, [0])
    o.step(1)
    ev = o.counters()["events"][4]
    ngas = d.p_Pa / (KB * d.T_gas)
    mu = ME * M_O2 / (ME + M_O2)
    numax = d.numax_safety * ngas * sig * math.sqrt(2 * cap * QE / mu)
    nu = ngas * sig * math.sqrt(2 * E0 * QE / mu)  # gas motion is negligible here
    p = (1 - math.exp(-numax * d.dt)) * nu / numax
    assert abs(ev - n * p) < 4 * math.sqrt(n * p * (1 - p))


def test_electron_energy_bin_index():
    # quarter octaves of the lab energy from 2^-6 eV: K = m 2^e, m in [1, 2),
    # bin = 4 (e + 6) + floor(4 (m - 1)), clamped to [0, 63]
    o = oracle.Oracle(_disch(), [_flat(4, 1e-19)])
    cases = {2.0 ** -6: 0, 2.0 ** -7: 0, 0.0: 0, 1.0: 24, 1.3: 25, 1.5: 26, 1.75: 27,
             1.99: 27, 2.0: 28, 10.0: 37, 700.0: 61, 800.0: 62, 1000.0: 63, 1e6: 63}
    for K, b in cases.items():
        assert o.bin_of(K) == b, (K, o.bin_of(K), b)


# largest gas-molecule speed a collision can draw, in thermal speeds
# sqrt(kT/M): two Box-Muller pairs whose radius sqrt(-2 ln r) is largest at
# the smallest FP64 uniform r = 2^-33, so |(n0, n1)| and |n2| are at most
# sqrt(66 ln 2) each
BM_MAX = math.sqrt(2 * 66 * math.log(2.0))


def _gas_frequency(o, tabs_idx, ngas, u, Ecm):
    nu = np.zeros(len(u))
    for k in tabs_idx:
        nu += ngas * np.array([o.sigma(k, e) for e in Ecm]) * u
    return nu


def test_electron_bin_bounds_cover_the_collision_frequency():
    # every bin's bound is at least sum_j n_j sigma_j(E_cm) u for electrons of
    # that bin against ANY gas molecule Box-Muller can draw (speeds up to
    # BM_MAX thermal speeds, including the worst case: at the top of the bin,
    # head on at the largest speed), and, the point of the bins, not much
    # larger than the largest such frequency
    d = _disch(p_Pa=20.0, ecap_override=1250.0)
    tabs = [t for t in inputs.xs_tables() if t["reaction"] in (4, 7, 8, 9, 10, 11, 12, 15, 18)]
    o = oracle.Oracle(d, tabs)
    ngas = d.p_Pa / (KB * d.T_gas)
    mu = ME * M_O2 / (ME + M_O2)
    vg = math.sqrt(KB * d.T_gas / M_O2)
    assert 9.5 < BM_MAX < 10.0
    rs = np.random.default_rng(21)
    gas_tabs = list(range(len(tabs)))
    for b in range(0, 63, 3):
        lo = 2.0 ** (-6 + b // 4) * (1 + (b % 4) / 4)
        hi = 2.0 ** (-6 + b // 4) * (1 + (b % 4 + 1) / 4)
        K = np.concatenate([rs.uniform(lo, hi, size=400), [hi * (1 - 1e-15)]])
        dirs = rs.normal(size=(401, 3))
        dirs /= np.linalg.norm(dirs, axis=1)[:, None]
        v = np.sqrt(2 * K * QE / ME)[:, None] * dirs
        # molecule speeds spread over the whole range Box-Muller can give
        gd = rs.normal(size=(401, 3))
        gd /= np.linalg.norm(gd, axis=1)[:, None]
        V = gd * vg * rs.uniform(0.0, BM_MAX, size=401)[:, None]
        V[-1] = -dirs[-1] * vg * BM_MAX  # head on, fastest molecule, top of the bin
        u = np.linalg.norm(v - V, axis=1)
        Ecm = 0.5 * mu * u * u / QE
        nu = _gas_frequency(o, gas_tabs, ngas, u, Ecm)
        bound = o.numax_bin(b)
        assert np.all(nu <= bound / d.numax_safety), (b, nu.max(), bound)
        assert bound <= o.numax(0) * 1.0000001 or hi > 1000.0
        if nu.max() > 0 and b >= 8:
            assert bound < 2.0 * nu.max(), (b, bound, nu.max())


@pytest.mark.parametrize("species", [0, 1, 2])
def test_numax_bounds_every_energy_up_to_the_cap(species):
    # nu_max of Sec. II's null-collision bound: no centre-of-mass energy in
    # [0, E_cap] has sum_j n_j sigma_j(E) sqrt(2E/mu) above it (the tables'
    # nodes, thresholds, points between them and random energies), and it is
    # the sup of that frequency within the width of a grid segment
    d = _disch(p_Pa=20.0, ecap_override=1250.0)
    tabs = [t for t in inputs.xs_tables() if t["reaction"] not in (13, 14, 19)]
    o = oracle.Oracle(d, tabs)
    # projectiles of Table I: O- for (5), (14), (16), (17), O2+ for (6), else the electron
    proj = {5: 1, 14: 1, 16: 1, 17: 1, 6: 2}
    idx = [k for k, t in enumerate(tabs) if proj.get(t["reaction"], 0) == species]
    assert idx
    ngas = d.p_Pa / (KB * d.T_gas)
    mu = MASS[species] * M_O2 / (MASS[species] + M_O2)
    cap = d.ecap_eV[species]
    pts = [0.0, cap]
    for k in idx:
        E = tabs[k]["E_eV"]
        E = E[E < cap]
        pts += list(E) + list(0.5 * (E[1:] + E[:-1])) + [tabs[k]["threshold_eV"]]
    rs = np.random.default_rng(5 + species)
    pts += list(rs.uniform(0.0, cap, 2000)) + list(np.exp(rs.uniform(math.log(1e-4), math.log(cap), 2000)))
    E = np.array(sorted(p for p in pts if 0.0 <= p <= cap))
    u = np.sqrt(2 * E * QE / mu)
    nu = np.zeros(len(E))
    for k in idx:
        s = np.array([o.sigma(k, e) for e in E])
        # (17) sees O2(a) at C n_O2 (Sec. III C), every other channel n_O2
        nj = ngas * (d.C_delta if tabs[k]["reaction"] == 17 else 1.0)
        nu += nj * s * u
    bound = o.numax(species) / d.numax_safety
    assert np.all(nu <= bound), (nu.max(), bound)
    assert bound < 1.15 * nu.max(), (bound, nu.max())


def test_binned_null_collision_real_event_fraction():
    # with an energy-dependent bound the real-event probability is
    # (1 - exp(-nu_b dt)) nu / nu_b for the bin's bound nu_b (the rejection
    # step of the null-collision method), and the bound is far below the
    # single bound at the cap
    sig, E0, cap = 1e-19, 10.0, 400.0
    d = _disch(ecap_override=cap, dt_override=5e-11, numax_bins=64)
    o = oracle.Oracle(d, [_flat(4, sig)])
    n = 200000
    rs = np.random.default_rng(13)
    dirs = rs.normal(size=(n, 3))
    dirs /= np.linalg.norm(dirs, axis=1)[:, None]
    v = math.sqrt(2 * E0 * QE / ME) * dirs
    o.set(0, np.full(n, 0.5), v[:, 0], v[:, 1], v[:, 2])
    _empty_others(o, [0])
    o.step(1)
    ev = o.counters()["events"][4]
    ngas = d.p_Pa / (KB * d.T_gas)
    mu = ME * M_O2 / (ME + M_O2)
    nu = ngas * sig * math.sqrt(2 * E0 * QE / mu)
    nub = o.numax_bin(o.bin_of(E0))
    assert nu < nub < 1.2 * nu and nub < 0.2 * o.numax(0)
    p = (1 - math.exp(-nub * d.dt)) * nu / nub
    assert abs(ev - n * p) < 4 * math.sqrt(n * p * (1 - p))


def test_channel_shares_follow_cross_sections():
    d = _disch(ecap_override=30.0, dt_override=1e-10)
    tabs = [_flat(4, 1e-19), _flat(9, 3e-20, th=6.4)]
    o = oracle.Oracle(d, tabs)
    n = 100000
    E0 = 20.0
    rs = np.random.default_rng(12)
    dirs = rs.normal(size=(n, 3))
    dirs /= np.linalg.norm(dirs, axis=1)[:, None]
    v = math.sqrt(2 * E0 * QE / ME) * dirs
    o.set(0, np.full(n, 0.5), v[:, 0], v[:, 1], v[:, 2])
    _empty_others(o, [0])
    o.step(1)
    ev = o.counters()["events"]
    tot = ev[4] + ev[9]
    frac = 3e-20 / 1.3e-19
    assert abs(ev[9] - tot * frac) < 4 * math.sqrt(tot * frac * (1 - frac))


@pytest.mark.parametrize("T0", [0.0259, 1.0])
def test_associative_detachment_decay_rate(T0):
    # sigma_ad u is energy independent (Eq. 9), so O- decays as
    # exp(-C n_O2 K_ad t) whatever its velocity distribution (Sec. IV)
    d = _disch(n_op=0, T0_eV=(0.0, T0, 0.0), dt_override=1e-7, ecap_override=5.0)
    o = oracle.Oracle(d, [_table(17)])
    n = 40000
    rs = np.random.default_rng(13)
    vt = math.sqrt(T0 * QE / M_OM)
    v = rs.normal(0, vt, size=(n, 3))
    o.set(1, rs.uniform(0.45, 0.55, n), v[:, 0], v[:, 1], v[:, 2])
    _empty_others(o, [1])
    steps = 100
    o.step(steps)
    mu = M_OM * M_O2 / (M_OM + M_O2)
    kad = 5.96e-16 * 1e-4 * math.sqrt(2 * QE / mu)
    nu = d.C_delta * d.p_Pa / (KB * d.T_gas) * kad
    surv = math.exp(-nu * steps * d.dt)
    alive = o.get(1)["alive"].sum()
    c = o.counters()
    assert abs(alive - n * surv) < 4 * math.sqrt(n * surv * (1 - surv))
    assert c["events"][17] == n - alive
    assert c["births"][0] == c["events"][17] and o.count(0) == c["births"][0]


@pytest.mark.parametrize("species,reaction", [(2, 6), (1, 5)])
def test_ion_relaxes_to_gas_maxwellian(species, reaction):
    # (6) and (5) conserve the pair's momentum and energy, so the ion
    # distribution relaxes to a Maxwellian at the gas temperature
    d = _disch(n_op=0, dt_override=2e-8 if reaction == 6 else 4e-8, ecap_override=5.0)
    o = oracle.Oracle(d, [_table(reaction)])
    n = 20000
    rs = np.random.default_rng(14)
    m = MASS[species]
    v = rs.normal(0, math.sqrt(0.5 * QE / m), size=(n, 3))
    o.set(species, rs.uniform(0.45, 0.55, n), v[:, 0], v[:, 1], v[:, 2])
    _empty_others(o, [species])
    o.step(400)
    st = o.get(species)
    assert st["alive"].all()
    kT = KB * d.T_gas
    ke = 0.5 * m * (st["vx"]**2 + st["vy"]**2 + st["vz"]**2)
    assert np.mean(ke) / (1.5 * kT) == pytest.approx(1.0, abs=0.03)
    assert stats.kstest(st["vx"] / math.sqrt(kT / m), "norm").pvalue > 1e-3


def _ke(m, v):
    return 0.5 * m * float(np.dot(v, v))


@pytest.mark.parametrize("reaction", [4, 5, 7, 8, 9, 10, 11, 12, 15, 16, 17, 18])
def test_gas_event_conservation(reaction):
    tabs = inputs.xs_tables()
    idx = [i for i, t in enumerate(tabs) if t["reaction"] == reaction][0]
    th = tabs[idx]["threshold_eV"]
    sp = {5: 1, 16: 1, 17: 1}.get(reaction, 0)
    o = oracle.Oracle(_disch(), tabs)
    rs = np.random.default_rng(reaction)
    for trial in range(20):
        m = MASS[sp]
        E = th + 1.0 + 30.0 * rs.random()
        dirn = rs.normal(size=3)
        dirn /= np.linalg.norm(dirn)
        v = math.sqrt(2 * E * QE / m) * dirn * (1.05 if sp == 0 else 1.0)
        V = rs.normal(0, 300.0, 3)
        r4 = rs.random(4)
        r2 = rs.random(2)
        vo, alive, prods, Vo = o.gas_event(sp, idx, v, V, r4, r2)
        p_in = m * v + M_O2 * V
        k_in = _ke(m, v) + _ke(M_O2, V)
        if reaction in (4, 5, 7, 8, 9, 10, 11, 12):
            assert alive and not prods
            assert np.allclose(m * vo + M_O2 * Vo, p_in, rtol=1e-12, atol=1e-12 * np.abs(p_in).max())
            dk = k_in - _ke(m, vo) - _ke(M_O2, Vo)
            assert dk == pytest.approx(th * QE, rel=1e-9, abs=1e-9 * k_in)
        elif reaction == 15:
            assert not alive and [p[0] for p in prods] == [1]
            vom = prods[0][1]
            vO = (p_in - M_OM * vom) / M_O
            dk = k_in - _ke(M_OM, vom) - _ke(M_O, vO)
            assert dk == pytest.approx(th * QE, rel=1e-9)
        elif reaction == 16:
            assert not alive and [p[0] for p in prods] == [0]
            assert _ke(ME, prods[0][1]) == pytest.approx(_ke(M_OM, v) / 10, rel=1e-12)
        elif reaction == 17:
            assert not alive and [p[0] for p in prods] == [0]
            vcm = p_in / (m + M_O2)
            mu = m * M_O2 / (m + M_O2)
            ecm = 0.5 * mu * float(np.dot(v - V, v - V))
            w = np.linalg.norm(prods[0][1] - vcm)
            assert w == pytest.approx(math.sqrt(2 * ecm / ME), rel=1e-12)
        elif reaction == 18:
            assert alive and [p[0] for p in prods] == [0, 2]
            ve2, vop = prods[0][1], prods[1][1]
            p_out = ME * vo + ME * ve2 + M_OP * vop
            assert np.allclose(p_out, p_in, rtol=1e-10, atol=1e-10 * np.abs(p_in).max())
            dk = k_in - _ke(ME, vo) - _ke(ME, ve2) - _ke(M_OP, vop)
            assert dk == pytest.approx(th * QE, rel=1e-8)


@pytest.mark.parametrize("reaction,sp", [(4, 0), (9, 0), (5, 1)])
def test_scattering_is_isotropic_in_the_cm_frame(reaction, sp):
    """Sec. III: the scattering of (4)-(12) is isotropic in the centre-of-mass
    frame.  With uniform random numbers, the cosine of the angle between the
    relative velocities before and after is uniform on [-1, 1] and the
    azimuth about the incoming one is uniform on [0, 2 pi); the outgoing
    speed is that of Eq. 5.  A half-range cosine, a doubled azimuth or a
    direction tied to the incoming one fails."""
    tabs = inputs.xs_tables()
    idx = [i for i, t in enumerate(tabs) if t["reaction"] == reaction][0]
    th = tabs[idx]["threshold_eV"]
    o = oracle.Oracle(_disch(), tabs)
    rs = np.random.default_rng(70 + reaction)
    m = MASS[sp]
    mu = m * M_O2 / (m + M_O2)
    g = np.array([0.3, -0.5, 0.81])
    g /= np.linalg.norm(g)
    Ecm = th + 4.0
    u = math.sqrt(2 * Ecm * QE / mu)
    V = np.array([120.0, -40.0, 75.0])
    v = V + u * g
    # a basis about g for the azimuth
    e1 = np.cross(g, [1.0, 0.0, 0.0])
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(g, e1)
    cosx, phi = [], []
    for _ in range(3000):
        vo, alive, prods, Vo = o.gas_event(sp, idx, v, V, rs.random(4), rs.random(2))
        gp = vo - Vo
        up = np.linalg.norm(gp)
        assert up == pytest.approx(math.sqrt(max(0.0, u * u - 2 * th * QE / mu)), rel=1e-9)
        n = gp / up
        cosx.append(float(np.dot(n, g)))
        phi.append(math.atan2(float(np.dot(n, e2)), float(np.dot(n, e1))) % (2 * math.pi))
    assert stats.kstest((np.array(cosx) + 1) / 2, "uniform").pvalue > 1e-3
    assert stats.kstest(np.array(phi) / (2 * math.pi), "uniform").pvalue > 1e-3


def test_charge_exchange_swaps_velocities():
    tabs = inputs.xs_tables()
    idx = [i for i, t in enumerate(tabs) if t["reaction"] == 6][0]
    o = oracle.Oracle(_disch(), tabs)
    v, V = np.array([1e3, -2e3, 5.0]), np.array([-300.0, 20.0, 110.0])
    vo, alive, prods, Vo = o.gas_event(2, idx, v, V, [0.3, 0.2, 0.7, 0.1])
    assert alive and not prods
    assert np.array_equal(vo, V) and np.array_equal(Vo, v)


def test_impact_detachment_event_conservation():
    tabs = inputs.xs_tables()
    idx = [i for i, t in enumerate(tabs) if t["reaction"] == 19][0]
    th = tabs[idx]["threshold_eV"]
    o = oracle.Oracle(_disch(), tabs)
    rs = np.random.default_rng(19)
    for _ in range(20):
        v = rs.normal(0, 3e6, 3)
        vt = rs.normal(0, 500, 3)
        v1, v2, vO = o.pair19_event(idx, v, vt, rs.random(2), rs.random(2))
        p_in = ME * v + M_OM * vt
        p_out = ME * v1 + ME * v2 + M_O * vO
        assert np.allclose(p_out, p_in, rtol=1e-10, atol=1e-10 * np.abs(p_in).max())
        dk = _ke(ME, v) + _ke(M_OM, vt) - _ke(ME, v1) - _ke(ME, v2) - _ke(M_O, vO)
        assert dk == pytest.approx(th * QE, rel=1e-8)


# -------------------------------------------------------- bookkeeping

def test_births_are_appended_after_the_survivors_in_parent_order():
    """Most electrons ionise (18) in one step (a cross section so large that
    the null-collision test always passes): the new electrons and O2+ follow
    the survivors of their species, one per ionising parent, in the parents'
    order, at the parents' positions.  Without a field the parents that did
    not collide keep their velocities bit for bit, which tells them apart."""
    d = _disch(L=0.01, dt_override=1e-11)
    E = inputs.geometric_grid(0.01, 1e3, 64)
    tab = dict(reaction=18, sub=0, E_eV=E, sigma_m2=np.full_like(E, 1e-15), threshold_eV=0.1)
    o = oracle.Oracle(d, [tab])
    rs = np.random.default_rng(17)
    n = 50
    x0 = rs.permutation(np.linspace(0.1, 0.9, n)) * d.L   # parents not sorted by position
    v = rs.normal(size=(n, 3)) * 1.5e6
    o.set(0, x0, v[:, 0], v[:, 1], v[:, 2])
    o.set(2, [0.5 * d.L], [0.0], [0.0], [0.0])           # one O2+ already there
    o.set(1, [], [], [], [])
    o.step(1)
    k = o.counters()["events"][18]
    e, op = o.get(0), o.get(2)
    hit = (e["vx"][:n] != v[:, 0]) | (e["vy"][:n] != v[:, 1]) | (e["vz"][:n] != v[:, 2])
    assert hit.sum() == k and k > n // 2 and k < n          # some parents did not collide
    assert len(e["x"]) == n + k and len(op["x"]) == 1 + k
    assert np.array_equal(e["x"][n:], e["x"][:n][hit])       # born where the parent is
    assert np.array_equal(op["x"][1:], e["x"][:n][hit])
    assert np.allclose(e["x"][:n], x0 + v[:, 0] * d.dt, rtol=0, atol=1e-12 * d.L)
    assert e["alive"].all() and op["alive"].all()


def test_particle_and_charge_bookkeeping_full_step_loop():
    d = inputs.cfg1(n_op=4000)
    o = oracle.Oracle(d, inputs.xs_tables())
    n0 = [o.count(s) for s in range(3)]
    o.step(300)
    c = o.counters()
    ev, ab = c["events"], c["absorbed"].sum(axis=1)
    live = [int(o.get(s)["alive"].sum()) for s in range(3)]
    de = -ev[13] - ev[15] + ev[16] + ev[17] + ev[18] + ev[19] - ab[0]
    dm = -ev[14] + ev[15] - ev[16] - ev[17] - ev[19] - ab[1]
    dp = -ev[13] - ev[14] + ev[18] - ab[2]
    assert live == [n0[0] + de, n0[1] + dm, n0[2] + dp]
    assert ev[4] > 0 and ev[18] > 0 and c["violations"][0] == 0
    q = live[2] - live[0] - live[1]
    assert q == (n0[2] - n0[0] - n0[1]) - ab[2] + ab[0] + ab[1]


def test_sort_is_stable_by_cell_and_drops_dead():
    d = _disch(L=0.01, n_cells=32, sort_interval=1)
    o = oracle.Oracle(d, [])
    rs = np.random.default_rng(21)
    n = 3000
    x = rs.uniform(0, d.L, n)
    vx = np.zeros(n)
    vx[:50] = -1e9  # leave through x = 0 in the first step
    tag = np.arange(n, dtype=float)  # carried in vy to follow each particle
    o.set(0, x, vx, tag, np.zeros(n))
    _empty_others(o, [0])
    o.step(1)
    st = o.get(0)
    cell = np.floor(x[50:] / (d.L / d.n_cells))
    order = np.argsort(cell, kind="stable") + 50
    assert np.array_equal(st["vy"], tag[order])
    assert st["alive"].all() and len(st["x"]) == n - 50


# ----------------------------------------------------------- pair pass

@pytest.mark.parametrize("weight", [2e14, 1e13])
def test_neutralisation_rate_matches_eq1(weight):
    # all O- and O2+ in one cell, zero net charge, one pass of (14); at the
    # smaller weight the bound B on P is below 1, so candidates are thinned
    # (probability B each) and accepted with P/B: the rate is Eq. 1's either way
    L, N = 0.064, 64
    dx = L / N
    n = 8000
    dt = 1e-9
    d = _disch(L=L, n_cells=N, n1=1, dt_override=dt, weight_override=weight)
    o = oracle.Oracle(d, [_table(14)])
    rs = np.random.default_rng(31)
    x = rs.uniform(10 * dx + 0.3 * dx, 10 * dx + 0.7 * dx, n)
    vm = rs.normal(0, math.sqrt(KB * 300 / M_OM), (n, 3))
    vp = rs.normal(0, math.sqrt(KB * 300 / M_OP), (n, 3))
    o.set(1, x, vm[:, 0], vm[:, 1], vm[:, 2])
    o.set(2, x, vp[:, 0], vp[:, 1], vp[:, 2])
    o.set(0, [], [], [], [])
    o.step(1)
    ev = o.counters()["events"][14]
    nT = n * d.weight / dx
    mu = M_OM * M_OP / (M_OM + M_OP)
    sub = rs.choice(n, 1500, replace=False)
    g = vm[sub][:, None, :] - vp[None, :, :]
    u = np.sqrt(np.sum(g * g, axis=2))
    E = 0.5 * mu * u * u / QE
    sig = 0.8 * (1 + 2.85 / E) * 1e-18
    p = np.minimum(nT * sig * u * dt, 1.0).mean()
    expect = n * p
    assert 40 < expect < 4000
    assert abs(ev - expect) < 4 * math.sqrt(expect) + 0.02 * expect


@pytest.mark.parametrize("reaction,target", [(13, 2), (19, 1)])
def test_electron_target_rate_matches_eq1(reaction, target):
    """Recombination (13) on O2+ and detachment (19) on O- with a cross
    section linear in the pair energy (exact under the tables' linear
    interpolation): every electron, at speed u on resting targets, reacts
    with P = n_T sigma(E) u tau of Eq. 1, E = mu u^2 / 2 with the pair's
    reduced mass; the projectiles are thinned (bound below 1).  A wrong mass,
    target density, speed or tau changes the count by far more than its
    binomial spread."""
    L, N = 0.064, 64
    dx = L / N
    ne, nt, w, dt, u = 20000, 4000, 1e6, 1e-12, 1e6
    E = inputs.geometric_grid(0.01, 10.0, 64)
    a = 4.4e-9  # m^2 per eV
    tab = dict(reaction=reaction, sub=0, E_eV=E, sigma_m2=a * E, threshold_eV=0.0)
    d = _disch(L=L, n_cells=N, n1=1, dt_override=dt, weight_override=w)
    o = oracle.Oracle(d, [tab])
    rs = np.random.default_rng(41 + reaction)
    x = rs.uniform(10.3 * dx, 10.7 * dx, ne)
    n = rs.normal(size=(ne, 3))
    v = u * n / np.linalg.norm(n, axis=1)[:, None]
    o.set(0, x, v[:, 0], v[:, 1], v[:, 2])
    o.set(target, x[:nt], np.zeros(nt), np.zeros(nt), np.zeros(nt))
    o.set(3 - target, [], [], [], [])
    o.step(1)
    ev = o.counters()["events"][reaction]
    mu = ME * MASS[target] / (ME + MASS[target])
    Ep = 0.5 * mu * u * u / QE
    P = nt * w / dx * a * Ep * u * dt
    assert 0.03 < P < 0.07
    expect = ne * P
    assert abs(ev - expect) < 4 * math.sqrt(expect * (1 - P))


def test_pair_pass_exhausts_targets_with_clamped_probability():
    L, N = 0.064, 64
    dx = L / N
    # a huge cross section (not a weight, whose field would scatter the
    # electrons) makes P = n sigma u tau >> 1 for every pair
    d = _disch(L=L, n_cells=N, n1=1, dt_override=1e-9, weight_override=1e6)
    o = oracle.Oracle(d, [_flat(13, 1e-2)])
    rs = np.random.default_rng(33)
    ne, nop = 300, 200
    x = rs.uniform(5.2 * dx, 5.8 * dx, ne)
    v = rs.normal(0, 1e3, (ne, 3))  # slow: everyone stays in cell 5
    o.set(0, x, v[:, 0], v[:, 1], v[:, 2])
    o.set(2, x[:nop], np.zeros(nop), np.zeros(nop), np.zeros(nop))
    o.set(1, [], [], [], [])
    o.step(1)
    c = o.counters()
    assert c["events"][13] == nop
    assert c["violations"][1] == nop
    assert o.get(2)["alive"].sum() == 0
    assert o.get(0)["alive"].sum() == ne - nop


def test_pair_pass_fast_projectile_reacts_with_eq1_probability():
    """A projectile far faster than the rest (here far above any energy cap
    of the discharge) reacts with P = n_T sigma u tau of Eq. 1, not with a
    bound computed for slower pairs: the thinning bound follows the largest
    speeds of the two species.  Recombination (13) with a flat cross section
    in 64 cells, each with 60 slow electrons, one fast electron and 20 O2+ at
    rest; 12 seeds."""
    L, N = 0.064, 64
    dx = L / N
    w, dt, sig = 1e6, 1e-12, 1.25e-6
    u_fast, u_slow = 2e7, 1e5
    fast = slow = 0
    n_fast = n_slow = 0
    for seed in range(1, 13):
        d = _disch(L=L, n_cells=N, n1=1, dt_override=dt, weight_override=w, seed=seed)
        o = oracle.Oracle(d, [_flat(13, sig)])
        rs = np.random.default_rng(100 + seed)
        xs, vs = [], []
        for c in range(N):
            x = (c + rs.uniform(0.4, 0.6, 61)) * dx
            dirs = rs.normal(size=(61, 3))
            dirs /= np.linalg.norm(dirs, axis=1)[:, None]
            sp = np.full(61, u_slow)
            sp[30] = u_fast
            xs.append(x)
            vs.append(dirs * sp[:, None])
        x, v = np.concatenate(xs), np.concatenate(vs)
        o.set(0, x, v[:, 0], v[:, 1], v[:, 2])
        xt = np.repeat((np.arange(N) + 0.5) * dx, 20)
        o.set(2, xt, np.zeros_like(xt), np.zeros_like(xt), np.zeros_like(xt))
        o.set(1, [], [], [], [])
        o.step(1)
        st = o.get(0)
        spd = np.sqrt(st["vx"] ** 2 + st["vy"] ** 2 + st["vz"] ** 2)
        isf = spd > 0.5 * u_fast
        assert isf.sum() == N
        fast += int((~st["alive"][isf]).sum())
        slow += int((~st["alive"][~isf]).sum())
        n_fast += N
        n_slow += int((~isf).sum())
        assert o.counters()["violations"][2] == 0
    nT = 20 * w / dx
    Pf = nT * sig * u_fast * dt
    Ps = nT * sig * u_slow * dt
    assert 0.4 < Pf < 0.6
    assert abs(fast - n_fast * Pf) < 4 * math.sqrt(n_fast * Pf * (1 - Pf)), (fast, n_fast * Pf)
    assert abs(slow - n_slow * Ps) < 4 * math.sqrt(n_slow * Ps * (1 - Ps)) + 2, (slow, n_slow * Ps)


# ------------------------------------------------------------- loading

def test_initial_load_statistics():
    d = inputs.cfg1(n_op=20000)
    o = oracle.Oracle(d, [])
    for s in range(3):
        st = o.get(s)
        assert len(st["x"]) == d.n_init[s]
        assert stats.kstest(st["x"] / d.L, "uniform").pvalue > 1e-3
        vt = math.sqrt(d.T0_eV[s] * QE / MASS[s])
        for comp in ("vx", "vy", "vz"):
            assert stats.kstest(st[comp] / vt, "norm").pvalue > 1e-3
