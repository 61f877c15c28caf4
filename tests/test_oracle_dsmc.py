"""Pins of the oracle's sequential gas-channel scheme (the paper's own
collision scheme, Sec. II "Method of simulation", with Eq. 1 for every
channel of Table I): the event count of a channel against Eq. 1 with
tau = n1 dt, no gas event between passes, the readmission of a product to
the later channels of the list (a chain (15) -> (16) in one pass) against
the probabilities of the chain, and the particle bookkeeping of Table I over
a discharge run.  Runs on the CPU only."""
import math

import numpy as np

import oracle
from paper_0705_0495_gb300 import inputs

QE = 1.602176634e-19
ME = 9.1093837015e-31
AMU = 1.66053906660e-27
KB = 1.380649e-23
M_O2 = 32 * AMU


def _disch(**kw):
    base = dict(L=1.0, n_cells=128, p_Pa=20.0, U_rf=0.0, n_op=0, n0_m3=0.0,
                weight_override=0.0, n1=10, sort_interval=0, diag_every=0,
                T0_eV=(0.0, 0.0, 0.0), dt_override=1e-10, gas_scheme=1)
    base.update(kw)
    return inputs.Discharge(**base)


def _table(reaction, sigma_of_E, th=0.0):
    E = inputs.geometric_grid(1e-4, 1e4, 801)
    return dict(reaction=reaction, sub=0, E_eV=E, sigma_m2=sigma_of_E(E), threshold_eV=th)


def _electrons(n, E0, seed):
    rs = np.random.default_rng(seed)
    dirs = rs.normal(size=(n, 3))
    dirs /= np.linalg.norm(dirs, axis=1)[:, None]
    return math.sqrt(2 * E0 * QE / ME) * dirs


def _setup(d, tabs, v):
    o = oracle.Oracle(d, tabs)
    n = len(v)
    o.set(0, np.full(n, 0.5), v[:, 0], v[:, 1], v[:, 2])
    o.set(1, [], [], [], [])
    o.set(2, [], [], [], [])
    return o


def test_channel_events_follow_eq1_once_per_pass():
    # flat elastic cross section, 5 eV electrons: P = n sigma u n1 dt with u
    # the speed relative to a gas molecule (300 K O2 moves ~300 m/s, 2e-4 of
    # the electron speed); events only at the pass, every n1 = 10 steps
    sig, E0, n = 1e-19, 5.0, 20000
    d = _disch()
    o = _setup(d, [_table(4, lambda E: np.full_like(E, sig))], _electrons(n, E0, 3))
    o.step(9)
    assert o.counters()["events"].sum() == 0
    o.step(1)
    ev = o.counters()["events"][4]
    ngas = d.p_Pa / (KB * d.T_gas)
    u = math.sqrt(2 * E0 * QE / ME)
    p = ngas * sig * u * d.n1 * d.dt
    assert 0.3 < p < 0.9
    assert abs(ev - n * p) < 4 * math.sqrt(n * p * (1 - p)) + 2e-3 * n * p
    o.step(10)
    ev2 = o.counters()["events"][4] - ev
    assert abs(ev2 - n * p) < 4 * math.sqrt(n * p * (1 - p)) + 2e-3 * n * p


def test_product_is_readmitted_to_later_channels():
    # sigma = K / sqrt(E) makes sigma u constant (u = sqrt(2 E / mu) in the
    # centre of mass), so (15) happens with probability P15 for every
    # electron and (16) with P16 for every O- it produces, whatever their
    # energies; in one pass an electron ends as itself (1 - P15), as an O-
    # (P15 (1 - P16)) or, readmitted, as a new electron (P15 P16)
    n, E0 = 40000, 5.0
    d = _disch()
    ngas = d.p_Pa / (KB * d.T_gas)
    tau = d.n1 * d.dt
    mu_e = ME * M_O2 / (ME + M_O2)
    m_om = 16 * AMU + ME
    mu_o = m_om * M_O2 / (m_om + M_O2)
    P15, P16 = 0.5, 0.4
    k15 = P15 / (ngas * tau * math.sqrt(2 * QE / mu_e))
    k16 = P16 / (ngas * tau * math.sqrt(2 * QE / mu_o))
    tabs = [_table(15, lambda E: k15 / np.sqrt(E)), _table(16, lambda E: k16 / np.sqrt(E))]
    o = _setup(d, tabs, _electrons(n, E0, 5))
    o.step(10)
    ev = o.counters()["events"]
    e_live = int(o.get(0)["alive"].sum())
    om_live = int(o.get(1)["alive"].sum())

    def near(x, p):
        return abs(x - n * p) < 4 * math.sqrt(n * p * (1 - p)) + 5e-3 * n * p

    assert near(ev[15], P15), ev[15]
    assert near(ev[16], P15 * P16), ev[16]
    assert near(om_live, P15 * (1 - P16)), om_live
    assert near(e_live, 1 - P15 + P15 * P16), e_live
    assert e_live + om_live == n


def test_bookkeeping_of_a_discharge_run():
    d = inputs.cfg1(n_op=4000, gas_scheme=1)
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
    assert ev[4] > 0 and ev[6] > 0 and ev[18] > 0
