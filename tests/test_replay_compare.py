"""The FP32 replay comparison (tests/replay.py) on synthetic states, on the
CPU: push-only particles are identified across a reordering and held to the
tolerance; each kind of decision flip is counted as one; an arithmetic error
of a push-only particle is never absorbed into the flips."""
import numpy as np

from paper_0705_0495_gb300 import inputs
from replay import compare_step, vth

TOL = 1e-5


def _states(n=2000, seed=3):
    d = inputs.cfg1(fp64=False, n_op=n)
    rs = np.random.default_rng(seed)
    v0 = vth(d, 0)
    pre = {"x": rs.uniform(0, d.L, n), "vx": rs.normal(0, v0, n), "vy": rs.normal(0, v0, n),
           "vz": rs.normal(0, v0, n), "alive": np.ones(n, bool)}
    # the GPU holds the injected state in FP32
    pre_g = {k: (v.astype(np.float32).astype(np.float64) if k != "alive" else v.copy())
             for k, v in pre.items()}
    dt = 1e-11
    o = {k: v.copy() for k, v in pre.items()}
    o["x"] = pre["x"] + pre["vx"] * dt
    g = {k: v.copy() for k, v in pre_g.items()}
    g["x"] = o["x"] * (1 + 1e-8)
    g["vx"] = o["vx"] * (1 + 2e-8)
    return d, pre, pre_g, g, o


def _perm(st, p):
    return {k: v[p] for k, v in st.items()}


def test_push_only_particles_are_matched_across_a_reordering():
    d, pre, pre_g, g, o = _states()
    p = np.random.default_rng(1).permutation(len(g["x"]))
    r = compare_step(d, 0, pre, pre_g, _perm(g, p), o, TOL)
    assert r.flips == 0 and r.compared == len(o["x"])
    assert 0 < r.worst < TOL


def test_each_kind_of_decision_flip_is_counted():
    d, pre, pre_g, g, o = _states()
    rs = np.random.default_rng(2)
    # absorbed on the GPU only
    g["alive"][10] = False
    # collided on the oracle's side only (new vy, vz)
    o["vy"][20], o["vz"][20] = rs.normal(0, vth(d, 0), 2)
    # collided on both sides with the same outcome: agrees
    for st in (g, o):
        st["vy"][30], st["vz"][30] = 1234.5, -987.25
    # collided on both sides with different outcomes: a flip
    o["vy"][40], o["vz"][40] = 555.0, 444.0
    g["vy"][40], g["vz"][40] = -555.0, 444.0
    r = compare_step(d, 0, pre, pre_g, g, o, TOL)
    assert r.flips == 3, r
    assert r.compared == len(o["x"]) - 1
    assert r.worst < TOL and r.worst_flip > TOL


def test_an_arithmetic_error_is_not_a_flip():
    d, pre, pre_g, g, o = _states()
    g["vx"][7] += 1e-3 * vth(d, 0)  # a push-only particle off by 1e-3 of the thermal speed
    r = compare_step(d, 0, pre, pre_g, g, o, TOL)
    assert r.flips == 0
    assert r.worst > 10 * TOL


def test_coulomb_cells_with_different_counts_are_left_out():
    d, pre, pre_g, g, o = _states()
    rs = np.random.default_rng(4)
    # every particle collided (Coulomb pass): no identities survive
    for st in (g, o):
        st["vy"] = st["vy"] + 1.0
    g["vy"] = o["vy"].copy()
    g["vz"] = o["vz"].copy()
    # one extra birth in some cell on the GPU side
    k = 5
    for key in g:
        g[key] = np.append(g[key], g[key][k])
    r = compare_step(d, 0, pre, pre_g, g, o, TOL, coulomb=True)
    assert r.recount_cells == 1 and r.flips == 0
    assert r.compared + r.excluded - 1 == len(o["x"])
    assert rs is not None


def test_align_skips_inserted_and_missing_particles():
    from replay import align
    rs = np.random.default_rng(5)
    x = rs.uniform(0, 1, 1000)
    xg = np.delete(x, [100, 500])          # the GPU lacks two
    xo = np.insert(x, 700, 0.123456789)    # the oracle holds one more
    pg, po, ug, uo = align(xg, xo, 1e-9)
    assert len(ug) == 0 and sorted(xo[uo].tolist()) == sorted([x[100], x[500], 0.123456789])
    assert np.array_equal(xg[pg], xo[po]) and len(pg) == 998


def test_a_membership_change_in_a_coulomb_cell_leaves_the_rest_aligned():
    # one particle sits in cell c on the GPU side and in cell c + 1 on the
    # oracle's (an edge flip), another the other way round: both cells keep
    # their counts, and a pairing by order within cells would misalign them
    # entirely; the alignment by position keeps the other cells compared
    d, pre, pre_g, g, o = _states()
    for st in (g, o):
        st["vy"] = st["vy"] + 1.0  # every particle collided (a Coulomb step)
    g["vy"], g["vz"] = o["vy"].copy(), o["vz"].copy()
    order = np.argsort(np.floor(o["x"] / (d.L / d.n_cells)), kind="stable")
    o = _perm(o, order)
    g = _perm(g, order)
    # move GPU particle 10 to the end of the sequence (another cell's bucket)
    p = np.r_[np.arange(10), np.arange(11, len(g["x"])), 10]
    g = _perm(g, p)
    r = compare_step(d, 0, pre, pre_g, g, o, TOL, coulomb=True)
    assert r.flips == 0 and 1 <= r.recount_cells <= 2
    assert r.compared >= len(o["x"]) - 60
