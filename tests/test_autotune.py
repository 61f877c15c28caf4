"""The autotuners of the sort interval and of the push grid: their
candidates on the CPU; on the GPU, tuning runs and the property the push
tuner rests on (the push grid does not change the results)."""
import numpy as np
import pytest

from paper_0705_0495_gb300 import autotune, inputs


def test_candidates_divide_the_particle_target_interval():
    assert autotune.candidates(10) == [0, 1, 2, 5, 10]
    assert autotune.candidates(7) == [0, 1, 7]
    assert all(k > 0 for k in autotune.candidates(0))


def test_push_candidates_are_every_count_that_fits():
    assert autotune.push_candidates(3) == [1, 2, 3]
    assert autotune.push_candidates(0) == [1]


def test_shape_candidates_cover_every_shape_and_count():
    shapes = [(256, 4, 3), (128, 8, 2), (512, 4, 1)]
    assert autotune.shape_candidates(shapes) == [(0, 1), (0, 2), (0, 3), (1, 1), (1, 2), (2, 1)]


def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()


@pytest.mark.gpu
def test_tuner_times_every_candidate_and_picks_the_fastest():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    best, ms = autotune.tune_sort_interval(inputs.cfg1(fp64=False), inputs.xs_tables(),
                                           warm_steps=20, timed_steps=40)
    assert set(ms) == set(autotune.candidates(10))
    assert best in ms and ms[best] == min(ms.values()) and all(v > 0 for v in ms.values())


@pytest.mark.gpu
def test_push_grid_does_not_change_fp32_results():
    """The FP32 state after 300 steps is bit for bit the same with one push
    block per SM, with the most that fit, and with the count changed twice in
    the run (each change drops the captured graph of a period)."""
    _gpu()
    from paper_0705_0495_gb300 import o2pic
    d = inputs.cfg1(fp64=False, n_op=40000)
    tabs = inputs.xs_tables()
    sims = [o2pic.Simulation([d], tabs) for _ in range(3)]
    mx = sims[0].launch()[1]
    assert sims[0].launch()[0] == mx >= 1
    sims[1].set_launch(1)
    assert sims[1].launch() == (1, mx)
    for s in sims[:2]:
        s.step(300)
    sims[2].step(100)
    sims[2].set_launch(1)
    sims[2].step(100)
    sims[2].set_launch(mx)
    sims[2].step(100)
    ref = [sims[0].get_state(0, s) for s in range(3)]
    gref = sims[0].diagnostics(0)
    assert gref["events"][18] > 0 and ref[0]["alive"].sum() > 0
    for sim in sims[1:]:
        for s in range(3):
            st = sim.get_state(0, s)
            for k in ("x", "vx", "vy", "vz", "alive"):
                assert np.array_equal(st[k], ref[s][k]), (s, k)
        g = sim.diagnostics(0)
        for k in ("events", "absorbed", "eedf", "iedf", "fm"):
            assert np.array_equal(g[k], gref[k]), k
        assert np.array_equal(g["dens_sum"], gref["dens_sum"])
    for s in sims:
        s.close()


@pytest.mark.gpu
def test_push_grid_out_of_range_is_rejected():
    _gpu()
    from paper_0705_0495_gb300 import o2pic
    sim = o2pic.Simulation([inputs.cfg1(fp64=False)], inputs.xs_tables())
    cur, mx = sim.launch()
    for bad in (0, mx + 1):
        with pytest.raises(o2pic.PicError) as e:
            sim.set_launch(bad)
        assert e.value.code == 1
    with pytest.raises(o2pic.PicError):
        sim.launch("coulomb")
    assert sim.launch() == (cur, mx)
    sim.close()


@pytest.mark.gpu
def test_push_tuner_times_every_count_and_keeps_the_fastest():
    _gpu()
    from paper_0705_0495_gb300 import o2pic
    sim = o2pic.Simulation([inputs.cfg1(fp64=False, n_op=40000)], inputs.xs_tables())
    best, ms = autotune.tune_push_blocks(sim, steps=40, rounds=1)
    _, mx = sim.launch()
    assert set(ms) == set(range(1, mx + 1))
    assert ms[best] == min(ms.values()) and all(v > 0 for v in ms.values())
    assert sim.launch()[0] == best
    sim.close()


@pytest.mark.gpu
def test_push_launch_shapes_do_not_change_fp32_results():
    """The FP32 state after 250 steps is bit for bit the same for every
    compiled launch shape of the push (threads per block, slots per thread)
    at its largest and at one block per SM, and with the shape switched in
    the middle of a run."""
    _gpu()
    from paper_0705_0495_gb300 import o2pic
    d = inputs.cfg1(fp64=False, n_op=40000)
    tabs = inputs.xs_tables()
    ref_sim = o2pic.Simulation([d], tabs)
    shapes = ref_sim.launch_shapes()
    assert len(shapes) >= 3 and {spt for _, spt, _ in shapes} >= {4, 8}
    assert len({nt for nt, _, _ in shapes}) >= 2
    ref_sim.step(250)
    ref = [ref_sim.get_state(0, s) for s in range(3)]
    gref = ref_sim.diagnostics(0)
    ref_sim.close()
    runs = [[(k, mx)] for k, (_, _, mx) in enumerate(shapes)] + [[(k, 1)] for k in range(len(shapes))]
    runs.append([(len(shapes) - 1, 1), (0, shapes[0][2])])
    for plan in runs:
        sim = o2pic.Simulation([d], tabs)
        per = 250 // len(plan)
        done = 0
        for i, (k, b) in enumerate(plan):
            sim.set_launch_shape(k, b)
            assert sim.launch_shape() == (k, b)
            n = per if i < len(plan) - 1 else 250 - done
            sim.step(n)
            done += n
        for s in range(3):
            st = sim.get_state(0, s)
            for key in ("x", "vx", "vy", "vz", "alive"):
                assert np.array_equal(st[key], ref[s][key]), (plan, s, key)
        g = sim.diagnostics(0)
        for key in ("events", "absorbed", "eedf", "iedf", "fm"):
            assert np.array_equal(g[key], gref[key]), (plan, key)
        assert np.array_equal(g["dens_sum"], gref["dens_sum"])
        sim.close()


@pytest.mark.gpu
def test_push_shape_tuner_times_every_shape_and_keeps_the_fastest():
    _gpu()
    from paper_0705_0495_gb300 import o2pic
    sim = o2pic.Simulation([inputs.cfg1(fp64=False, n_op=40000)], inputs.xs_tables())
    best, ms = autotune.tune_push_shape(sim, steps=20, rounds=1)
    shapes = sim.launch_shapes()
    assert len(ms) == sum(mx for _, _, mx in shapes)
    key = f"{best[0]}x{best[1]}@{best[2]}"
    assert ms[key] == min(ms.values())
    k, b = sim.launch_shape()
    assert (shapes[k][0], shapes[k][1], b) == best
    with pytest.raises(o2pic.PicError):
        sim.set_launch_shape(len(shapes), 1)
    with pytest.raises(o2pic.PicError):
        sim.set_launch_shape(0, shapes[0][2] + 1)
    assert sim.launch_shape() == (k, b)
    # the tuner ends on a whole RF cycle: a cycle's steps are one graph launch
    g0 = sim.diagnostics(0)
    c = g0["graph_cycle_steps"]
    assert c > 0 and g0["steps"] % c == 0
    sim.step(2 * c)
    g1 = sim.diagnostics(0)
    assert g1["graph_launch_calls"] - g0["graph_launch_calls"] == 2
    assert sim.align_to_cycle() == 0
    sim.step(3)
    assert sim.align_to_cycle() == c - 3
    sim.close()
