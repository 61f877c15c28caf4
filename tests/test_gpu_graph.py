"""One RF cycle as one CUDA graph: pic_step over a whole cycle is a single
graph launch, and the graph replays exactly the work of launching the steps
one by one (FP32 state bit for bit, every counter and histogram)."""
import numpy as np
import pytest

from paper_0705_0495_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()


def test_one_rf_cycle_is_one_graph_launch_with_the_same_results():
    from paper_0705_0495_gb300 import o2pic
    d = inputs.cfg1(fp64=False, n_op=20000)
    spc = d.steps_per_cycle
    tabs = inputs.xs_tables()
    a = o2pic.Simulation([d], tabs)
    b = o2pic.Simulation([d], tabs)
    g0 = a.diagnostics(0)["graph_launch_calls"]
    a.step(spc)
    ga = a.diagnostics(0)
    assert ga["graph_cycle_steps"] == spc
    assert ga["graph_launch_calls"] - g0 == 1
    a.step(2 * spc + 30)  # two cycles, then three periods of 10 steps
    assert a.diagnostics(0)["graph_launch_calls"] - g0 == 1 + 2 + 3
    # the same steps launched one by one (timing mode captures nothing)
    b.set_timing(True)
    b.step(3 * spc + 30)
    b.set_timing(False)
    assert b.diagnostics(0)["graph_launch_calls"] == 0
    for s in range(3):
        sa, sb = a.get_state(0, s), b.get_state(0, s)
        for k in ("x", "vx", "vy", "vz", "alive"):
            assert np.array_equal(sa[k], sb[k]), (s, k)
    da, db = a.diagnostics(0), b.diagnostics(0)
    for k in ("events", "absorbed", "eedf", "iedf", "fm", "dens_sum", "phi_sum"):
        assert np.array_equal(da[k], db[k]), k
    assert da["events"][18] > 0
    a.close()
    b.close()


def test_a_cycle_that_is_no_whole_number_of_periods_uses_period_graphs():
    from paper_0705_0495_gb300 import o2pic
    import math
    d = inputs.cfg1(fp64=False, n_op=2000, n1=7, sort_interval=7)
    period = math.lcm(2, d.n1, d.sort_interval, d.diag_every)  # 70: no divisor of the 1000-step cycle
    sim = o2pic.Simulation([d], inputs.xs_tables())
    sim.step(1000)
    g = sim.diagnostics(0)
    assert g["graph_cycle_steps"] == 0
    assert g["graph_launch_calls"] == 1000 // period
    sim.close()
