"""The sort-interval autotuner: its candidates on the CPU, a tuning run on
the GPU."""
import pytest

from paper_0705_0495_gb300 import autotune, inputs


def test_candidates_divide_the_particle_target_interval():
    assert autotune.candidates(10) == [0, 1, 2, 5, 10]
    assert autotune.candidates(7) == [0, 1, 7]
    assert all(k > 0 for k in autotune.candidates(0))


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
