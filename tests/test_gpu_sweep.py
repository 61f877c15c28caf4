"""The 13.8 Pa workload of Sec. IV on the GPU: associative detachment (17)
with C = 1/6 removes O- on a time scale of (C n_O2 sigma u)^-1, about 7 us or
100 RF cycles; without it (C = 0, Fig. Profiles) the negative ions pile up.
After 150 cycles from the same load the bulk O- density without (17) must
be well above the one with it (the paper reports an order of magnitude at
quasi-stationarity, after about 10^3 cycles)."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()


def test_associative_detachment_contrast_at_150V():
    from paper_0705_0495_gb300 import sweep
    res, _ = sweep.run(cycles=150, average_cycles=20, n_op=20000)
    rows = {(r["U_rf"], r["C"]): r for r in res["rows"]}
    with_ad, without = rows[(150.0, 1.0 / 6.0)], rows[(150.0, 0.0)]
    assert without["events"][17] == 0 and with_ad["events"][17] > 0
    assert without["n_O-"] > 2.0 * with_ad["n_O-"], (without["n_O-"], with_ad["n_O-"])
    # every discharge keeps its plasma
    assert all(min(r["superparticles"]) > 100 for r in res["rows"]), res["rows"]
