"""pic_field_solve_static: the charge deposit and field solve for callers that
cannot allocate device memory (their scratch is a fixed array inside the
library), checked against pic_fields() of a simulation holding the same
particles.  Kept in a file collected last."""
import math

import numpy as np
import pytest

from paper_0705_0495_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-11  # relative to the largest value, as the GPU field parity tests use


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()


def _device_arrays(sim, d, fp64):
    """the simulation's particles as the caller-owned (cell, offset) arrays"""
    dx = d.L / d.n_cells
    cells, offs, counts = [], [], []
    for s in range(3):
        st = sim.get_state(0, s)
        xx = st["x"] / dx
        c = np.where(st["alive"], np.floor(xx), -1).astype(np.int64)
        c = np.minimum(c, d.n_cells - 1)
        off = np.where(st["alive"], xx - c, 0.0)
        if not fp64:
            off = off.astype(np.float32)
            up = off >= np.float32(1.0)
            c = np.where(up, c + 1, c)
            off = np.where(up, np.float32(0.0), off).astype(np.float32)
        cells.append(torch.from_numpy(c.astype(np.int32)).cuda())
        offs.append(torch.from_numpy(np.ascontiguousarray(off)).cuda())
        counts.append(len(c))
    return cells, offs, counts


@pytest.mark.parametrize("fp64", [False, True])
def test_static_field_solve_matches_pic_fields_twice(fp64):
    from paper_0705_0495_gb300 import o2pic
    d = inputs.cfg1(fp64=fp64, n_op=8000)
    sim = o2pic.Simulation([d], inputs.xs_tables())
    cfg = o2pic.make_config(d)
    N = d.n_cells
    for steps in (7, 5):  # two calls in a row, on two different states
        sim.step(steps)
        rho_ref, phi_ref, E_ref = sim.fields(0)
        step = sim.diagnostics(0)["steps"]
        cells, offs, counts = _device_arrays(sim, d, fp64)
        out = [torch.full((N + 1,), math.nan, dtype=torch.float64, device="cuda") for _ in range(3)]
        stream = torch.cuda.current_stream()
        o2pic.field_solve_static(cfg, step, [t.data_ptr() for t in cells], [t.data_ptr() for t in offs],
                                 counts, out[0].data_ptr(), out[1].data_ptr(), out[2].data_ptr(),
                                 stream.cuda_stream)
        torch.cuda.synchronize()
        rho, phi, E = (t.cpu().numpy() for t in out)
        for got, ref in ((rho, rho_ref), (phi, phi_ref), (E, E_ref)):
            assert np.all(np.isfinite(got))
            assert np.max(np.abs(got - ref)) <= TOL * np.max(np.abs(ref)), (steps, fp64)


def test_static_field_solve_rejects_grids_beyond_its_scratch():
    from paper_0705_0495_gb300 import o2pic
    d = inputs.cfg1(n_cells=5000)
    cfg = o2pic.make_config(d)
    dummy = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(o2pic.PicError, match="4096"):
        o2pic.field_solve_static(cfg, 0, [0, 0, 0], [0, 0, 0], [0, 0, 0], dummy.data_ptr(),
                                 dummy.data_ptr(), dummy.data_ptr())
