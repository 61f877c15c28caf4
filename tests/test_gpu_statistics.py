"""Long-run agreement of the FP32 GPU path with the FP64 oracle.

After the first steps the two paths are different realisations of the same
stochastic process (FP32 rounding changes single decisions, which then
diverge), so they are compared as ensembles: the time-averaged densities of
e, O- and O2+, the potential, the EEDF at L/2 and the O2+ energy distribution
at the electrodes, each averaged over independent seeds, must agree within
3 standard errors of the seed-to-seed scatter: with
z = (m_gpu - m_orc) / sqrt(s_gpu^2/n + s_orc^2/n) for every node and every
histogram bin holding at least 100 counts on both sides, the mean of z^2 is
at most 3, at most 10% of the values exceed 3 and none exceeds 6.  Neighbouring
nodes are strongly correlated, so exceedances come in clusters: two oracle
ensembles of 12 independent seeds each gave mean z^2 between 1.2 and 2.1, up
to 4.6% of the values beyond 3 and at most 4.2 (four trials).  The same test
runs with the paper's sequential gas scheme and with intra- and inter-species
Coulomb collisions."""
import multiprocessing
import os
import sys

import numpy as np
import pytest

import oracle
from paper_0705_0495_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SEEDS = 12
STEPS = 2000  # two RF cycles of the cfg1 discharge
# cfg1 with twice the superparticles and 2 energy bins per electrode for the
# O2+ distribution, so that its bins hold more than 100 counts
KW = dict(n_op=40000, iedf_bins=2)
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


# the discharge as loaded, with the paper's sequential gas scheme instead
# of the null-collision test, and with intra- and inter-species Coulomb
# collisions every 10 steps (ln Gamma raised so that they matter)
VARIANTS = {"null_collision": {}, "sequential_gas": {"gas_scheme": 1},
            "coulomb": {"n2": 10, "coulomb_log": 1e3, "coulomb_inter": True}}


def _oracle_run(args):
    seed, extra = args
    sys.path.insert(0, ROOT)
    import oracle as orc
    from paper_0705_0495_gb300 import inputs as inp
    o = orc.Oracle(inp.cfg1(seed=seed, **KW, **extra), inp.xs_tables())
    o.step(STEPS)
    return _averages(o.diag())


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()


def _averages(g):
    ns = g["n_samples"]
    return {"dens": g["dens_sum"] / ns, "phi": g["phi_sum"] / ns,
            "eedf": g["eedf"].astype(float), "iedf": g["iedf"].astype(float).ravel()}


def _z(a, b):
    a, b = np.asarray(a), np.asarray(b)
    n = a.shape[0]
    # values the seeds do not change (the driven electrode's potential) would
    # have no scatter: the error gets a floor of 1e-6 of the quantity's RMS,
    # far above FP32/FP64 rounding and far below the statistical scatter
    floor = 1e-6 * np.sqrt(np.mean(b.mean(axis=0) ** 2))
    se = np.sqrt(a.var(axis=0, ddof=1) / n + b.var(axis=0, ddof=1) / n + floor ** 2)
    diff = a.mean(axis=0) - b.mean(axis=0)
    return diff / np.where(se > 0, se, 1.0)


@pytest.mark.parametrize("variant", sorted(VARIANTS))
def test_fp32_gpu_ensemble_matches_fp64_oracle_ensemble(variant):
    from paper_0705_0495_gb300 import o2pic
    oracle.build()
    extra = VARIANTS[variant]
    # independent realisations on the oracle side, run in parallel on the
    # host cores (a spawned pool: no process is forked from a CUDA process)
    pool = multiprocessing.get_context("spawn").Pool(min(SEEDS, os.cpu_count() or 1))
    pending = pool.map_async(_oracle_run, [(101 + k, extra) for k in range(SEEDS)])
    tabs = inputs.xs_tables()
    gpu = []
    for k in range(SEEDS):
        sim = o2pic.Simulation([inputs.cfg1(fp64=False, seed=1 + k, **KW, **extra)], tabs)
        sim.step(STEPS)
        gpu.append(_averages(sim.diagnostics(0)))
        sim.close()
    orc = pending.get(timeout=1800)
    pool.close()
    pool.join()
    zs = compare(gpu, orc)
    top = np.sort(np.abs(zs))[-5:]
    assert np.mean(zs ** 2) <= 3.0, (np.mean(zs ** 2), top)
    assert np.mean(np.abs(zs) > 3.0) <= 0.10, (np.mean(np.abs(zs) > 3.0), top)
    assert np.all(np.abs(zs) <= 6.0), top


def compare(gpu, orc):
    """z of every node of the densities and potential, and of every EEDF and
    IEDF bin with at least 100 counts on both sides"""
    zs = []
    for key in ("dens", "phi"):
        zs.append(_z([g[key] for g in gpu], [o[key] for o in orc]).ravel())
    for key in ("eedf", "iedf"):
        a = np.array([g[key] for g in gpu])
        b = np.array([o[key] for o in orc])
        keep = (a.mean(axis=0) >= 100) & (b.mean(axis=0) >= 100)
        assert keep.sum() >= 2, key
        zs.append(_z(a[:, keep], b[:, keep]).ravel())
    return np.concatenate(zs)
