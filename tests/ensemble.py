"""Seed-ensemble comparison of time-averaged profiles and distributions.

Two ensembles of independent runs (different seeds) of the same discharge
are compared quantity by quantity (every node of the densities and of the
potential, every EEDF and IEDF bin holding at least 100 counts on both
sides): Welch's t of the two ensemble means, with the Welch-Satterthwaite
degrees of freedom, converted to the normal deviate of the same tail
probability, so that "within 3 sigma" means a two-sided tail of 0.27 % of a
standard normal whatever the number of seeds (with 8 seeds a raw t beyond 3
is about four times as likely as a normal deviate beyond 3).  The bar: at
least 99 % of the quantities within 3.
"""
from __future__ import annotations

import numpy as np
from scipy import stats

MIN_COUNTS = 100


def averages(g):
    """time averages of one run's diagnostics (GPU dict or oracle dict)"""
    ns = max(g["n_samples"], 1)
    return {"dens": g["dens_sum"] / ns, "phi": g["phi_sum"] / ns,
            "eedf": np.asarray(g["eedf"], dtype=float).ravel(),
            "iedf": np.asarray(g["iedf"], dtype=float).ravel()}


def welch_z(a, b):
    """normal-equivalent deviate of Welch's t for every column of a and b
    (runs along axis 0); a column with no scatter on either side beyond
    rounding (standard error below 1e-12 of the quantity's scale: the driven
    electrode's potential, a time average of the drive alone) gives 0 when
    the means agree to 1e-9 of the scale"""
    a, b = np.asarray(a, dtype=float), np.asarray(b, dtype=float)
    na, nb = a.shape[0], b.shape[0]
    va, vb = a.var(axis=0, ddof=1) / na, b.var(axis=0, ddof=1) / nb
    diff = a.mean(axis=0) - b.mean(axis=0)
    se2 = va + vb
    scale = np.sqrt(np.mean(b.mean(axis=0) ** 2)) + 1e-300
    z = np.zeros_like(diff)
    ok = se2 > (1e-12 * scale) ** 2
    t = diff[ok] / np.sqrt(se2[ok])
    dof = se2[ok] ** 2 / (va[ok] ** 2 / (na - 1) + vb[ok] ** 2 / (nb - 1))
    # the same two-sided tail probability under a standard normal
    p = 2.0 * stats.t.sf(np.abs(t), dof)
    z[ok] = np.sign(t) * stats.norm.isf(np.maximum(p, 1e-300) / 2.0)
    z[~ok] = np.where(np.abs(diff[~ok]) <= 1e-9 * scale, 0.0, np.inf)
    return z


def compare_labeled(ens_a, ens_b, min_iedf_bins=1):
    """z of every node of the densities and potential and of every EEDF and
    IEDF bin with at least MIN_COUNTS counts on both sides; returns
    (z array, {part: number of quantities}, [(part, index) of each z])"""
    zs, sizes, labels = [], {}, []
    for key in ("dens", "phi"):
        z = welch_z([g[key].ravel() for g in ens_a], [o[key].ravel() for o in ens_b])
        zs.append(z)
        sizes[key] = len(z)
        labels += [(key, i) for i in range(len(z))]
    for key in ("eedf", "iedf"):
        a = np.array([g[key] for g in ens_a])
        b = np.array([o[key] for o in ens_b])
        keep = (a.mean(axis=0) >= MIN_COUNTS) & (b.mean(axis=0) >= MIN_COUNTS)
        need = min_iedf_bins if key == "iedf" else 2
        assert keep.sum() >= need, (key, int(keep.sum()), need)
        z = welch_z(a[:, keep], b[:, keep])
        zs.append(z)
        sizes[key] = len(z)
        labels += [(key, int(i)) for i in np.flatnonzero(keep)]
    return np.concatenate(zs), sizes, labels


def compare(ens_a, ens_b, min_iedf_bins=1):
    """compare_labeled without the labels"""
    z, sizes, _ = compare_labeled(ens_a, ens_b, min_iedf_bins)
    return z, sizes


def worst(ens_a, ens_b, n=5, min_iedf_bins=1):
    """the n quantities of largest |z|: part, flat index, z and each
    ensemble's mean and standard deviation there"""
    z, _, labels = compare_labeled(ens_a, ens_b, min_iedf_bins)
    out = []
    for j in np.argsort(-np.abs(z))[:n]:
        key, i = labels[j]
        a = np.array([np.asarray(g[key], dtype=float).ravel()[i] for g in ens_a])
        b = np.array([np.asarray(o[key], dtype=float).ravel()[i] for o in ens_b])
        out.append({"part": key, "index": i, "z": float(z[j]), "mean_a": float(a.mean()),
                    "sd_a": float(a.std(ddof=1)), "mean_b": float(b.mean()), "sd_b": float(b.std(ddof=1))})
    return out


def within_3(zs):
    """fraction of the quantities with |z| <= 3"""
    return float(np.mean(np.abs(zs) <= 3.0))
