"""One step of an FP32 replay compared particle by particle, with decision
flips told apart from arithmetic error.

In a replay step the GPU and the oracle both start from the oracle's state
and take one step.  A particle that meets no collision keeps vy and vz (the
push changes only x and vx), so its (vy, vz) before the step identifies it
after the step on each side, whatever the sort did to the slot order: exactly
on the oracle's side, and as the GPU holds it (FP32) on the GPU's side.

* Push-only particles (identified on both sides, alive on both): their error
  is arithmetic error alone and must stay within the tolerance; there is no
  decision that could explain more.
* A particle identified on both sides but alive on one only took a different
  decision (absorption, a kill in the particle-target pass): a flip.
* The remaining live particles of each side (collided, newborn) are paired
  in slot order, aligned by position (a collision does not move a
  particle); a pair beyond the tolerance took a different collision outcome
  (channel, partner) and is a flip, as is a particle left without a partner.
  When a Coulomb pass ran, a cell whose particles differ between the sides
  is re-paired as a whole: such cells are counted and left out instead.

Errors: |dx| / L for the position; |dv| / max(v_th, |v|) per component for
the velocity, i.e. relative to the particle's own speed once it is faster
than thermal (FP32 holds a velocity to 6e-8 of itself, so a sheath ion at
over 80 thermal speeds cannot be held to 1e-5 of the thermal speed).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

QE = 1.602176634e-19
AMU = 1.66053906660e-27
ME = 9.1093837015e-31
MASS = (ME, 16 * AMU + ME, 32 * AMU - ME)


def vth(d, s):
    return math.sqrt(max(d.T0_eV[s], 0.0259) * QE / MASS[s])


@dataclasses.dataclass
class StepResult:
    compared: int = 0        # particles compared (push-only and paired collided ones)
    flips: int = 0           # particles whose discrete decision differs
    worst: float = 0.0       # largest error of the push-only particles (must be < tol)
    worst_paired: float = 0.0  # largest error of the collided pairs within tol
    worst_flip: float = 0.0  # largest error among paired flips (reported)
    recount_cells: int = 0   # cells re-paired by a Coulomb pass (count differs)
    excluded: int = 0        # particles in those cells
    # flips by kind: alive on one side only, (unused), paired with an error
    # in [tol, 10 tol), [10 tol, 100 tol), beyond, unpaired
    kinds: tuple = (0, 0, 0, 0, 0, 0)

    def add(self, o: "StepResult") -> "StepResult":
        return StepResult(self.compared + o.compared, self.flips + o.flips, max(self.worst, o.worst),
                          max(self.worst_paired, o.worst_paired), max(self.worst_flip, o.worst_flip),
                          self.recount_cells + o.recount_cells, self.excluded + o.excluded,
                          tuple(a + b for a, b in zip(self.kinds, o.kinds)))


def _keys(st):
    return np.asarray(st["vy"], dtype=np.float64) + 1j * np.asarray(st["vz"], dtype=np.float64)


def _identify(pre, post):
    """index into `pre` of every particle of `post` carrying a (vy, vz) that
    occurs exactly once in `pre`; -1 otherwise"""
    kp = _keys(pre)
    order = np.argsort(kp, kind="stable")
    sk = kp[order]
    uniq = np.ones(len(sk), dtype=bool)
    if len(sk) > 1:
        dup = sk[1:] == sk[:-1]
        uniq[1:] &= ~dup
        uniq[:-1] &= ~dup
    kq = _keys(post)
    if len(sk) == 0:
        return np.full(len(kq), -1, dtype=np.int64)
    pos = np.clip(np.searchsorted(sk, kq), 0, len(sk) - 1)
    hit = (sk[pos] == kq) & uniq[pos]
    return np.where(hit, order[pos], -1)


def _err(d, s, a, ia, b, ib):
    """error of particles a[ia] against b[ib] (b is the oracle's side)"""
    ex = np.abs(a["x"][ia] - b["x"][ib]) / d.L
    vb = np.sqrt(b["vx"][ib] ** 2 + b["vy"][ib] ** 2 + b["vz"][ib] ** 2)
    scale = np.maximum(vth(d, s), vb)
    e = ex
    for c in ("vx", "vy", "vz"):
        e = np.maximum(e, np.abs(a[c][ia] - b[c][ib]) / scale)
    return e


# positions of one particle on the two sides agree to FP32 rounding of the
# offset (below 1e-6 of a cell); unrelated particles are this close with a
# chance of about 1e-5
X_MATCH = 1e-5


def align(xg, xo, tol_x, look=8):
    """Align two sequences of positions that are equal up to a few inserted
    or missing elements: returns (paired indices of xg, of xo, unpaired of
    xg, unpaired of xo).  Runs of agreeing elements are taken whole; at a
    disagreement the nearer of a skip on either side (up to `look` ahead)
    that restores agreement is taken, else both elements stay unpaired."""
    ng, no = len(xg), len(xo)
    pg, po, ug, uo = [], [], [], []
    i = j = 0
    while i < ng and j < no:
        m = min(ng - i, no - j)
        agree = np.abs(xg[i:i + m] - xo[j:j + m]) <= tol_x
        k = int(np.argmin(agree)) if not agree.all() else m
        pg.append(np.arange(i, i + k))
        po.append(np.arange(j, j + k))
        i += k
        j += k
        if k == m:
            break
        skip = None
        for t in range(1, look + 1):
            if j + t < no and abs(xg[i] - xo[j + t]) <= tol_x:
                skip = ("o", t)
                break
            if i + t < ng and abs(xg[i + t] - xo[j]) <= tol_x:
                skip = ("g", t)
                break
        if skip is None:
            ug.append(np.array([i]))
            uo.append(np.array([j]))
            i += 1
            j += 1
        elif skip[0] == "o":
            uo.append(np.arange(j, j + skip[1]))
            j += skip[1]
        else:
            ug.append(np.arange(i, i + skip[1]))
            i += skip[1]
    ug.append(np.arange(i, ng))
    uo.append(np.arange(j, no))
    cat = lambda v: np.concatenate(v).astype(np.int64) if v else np.zeros(0, np.int64)
    return cat(pg), cat(po), cat(ug), cat(uo)


def compare_step(d, s, pre_o, pre_g, g, o, tol, coulomb=False) -> StepResult:
    """Species s after one replay step: pre_o / pre_g the oracle's and the
    GPU's state before it, g / o after it (dicts of x, vx, vy, vz, alive)."""
    r = StepResult()
    ga, oa = np.asarray(g["alive"], bool), np.asarray(o["alive"], bool)
    gid, oid = _identify(pre_g, g), _identify(pre_o, o)
    npre = len(pre_o["x"])
    # pre index -> post index on each side
    gpos = np.full(npre, -1, dtype=np.int64)
    opos = np.full(npre, -1, dtype=np.int64)
    gpos[gid[gid >= 0]] = np.flatnonzero(gid >= 0)
    opos[oid[oid >= 0]] = np.flatnonzero(oid >= 0)
    both = (gpos >= 0) & (opos >= 0)
    gal = np.zeros(npre, bool)
    oal = np.zeros(npre, bool)
    gal[gid[gid >= 0]] = ga[gid >= 0]
    oal[oid[oid >= 0]] = oa[oid >= 0]
    push_only = both & gal & oal
    kinds = [0] * 6
    # identified on both sides but alive on one only: absorption or kill
    kinds[0] = int(np.sum(both & (gal != oal)))
    if push_only.any():
        e = _err(d, s, g, gpos[push_only], o, opos[push_only])
        r.worst = float(e.max())
        r.compared += int(push_only.sum())
    # the rest: live particles without a common identity (collided on either
    # side, newborn; a collision on one side only, or a kick below FP32
    # resolution, leaves the identity on one side), in slot order on each side.  Both sides order them alike (births in
    # parent order, a stable sort by cell), except around a particle that
    # only one side holds (a decision that differs) or that sits in another
    # cell; the two sequences are aligned by position, which a collision
    # does not change.
    gi_used = np.zeros(len(ga), bool)
    oi_used = np.zeros(len(oa), bool)
    gi_used[gpos[both]] = True
    oi_used[opos[both]] = True
    grest = np.flatnonzero(ga & ~gi_used)
    orest = np.flatnonzero(oa & ~oi_used)
    N, dx = d.n_cells, d.L / d.n_cells
    pg, po, ug, uo = align(np.asarray(g["x"])[grest], np.asarray(o["x"])[orest], X_MATCH * dx)
    pg, po = grest[pg], orest[po]
    ug, uo = grest[ug], orest[uo]
    if coulomb:
        # a cell whose particles differ between the sides is re-paired by
        # the Coulomb pass: all of its particles are left out
        cell = lambda st, i: np.clip(np.floor(np.asarray(st["x"])[i] / dx).astype(np.int64), 0, N - 1)
        bad = np.zeros(N, bool)
        bad[cell(g, ug)] = True
        bad[cell(o, uo)] = True
        keep = ~bad[cell(o, po)]
        r.recount_cells = int(bad.sum())
        r.excluded = int(len(po) - keep.sum() + len(ug) + len(uo))
        pg, po = pg[keep], po[keep]
    else:
        kinds[5] += int(len(ug) + len(uo))
    if len(pg):
        e = _err(d, s, g, pg, o, po)
        ok = e <= tol
        r.compared += int(len(e))
        kinds[2] += int(np.sum(~ok & (e < 10 * tol)))
        kinds[3] += int(np.sum((e >= 10 * tol) & (e < 100 * tol)))
        kinds[4] += int(np.sum(e >= 100 * tol))
        r.worst_paired = float(e[ok].max(initial=0.0))
        r.worst_flip = float(e[~ok].max(initial=0.0))
    r.kinds = tuple(kinds)
    r.flips = sum(kinds)
    return r
