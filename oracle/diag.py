"""Oracle of the end-of-run observables (test infrastructure: only tests, the smoke check and
the benchmark's CPU baseline use this package).

Follows the post-processing of the paper's VB algorithm (Sec. IV, the algorithm "VB effect
in SLIPs"): select a detection basis, rotate each photon's Stokes parameters from its own
basis to it with Eq. (rotation), and average per detector cell; and the spectra / mean spin
/ yield read-outs of Sec. IV.  Plain numpy in float64: per-particle values, then
``np.add.at`` into the bins.

Conventions (the same as the step's): a photon's basis vector P1 lies at angle theta from
e1 of the canonical frame of n = k/|k| (e1 = unit(y x n), or unit(n x x) within 1e-10 of
+-y; e2 = n x e1).  The detection basis is d1 = unit(ref - (ref.n) n), d2 = n x d1; the
Stokes parameters go from the angle theta to the angle of d1 by ROT(psi), psi = theta_d1 -
theta, with P1' = P1 cos psi + P2 sin psi (Sec. III D).
"""
from __future__ import annotations

import numpy as np

SPECTRUM, DETECTOR = 0, 1


def canonical_frame(n: np.ndarray):
    """e1, e2 of the canonical transverse frame of unit directions n [N, 3]."""
    a, b, c = n[:, 2].copy(), np.zeros(len(n)), -n[:, 0]
    m2 = a * a + c * c
    near_y = m2 < 1e-20
    a[near_y], b[near_y], c[near_y] = 0.0, n[near_y, 2], -n[near_y, 1]
    m2 = a * a + b * b + c * c
    e1 = np.stack([a, b, c], 1) / np.sqrt(m2)[:, None]
    e2 = np.cross(n, e1)
    return e1, e2


def rot(psi: np.ndarray, xi: np.ndarray) -> np.ndarray:
    """Eq. (rotation): Stokes parameters w.r.t. the basis turned by psi."""
    c2, s2 = np.cos(2 * psi), np.sin(2 * psi)
    return np.stack([xi[:, 0] * c2 - xi[:, 2] * s2, xi[:, 1], xi[:, 0] * s2 + xi[:, 2] * c2], 1)


def detector_stokes(k: np.ndarray, theta: np.ndarray, xi: np.ndarray, ref=(1.0, 0.0, 0.0)) -> np.ndarray:
    n = k / np.linalg.norm(k, axis=1)[:, None]
    e1, e2 = canonical_frame(n)
    r = np.asarray(ref, dtype=np.float64)
    d1 = r[None, :] - (n @ r)[:, None] * n
    dd = np.einsum("ij,ij->i", d1, d1)
    th_d = np.where(dd < 1e-20, 0.0, np.arctan2(np.einsum("ij,ij->i", d1, e2), np.einsum("ij,ij->i", d1, e1)))
    return rot(th_d - theta, xi)


def diag(d: dict, kind: int, nx: int, ny: int = 1, lo_x=1.0, hi_x=2.0, lo_y=0.0, hi_y=1.0,
         ref=(0.0, 0.0, 0.0), photon: bool = False) -> dict:
    """Bins [ny, nx, 5] of {sum w, sum w o1, sum w o2, sum w o3, count}, the same five over the
    whole set, and sum w below / above the range (detector: outside counts as above)."""
    n = len(d["id"])
    w = np.asarray(d["w"], dtype=np.float64)
    p = np.stack([d["px"], d["py"], d["pz"]], 1).astype(np.float64)
    o = np.stack([d["s1"], d["s2"], d["s3"]], 1).astype(np.float64)
    if photon:
        energy = np.linalg.norm(p, axis=1)
        r = np.asarray(ref, dtype=np.float64)
        if not np.any(r):
            r = np.array([1.0, 0.0, 0.0])
        ok = energy > 0
        if ok.any():
            o[ok] = detector_stokes(p[ok], np.asarray(d["theta"], dtype=np.float64)[ok], o[ok], r)
    else:
        energy = np.sqrt(1.0 + np.einsum("ij,ij->i", p, p))
    vals = np.concatenate([w[:, None], w[:, None] * o, np.ones((n, 1))], 1)
    bins = np.zeros((ny * nx, 5))
    below = above = 0.0
    if kind == SPECTRUM:
        with np.errstate(divide="ignore"):
            t = np.where(energy > 0, (np.log(energy) - np.log(lo_x)) * (nx / (np.log(hi_x) - np.log(lo_x))), -1.0)
        lo_m, hi_m = t < 0, t >= nx
        inside = ~(lo_m | hi_m)
        idx = np.minimum(t[inside].astype(np.int64), nx - 1)
        below, above = float(w[lo_m].sum()), float(w[hi_m].sum())
    else:
        tx = (np.asarray(d["x"], dtype=np.float64) - lo_x) * (nx / (hi_x - lo_x))
        ty = (np.asarray(d["y"], dtype=np.float64) - lo_y) * (ny / (hi_y - lo_y))
        inside = (tx >= 0) & (ty >= 0) & (tx < nx) & (ty < ny)
        idx = np.minimum(tx[inside].astype(np.int64), nx - 1) + nx * np.minimum(ty[inside].astype(np.int64), ny - 1)
        above = float(w[~inside].sum())
    np.add.at(bins, idx, vals[inside])
    return {"bins": bins.reshape(ny, nx, 5), "total": vals.sum(0), "below": below, "above": above}
