"""The near-tie rule of the GPU-vs-oracle parity tests.

Every Monte Carlo decision of the step compares a uniform draw r with a threshold: the
emission or decay probability W dt (Secs. III C, D), the spin-collapse probabilities
(1 + |S|)/2 and (1 + |g|/c0)/2, the photon pure-state probability (1 + |F|/F0)/2, the
weights of the energy mixtures and the cumulative weights of the four pair-spin outcomes.
An implementation whose threshold carries a relative error e can take the other branch
only where |r - thr| < e thr.  The oracle logs every decision of a step whose draw lies
within ``LOG_TOL`` relative of its threshold (kind, id, step, margin = |r - thr|/thr);
a GPU particle that differs from the oracle is exempted only when one of its logged
margins lies below the bound of its path:

* FP64 path: ``NEAR_FP64`` = 1e-6, the rule stated for the FP64 step (its thresholds agree
  with the oracle's to ~1e-12, so in practice nothing is exempted).
* Mixed path: ``NEAR_MIXED`` = 1e-4.  Its thresholds are formed in FP32 from FP32 state:
  the field phase and envelope argument are float sums of values up to ~100 (relative
  error ~1e-5 of chi for a circularly polarised pulse), the rate tables are float cubics
  (~1e-6), and over a multi-step run the state itself drifts from the oracle's by up to
  the 2e-5 per-particle tolerance, which a threshold (linear to ~chi^(2/3..1) in it)
  carries at most twice.  1e-4 covers 2.5x that budget.

Everything else must agree: no other mismatch is allowed.  The tests report the number of
particles exempted and the largest margin among them.
"""
from __future__ import annotations

import numpy as np

LOG_TOL = 1e-3
NEAR_FP64 = 1e-6
NEAR_MIXED = 1e-4


def bound(mixed: bool) -> float:
    return NEAR_MIXED if mixed else NEAR_FP64


def near_margins(orc, step=None) -> dict:
    """id -> smallest logged margin (over the decisions of `step`, or of every step)."""
    ids, steps, _kinds, m = orc.near_log()
    if step is not None:
        sel = steps == step
        ids, m = ids[sel], m[sel]
    out: dict = {}
    for i, v in zip(ids.tolist(), m.tolist()):
        if v < out.get(i, np.inf):
            out[i] = v
    return out


def exemptions(mismatched_ids, margins: dict, mixed: bool):
    """Split mismatched particle ids into (exempted, unexplained) and return the largest
    margin among the exempted ones (0 if none)."""
    b = bound(mixed)
    ex, bad, worst = [], [], 0.0
    for i in mismatched_ids:
        m = margins.get(int(i), np.inf)
        if m < b:
            ex.append(int(i))
            worst = max(worst, m)
        else:
            bad.append((int(i), m))
    return ex, bad, worst
