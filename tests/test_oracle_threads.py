"""The oracle's optional OpenMP particle loops (used for the all-core CPU baseline) give
the same step as the single-threaded oracle: every particle's outcome goes to its own slot
and births are appended in index order afterwards.  Every array, the counters and the set
of logged near-tie decisions must agree exactly."""
import math
import os

import numpy as np

import oracle
import workloads


def _run(orc, threads, steps=60):
    orc.set_threads(threads)
    wl = workloads.c2(n=1500, seed=23)
    shift = 8.5 * math.pi
    wl["e"]["z"] = wl["e"]["z"] + shift
    wl["t0"], wl["step0"] = shift, int(round(shift / wl["dt"]))
    s = oracle.Sim(orc, wl)
    orc.set_near_tol(1e-3)
    try:
        st = s.run(steps, oracle.F_NCS | oracle.F_NBW | oracle.F_VB | oracle.F_SPIN)
        ids, steps_, kinds, m = orc.near_log()
    finally:
        orc.set_near_tol(1e-6)
        orc.set_threads(1)
    log = sorted(zip(ids.tolist(), steps_.tolist(), kinds.tolist(), m.tolist()))
    return s.state(), st, log


def test_threaded_step_equals_serial(orc):
    n = max(2, min(os.cpu_count() or 2, 8))
    a, sa, la = _run(orc, 1)
    b, sb, lb = _run(orc, n)
    assert sa == sb and sa["n_nbw"] > 0 and sa["n_ncs_p"] > 0
    assert a["next_id"] == b["next_id"]
    for sp in ("e", "pos", "ph"):
        for k in a[sp]:
            assert np.array_equal(a[sp][k], b[sp][k]), (sp, k)
    assert la == lb and len(la) > 0
