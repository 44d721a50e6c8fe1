"""Bremsstrahlung and Bethe-Heitler pair creation in matter (paper Sec. III E) on the GPU,
against the oracle through the C ABI.

* The medium tables built on the device equal the oracle's (both follow one table
  specification, each with its own code).
* FP64 path, a 1 GeV electron beam through a gold slab (the paper's test geometry, no
  field): every bremsstrahlung photon, every pair and every particle agree with the
  oracle -- ids and counts exactly, momenta, spins and positions to 1e-10.
* FP64 path, matter and field together (a crossed field inside a gold slab, e-, e+
  and photons, every process on): the one-event-per-step rule between NCS and
  bremsstrahlung and between NBW and pairs is the oracle's.
* Mixed path: every primary electron within 2e-5 over 60 steps (near-tie rule), and the
  photon and pair counts of the two within 3 sigma.
* Validation: matter flags without a medium, a medium outside Tsai's range, batches.
"""
import math

import numpy as np
import pytest

import oracle
import parity_rules
import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2306_11288_gb300 as q  # noqa: E402

MED = q.QED_F_BREMS | q.QED_F_BH
ALL = q.QED_F_NCS | q.QED_F_NBW | q.QED_F_VB | q.QED_F_SPIN


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    q.build()
    c = q.qed_init_tables()
    yield c
    torch.cuda.synchronize()


def _by_id(d):
    o = np.argsort(d["id"], kind="stable")
    return {k: v[o] for k, v in d.items()}


def _compare(g, o, tol):
    for sp in ("e", "pos", "ph"):
        a, b = _by_id(g[sp]), _by_id(o[sp])
        assert np.array_equal(a["id"], b["id"]), (sp, len(a["id"]), len(b["id"]))
        for k in ("px", "py", "pz", "s1", "s2", "s3", "x", "y", "z"):
            assert np.all(np.abs(a[k] - b[k]) <= tol * np.maximum(np.abs(b[k]), 1.0)), (sp, k)
        assert np.array_equal(a["w"], b["w"])


def test_medium_tables_match_oracle(orc, ctx):
    med = workloads.medium("Au", k_min=1.0)
    q.qed_set_medium(ctx, med)
    orc.set_medium(med)
    g = q.qed_copy_medium_table(ctx).reshape(2, 256, 512)
    o = orc.table(7).reshape(2, 256, 512)
    scale = np.maximum(o[:, :, -1:], 1e-300)
    assert (np.abs(g - o) / scale).max() < 1e-11
    assert o[0, 100, -1] > 0 and o[1, 200, -1] > 0
    q.qed_set_medium(ctx, None)
    orc.set_medium(None)


def _caps(n):
    return {"cap_e": 3 * n + 1024, "cap_p": 2 * n + 1024, "cap_ph": 40 * n + 1024}


def test_slab_fp64_matches_oracle(orc, ctx):
    """1 GeV electrons, 5 um steps through 5 mm of gold: 120 steps (0.6 mm)."""
    n = 3000
    wl = workloads.slab(n=n, seed=8)
    sim = q.Simulation(wl, prec=q.QED_PREC_F64, ctx=ctx, **_caps(n))
    osim = oracle.Sim(orc, wl, **_caps(n))
    sim.run(120, MED)
    ost = osim.run(120, MED)
    c = sim.counters()
    assert c["n_brems_e"] == ost["n_brems_e"] > 1000 and c["n_bh"] == ost["n_bh"] > 0
    assert c["n_brems_p"] == ost["n_brems_p"]
    assert sim.status() == 0
    g, o = sim.state(), osim.state()
    assert g["next_id"] == o["next_id"]
    _compare(g, o, 1e-10)
    sim.close()


def test_matter_with_field_fp64_matches_oracle(orc, ctx):
    """e-, e+ and polarised photons in a strong crossed field inside a (20x denser) gold
    slab, every process on: NCS or bremsstrahlung (one event per lepton per step), NBW or
    pairs (one decay per photon per step); the pairs' leptons start unpolarised (S = 0)."""
    rng = np.random.default_rng(4)

    def lep(n, first):
        s = rng.normal(size=(n, 3))
        s /= np.linalg.norm(s, axis=1, keepdims=True)
        p = rng.normal(size=(n, 3)) * 30 + np.array([0, 0, 4000.0])
        return {"x": rng.normal(size=n), "y": rng.normal(size=n), "z": rng.uniform(0, 6e3, n),
                "px": p[:, 0], "py": p[:, 1], "pz": p[:, 2], "s1": s[:, 0], "s2": s[:, 1], "s3": s[:, 2],
                "w": rng.uniform(0.5, 2, n), "id": np.arange(first, first + n, dtype=np.uint64)}
    e, pos = lep(1500, 0), lep(700, 1500)
    nph = 3000
    k = rng.normal(size=(nph, 3)) * 50 + np.array([0, 0, 3000.0])
    xi = rng.normal(size=(nph, 3))
    xi *= rng.uniform(0, 1, (nph, 1)) / np.linalg.norm(xi, axis=1, keepdims=True)
    ph = {"x": rng.normal(size=nph), "y": rng.normal(size=nph), "z": rng.uniform(0, 6e3, nph), "px": k[:, 0],
          "py": k[:, 1], "pz": k[:, 2], "s1": xi[:, 0], "s2": xi[:, 1], "s3": xi[:, 2],
          "theta": rng.uniform(-3, 3, nph), "w": np.ones(nph), "id": np.arange(2200, 2200 + nph, dtype=np.uint64)}
    E0 = 40.0
    med = workloads.medium("Au", thickness_mm=1.0, k_min=2.0)
    med["n"] *= 20   # a denser gold, so that matter events compete with the field's in 40 steps
    wl = {"e": e, "pos": pos, "ph": ph, "field": {"kind": "uniform", "E": (E0, 0, 0), "B": (0, -E0, 0)},
          "dt": 0.3, "seed": 12, "next_id": 2200 + nph, "medium": med}
    caps = _caps(6000)
    sim = q.Simulation(wl, prec=q.QED_PREC_F64, ctx=ctx, **caps)
    osim = oracle.Sim(orc, wl, **caps)
    sim.run(40, ALL | MED)
    ost = osim.run(40, ALL | MED)
    c = sim.counters()
    for key in ("n_ncs_e", "n_ncs_p", "n_nbw", "n_brems_e", "n_brems_p", "n_bh"):
        assert c[key] == ost[key], key
    assert c["n_ncs_e"] > 0 and c["n_brems_e"] > 0 and c["n_brems_p"] > 0 and c["n_nbw"] > 0 and c["n_bh"] > 0
    assert sim.status() == 0
    g, o = sim.state(), osim.state()
    assert g["next_id"] == o["next_id"]
    _compare(g, o, 1e-10)
    sim.close()


def test_slab_mixed_per_particle_and_counts(orc, ctx):
    """Mixed path, 60 steps of the gold slab: every primary electron within 2e-5 (momentum,
    spin, position) unless the oracle logged one of its decisions within the mixed-path
    bound of its threshold; bremsstrahlung and pair counts within 3 sigma of the FP64
    oracle's."""
    n = 6000
    wl = workloads.slab(n=n, seed=9)
    sim = q.Simulation(wl, prec=q.QED_PREC_MIXED, ctx=ctx, **_caps(n))
    osim = oracle.Sim(orc, wl, **_caps(n))
    orc.set_near_tol(parity_rules.LOG_TOL)
    try:
        sim.run(60, MED)
        ost = osim.run(60, MED)
        margins = parity_rules.near_margins(orc)
    finally:
        orc.set_near_tol(parity_rules.NEAR_FP64)
    c = sim.counters()
    for key in ("n_brems_e", "n_bh"):
        assert abs(c[key] - ost[key]) <= 3 * math.sqrt(c[key] + ost[key] + 1), key
    g, o = _by_id(sim.state()["e"]), _by_id(osim.state()["e"])
    prim = np.arange(n, dtype=np.uint64)
    g = {k: v[np.isin(g["id"], prim)] for k, v in g.items()}
    o = {k: v[np.isin(o["id"], prim)] for k, v in o.items()}
    assert np.array_equal(g["id"], o["id"])
    pg, po = (np.stack([d["px"], d["py"], d["pz"]], 1) for d in (g, o))
    dp = np.linalg.norm(pg - po, axis=1) / np.linalg.norm(po, axis=1)
    ds = np.abs(np.stack([g[k] - o[k] for k in ("s1", "s2", "s3")], 1)).max(1)
    dx = np.abs(np.stack([(g[k] - o[k]) / (np.abs(o[k]) + 1.0) for k in ("x", "y", "z")], 1)).max(1)
    bad = (dp > 2e-5) | (ds > 2e-5) | (dx > 2e-5)
    ex, unexplained, worst = parity_rules.exemptions(g["id"][bad], margins, mixed=True)
    print(f"mixed slab: {len(ex)} exempted, max dp {dp[~bad].max():.2e}")
    assert not unexplained, unexplained[:10]
    sim.close()


def test_matter_validation(ctx):
    wl = workloads.slab(n=64, seed=1)
    wl_no = dict(wl)
    wl_no.pop("medium")
    sim = q.Simulation(wl_no, prec=q.QED_PREC_F64, ctx=ctx, **_caps(64))
    q.qed_set_medium(sim.ctx, None)
    with pytest.raises(q.QedError, match="medium"):
        sim.run(1, q.QED_F_BREMS)
    with pytest.raises(q.QedError, match="Z"):
        q.qed_set_medium(sim.ctx, dict(workloads.medium("Al"), Z=3))
    with pytest.raises(q.QedError, match="radiative pusher"):
        q.qed_set_medium(sim.ctx, workloads.medium("Al"))
        sim.run(1, q.QED_F_BREMS | q.QED_F_MLL)
    q.qed_set_medium(sim.ctx, None)
    sim.close()
