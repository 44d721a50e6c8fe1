"""Parity at full size, in the launch configuration the benchmark times.

1. Ragged e-, e+ and photon counts spanning several tiles per block in a strong crossed
   field: the FP64 path against the oracle particle by particle (ids, births, values to
   1e-10), and the mixed path run twice, bit for bit.
2. The 1e6-electron focused-pulse workload at its benchmark state (150 steps in, the
   beam at the focus): after one more GPU step, a random sample of particles is stepped
   by the oracle from the same pre-step state (the random numbers of a particle depend
   only on its id, the step and the seed) and compared one by one.  FP64 path: decisions
   exact, values within 1e-10.  Mixed path: values within 2e-5.  On either path a particle
   may differ only where the oracle logged a decision whose draw lay within the path's
   near-tie bound of its threshold (``parity_rules``); no other mismatch is allowed.
3. The grid workload at its full size (3e7 electrons, 4096 x 2048 FP32 Yee grid, TSC
   gather): the same sampled comparison, 12 steps in, drawn mostly from the particles
   inside the reflected pulse."""
import math

import numpy as np
import pytest

import oracle
import parity_rules
import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2306_11288_gb300 as q  # noqa: E402

ALL = q.QED_F_NCS | q.QED_F_NBW | q.QED_F_VB | q.QED_F_SPIN


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    q.build()
    c = q.qed_init_tables()
    yield c
    torch.cuda.synchronize()


def _crossed_field_sets(ne, npos, nph, seed):
    rng = np.random.default_rng(seed)

    def lep(n, first):
        s = rng.normal(size=(n, 3))
        s /= np.linalg.norm(s, axis=1, keepdims=True)
        p = rng.normal(size=(n, 3)) * 30 + np.array([0, 0, 4000.0])
        return {"x": rng.normal(size=n), "y": rng.normal(size=n), "z": rng.normal(size=n),
                "px": p[:, 0], "py": p[:, 1], "pz": p[:, 2], "s1": s[:, 0], "s2": s[:, 1], "s3": s[:, 2],
                "w": rng.uniform(0.5, 2, n), "id": np.arange(first, first + n, dtype=np.uint64)}

    e, pos = lep(ne, 0), lep(npos, ne)
    k = rng.normal(size=(nph, 3)) * 50 + np.array([0, 0, 3000.0])
    xi = rng.normal(size=(nph, 3))
    xi *= rng.uniform(0, 1, (nph, 1)) / np.linalg.norm(xi, axis=1, keepdims=True)
    first = ne + npos
    ph = {"x": rng.normal(size=nph), "y": rng.normal(size=nph), "z": rng.normal(size=nph), "px": k[:, 0],
          "py": k[:, 1], "pz": k[:, 2], "s1": xi[:, 0], "s2": xi[:, 1], "s3": xi[:, 2],
          "theta": rng.uniform(-3, 3, nph), "w": np.ones(nph), "id": np.arange(first, first + nph, dtype=np.uint64)}
    E0 = 150.0
    return {"e": e, "pos": pos, "ph": ph, "field": {"kind": "uniform", "E": (E0, 0, 0), "B": (0, -E0, 0)},
            "dt": math.pi / 100, "seed": 9, "next_id": first + nph}


def _ragged_sizes(blocks_per_sm):
    per = torch.cuda.get_device_properties(0).multi_processor_count * blocks_per_sm * 256
    return 3 * per + 1234, per + 77, 4 * per + 99   # several tiles per block, ragged tails


def _by_id(d):
    o = np.argsort(d["id"], kind="stable")
    return {k: v[o] for k, v in d.items()}


def test_many_tiles_per_block_fp64_matches_oracle(orc, ctx):
    """FP64 grid (2 blocks per SM): every particle, id and birth against the oracle."""
    wl = _crossed_field_sets(*_ragged_sizes(2), seed=62)
    sim = q.Simulation(wl, prec=q.QED_PREC_F64, ctx=ctx)
    osim = oracle.Sim(orc, wl)
    sim.run(3, ALL)
    ost = osim.run(3, ALL)
    c = sim.counters()
    assert c["n_ncs_e"] == ost["n_ncs_e"] > 0 and c["n_ncs_p"] == ost["n_ncs_p"] > 0
    assert c["n_nbw"] == ost["n_nbw"] > 0 and sim.status() == 0
    g, o = sim.state(), osim.state()
    assert g["next_id"] == o["next_id"]
    for sp in ("e", "pos", "ph"):
        a, b = _by_id(g[sp]), _by_id(o[sp])
        assert np.array_equal(a["id"], b["id"]), sp
        for k in ("px", "py", "pz", "s1", "s2", "s3", "x", "y", "z"):
            assert np.all(np.abs(a[k] - b[k]) <= 1e-10 * np.maximum(np.abs(b[k]), 1.0)), (sp, k)
        assert np.array_equal(a["w"], b["w"])
    sim.close()


def test_many_tiles_per_block_mixed_is_deterministic(ctx):
    """Mixed grid (4 blocks per SM): the event log fills in a different order on every run
    (atomics), the ranks do not depend on it, so two runs agree bit for bit."""
    wl = _crossed_field_sets(*_ragged_sizes(4), seed=61)
    runs = []
    for _ in range(2):
        sim = q.Simulation(wl, prec=q.QED_PREC_MIXED, ctx=ctx)
        sim.run(6, ALL)
        runs.append((sim.state(), sim.counters(), sim.status()))
        sim.close()
    (a, ca, sa), (b, cb, sb) = runs
    assert sa == 0 and sb == 0
    assert ca == cb and ca["n_ncs_e"] > 0 and ca["n_ncs_p"] > 0 and ca["n_nbw"] > 0
    assert a["next_id"] == b["next_id"]
    for sp in ("e", "pos", "ph"):
        for k in a[sp]:
            assert np.array_equal(a[sp][k], b[sp][k]), (sp, k)


# ---------------------------------------------------------------------------------------
N_BENCH, PRE_STEPS, T_SHIFT = 1_000_000, 150, 8.5 * math.pi   # the benchmark's workload
N_GRID, PRE_GRID = 30_000_000, 12                             # the grid workload at size


def _bench_workload():
    wl = workloads.c2(n=N_BENCH, seed=2)
    wl["e"]["z"] = wl["e"]["z"] + T_SHIFT
    wl["t0"] = T_SHIFT
    wl["step0"] = int(round(T_SHIFT / wl["dt"]))
    return wl


def _take(d, ids):
    o = np.argsort(d["id"])
    pos = np.searchsorted(d["id"], ids, sorter=o)
    pos = np.clip(pos, 0, len(o) - 1) if len(o) else pos
    idx = o[pos] if len(o) else np.zeros(0, dtype=np.int64)
    found = (d["id"][idx] == ids) if len(o) else np.zeros(len(ids), dtype=bool)
    return {k: v[idx] for k, v in d.items()}, found


def _rows_at(sp, idx):
    """rows `idx` (device index tensor) of one species, copied to the host"""
    out = {}
    for k, v in sp.t.items():
        a = v[idx].cpu().numpy()
        out[k] = a.view(np.uint64) if k == "id" else a.astype(np.float64)
    return out


def _rows_of_ids(sp, ids):
    """the live rows whose id is in `ids` (selected on the device: no full-state copy)"""
    n = sp.count()
    want = torch.as_tensor(np.asarray(ids, dtype=np.uint64).view(np.int64), device="cuda")
    idx = torch.nonzero(torch.isin(sp.t["id"][:n], want)).flatten()
    return _rows_at(sp, idx)


def _pick(sp, k, rng, cand=None):
    """k random live rows of a species (from the candidate index tensor if given)"""
    n = sp.count()
    if cand is None:
        cand = torch.arange(n, device="cuda")
    m = int(cand.numel())
    sel = np.sort(rng.choice(m, size=min(k, m), replace=False)).astype(np.int64)
    return _rows_at(sp, cand[torch.as_tensor(sel, device="cuda")])


def _sample_parity(orc, sim, wl, pre, tol, mixed):
    """Step the GPU set once more; step the sampled pre-step rows `pre` once with the
    oracle from the same state; compare the sampled particles one by one."""
    t, step = sim.t, sim.step_no
    qed_next_id = q.qed_get_next_id(sim.ctx)
    sim.run(1, ALL)
    torch.cuda.synchronize()
    assert sim.status() == 0
    return _compare_sample(orc, sim, wl, pre, t, step, qed_next_id, tol, mixed)


def _compare_sample(orc, sim, wl, pre, t, step, qed_next_id, tol, mixed):
    """the sampled rows `pre` (state at (t, step)) stepped once by the oracle, against the
    rows of the same ids in the GPU set after its step"""
    pick = {sp: np.sort(pre[sp]["id"]) for sp in ("e", "pos", "ph")}
    post = {sp: _rows_of_ids(getattr(sim, sp), pick[sp]) for sp in ("e", "pos", "ph")}
    owl = {"field": wl["field"], "dt": wl["dt"], "seed": wl["seed"], "t0": t, "step0": step,
           "next_id": int(qed_next_id)}
    if "grid" in wl:
        owl["grid"] = wl["grid"]
    for sp in ("e", "pos", "ph"):
        owl[sp] = pre[sp]
    osim = oracle.Sim(orc, owl)
    orc.set_near_tol(parity_rules.LOG_TOL)
    try:
        ost = osim.run(1, ALL)
        margins = parity_rules.near_margins(orc, step)
    finally:
        orc.set_near_tol(parity_rules.NEAR_FP64)
    ostate = osim.state()

    total, exempt, unexplained, worst = 0, 0, [], 0.0
    for sp in ("e", "pos", "ph"):
        if not len(pick[sp]):
            continue
        g, gf = _take(post[sp], pick[sp])
        o, of = _take(ostate[sp], pick[sp])
        if sp != "ph":
            assert gf.all() and of.all()
        ok = gf & of
        # photons: decayed on one side only is a decision mismatch
        dec_mis = (gf != of)
        p_g = np.stack([g["px"], g["py"], g["pz"]], 1)
        p_o = np.stack([o["px"], o["py"], o["pz"]], 1)
        dp = np.linalg.norm(p_g - p_o, axis=1) / np.maximum(np.linalg.norm(p_o, axis=1), 1.0)
        ds = np.abs(np.stack([g[k] - o[k] for k in ("s1", "s2", "s3")], 1)).max(1)
        dx = np.abs(np.stack([(g[k] - o[k]) / (np.abs(o[k]) + 1.0) for k in ("x", "y", "z")], 1)).max(1)
        bad = dec_mis | (ok & ((dp > tol) | (ds > tol) | (dx > tol)))
        ex, un, w = parity_rules.exemptions(pick[sp][bad], margins, mixed)
        exempt += len(ex)
        unexplained += [(sp,) + u for u in un]
        worst = max(worst, w)
        total += len(pick[sp])
        good = ok & ~bad
        assert good.sum() > 0.9 * len(pick[sp]), sp
        assert np.array_equal(g["w"][good], o["w"][good])
    print(f"sampled parity ({'mixed' if mixed else 'FP64'}): {total} particles, {exempt} exempted "
          f"near-ties (largest margin {worst:.2e})")
    assert not unexplained, f"particles that differ without a near-tie (species, id, margin): {unexplained[:10]}"
    return ost


def _sample_step(orc, ctx, prec, tol):
    wl = _bench_workload()
    sim = q.Simulation(wl, prec=prec, ctx=ctx, cap_e=N_BENCH + 2_000_000, cap_p=2_000_000, cap_ph=10_000_000)
    sim.run(PRE_STEPS, ALL)
    torch.cuda.synchronize()
    assert sim.ph.count() > N_BENCH and sim.pos.count() > N_BENCH // 1000
    rng = np.random.default_rng(5)
    pre = {sp: _pick(getattr(sim, sp), n, rng) for sp, n in (("e", 4000), ("pos", 2000), ("ph", 6000))}
    ost = _sample_parity(orc, sim, wl, pre, tol, prec == q.QED_PREC_MIXED)
    assert ost["n_ncs_e"] > 0 and ost["n_nbw"] > 0
    sim.close()


def test_bench_workload_sampled_parity_fp64(orc, ctx):
    _sample_step(orc, ctx, q.QED_PREC_F64, 1e-10)


def test_bench_workload_sampled_parity_mixed(orc, ctx):
    _sample_step(orc, ctx, q.QED_PREC_MIXED, 2e-5)


@pytest.fixture(scope="module")
def grid_wl():
    return workloads.c3(n=N_GRID, seed=3)


def _grid_sample_step(orc, ctx, wl, prec, tol):
    """Config 3 at full size: 3e7 electrons on the 4096 x 2048 Yee grid (TSC gather),
    12 steps in (photons and pairs exist); the sample is drawn mostly from particles
    inside the reflected pulse, where every process is active."""
    sim = q.Simulation(wl, prec=prec, ctx=ctx, cap_e=N_GRID + 2_000_000, cap_p=2_000_000, cap_ph=20_000_000)
    sim.run(PRE_GRID, ALL)
    torch.cuda.synchronize()
    assert sim.ph.count() > 10_000
    rng = np.random.default_rng(6)
    x_lo = wl["grid"]["xs"] - 4.5 * 2 * math.pi   # the pulse reaches 4 wavelengths in front of the slab
    pre = {}
    for sp, n_in, n_any in (("e", 4000, 1000), ("pos", 1000, 0), ("ph", 4000, 1000)):
        s = getattr(sim, sp)
        n = s.count()
        hot = torch.nonzero(s.t["x"][:n] > x_lo).flatten()
        a = _pick(s, n_in, rng, hot)
        if n_any:
            b = _pick(s, n_any, rng)
            keep = ~np.isin(b["id"], a["id"])
            a = {k: np.concatenate([a[k], b[k][keep]]) for k in a}
        pre[sp] = a
    ost = _sample_parity(orc, sim, wl, pre, tol, prec == q.QED_PREC_MIXED)
    assert ost["n_ncs_e"] > 0
    sim.close()


def test_grid_workload_sampled_parity_fp64(orc, ctx, grid_wl):
    _grid_sample_step(orc, ctx, grid_wl, q.QED_PREC_F64, 1e-10)


def test_grid_workload_sampled_parity_mixed(orc, ctx, grid_wl):
    _grid_sample_step(orc, ctx, grid_wl, q.QED_PREC_MIXED, 2e-5)


def test_batch_workload_sampled_parity_mixed(orc, ctx):
    """The 64-ensemble batch at its full size (sizes 10^U(3,6), a0 10-200, gamma0 500-2e4,
    LP/CP, every fourth a gamma beam) in the benchmark's launch configuration (graph replay
    of one batched step): 150 steps in, one more batched step, and for eight ensembles a
    sample of their particles stepped by the oracle from the same pre-step state (each
    ensemble's own field, seed and clock), compared one by one (mixed path: 2e-5; only
    logged near-ties may differ)."""
    import bench
    wls = bench.c4_workload()
    caps = []
    for wl in wls:
        n = len(wl["e"]["id"]) + len(wl["ph"]["id"])
        caps.append({"cap_e": n + n // 2 + 4096, "cap_p": n // 2 + 4096, "cap_ph": 24 * n + 4096})
    b = q.Batch(wls, prec=q.QED_PREC_MIXED, flags=ALL, ctx=ctx, caps=caps)
    b.run(bench.C4_PRE)
    torch.cuda.synchronize()
    sizes = np.array([len(w["e"]["id"]) + len(w["ph"]["id"]) for w in wls])
    order = np.argsort(sizes)
    chosen = list(order[-4:]) + list(order[len(order) // 2: len(order) // 2 + 2]) + [3, 7]   # big, middle, gamma beams
    rng = np.random.default_rng(8)
    pres, clocks = {}, b.clocks()
    for k in chosen:
        s = b.sims[k]
        pres[k] = ({sp: _pick(getattr(s, sp), n, rng) for sp, n in (("e", 1500), ("pos", 500), ("ph", 2000))},
                   q.qed_get_next_id(s.ctx))
    b.run(1)
    torch.cuda.synchronize()
    assert q.qed_read_status(b.ctx) == 0
    total_nbw = total_ncs = 0
    for k in chosen:
        pre, nid = pres[k]
        t, step = clocks[k]
        ost = _compare_sample(orc, b.sims[k], wls[k], pre, t, step, nid, 2e-5, True)
        total_ncs += ost["n_ncs_e"]
        total_nbw += ost["n_nbw"]
    assert total_ncs > 0 and total_nbw > 0
    b.close()
