"""Batches of independent ensembles (qed_batch_*) through the C ABI.

An ensemble stepped in a batch must end exactly where it ends when stepped alone with
qed_step (same arrays bit for bit, same ids, counts, statistics and clock), whatever the
launch shape (the autotuner steps the batch under every candidate) and whether the steps
come from direct launches or from the replayed CUDA graph.  The FP64 batch is also checked
against the oracle.  Ensembles follow the many-collisions recipe (sizes, a0, gamma0,
polarisation and spin states vary; every fourth one is a gamma beam), moved close to the
focus so that every process fires, with different clocks and step counters."""
import math

import numpy as np
import pytest

import oracle
import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2306_11288_gb300 as q  # noqa: E402

ALL = q.QED_F_NCS | q.QED_F_NBW | q.QED_F_VB | q.QED_F_SPIN


@pytest.fixture(scope="module")
def parent():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    q.build()
    return q.qed_init_tables()


def _ensembles(n_ens, cap_each, seed):
    wls = workloads.c4(n_ens=n_ens, seed=seed, cap_each=cap_each)
    for k, wl in enumerate(wls):
        m = max(1, int(cap_each * (0.15 + 0.85 * ((k * 37) % 11) / 10)))   # uneven sizes
        for sp in ("e", "ph"):
            if len(wl[sp]["id"]):
                wl[sp] = {key: v[:m] for key, v in wl[sp].items()}
        wl["next_id"] = m
        shift = (8.0 + 0.3 * (k % 5)) * math.pi
        for sp in ("e", "ph"):
            if len(wl[sp]["id"]):
                wl[sp]["z"] = wl[sp]["z"] + shift
        wl["t0"] = shift
        wl["step0"] = int(round(shift / wl["dt"])) + 7 * k
    empty = workloads.c2(n=0, seed=99)
    empty["t0"], empty["step0"] = 0.5, 3
    wls.insert(2, empty)          # an ensemble with no particles at all
    return wls


def _caps(wl):
    n = len(wl["e"]["id"]) + len(wl["ph"]["id"])
    return {"cap_e": 4 * n + 64, "cap_p": 4 * n + 64, "cap_ph": 8 * n + 64}


def _alone(parent, wl, prec, steps):
    c = q.qed_ctx_share(parent)
    sim = q.Simulation(wl, prec=prec, ctx=c, **_caps(wl))
    processed = 0
    for _ in range(steps):
        processed += sim.e.count() + sim.pos.count() + sim.ph.count()
        sim.run(1, ALL)
    assert sim.counters()["n_processed"] == processed   # particle-steps counted on the device
    out = (sim.state(), sim.counters(), sim.t, sim.step_no)
    sim.close()
    q.qed_destroy(c)
    return out


def _same(bs, alone, clock):
    st, cnt, t, step = alone
    g = bs.state()
    assert g["next_id"] == st["next_id"]
    for sp in ("e", "pos", "ph"):
        for k in st[sp]:
            assert np.array_equal(g[sp][k], st[sp][k]), (sp, k)
    assert bs.counters() == cnt
    assert clock == (t, step)


@pytest.mark.parametrize("prec", [q.QED_PREC_MIXED, q.QED_PREC_F64])
def test_batch_equals_each_ensemble_alone(parent, prec):
    wls = _ensembles(7, 2500, seed=41)
    steps = 30
    b = q.Batch(wls, prec=prec, ctx=parent, caps=[_caps(w) for w in wls])
    b.step(steps)
    clocks = b.clocks()
    assert q.qed_read_status(parent) == 0
    fired = {"ncs": 0, "nbw": 0}
    for k, wl in enumerate(wls):
        alone = _alone(parent, wl, prec, steps)
        _same(b.sims[k], alone, clocks[k])
        fired["ncs"] += alone[1]["n_ncs_e"]
        fired["nbw"] += alone[1]["n_nbw"]
    assert fired["ncs"] > 0 and fired["nbw"] > 0
    b.close()


def test_graph_replay_and_every_tuned_shape_equal_alone(parent):
    wls = _ensembles(5, 2000, seed=43)
    b = q.Batch(wls, prec=q.QED_PREC_MIXED, ctx=parent, caps=[_caps(w) for w in wls])
    b.run(12)                                  # CUDA graph of one step, replayed
    cfg, rate = q.qed_batch_tune(b.b, 1)       # every candidate shape steps the batch
    assert rate > 0 and 1 <= cfg["stream_blocks_per_sm"] <= 4
    b.run(5)                                   # graph recaptured for the chosen shape
    clocks = b.clocks()
    for k, wl in enumerate(wls):
        steps = clocks[k][1] - wl["step0"]
        assert steps > 17
        _same(b.sims[k], _alone(parent, wl, q.QED_PREC_MIXED, steps), clocks[k])
    b.close()


def test_fp64_batch_matches_oracle(parent, orc):
    wls = _ensembles(3, 400, seed=45)
    b = q.Batch(wls, prec=q.QED_PREC_F64, ctx=parent, caps=[_caps(w) for w in wls])
    steps = 40
    b.step(steps)
    for k, wl in enumerate(wls):
        osim = oracle.Sim(orc, wl, **_caps(wl))
        ost = osim.run(steps, ALL)
        c = b.sims[k].counters()
        assert (c["n_ncs_e"], c["n_nbw"]) == (ost["n_ncs_e"], ost["n_nbw"])
        g, o = b.sims[k].state(), osim.state()
        assert g["next_id"] == o["next_id"]
        for sp in ("e", "pos", "ph"):
            og = np.argsort(g[sp]["id"])
            oo = np.argsort(o[sp]["id"])
            assert np.array_equal(g[sp]["id"][og], o[sp]["id"][oo])
            for key in ("px", "py", "pz", "s1", "s2", "s3", "x", "y", "z"):
                a, r = g[sp][key][og], o[sp][key][oo]
                assert np.all(np.abs(a - r) <= 1e-10 * np.maximum(np.abs(r), 1.0)), (k, sp, key)
    b.close()


def test_batch_validation(parent):
    wl = _ensembles(2, 300, seed=47)
    c1, c2 = q.qed_ctx_share(parent), q.qed_ctx_share(parent)
    s1 = q.Simulation(wl[0], prec=q.QED_PREC_F64, ctx=c1)
    s2 = q.Simulation(wl[1], prec=q.QED_PREC_MIXED, ctx=c2)

    def ens(s):
        return q.qed_ensemble(s.ctx, s.e.handle, s.pos.handle, s.ph.handle, s.fields, s.t, s.step_no, s.seed, None)

    with pytest.raises(q.QedError, match="mixed precisions"):
        q.qed_batch_create(parent, [ens(s1), ens(s2)], s1.dt, ALL)
    with pytest.raises(q.QedError, match="share a context"):
        q.qed_batch_create(parent, [ens(s1), ens(s1)], s1.dt, ALL)
    with pytest.raises(q.QedError, match="n_ens"):
        q.qed_batch_create(parent, [], s1.dt, ALL)
    own = q.Simulation(wl[0], prec=q.QED_PREC_F64, ctx=parent)
    with pytest.raises(q.QedError, match="own context"):
        q.qed_batch_create(parent, [ens(own)], own.dt, ALL)
    for s in (s1, s2, own):
        s.close()
    q.qed_destroy(c1)
    q.qed_destroy(c2)


def _event_heavy(n_e, n_ph, orc):
    """Photons (omega = 4000, chi_gamma = 1) of which ~30% decay in one step and electrons
    (gamma = 4000, chi_e = 1) that all emit, in a uniform crossed field: the one-step NBW
    geometry of the oracle's statistics, with a lepton beam added."""
    xil, alpha = 2.42631023867e-6, 7.2973525693e-3
    om, chig = 4000.0, 1.0
    E0 = chig / (xil * om * 2)
    xi = np.array([0.3, -0.4, 0.5])
    rng = np.random.default_rng(61)

    def beam(n, px, stokes):
        d = {"x": rng.uniform(-1, 1, n), "y": rng.uniform(-1, 1, n), "z": rng.uniform(-1, 1, n),
             "px": np.full(n, px), "py": np.zeros(n), "pz": np.zeros(n), "w": np.ones(n)}
        if stokes is None:   # spins: random directions, |S| uniform in [0, 1)
            s = rng.normal(size=(n, 3))
            s *= rng.uniform(0.0, 1.0, (n, 1)) / np.linalg.norm(s, axis=1, keepdims=True)
        else:
            s = np.tile(stokes, (n, 1))
        d["s1"], d["s2"], d["s3"] = s[:, 0], s[:, 1], s[:, 2]
        return d

    e = beam(n_e, math.sqrt(om * om - 1.0), None)
    e["id"] = np.arange(n_e, dtype=np.uint64)
    ph = beam(n_ph, om, xi)
    ph["theta"] = np.zeros(n_ph)
    ph["id"] = np.arange(n_e, n_e + n_ph, dtype=np.uint64)
    empty = {k: np.zeros(0) for k in ("x", "y", "z", "px", "py", "pz", "s1", "s2", "s3", "w")}
    empty["id"] = np.zeros(0, dtype=np.uint64)
    T = orc.nbw_rates(chig)
    rate = alpha / (math.sqrt(3) * math.pi * xil * om) * (T[0] + xi[2] * T[1])
    return {"e": e, "pos": empty, "ph": ph, "dt": 0.3 / rate, "seed": 23, "next_id": n_e + n_ph,
            "field": {"kind": "uniform", "E": (0, E0, 0), "B": (0, 0, -E0)}}


@pytest.mark.parametrize("prec", [q.QED_PREC_MIXED, q.QED_PREC_F64])
def test_more_events_than_event_threads_equal_alone(parent, orc, prec):
    """A step with more emissions and more decays than the event kernel has threads (one
    event block of 256 threads per SM): a thread samples its first event before the scan has
    finished and takes the rest after it, and here every decay is such a later task.  The
    batch ends exactly where the ensemble ends when stepped alone by qed_step (whose wider
    event grid gives most events a thread of their own), and on FP64 where the oracle ends."""
    threads = torch.cuda.get_device_properties(0).multi_processor_count * 256
    n_e, n_ph = int(1.3 * threads), 4 * threads
    wl = _event_heavy(n_e, n_ph, orc)
    caps = {"cap_e": n_e + n_ph, "cap_p": n_ph, "cap_ph": n_ph + 3 * n_e}
    steps = 2
    b = q.Batch([wl], prec=prec, ctx=parent, caps=[caps])
    q.qed_batch_set_config(b.b, 4, 1, 0)
    b.step(1)
    c1 = b.sims[0].counters()
    assert c1["n_ncs_e"] > threads and c1["n_nbw"] > threads   # later tasks of both kinds
    b.step(steps - 1)
    assert q.qed_read_status(parent) == 0
    _same(b.sims[0], _alone(parent, wl, prec, steps), b.clocks()[0])
    if prec == q.QED_PREC_F64:
        osim = oracle.Sim(orc, wl, **caps)
        ost = osim.run(steps, ALL)
        c = b.sims[0].counters()
        assert (c["n_ncs_e"], c["n_nbw"]) == (ost["n_ncs_e"], ost["n_nbw"])
        g, o = b.sims[0].state(), osim.state()
        assert g["next_id"] == o["next_id"]
        for sp in ("e", "pos", "ph"):
            og, oo = np.argsort(g[sp]["id"]), np.argsort(o[sp]["id"])
            assert np.array_equal(g[sp]["id"][og], o[sp]["id"][oo])
            for key in ("px", "py", "pz", "s1", "s2", "s3", "x", "y", "z"):
                a, r = g[sp][key][og], o[sp][key][oo]
                assert np.all(np.abs(a - r) <= 1e-10 * np.maximum(np.abs(r), 1.0)), (sp, key)
    b.close()
