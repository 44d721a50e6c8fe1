"""Checkpoint/resume, out-of-range inputs and host-side rejection, through the C ABI.

* Resume: the state of a run is its particle arrays plus (seed, step, time, next id); the
  random numbers of a particle depend only on (seed, id, step), so N steps, a round trip
  of the whole state through host memory (an .npz file) into fresh device sets and a new
  context, and N more steps give the same arrays, bit for bit, as 2N steps in one go.
* chi_e beyond the tables' upper edge (1e3): the step clamps chi, counts the particle in
  n_range, raises QED_STATUS_TABLE_RANGE, and still matches the oracle, which clamps the
  same way (FP64 path, 1e-10).
* Non-finite field parameters are rejected before any launch; a particle whose momentum
  is NaN does not disturb the others (every other particle matches the oracle)."""
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
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    q.build()
    c = q.qed_init_tables()
    yield c
    torch.cuda.synchronize()


def _at_focus(n, seed):
    wl = workloads.c2(n=n, seed=seed)
    shift = 9.0 * math.pi
    wl["e"]["z"] = wl["e"]["z"] + shift
    wl["t0"] = shift
    wl["step0"] = 900
    return wl


@pytest.mark.parametrize("prec", [q.QED_PREC_MIXED, q.QED_PREC_F64])
def test_resume_from_host_checkpoint_is_bit_exact(ctx, prec, tmp_path):
    wl = _at_focus(3000, seed=61)
    caps = dict(cap_e=20000, cap_p=20000, cap_ph=200000)
    n = 25
    full = q.Simulation(wl, prec=prec, ctx=ctx, **caps)
    full.run(2 * n, ALL)
    ref = full.state()
    assert full.status() == 0
    full.close()

    first = q.Simulation(wl, prec=prec, ctx=ctx, **caps)
    first.run(n, ALL)
    st = first.state()
    path = tmp_path / "ckpt.npz"
    flat = {f"{sp}.{k}": v for sp in ("e", "pos", "ph") for k, v in st[sp].items()}
    np.savez(path, t=first.t, step=first.step_no, next_id=st["next_id"], seed=first.seed, **flat)
    first.close()

    z = np.load(path)
    wl2 = {"field": wl["field"], "dt": wl["dt"], "seed": int(z["seed"]), "t0": float(z["t"]),
           "step0": int(z["step"]), "next_id": int(z["next_id"])}
    for sp in ("e", "pos", "ph"):
        wl2[sp] = {k.split(".", 1)[1]: z[k] for k in z.files if k.startswith(sp + ".")}
    ctx2 = q.qed_init_tables()   # a fresh context: nothing carried over on the device
    second = q.Simulation(wl2, prec=prec, ctx=ctx2, **caps)
    second.run(n, ALL)
    got = second.state()
    assert second.status() == 0
    second.close()
    q.qed_destroy(ctx2)
    assert got["next_id"] == ref["next_id"]
    assert len(ref["ph"]["id"]) > 0 and len(ref["pos"]["id"]) > 0
    for sp in ("e", "pos", "ph"):
        for k in ref[sp]:
            assert np.array_equal(got[sp][k], ref[sp][k]), (sp, k)


def test_chi_beyond_table_range(orc, ctx):
    gamma, E0 = 1.0e5, 1.0e4            # head-on: chi = 2 gamma E0 xi_L ~ 4.9e3 > 1e3
    n = 300
    rng = np.random.default_rng(4)
    pz = -math.sqrt(gamma * gamma - 1)
    s = rng.normal(size=(n, 3))
    s /= np.linalg.norm(s, axis=1, keepdims=True)
    e = {"x": np.zeros(n), "y": np.zeros(n), "z": np.zeros(n), "px": np.zeros(n), "py": np.zeros(n),
         "pz": np.full(n, pz), "s1": s[:, 0], "s2": s[:, 1], "s3": s[:, 2], "w": np.ones(n),
         "id": np.arange(n, dtype=np.uint64)}
    wl = {"e": e, "pos": workloads.empty(), "ph": workloads.empty(True),
          "field": {"kind": "uniform", "E": (E0, 0, 0), "B": (0, E0, 0)}, "dt": 1e-4, "seed": 3, "next_id": n}
    flags = q.QED_F_NCS | q.QED_F_SPIN
    sim = q.Simulation(wl, prec=q.QED_PREC_F64, ctx=ctx)
    sim.run(3, flags)
    osim = oracle.Sim(orc, wl)
    ost = osim.run(3, flags)
    c = sim.counters()
    assert c["n_range"] == ost["n_range"] > 0
    assert sim.status() & q.QED_STATUS_TABLE_RANGE
    g, o = sim.state(), osim.state()
    assert g["next_id"] == o["next_id"]
    for sp in ("e", "ph"):
        a, b = g[sp], o[sp]
        ia, ib = np.argsort(a["id"]), np.argsort(b["id"])
        assert np.array_equal(a["id"][ia], b["id"][ib])
        pa = np.stack([a["px"], a["py"], a["pz"]], 1)[ia]
        pb = np.stack([b["px"], b["py"], b["pz"]], 1)[ib]
        if len(pb):
            assert (np.linalg.norm(pa - pb, axis=1) / np.linalg.norm(pb, axis=1)).max() < 1e-10
    sim.close()


def test_non_finite_inputs(orc, ctx):
    wl = workloads.c1(n=1000, seed=5)
    sim = q.Simulation(wl, prec=q.QED_PREC_F64, ctx=ctx)
    bad = [q.fields_from_spec({"kind": "uniform", "E": (float("nan"), 0, 0), "B": (0, 0, 0)}),
           q.fields_from_spec({"kind": "plane", "a0": float("inf"), "len": 8 * math.pi}),
           q.fields_from_spec({"kind": "gauss", "a0": 10.0, "len": 8 * math.pi, "w0": float("nan")})]
    for f in bad:
        with pytest.raises(q.QedError, match="non-finite"):
            q.qed_step(sim.ctx, sim.e.handle, sim.pos.handle, sim.ph.handle, f, sim.t, sim.dt, sim.seed,
                       sim.step_no, q.QED_F_NCS)
    sim.close()
    # a NaN momentum: that particle goes NaN, every other one is untouched by it
    wl = workloads.c1(n=1000, seed=5)
    wl["e"]["px"][417] = float("nan")
    flags = q.QED_F_NCS | q.QED_F_SPIN
    sim = q.Simulation(wl, prec=q.QED_PREC_F64, ctx=ctx)
    sim.run(300, flags)
    osim = oracle.Sim(orc, wl)
    ost = osim.run(300, flags)
    assert sim.counters()["n_ncs_e"] == ost["n_ncs_e"] > 0
    g, o = sim.state(), osim.state()
    assert g["next_id"] == o["next_id"]
    a, b = g["e"], o["e"]
    assert np.array_equal(a["id"], b["id"])
    ok = a["id"] != 417
    pa = np.stack([a["px"], a["py"], a["pz"]], 1)[ok]
    pb = np.stack([b["px"], b["py"], b["pz"]], 1)[ok]
    assert (np.linalg.norm(pa - pb, axis=1) / np.linalg.norm(pb, axis=1)).max() < 1e-10
    assert np.isnan(a["px"][~ok]).all()
    sim.close()
