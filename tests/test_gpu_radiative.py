"""The radiative pusher (QED_F_LL, QED_F_MLL, QED_F_MBMT: Sec. III A Landau-Lifshitz and
its quantum correction, Sec. III B radiative T-BMT) through the C ABI against the oracle,
on identical inputs.  The pusher is deterministic, so every particle is compared: FP64
path within 1e-10 relative, mixed path within 2e-5.  Also: flag validation, the
grid-gathered workload, and a batch of ensembles against the same ensembles alone."""
import math

import numpy as np
import pytest

import oracle
import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2306_11288_gb300 as q  # noqa: E402

MLL = q.QED_F_MLL | q.QED_F_MBMT | q.QED_F_SPIN
LL = q.QED_F_LL | q.QED_F_MBMT | q.QED_F_SPIN


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


def _max_diffs(g, o):
    g, o = _by_id(g), _by_id(o)
    assert np.array_equal(g["id"], o["id"])
    if not len(o["id"]):
        return 0.0, 0.0, 0.0
    pg = np.stack([g["px"], g["py"], g["pz"]], 1)
    po = np.stack([o["px"], o["py"], o["pz"]], 1)
    dp = (np.linalg.norm(pg - po, axis=1) / np.maximum(np.linalg.norm(po, axis=1), 1.0)).max()
    ds = np.abs(np.stack([g[k] - o[k] for k in ("s1", "s2", "s3")], 1)).max()
    dx = np.abs(np.stack([(g[k] - o[k]) / (np.abs(o[k]) + 1.0) for k in ("x", "y", "z")], 1)).max()
    return dp, ds, dx


def _run(orc, ctx, wl, steps, flags, prec):
    sim = q.Simulation(wl, prec=prec, ctx=ctx)
    sim.run(steps, flags)
    osim = oracle.Sim(orc, wl)
    osim.run(steps, flags)
    g, o = sim.state(), osim.state()
    assert sim.status() == 0
    sim.close()
    return g, o


def _crossed(ne, npos, seed, E0=150.0):
    """e- and e+ (ragged counts) head-on with a static crossed field, random spins"""
    rng = np.random.default_rng(seed)

    def lep(n, first):
        s = rng.normal(size=(n, 3))
        s /= np.linalg.norm(s, axis=1, keepdims=True)
        p = rng.normal(size=(n, 3)) * 30 + np.array([0, 0, 4000.0])
        return {"x": rng.normal(size=n), "y": rng.normal(size=n), "z": rng.normal(size=n),
                "px": p[:, 0], "py": p[:, 1], "pz": p[:, 2], "s1": s[:, 0], "s2": s[:, 1], "s3": s[:, 2],
                "w": np.ones(n), "id": np.arange(first, first + n, dtype=np.uint64)}

    return {"e": lep(ne, 0), "pos": lep(npos, ne), "ph": workloads.empty(True),
            "field": {"kind": "uniform", "E": (E0, 0, 0), "B": (0, -E0, 0)}, "dt": math.pi / 100, "seed": 5,
            "next_id": ne + npos}


@pytest.mark.parametrize("flags", [MLL, LL, q.QED_F_MLL, q.QED_F_MBMT], ids=["mll+mbmt", "ll+mbmt", "mll", "mbmt"])
def test_plane_wave_full_crossing_fp64(orc, ctx, flags):
    """Config 1 (a0 = 20, gamma0 = 2000, chi up to ~0.2) over the 450-step crossing."""
    wl = workloads.c1(n=1500, seed=17)
    g, o = _run(orc, ctx, wl, 450, flags, q.QED_PREC_F64)
    dp, ds, dx = _max_diffs(g["e"], o["e"])
    assert dp < 1e-10 and ds < 1e-10 and dx < 1e-10, (dp, ds, dx)
    # radiation reaction acted: the beam lost energy (LL/MLL) or the spin left the unit sphere (MBMT)
    gam = np.sqrt(1 + g["e"]["px"] ** 2 + g["e"]["py"] ** 2 + g["e"]["pz"] ** 2)
    if flags & (q.QED_F_LL | q.QED_F_MLL):
        assert gam.mean() < 0.99 * 2000.0
    if flags & q.QED_F_MBMT:
        sn = np.sqrt(g["e"]["s1"] ** 2 + g["e"]["s2"] ** 2 + g["e"]["s3"] ** 2)
        assert sn.max() < 1 - 1e-6
    assert len(g["ph"]["id"]) == 0   # no photons: the pusher replaces the Monte Carlo


def test_both_species_crossed_field_fp64(orc, ctx):
    """e- and e+ with ragged counts in a strong crossed field (chi ~ 3)."""
    wl = _crossed(1031, 517, seed=3)
    g, o = _run(orc, ctx, wl, 80, MLL, q.QED_PREC_F64)
    for sp in ("e", "pos"):
        dp, ds, dx = _max_diffs(g[sp], o[sp])
        assert dp < 1e-10 and ds < 1e-10 and dx < 1e-10, (sp, dp, ds, dx)


@pytest.mark.parametrize("flags", [MLL, LL], ids=["mll+mbmt", "ll+mbmt"])
def test_mixed_path_per_particle(orc, ctx, flags):
    """Mixed path: every particle within 2e-5 of the FP64 oracle after 100 steps of the
    crossed-field set and 200 steps of config 1 (no stochastic decisions to exempt)."""
    for wl, steps in ((_crossed(2000, 700, seed=9), 100), (workloads.c1(n=3000, seed=19), 200)):
        g, o = _run(orc, ctx, wl, steps, flags, q.QED_PREC_MIXED)
        for sp in ("e", "pos"):
            dp, ds, dx = _max_diffs(g[sp], o[sp])
            assert dp < 2e-5 and ds < 2e-5 and dx < 2e-5, (sp, dp, ds, dx)


def test_grid_workload_fp64(orc, ctx):
    """The config-3 style grid (256 x 128 Yee cells, TSC gather) with MLL + M-BMT."""
    g3 = workloads.c3_grid(nx=256, ny=128, a0=150.0)
    wl = workloads.c3(n=3000, seed=13, nx=256, ny=128, grid=g3)
    g, o = _run(orc, ctx, wl, 40, MLL, q.QED_PREC_F64)
    dp, ds, dx = _max_diffs(g["e"], o["e"])
    assert dp < 1e-9 and ds < 1e-9 and dx < 1e-9, (dp, ds, dx)


def test_flag_validation(ctx):
    wl = workloads.c1(n=10, seed=1)
    sim = q.Simulation(wl, prec=q.QED_PREC_F64, ctx=ctx)
    for bad in (q.QED_F_NCS | q.QED_F_MLL, q.QED_F_NCS | q.QED_F_MBMT, q.QED_F_LL | q.QED_F_MLL, 1 << 12):
        with pytest.raises(q.QedError):
            q.qed_step(sim.ctx, sim.e.handle, sim.pos.handle, sim.ph.handle, sim.fields, sim.t, sim.dt, sim.seed,
                       sim.step_no, bad)
    sim.close()


def test_batch_equals_each_ensemble_alone(ctx):
    """A batch stepped with the radiative pusher equals each ensemble stepped alone, bit
    for bit (mixed path)."""
    wls = workloads.c4(n_ens=6, seed=8, cap_each=3000)
    wls = [w for w in wls if len(w["e"]["id"])]
    for w in wls:
        shift = 9.0 * math.pi
        w["e"]["z"] = w["e"]["z"] + shift
        w["t0"] = shift
    b = q.Batch(wls, prec=q.QED_PREC_MIXED, flags=MLL, ctx=ctx)
    b.run(30)
    got = [s.state() for s in b.sims]
    b.close()
    for w, gb in zip(wls, got):
        sc = q.qed_ctx_share(ctx)
        sim = q.Simulation(w, prec=q.QED_PREC_MIXED, ctx=sc)
        sim.run(30, MLL)
        ga = sim.state()
        sim.close()
        q.qed_destroy(sc)
        for k in ga["e"]:
            assert np.array_equal(ga["e"][k], gb["e"][k]), k
