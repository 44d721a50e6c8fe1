"""GPU (sm_103a) vs oracle parity through the C ABI, on identical seeded inputs.

FP64 path: event counts and ids bit-exact; per-particle momenta, spins, Stokes and
positions within 1e-10 relative.  Mixed path: every electron within 2e-5 (momentum, spin,
position) over a 200-step run, except those with a logged near-tie decision (the rule of
``parity_rules``); photon spectra, photon Stokes parameters in a detection basis, pair
yield and positron spin within 3 sigma of the statistical error (independent seeds), on
the plane-wave workload and on the focused-pulse workload with every process on."""
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


@pytest.fixture(scope="session")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    q.build()
    c = q.qed_init_tables()
    yield c
    torch.cuda.synchronize()


def _run_both(orc, ctx, wl, steps, flags, prec=q.QED_PREC_F64, caps=None):
    caps = caps or {}
    sim = q.Simulation(wl, prec=prec, ctx=ctx, **caps)
    osim = oracle.Sim(orc, wl, **caps)
    sim.run(steps, flags)
    ost = osim.run(steps, flags)
    return sim, osim, ost


def _by_id(d):
    o = np.argsort(d["id"], kind="stable")
    return {k: v[o] for k, v in d.items()}


def _compare(g, o, species, tol, pos_tol, photon=False, exclude=()):
    g, o = _by_id(g), _by_id(o)
    assert np.array_equal(g["id"], o["id"]), f"{species}: id sets differ ({len(g['id'])} vs {len(o['id'])})"
    keep = ~np.isin(o["id"], np.asarray(list(exclude), dtype=np.uint64))
    p_g = np.stack([g["px"], g["py"], g["pz"]], 1)[keep]
    p_o = np.stack([o["px"], o["py"], o["pz"]], 1)[keep]
    if len(p_o) == 0:
        return 0.0
    scale = np.maximum(np.linalg.norm(p_o, axis=1), 1.0)
    dp = (np.linalg.norm(p_g - p_o, axis=1) / scale).max()
    s_g = np.stack([g["s1"], g["s2"], g["s3"]], 1)[keep]
    s_o = np.stack([o["s1"], o["s2"], o["s3"]], 1)[keep]
    ds = np.abs(s_g - s_o).max()
    x_g = np.stack([g["x"], g["y"], g["z"]], 1)[keep]
    x_o = np.stack([o["x"], o["y"], o["z"]], 1)[keep]
    dx = (np.abs(x_g - x_o) / (np.abs(x_o) + 1.0)).max()
    assert dp < tol, f"{species}: momentum rel diff {dp:.3e}"
    assert ds < tol, f"{species}: spin/Stokes diff {ds:.3e}"
    assert dx < pos_tol, f"{species}: position diff {dx:.3e}"
    assert np.array_equal(g["w"][keep], o["w"][keep]) or np.allclose(g["w"][keep], o["w"][keep], rtol=1e-7)
    if photon:
        dth = np.angle(np.exp(2j * (g["theta"][keep] - o["theta"][keep]))) / 2
        assert np.abs(dth).max() < tol * 10, f"{species}: basis angle diff {np.abs(dth).max():.3e}"
    return max(dp, ds)


def _compare_all(sim, osim, tol, pos_tol):
    gs, os_ = sim.state(), osim.state()
    assert gs["next_id"] == os_["next_id"]
    out = {}
    for sp in ("e", "pos", "ph"):
        out[sp] = _compare(gs[sp], os_[sp], sp, tol, pos_tol, photon=(sp == "ph"))
    return out


# ---------------------------------------------------------------------------------------
def test_tables_match_oracle(orc, ctx):
    """Each side builds its tables with its own quadrature; they agree to rounding."""
    names = {0: "K", 1: "ncs rate", 2: "ncs invcdf", 3: "nbw rate", 4: "nbw invcdf", 5: "vb", 6: "radiative pusher"}
    for w, name in names.items():
        g = q.qed_copy_table(ctx, w)
        o = orc.table(w)
        assert g.shape == o.shape, name
        half = len(g) // 2
        if w == 0:
            # values relative; d/dlnx = x(K13 - K23) - ... cancels at large x, so it is
            # compared on the scale of the values (what the Hermite step h d contributes)
            assert (np.abs(g[:half] - o[:half]) / o[:half]).max() < 1e-11, name
            assert (np.abs(g[half:] - o[half:]) / o[:half]).max() < 1e-9, name
        elif w in (2, 4):
            # values (ln u, ln delta): absolute; slopes: relative
            assert np.abs(g[:half] - o[:half]).max() < 2e-11, name
            assert (np.abs(g[half:] - o[half:]) / np.abs(o[half:])).max() < 1e-8, name
        elif w == 5:
            # M_par, M_perp cross zero near chi_gamma ~ 15: compare on their natural scale
            err = np.abs(g - o) / np.maximum(np.abs(o), 1.0)
            assert err.max() < 1e-11, (name, err.max(), int(err.argmax()))
        else:
            rel = np.abs(g - o) / np.maximum(np.abs(o), 1e-300)
            assert rel.max() < 1e-11, (name, rel.max(), int(rel.argmax()))


def test_interval_cubics_pass_through_the_oracle_nodes(orc, ctx):
    """The mixed path holds each 1-D table as the cubic of every node interval; a cubic is
    fixed by four points, so each row must reproduce the oracle's four nodes around its
    interval (f = -1, 0, 1, 2) up to the float rounding of its coefficients."""
    blk = q.qed_copy_table(ctx, 7)
    ncs, nbw, vb, rr = orc.table(1).reshape(2, -1), orc.table(3).reshape(2, -1), orc.table(5).reshape(2, -1), \
        orc.table(6).reshape(4, -1)
    layout = [("vb", [vb[0] - vb[1]]), ("nbw", [nbw[0], nbw[1]]), ("ncs", [ncs[0], ncs[1]]),
              ("radiative pusher", [rr[0], rr[1], rr[2], rr[3]])]
    off = 0
    fs = np.array([-1.0, 0.0, 1.0, 2.0])
    powers = np.stack([fs ** 0, fs, fs ** 2, fs ** 3], 1)          # [4 f][4 coefficients]
    for name, tables in layout:
        n = len(tables[0])
        rows = n - 3
        c = blk[off:off + rows * 4 * len(tables)].reshape(rows, len(tables), 4)
        off += rows * 4 * len(tables)
        for k, y in enumerate(tables):
            nodes = np.stack([y[r:r + 4] for r in range(rows)])      # y(i-1) .. y(i+2), i = r + 1
            vals = c[:, k, :] @ powers.T                             # p(-1), p(0), p(1), p(2)
            scale = np.abs(nodes).max(1, keepdims=True) + 1e-300
            err = (np.abs(vals - nodes) / scale).max()
            assert err < 2e-6, (name, k, err)
    assert off == len(blk)


def test_c1_plane_wave_fp64_full_crossing(orc, ctx):
    """Config 1 at 2000 electrons over the full 450-step crossing: NCS + T-BMT."""
    wl = workloads.c1(n=2000, seed=11)
    sim, osim, ost = _run_both(orc, ctx, wl, 450, q.QED_F_NCS | q.QED_F_SPIN)
    c = sim.counters()
    assert c["n_ncs_e"] == ost["n_ncs_e"] and c["n_ncs_e"] > 1000
    assert c["n_coarse"] == ost["n_coarse"] == 0   # W dt stays well below 0.1 at dt = T0/200
    assert sim.status() == 0
    d = _compare_all(sim, osim, 1e-10, 1e-10)
    print("max diffs", d)


def _c2_at_focus(n, seed, a0=100.0, gamma0=2e4, t_shift=8.5 * math.pi):
    wl = workloads.c2(n=n, seed=seed, a0=a0, gamma0=gamma0)
    wl["e"]["z"] = wl["e"]["z"] + t_shift
    wl["t0"] = t_shift
    wl["step0"] = int(round(t_shift / wl["dt"]))
    return wl


def test_c2_full_physics_fp64(orc, ctx):
    """Config 2 at 300 electrons through the focus: NCS + NBW + VB + T-BMT, compaction."""
    wl = _c2_at_focus(300, seed=21)
    sim, osim, ost = _run_both(orc, ctx, wl, 200, ALL)
    c = sim.counters()
    assert c["n_ncs_e"] == ost["n_ncs_e"] and c["n_nbw"] == ost["n_nbw"] and c["n_ncs_p"] == ost["n_ncs_p"]
    assert c["n_nbw"] > 0, "no pair was created: the workload does not exercise NBW"
    assert sim.status() == 0
    _compare_all(sim, osim, 1e-10, 1e-10)


def test_both_species_crossed_field_fp64(orc, ctx):
    """Electrons, positrons and polarised photons together in a static crossed field;
    ragged counts (not multiples of the 256-particle tile)."""
    rng = np.random.default_rng(3)
    def lep(n, first):
        s = rng.normal(size=(n, 3)); s /= np.linalg.norm(s, axis=1, keepdims=True)
        p = rng.normal(size=(n, 3)) * 30 + np.array([0, 0, 4000.0])
        return {"x": rng.normal(size=n), "y": rng.normal(size=n), "z": rng.normal(size=n),
                "px": p[:, 0], "py": p[:, 1], "pz": p[:, 2], "s1": s[:, 0], "s2": s[:, 1], "s3": s[:, 2],
                "w": rng.uniform(0.5, 2, n), "id": np.arange(first, first + n, dtype=np.uint64)}
    e, pos = lep(517, 0), lep(259, 517)
    nph = 301
    k = rng.normal(size=(nph, 3)) * 50 + np.array([0, 0, 3000.0])
    xi = rng.normal(size=(nph, 3)); xi *= rng.uniform(0, 1, (nph, 1)) / np.linalg.norm(xi, axis=1, keepdims=True)
    ph = {"x": rng.normal(size=nph), "y": rng.normal(size=nph), "z": rng.normal(size=nph), "px": k[:, 0],
          "py": k[:, 1], "pz": k[:, 2], "s1": xi[:, 0], "s2": xi[:, 1], "s3": xi[:, 2],
          "theta": rng.uniform(-3, 3, nph), "w": np.ones(nph), "id": np.arange(776, 776 + nph, dtype=np.uint64)}
    E0 = 150.0
    wl = {"e": e, "pos": pos, "ph": ph, "field": {"kind": "uniform", "E": (E0, 0, 0), "B": (0, -E0, 0)},
          "dt": math.pi / 100, "seed": 5, "next_id": 776 + nph}
    sim, osim, ost = _run_both(orc, ctx, wl, 60, ALL)
    c = sim.counters()
    assert c["n_nbw"] == ost["n_nbw"] > 0
    assert c["n_ncs_p"] == ost["n_ncs_p"] > 0
    _compare_all(sim, osim, 1e-10, 1e-10)


@pytest.mark.parametrize("n", [0, 1, 255, 256, 257])
def test_edge_sizes_fp64(orc, ctx, n):
    wl = _c2_at_focus(n, seed=31)
    sim, osim, ost = _run_both(orc, ctx, wl, 40, ALL)
    _compare_all(sim, osim, 1e-10, 1e-10)


def test_capacity_overflow_flags_and_matches(orc, ctx):
    """Births beyond the photon capacity are dropped on both sides and flagged."""
    wl = _c2_at_focus(200, seed=41)
    caps = {"cap_ph": 60}
    sim, osim, ost = _run_both(orc, ctx, wl, 30, q.QED_F_NCS | q.QED_F_SPIN, caps=caps)
    c = sim.counters()
    assert c["n_drop"] == ost["n_drop"] > 0
    assert sim.status() & q.QED_STATUS_CAPACITY
    gs, os_ = sim.state(), osim.state()
    assert len(gs["ph"]["id"]) == 60 and np.array_equal(np.sort(gs["ph"]["id"]), np.sort(os_["ph"]["id"]))
    _compare(gs["e"], os_["e"], "e", 1e-10, 1e-10)


def test_mass_decay_step_logs_every_event_fp64(orc, ctx):
    """30 % of 200,000 photons decay in one step (chi_gamma = 1, dt = 0.3 / rate; the
    geometry of the oracle's one-step NBW statistics): one event per photon is the most a
    step can log, and the logs hold that many, so nothing is dropped -- pair count, ids
    and every particle agree with the oracle (FP64, 1e-10) and the status word stays 0."""
    xil, alpha = 2.42631023867e-6, 7.2973525693e-3
    om, chig, N = 4000.0, 1.0, 200_000
    E0 = chig / (xil * om * 2)
    xi = np.array([0.3, -0.4, 0.5])
    ph = {"x": np.zeros(N), "y": np.zeros(N), "z": np.zeros(N), "px": np.full(N, om), "py": np.zeros(N),
          "pz": np.zeros(N), "s1": np.full(N, xi[0]), "s2": np.full(N, xi[1]), "s3": np.full(N, xi[2]),
          "theta": np.zeros(N), "w": np.ones(N), "id": np.arange(N, dtype=np.uint64)}
    T = orc.nbw_rates(chig)
    rate = alpha / (math.sqrt(3) * math.pi * xil * om) * (T[0] + xi[2] * T[1])
    empty = {k: np.zeros(0) for k in ("x", "y", "z", "px", "py", "pz", "s1", "s2", "s3", "w")}
    empty["id"] = np.zeros(0, dtype=np.uint64)
    wl = {"e": empty, "pos": dict(empty), "ph": ph, "dt": 0.3 / rate, "seed": 17, "next_id": N,
          "field": {"kind": "uniform", "E": (0, E0, 0), "B": (0, 0, -E0)}}
    caps = {"cap_e": N, "cap_p": N, "cap_ph": N}
    sim, osim, ost = _run_both(orc, ctx, wl, 1, q.QED_F_NBW | q.QED_F_VB, caps=caps)
    c = sim.counters()
    assert c["n_nbw"] == ost["n_nbw"] and 0.28 * N < c["n_nbw"] < 0.32 * N
    assert sim.status() == 0
    # every decision had T dt = 0.3 > 0.1: counted as a coarse step on both sides
    assert c["n_coarse"] == ost["n_coarse"] == N
    _compare_all(sim, osim, 1e-10, 1e-10)


def test_uniform_field_grid_matches_analytic_gather(orc, ctx):
    """Config-3 style TSC gather: a uniform grid field reproduces the field exactly and
    the FP64 step matches the oracle on a small synthetic grid."""
    g = workloads.c3_grid(nx=256, ny=128, a0=150.0)
    wl = workloads.c3(n=3000, seed=13, nx=256, ny=128, grid=g)
    sim, osim, ost = _run_both(orc, ctx, wl, 40, ALL)
    assert sim.counters()["n_ncs_e"] == ost["n_ncs_e"] > 0
    _compare_all(sim, osim, 1e-9, 1e-9)


@pytest.mark.parametrize("periodic", [0, 1])
def test_grid_gather_independent_of_particle_order(ctx, periodic):
    """Mixed path: the same particles tile-sorted and shuffled (every tile then spans the
    grid) give the same momenta, spins and positions bit for bit (push and spin only: no
    events, so nothing may depend on the order); bounded and periodic grids."""
    g = workloads.c3_grid(nx=256, ny=128, a0=150.0)
    g["periodic"] = periodic
    wl = workloads.c3(n=20000, seed=14, nx=256, ny=128, grid=g)
    rng = np.random.default_rng(2)
    perm = rng.permutation(len(wl["e"]["id"]))
    wl2 = dict(wl, e={k: v[perm] for k, v in wl["e"].items()})
    out = []
    for w in (wl, wl2):
        sim = q.Simulation(w, prec=q.QED_PREC_MIXED, ctx=ctx)
        sim.run(15, q.QED_F_SPIN)
        out.append(_by_id(sim.state()["e"]))
        sim.close()
    moved = np.abs(out[0]["py"]).max()
    assert moved > 1.0   # the fields acted
    for k in out[0]:
        assert np.array_equal(out[0][k], out[1][k]), k


# ---------------------------------------------------------------------------------------
def test_mixed_precision_short_run_per_particle(orc, ctx):
    """Mixed path against the FP64 oracle over 200 steps of config 1 (NCS + T-BMT): every
    electron within 2e-5 in momentum (relative), in each spin component and in position,
    except electrons with a decision whose draw lay within the mixed-path bound of its
    threshold at some step (their trajectories branch there); no other exception."""
    wl = workloads.c1(n=4000, seed=12)
    sim = q.Simulation(wl, prec=q.QED_PREC_MIXED, ctx=ctx)
    osim = oracle.Sim(orc, wl)
    orc.set_near_tol(parity_rules.LOG_TOL)
    steps = 200
    try:
        sim.run(steps, q.QED_F_NCS | q.QED_F_SPIN)
        ost = osim.run(steps, q.QED_F_NCS | q.QED_F_SPIN)
        margins = parity_rules.near_margins(orc)
    finally:
        orc.set_near_tol(parity_rules.NEAR_FP64)
    assert ost["n_ncs_e"] > 1000
    gs, os_ = sim.state(), osim.state()
    ge, oe = _by_id(gs["e"]), _by_id(os_["e"])
    assert np.array_equal(ge["id"], oe["id"])
    pg = np.stack([ge["px"], ge["py"], ge["pz"]], 1)
    po = np.stack([oe["px"], oe["py"], oe["pz"]], 1)
    dp = np.linalg.norm(pg - po, axis=1) / np.linalg.norm(po, axis=1)
    ds = np.abs(np.stack([ge[k] - oe[k] for k in ("s1", "s2", "s3")], 1)).max(1)
    dx = np.abs(np.stack([(ge[k] - oe[k]) / (np.abs(oe[k]) + 1.0) for k in ("x", "y", "z")], 1)).max(1)
    bad = (dp > 2e-5) | (ds > 2e-5) | (dx > 2e-5)
    ex, unexplained, worst = parity_rules.exemptions(ge["id"][bad], margins, mixed=True)
    print(f"mixed 200-step run: {len(ex)} of {len(dp)} electrons exempted (largest margin {worst:.2e}); "
          f"max dp {dp[~bad].max():.2e}, ds {ds[~bad].max():.2e}, dx {dx[~bad].max():.2e}")
    assert not unexplained, f"electrons beyond 2e-5 without a near-tie (id, margin): {unexplained[:10]}"
    assert len(ex) <= 0.01 * len(dp)


def _spectrum(ph, bins):
    om = np.sqrt(ph["px"] ** 2 + ph["py"] ** 2 + ph["pz"] ** 2)
    h, _ = np.histogram(om, bins=bins, weights=ph["w"])
    h3, _ = np.histogram(om, bins=bins, weights=ph["w"] * ph["s3"])
    h33, _ = np.histogram(om, bins=bins, weights=ph["w"] * ph["s3"] ** 2)
    return h, h3, h33


def test_mixed_precision_spectra_within_3_sigma(orc, ctx):
    """Mixed path vs FP64 oracle (independent seeds) after the full config-1 crossing:
    photon counts per energy bin within 3 sigma (Poisson; at chi ~ 0.2 an emission takes a
    small fraction of the electron's energy, so one electron's emissions are nearly
    independent), and the mean xi3 of every bin with more than 200 photons within 3 sigma
    of its standard error (sample variance of xi3 in the bin)."""
    n = 4000
    wl = workloads.c1(n=n, seed=14)
    sim = q.Simulation(wl, prec=q.QED_PREC_MIXED, ctx=ctx)
    sim.run(450, q.QED_F_NCS | q.QED_F_SPIN)
    wl2 = workloads.c1(n=n, seed=15)
    osim = oracle.Sim(orc, wl2)
    osim.run(450, q.QED_F_NCS | q.QED_F_SPIN)
    g, o = sim.state()["ph"], osim.state()["ph"]
    bins = np.geomspace(1.0, 2000.0, 13)
    hg, h3g, h33g = _spectrum(g, bins)
    ho, h3o, h33o = _spectrum(o, bins)
    m = (hg > 0) | (ho > 0)
    pull = (hg - ho)[m] / np.sqrt(hg + ho)[m]
    print("photon spectrum pulls", np.round(pull, 2))
    assert np.all(np.abs(pull) <= 3.0), (hg, ho)
    m = (hg > 200) & (ho > 200)
    xg, xo = h3g[m] / hg[m], h3o[m] / ho[m]
    var_g = (h33g[m] / hg[m] - xg ** 2) / hg[m]
    var_o = (h33o[m] / ho[m] - xo ** 2) / ho[m]
    pull3 = (xg - xo) / np.sqrt(var_g + var_o)
    print("mean xi3 pulls", np.round(pull3, 2))
    assert np.all(np.abs(pull3) <= 3.0)


# ---------------------------------------------------------------------------------------
# Focused-pulse workload with every process on: the observables of the paper's read-out
# (Sec. IV: spectra, Stokes parameters in a detection basis after Eq. (rotation), pair
# yield, mean positron spin), mixed GPU path against the oracle with independent seeds.
N_BATCH, E_PER_BATCH, C2_STEPS = 10, 4000, 200
SPEC_LO, SPEC_HI, SPEC_NX = 10.0, 3.0e4, 8


def _observables(ph, pos, spec_fn):
    """Per-run observables: photon weight per ln-energy bin, Stokes means in the detection
    basis x (all photons), positron count and mean spin."""
    sp = spec_fn(ph)
    bins, tot = sp["bins"][0], sp["total"]
    out = {"spec": bins[:, 0], "xi": tot[1:4] / tot[0], "n_ph": tot[0]}
    out["pairs"] = float(len(pos["id"]))
    s = np.stack([pos["s1"], pos["s2"], pos["s3"]], 1)
    out["pos_S"] = s.mean(0) if len(s) else np.zeros(3)
    return out


def _batch_stats(runs):
    """Mean and standard error of every observable over independent runs."""
    out = {}
    for k in runs[0]:
        a = np.array([np.atleast_1d(r[k]) for r in runs], dtype=np.float64)
        out[k] = (a.mean(0), a.std(0, ddof=1) / math.sqrt(len(runs)))
    return out


def test_mixed_focused_pulse_observables_within_3_sigma(orc, ctx):
    """Config 2 through the focus (NCS + NBW + VB + T-BMT) on the mixed GPU path and on the
    oracle, each as 10 independent runs of 4000 electrons (GPU seeds 100.., oracle seeds
    200..): photon weight per ln-energy bin, the mean Stokes parameters xi1..3 of all photons
    in the detection basis (x, y) (qed_diag on the GPU, the oracle's read-out on the CPU),
    the number of pairs, and the mean positron spin.  The error of each observable is the
    standard error over its runs (photons and pairs of one electron are correlated, so
    Poisson errors would be too small); every pull within 3 sigma, with no added slack."""
    spec = q.diag_spec(q.QED_DIAG_SPECTRUM, SPEC_NX, 1, SPEC_LO, SPEC_HI, ref=(1.0, 0.0, 0.0))
    g_runs, o_runs = [], []
    for b in range(N_BATCH):
        wl = _c2_at_focus(E_PER_BATCH, seed=100 + b)
        sim = q.Simulation(wl, prec=q.QED_PREC_MIXED, ctx=ctx)
        sim.run(C2_STEPS, ALL)
        assert sim.status() == 0
        pos = sim.state()["pos"]
        g_runs.append(_observables(None, pos, lambda _ph, s=sim: q.diag(s.ph, spec)))
        sim.close()
        wlo = _c2_at_focus(E_PER_BATCH, seed=200 + b)
        osim = oracle.Sim(orc, wlo)
        osim.run(C2_STEPS, ALL)
        st = osim.state()
        from oracle import diag as odiag
        o_runs.append(_observables(st["ph"], st["pos"], lambda ph: odiag.diag(
            ph, odiag.SPECTRUM, SPEC_NX, 1, SPEC_LO, SPEC_HI, ref=(1.0, 0.0, 0.0), photon=True)))
    G, O = _batch_stats(g_runs), _batch_stats(o_runs)
    checked = 0
    for k in ("spec", "xi", "n_ph", "pairs", "pos_S"):
        (mg, eg), (mo, eo) = G[k], O[k]
        sig = np.sqrt(eg ** 2 + eo ** 2)
        use = sig > 0
        if k == "spec":   # bins with a few hundred photons per run
            use &= (mg > 200) & (mo > 200)
        pull = (mg - mo)[use] / sig[use]
        print(k, "gpu", np.round(mg, 4), "oracle", np.round(mo, 4), "pulls", np.round(pull, 2))
        assert np.all(np.abs(pull) <= 3.0), (k, mg, mo, sig)
        checked += int(use.sum())
    assert G["pairs"][0][0] > 100 and checked >= 12
