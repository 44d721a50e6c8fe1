"""The self-consistent PIC loop around the step (Secs. II B, II C, II F) through the C ABI:
qed_fdtd_advance (Yee curl updates) and QED_F_DEPOSIT (Esirkepov current of every lepton
move), against the oracle on identical inputs.

The grid is FP32 by specification (the library evolves float E, B, J; the oracle evolves
double arrays and gathers from their float copies), and the current is summed with float
atomics, so the comparisons use float tolerances: 1e-5 of the field or current scale per
launch, growing with the number of steps.  Charge conservation and Gauss's law are checked
on the library's own output."""
import math

import numpy as np
import pytest

import oracle
import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2306_11288_gb300 as q  # noqa: E402

NAMES = ("Ex", "Ey", "Ez", "Bx", "By", "Bz")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    q.build()
    c = q.qed_init_tables()
    yield c
    torch.cuda.synchronize()


def _grid_pair(nx, ny, dx, dy, periodic, fields):
    """the library's float Yee grid and the oracle's double one, same (float) start"""
    f32 = {k: np.asarray(v, dtype=np.float32) for k, v in fields.items()}
    t = {k: torch.zeros((ny, nx), dtype=torch.float32, device="cuda") for k in NAMES + ("Jx", "Jy", "Jz")}
    for k, v in f32.items():
        t[k].copy_(torch.from_numpy(v))
    g = q.qed_grid2d()
    for k, v in t.items():
        setattr(g, k, v.data_ptr())
    g.nx, g.ny, g.dx, g.dy, g.periodic = nx, ny, dx, dy, periodic
    og = oracle.YeeGrid(nx, ny, dx, dy, periodic=periodic, fields={k: v.astype(np.float64) for k, v in f32.items()})
    return t, g, og


@pytest.mark.parametrize("periodic", [1, 0])
def test_fdtd_matches_oracle(ctx, periodic):
    """Random fields in every component (and a random current): 100 leapfrog steps."""
    nx, ny, dx, dy, dt = 200, 120, 0.4, 0.5, 0.2
    rng = np.random.default_rng(7 + periodic)
    fields = {k: rng.normal(size=(ny, nx)) for k in NAMES}
    t, g, og = _grid_pair(nx, ny, dx, dy, periodic, fields)
    J = {k: 0.1 * rng.normal(size=(ny, nx)).astype(np.float32) for k in ("Jx", "Jy", "Jz")}
    for step in range(100):
        q.qed_fdtd_advance(g, q.QED_FDTD_B, dt)
        if step == 0:   # one current pulse: the E update consumes it and clears J
            for k, v in J.items():
                t[k].copy_(torch.from_numpy(v))
                og.a[k][...] = v
        q.qed_fdtd_advance(g, q.QED_FDTD_E, dt)
        og.advance_b(dt)
        og.advance_e(dt)
        for k in ("Jx", "Jy", "Jz"):
            og.a[k][...] = 0.0
    torch.cuda.synchronize()
    for k in NAMES:
        a = t[k].cpu().numpy().astype(np.float64)
        assert np.abs(a - og.a[k]).max() < 2e-5 * np.abs(og.a[k]).max(), k
    for k in ("Jx", "Jy", "Jz"):
        assert float(t[k].abs().max()) == 0.0


def _leptons(n, rng, box, vmax, first=0):
    (xa, xb), (ya, yb) = box
    p = rng.uniform(-vmax, vmax, (n, 3))
    s = rng.normal(size=(n, 3))
    s /= np.linalg.norm(s, axis=1, keepdims=True)
    return {"x": rng.uniform(xa, xb, n), "y": rng.uniform(ya, yb, n), "z": np.zeros(n),
            "px": p[:, 0], "py": p[:, 1], "pz": p[:, 2], "s1": s[:, 0], "s2": s[:, 1], "s3": s[:, 2],
            "w": rng.uniform(0.5, 2.0, n), "id": np.arange(first, first + n, dtype=np.uint64)}


def _div_j(J, dx, dy, periodic):
    jx, jy = J["Jx"], J["Jy"]
    if periodic:
        return (jx - np.roll(jx, 1, 1)) / dx + (jy - np.roll(jy, 1, 0)) / dy
    d = jx / dx
    d[:, 1:] -= jx[:, :-1] / dx
    d = d + jy / dy
    d[1:, :] -= jy[:-1, :] / dy
    return d


def _cell_sorted(d, dx, dy):
    o = np.lexsort((np.floor(d["x"] / dx), np.floor(d["y"] / dy)))
    return {k: v[o] for k, v in d.items()}


@pytest.mark.parametrize("prec", [q.QED_PREC_F64, q.QED_PREC_MIXED])
@pytest.mark.parametrize("periodic", [1, 0])
@pytest.mark.parametrize("order", ["random", "cell-sorted"])
def test_deposit_matches_oracle_and_conserves_charge(orc, ctx, prec, periodic, order):
    """One step of e- and e+ (ragged counts, several tiles) with zero fields: the deposited
    current against the oracle's, and the continuity equation on the library's current.
    Random order: every tile spans the grid (direct atomic adds to the grid); cell-sorted:
    each tile's stencils fit the shared-memory window (summed there, then added)."""
    nx, ny, dx, dy, dt = 64, 48, 0.3, 0.25, 0.11
    rng = np.random.default_rng(5 + periodic)
    m = 0.0 if periodic else 3.0
    box = ((m * dx, (nx - m) * dx), (m * dy, (ny - m) * dy))
    e = _leptons(3001, rng, box, 3.0)
    pos = _leptons(1299, rng, box, 3.0, first=3001)
    if order == "cell-sorted":
        e, pos = _cell_sorted(e, dx, dy), _cell_sorted(pos, dx, dy)
    wl = {"e": e, "pos": pos, "ph": workloads.empty(True), "dt": dt, "seed": 1, "next_id": 4300}
    sim = q.PicSimulation(wl, nx, ny, dx, dy, periodic=periodic, prec=prec, ctx=ctx)
    # the deposit alone: one qed_step with QED_F_DEPOSIT on the zero grid (no FDTD)
    q.qed_step(sim.ctx, sim.e.handle, sim.pos.handle, sim.ph.handle, sim.fields, sim.t, sim.dt, sim.seed,
               sim.step_no, q.QED_F_DEPOSIT, sim.stats.data_ptr())
    st = sim.state()
    J = sim.field_arrays()
    og = oracle.YeeGrid(nx, ny, dx, dy, periodic=periodic)
    osim = oracle.PicSim(orc, wl, og)
    og.advance_b = lambda dt: None
    og.advance_e = lambda dt: None
    osim.run(1, 0)
    for k in ("Jx", "Jy", "Jz"):
        scale = np.abs(og.a[k]).max()
        assert np.abs(J[k] - og.a[k]).max() < 2e-5 * scale, (k, np.abs(J[k] - og.a[k]).max() / scale)
    rho0 = og.charge(np.r_[e["x"], pos["x"]], np.r_[e["y"], pos["y"]], np.r_[-e["w"], pos["w"]])
    rho1 = og.charge(np.r_[st["e"]["x"], st["pos"]["x"]], np.r_[st["e"]["y"], st["pos"]["y"]],
                     np.r_[-st["e"]["w"], st["pos"]["w"]])
    resid = (rho1 - rho0) / dt + _div_j(J, dx, dy, periodic)
    assert np.abs(resid).max() < 2e-5 * np.abs(rho0).max() / dt
    sim.close()


@pytest.mark.parametrize("prec", [q.QED_PREC_F64, q.QED_PREC_MIXED])
@pytest.mark.parametrize("heavy", [1.0e4, 3.0])
def test_deposit_keeps_light_particles_of_a_mixed_weight_tile(orc, ctx, prec, heavy):
    """One tile of 256 electrons in a 16 x 8-cell patch: light ones (w = 1) everywhere, a
    few of weight `heavy` in its right quarter.  Where no heavy stencil reaches, the current
    must match the oracle's to 1e-5 of the light particles' own scale: a tile whose weights
    spread by 1e4 must not round the light terms to the heavy ones' resolution."""
    nx, ny, dx, dy, dt = 64, 48, 0.3, 0.25, 0.11
    rng = np.random.default_rng(17)
    n = 256
    i0, j0 = 20, 20
    d = _leptons(n, rng, ((i0 * dx, (i0 + 16) * dx), (j0 * dy, (j0 + 8) * dy)), 0.5)
    d["w"] = np.ones(n)
    hv = rng.choice(n, 24, replace=False)
    d["x"][hv] = rng.uniform((i0 + 13) * dx, (i0 + 16) * dx, len(hv))
    d["w"][hv] = heavy
    d = _cell_sorted(d, dx, dy)
    wl = {"e": d, "pos": workloads.empty(), "ph": workloads.empty(True), "dt": dt, "seed": 1, "next_id": n}
    sim = q.PicSimulation(wl, nx, ny, dx, dy, periodic=0, prec=prec, ctx=ctx)
    q.qed_step(sim.ctx, sim.e.handle, sim.pos.handle, sim.ph.handle, sim.fields, sim.t, sim.dt, sim.seed,
               sim.step_no, q.QED_F_DEPOSIT, sim.stats.data_ptr())
    J = sim.field_arrays()
    og = oracle.YeeGrid(nx, ny, dx, dy, periodic=0)
    osim = oracle.PicSim(orc, wl, og)
    og.advance_b = lambda dt: None
    og.advance_e = lambda dt: None
    osim.run(1, 0)
    light = np.s_[:, : i0 + 9]      # heavy stencils start at column i0 + 13 - 3
    for k in ("Jx", "Jy", "Jz"):
        scale = np.abs(og.a[k][light]).max()
        assert scale > 0
        err = np.abs(J[k][light] - og.a[k][light]).max() / scale
        assert err < 1e-5, (k, err)
    sim.close()


def _plasma(nx, ny, dx, dy, ppc, n0, amp, seed):
    Lx = nx * dx
    k = 2 * math.pi / Lx
    N = nx * ny * ppc
    rng = np.random.default_rng(seed)
    xq = (np.arange(N) % (nx * ppc) + 0.5) * (Lx / (nx * ppc))
    x = xq + amp * np.sin(k * xq)
    y = rng.uniform(0, ny * dy, N)
    e = {"x": x, "y": y, "z": np.zeros(N), "px": np.zeros(N), "py": np.zeros(N), "pz": np.zeros(N),
         "s1": np.zeros(N), "s2": np.ones(N), "s3": np.zeros(N), "w": np.full(N, n0 * dx * dy / ppc),
         "id": np.arange(N, dtype=np.uint64)}
    og = oracle.YeeGrid(nx, ny, dx, dy, periodic=1)
    rho = og.charge(x, y, -e["w"]) + n0
    ex = np.cumsum(rho.mean(0)) * dx
    ex -= ex.mean()
    return e, np.repeat(ex[None, :], ny, 0), k


def test_pic_loop_matches_oracle_and_keeps_gauss(orc, ctx):
    """A warm plasma of e- and e+ with random momenta in a periodic box, 120 steps of the
    full loop (FDTD halves, step, deposit) on both sides: fields and particles agree to
    float accuracy, and div E - rho keeps its initial value on the library's arrays."""
    nx, ny, dx, dy, dt = 48, 40, 0.5, 0.5, 0.2
    rng = np.random.default_rng(13)
    box = ((0, nx * dx), (0, ny * dy))
    e = _leptons(4000, rng, box, 0.5)
    pos = _leptons(2000, rng, box, 0.5, first=4000)
    for d in (e, pos):
        d["w"] *= 0.05
    wl = {"e": e, "pos": pos, "ph": workloads.empty(True), "dt": dt, "seed": 3, "next_id": 6000}
    f0 = {"Ez": 0.05 * rng.normal(size=(ny, nx)).astype(np.float32)}
    sim = q.PicSimulation(wl, nx, ny, dx, dy, periodic=1, fields=f0, prec=q.QED_PREC_F64, ctx=ctx)
    og = oracle.YeeGrid(nx, ny, dx, dy, periodic=1, fields={"Ez": f0["Ez"].astype(np.float64)})
    osim = oracle.PicSim(orc, wl, og)

    def gauss(F, st):
        rho = og.charge(np.r_[st["e"]["x"], st["pos"]["x"]], np.r_[st["e"]["y"], st["pos"]["y"]],
                        np.r_[-st["e"]["w"], st["pos"]["w"]])
        return (F["Ex"] - np.roll(F["Ex"], 1, 1)) / dx + (F["Ey"] - np.roll(F["Ey"], 1, 0)) / dy - rho

    g0 = gauss(sim.field_arrays(), sim.state())
    flags = q.QED_F_SPIN
    sim.run(120, flags)
    osim.run(120, flags)
    F, st, ost = sim.field_arrays(), sim.state(), osim.state()
    g1 = gauss(F, st)
    assert np.abs(g1 - g0).max() < 1e-4 * np.abs(g0).max()
    for k in NAMES:
        scale = max(np.abs(og.a[k]).max(), 1e-6)
        assert np.abs(F[k] - og.a[k]).max() < 1e-3 * scale, (k, np.abs(F[k] - og.a[k]).max() / scale)
    for sp in ("e", "pos"):
        a, b = st[sp], ost[sp]
        assert np.array_equal(a["id"], b["id"])
        pa = np.stack([a["px"], a["py"], a["pz"]], 1)
        pb = np.stack([b["px"], b["py"], b["pz"]], 1)
        assert np.abs(pa - pb).max() < 1e-4 * np.abs(pb).max()
        assert np.abs(a["x"] - b["x"]).max() < 1e-5 * nx * dx
    assert float(np.abs(F["Bz"]).max()) > 1e-4   # the fields evolved
    sim.close()


@pytest.mark.parametrize("prec", [q.QED_PREC_F64, q.QED_PREC_MIXED])
def test_cold_plasma_frequency(ctx, prec):
    """The library's loop alone: a cold plasma oscillates at w_p = sqrt(n0) (3%)."""
    nx, ny, dx, dy, dt, n0 = 32, 4, 0.5, 0.5, 0.2, 0.01
    e, ex, k = _plasma(nx, ny, dx, dy, 16, n0, 0.02, seed=2)
    wl = {"e": e, "pos": workloads.empty(), "ph": workloads.empty(True), "dt": dt, "seed": 1,
          "next_id": len(e["id"])}
    sim = q.PicSimulation(wl, nx, ny, dx, dy, periodic=1, fields={"Ex": ex}, prec=prec, ctx=ctx)
    mode = np.sin(k * (np.arange(nx) + 0.5) * dx)
    prev = (sim.field_arrays()["Ex"].mean(0) * mode).sum()
    t_zero = None
    for step in range(1, 200):
        sim.run(1, 0)
        cur = (sim.field_arrays()["Ex"].mean(0) * mode).sum()
        if prev * cur < 0:
            t_zero = (step - 1 + prev / (prev - cur)) * dt
            break
        prev = cur
    sim.close()
    assert t_zero is not None
    assert t_zero == pytest.approx(math.pi / (2 * math.sqrt(n0)), rel=0.03)


def test_deposit_validation(ctx):
    wl = workloads.c1(n=10, seed=1)
    sim = q.Simulation(wl, prec=q.QED_PREC_F64, ctx=ctx)
    with pytest.raises(q.QedError, match="QED_F_DEPOSIT"):
        q.qed_step(sim.ctx, sim.e.handle, sim.pos.handle, sim.ph.handle, sim.fields, sim.t, sim.dt, sim.seed,
                   sim.step_no, q.QED_F_DEPOSIT)
    sim.close()
