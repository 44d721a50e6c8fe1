"""Pins of the oracle's field solver and current deposition (Secs. II B, II C, II F): the
self-consistent PIC loop around the QED step.

* Esirkepov deposition conserves charge on the grid exactly: (rho^{n+1} - rho^n)/dt +
  div J = 0 to rounding, with rho from the TSC charge assignment of Sec. II E (periodic and
  bounded grids, both charges, moves across cell boundaries); the summed current is
  sum q w v.
* The 2D Yee update propagates vacuum plane waves (each polarisation, along x and y)
  exactly as the discrete solution cos(k x - w t) with sin(w dt/2)/dt = sin(k dx/2)/dx.
* In the full loop, div E - rho and div B do not change (Gauss's law is embedded, the
  statement of Sec. II B), and a cold plasma oscillates at the plasma frequency."""
import math

import numpy as np
import pytest

import oracle
import workloads

F_DEP = oracle.F_DEPOSIT


def _leptons(n, rng, box, vmax, first=0):
    (xa, xb), (ya, yb) = box
    p = rng.uniform(-vmax, vmax, (n, 3))
    s = rng.normal(size=(n, 3))
    s /= np.linalg.norm(s, axis=1, keepdims=True)
    return {"x": rng.uniform(xa, xb, n), "y": rng.uniform(ya, yb, n), "z": np.zeros(n),
            "px": p[:, 0], "py": p[:, 1], "pz": p[:, 2], "s1": s[:, 0], "s2": s[:, 1], "s3": s[:, 2],
            "w": rng.uniform(0.5, 2.0, n), "id": np.arange(first, first + n, dtype=np.uint64)}


def _wl(e, pos, dt):
    return {"e": e, "pos": pos, "ph": workloads.empty(True), "field": {"kind": "grid2d"}, "dt": dt, "seed": 1,
            "next_id": len(e["id"]) + len(pos["id"])}


def _div_j(g, a):
    jx, jy = a["Jx"], a["Jy"]
    if g.periodic:
        return (jx - np.roll(jx, 1, 1)) / g.dx + (jy - np.roll(jy, 1, 0)) / g.dy
    d = jx / g.dx
    d[:, 1:] -= jx[:, :-1] / g.dx
    d = d + jy / g.dy
    d[1:, :] -= jy[:-1, :] / g.dy
    return d


@pytest.mark.parametrize("periodic", [1, 0])
def test_esirkepov_charge_conservation(orc, periodic):
    nx, ny, dx, dy, dt = 24, 18, 0.3, 0.25, 0.11
    rng = np.random.default_rng(3 + periodic)
    margin = 0.0 if periodic else 3.0
    box = ((margin * dx, (nx - margin) * dx), (margin * dy, (ny - margin) * dy))
    # momenta up to 3: speeds near 1, moves up to 0.44 of a cell; wrapping across the
    # periodic edges is exercised by particles near them
    e = _leptons(700, rng, box, 3.0)
    pos = _leptons(300, rng, box, 3.0, first=700)
    grid = oracle.YeeGrid(nx, ny, dx, dy, periodic=periodic)
    sim = oracle.PicSim(orc, _wl(e, pos, dt), grid)
    x0 = {sp: (d["x"].copy(), d["y"].copy()) for sp, d in (("e", e), ("pos", pos))}
    # one step of the deposit alone (no fields, no QED): the step zeroes J, deposits
    grid.advance_b = lambda dt: None
    grid.advance_e = lambda dt: None
    sim.run(1, 0)
    st = sim.state()
    rho0 = grid.charge(np.r_[x0["e"][0], x0["pos"][0]], np.r_[x0["e"][1], x0["pos"][1]],
                       np.r_[-e["w"], pos["w"]])
    rho1 = grid.charge(np.r_[st["e"]["x"], st["pos"]["x"]], np.r_[st["e"]["y"], st["pos"]["y"]],
                       np.r_[-st["e"]["w"], st["pos"]["w"]])
    resid = (rho1 - rho0) / dt + _div_j(grid.g, grid.a)
    scale = np.abs(rho0).max() / dt
    assert np.abs(resid).max() < 1e-12 * scale, np.abs(resid).max() / scale
    # the total current is sum q w v
    for k, axis in (("Jx", "x"), ("Jy", "y")):
        tot = grid.a[k].sum() * dx * dy
        mv = (-(st["e"][axis] - x0["e"][0 if axis == "x" else 1]) * e["w"]).sum() + \
             ((st["pos"][axis] - x0["pos"][0 if axis == "x" else 1]) * pos["w"]).sum()
        assert tot == pytest.approx(mv / dt, rel=1e-12, abs=1e-12 * scale)
    vz = lambda d: d["pz"] / np.sqrt(1 + d["px"] ** 2 + d["py"] ** 2 + d["pz"] ** 2)
    jz = (-(vz(st["e"]) * st["e"]["w"]).sum() + (vz(st["pos"]) * st["pos"]["w"]).sum())
    assert grid.a["Jz"].sum() * dx * dy == pytest.approx(jz, rel=1e-12)


@pytest.mark.parametrize("mode", ["Ey-Bz along x", "Ez-By along x", "Ex-Bz along y", "Ez-Bx along y"])
def test_yee_vacuum_plane_wave_is_the_discrete_solution(mode):
    """A periodic vacuum plane wave: after N leapfrog steps the fields equal the exact
    discrete wave, frequency from the Yee dispersion relation."""
    nx, ny, dx, dy, dt, m = 48, 40, 0.4, 0.5, 0.18, 3
    along_x = mode.endswith("x")
    L, h = (nx * dx, dx) if along_x else (ny * dy, dy)
    k = 2 * math.pi * m / L
    w = 2 / dt * math.asin(dt / h * math.sin(k * h / 2))
    I, J = np.meshgrid(np.arange(nx), np.arange(ny))
    s = 1.0 if along_x else -1.0   # orientation of the transverse pair

    def wave(comp, t, half_x, half_y):
        pos = (I + 0.5 * half_x) * dx if along_x else (J + 0.5 * half_y) * dy
        return np.cos(k * pos - w * t)

    # staggering: Ex (1/2,0) Ey (0,1/2) Ez (0,0) Bx (0,1/2) By (1/2,0) Bz (1/2,1/2)
    stag = {"Ex": (1, 0), "Ey": (0, 1), "Ez": (0, 0), "Bx": (0, 1), "By": (1, 0), "Bz": (1, 1)}
    e_comp, b_comp = {"Ey-Bz along x": ("Ey", "Bz"), "Ez-By along x": ("Ez", "By"),
                      "Ex-Bz along y": ("Ex", "Bz"), "Ez-Bx along y": ("Ez", "Bx")}[mode]
    # sign of B for a wave along +axis: Ey->Bz (+), Ez->By (-), Ex->Bz (-), Ez->Bx (+)
    bs = {"Ey-Bz along x": 1.0, "Ez-By along x": -1.0, "Ex-Bz along y": -1.0, "Ez-Bx along y": 1.0}[mode]
    del s
    g = oracle.YeeGrid(nx, ny, dx, dy, periodic=1)
    g.a[e_comp][...] = wave(e_comp, 0.0, *stag[e_comp])
    g.a[b_comp][...] = bs * wave(b_comp, -0.5 * dt, *stag[b_comp])
    nstep = 150
    for _ in range(nstep):
        g.advance_b(dt)      # B^{n-1/2} -> B^{n+1/2}
        g.advance_e(dt)      # E^n -> E^{n+1}
    t = nstep * dt
    assert np.abs(g.a[e_comp] - wave(e_comp, t, *stag[e_comp])).max() < 1e-11
    assert np.abs(g.a[b_comp] - bs * wave(b_comp, t - 0.5 * dt, *stag[b_comp])).max() < 1e-11
    for other in ("Ex", "Ey", "Ez", "Bx", "By", "Bz"):
        if other not in (e_comp, b_comp):
            assert np.abs(g.a[other]).max() == 0.0


def test_gauss_law_embedded_in_the_loop(orc):
    """Sec. II B: with the charge-conserving deposition the solver needs only the curl
    equations; div E - rho keeps its initial value and div B stays zero."""
    nx, ny, dx, dy, dt = 20, 16, 0.5, 0.5, 0.2
    rng = np.random.default_rng(11)
    box = ((0, nx * dx), (0, ny * dy))
    e = _leptons(600, rng, box, 0.8)
    pos = _leptons(200, rng, box, 0.8, first=600)
    grid = oracle.YeeGrid(nx, ny, dx, dy, periodic=1)
    grid.a["Ez"][...] = 0.2 * rng.normal(size=(ny, nx))    # a divergence-free start for B (B = 0)
    sim = oracle.PicSim(orc, _wl(e, pos, dt), grid)

    def rho(st):
        return grid.charge(np.r_[st["e"]["x"], st["pos"]["x"]], np.r_[st["e"]["y"], st["pos"]["y"]],
                           np.r_[-st["e"]["w"], st["pos"]["w"]])

    g0 = grid.div_e() - rho(sim.state())
    for _ in range(5):
        sim.run(20, oracle.F_SPIN)
        g1 = grid.div_e() - rho(sim.state())
        assert np.abs(g1 - g0).max() < 1e-10 * max(np.abs(g0).max(), 1.0)
    # Bx(i, j+1/2) and By(i+1/2, j): div B at the cell centres (i+1/2, j+1/2)
    bx, by = grid.a["Bx"], grid.a["By"]
    divb = (np.roll(bx, -1, 1) - bx) / dx + (np.roll(by, -1, 0) - by) / dy
    assert np.abs(divb).max() < 1e-10 * max(np.abs(bx).max() + np.abs(by).max(), 1e-3)
    assert np.abs(bx).max() > 1e-4   # the fields did evolve


def test_cold_plasma_oscillates_at_the_plasma_frequency(orc):
    """Electrons with a small sinusoidal displacement over a fixed neutralising background
    (initial E from Gauss's law): E_x oscillates at w_p = sqrt(n0) (n0 in n_c, Sec. II B
    normalisation).  Quarter period from the first zero of the mode amplitude."""
    nx, ny, dx, dy, dt = 32, 4, 0.5, 0.5, 0.2
    ppc = 16
    n0 = 0.01
    Lx = nx * dx
    k = 2 * math.pi / Lx
    N = nx * ny * ppc
    w = n0 * dx * dy / ppc            # density w/(dx dy) n_c per particle and cell
    rng = np.random.default_rng(2)
    xq = (np.arange(N) % (nx * ppc) + 0.5) * (Lx / (nx * ppc))
    amp = 0.02
    x = xq + amp * np.sin(k * xq)
    y = rng.uniform(0, ny * dy, N)
    e = {"x": x, "y": y, "z": np.zeros(N), "px": np.zeros(N), "py": np.zeros(N), "pz": np.zeros(N),
         "s1": np.zeros(N), "s2": np.ones(N), "s3": np.zeros(N), "w": np.full(N, w),
         "id": np.arange(N, dtype=np.uint64)}
    grid = oracle.YeeGrid(nx, ny, dx, dy, periodic=1)
    rho = grid.charge(x, y, -e["w"]) + n0
    # Gauss along x: Ex(i+1/2) - Ex(i-1/2) = dx rho(i), zero mean
    ex = np.cumsum(rho.mean(0)) * dx
    ex -= ex.mean()
    grid.a["Ex"][...] = ex[None, :]
    sim = oracle.PicSim(orc, _wl(e, workloads.empty(), dt), grid)
    mode = np.sin(k * (np.arange(nx) + 0.5) * dx)   # the displacement goes as sin(kx): so does E_x
    a0 = (grid.a["Ex"].mean(0) * mode).sum()
    t_zero = None
    prev = a0
    for step in range(1, 200):
        sim.run(1, 0)
        cur = (grid.a["Ex"].mean(0) * mode).sum()
        if prev * cur < 0:
            t_zero = (step - 1 + prev / (prev - cur)) * dt
            break
        prev = cur
    assert t_zero is not None
    wp = math.sqrt(n0)
    assert t_zero == pytest.approx(math.pi / (2 * wp), rel=0.03)
