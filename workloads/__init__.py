"""Seeded synthetic inputs shaped like the paper's workloads.

This module draws initial particle states (numpy, seeded) and describes the external
fields by their parameters.  It holds none of the method's arithmetic: the field
formulas, pushes and QED processes are evaluated separately by the CUDA library and
by the oracle.  Both sides are fed from here.

Units: t in 1/omega0, x in 1/k0 (lambda = 2 pi), p in m c, fields in m c omega0 / e.
"""
from __future__ import annotations

import math

import numpy as np

TWO_PI = 2.0 * math.pi
T0 = TWO_PI                    # laser period
DT_200 = T0 / 200.0            # pi/100


def _ids(n, first=0):
    return np.arange(first, first + n, dtype=np.uint64)


def _sphere(rng, n):
    v = rng.normal(size=(n, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return v


def empty(photon=False):
    d = {k: np.zeros(0) for k in ("x", "y", "z", "px", "py", "pz", "s1", "s2", "s3", "w")}
    if photon:
        d["theta"] = np.zeros(0)
    d["id"] = np.zeros(0, dtype=np.uint64)
    return d


# ---------------------------------------------------------------------------------
# Config 1: plain NCS, LP plane wave, monoenergetic polarised electrons
# ---------------------------------------------------------------------------------
def c1(n=10_000, seed=1, gamma0=2000.0, a0=20.0, cycles=4, z0=-0.5):
    """1e4 e-, gamma0 = 2000 along +z, S = +y, all at (0, 0, z0) just outside an LP
    (E along x) plane wave moving along -z with a sin^2 envelope of `cycles` periods
    starting at phase t + z = 0; dt = T0/200; 450 steps cover the crossing."""
    pz = math.sqrt(gamma0 * gamma0 - 1.0)
    e = {"x": np.zeros(n), "y": np.zeros(n), "z": np.full(n, z0),
         "px": np.zeros(n), "py": np.zeros(n), "pz": np.full(n, pz),
         "s1": np.zeros(n), "s2": np.ones(n), "s3": np.zeros(n),
         "w": np.ones(n), "id": _ids(n)}
    field = {"kind": "plane", "circular": 0, "a0": a0, "phi0": 0.0, "len": cycles * T0}
    return {"e": e, "pos": empty(), "ph": empty(True), "field": field, "dt": DT_200,
            "t0": 0.0, "steps": 450, "seed": seed, "next_id": n,
            "name": f"c1_plane_lp_a{a0:g}_g{gamma0:g}_n{n}"}


# ---------------------------------------------------------------------------------
# Config 2: full NCS + NBW + VB, CP paraxial Gaussian, Gaussian beam, random spins
# ---------------------------------------------------------------------------------
def c2(n=1_000_000, seed=2, gamma0=2.0e4, spread=0.05, a0=100.0, w0_um=3.0, cycles=10,
       sigma_r_um=1.0, sigma_z_um=1.0):
    """e- beam with gamma ~ N(gamma0, spread*gamma0) along +z, transverse and longitudinal
    rms 1 um, spins uniform on the sphere; CP paraxial Gaussian (a0 per component,
    w0 = 3 um) moving along -z with a 10-cycle sin^2 envelope over t + z in [0, 20 pi].
    The beam centre starts at z = -10 pi (outside the pulse) and meets the pulse centre at
    the focus z = 0, t = 10 pi.  dt = T0/200; steps 200..1800 span the collision."""
    rng = np.random.default_rng(seed)
    um = TWO_PI  # 1 um in units of 1/k0
    L = cycles * T0
    zc = -0.5 * L
    g = rng.normal(gamma0, spread * gamma0, n)
    g = np.maximum(g, 2.0)
    pz = np.sqrt(g * g - 1.0)
    s = _sphere(rng, n)
    e = {"x": rng.normal(0, sigma_r_um * um, n), "y": rng.normal(0, sigma_r_um * um, n),
         "z": zc + rng.normal(0, sigma_z_um * um, n),
         "px": np.zeros(n), "py": np.zeros(n), "pz": pz,
         "s1": s[:, 0], "s2": s[:, 1], "s3": s[:, 2], "w": np.ones(n), "id": _ids(n)}
    field = {"kind": "gauss", "circular": 1, "a0": a0, "phi0": 0.0, "len": L,
             "w0": w0_um * um, "zf": 0.0}
    return {"e": e, "pos": empty(), "ph": empty(True), "field": field, "dt": DT_200,
            "t0": 0.0, "steps": 1800, "seed": seed, "next_id": n,
            "name": f"c2_gauss_cp_a{a0:g}_g{gamma0:g}_n{n}"}


# ---------------------------------------------------------------------------------
# Config 3: 2D3V Yee grid snapshot of an LP pulse reflected off a dense slab
# ---------------------------------------------------------------------------------
def c3_grid(nx=4096, ny=2048, a0=150.0, ncrit=100.0, seed=3):
    """FP32 Yee arrays (cells of lambda/32) holding an LP pulse (E along y, 8 cycles) moving
    along +x whose centre has reached a slab at x_s = 3/4 of the box (plasma frequency
    sqrt(ncrit) omega0): in front of the slab the incident field plus its reflection (pi
    phase, the mirror image of the part beyond x_s); inside, decay as exp(-(x-x_s) w_p).
    A single frozen snapshot, taken an eighth of a period after the instant at which the
    standing wave in front of the slab has no electric field (x_s is a whole number of
    wavelengths), so that E and B are both present; Ez = Bx = By = 0 (2D TE-like, z
    squeezed)."""
    dx = TWO_PI / 32.0
    dy = dx
    xs = 0.75 * nx * dx
    wp = math.sqrt(ncrit)
    L = 8 * T0                      # pulse length (phase)
    wy = 0.25 * ny * dy             # transverse Gaussian width
    yc = 0.5 * ny * dy

    def profile(xp):  # incident pulse centred on the slab surface: half already reflected
        ph = xp - xs
        env = np.where(np.abs(ph) < 0.5 * L, np.cos(math.pi * ph / L) ** 2, 0.0)
        return env

    i = np.arange(nx)
    j = np.arange(ny)
    xh = (i + 0.5) * dx               # half-grid x
    xg = i * dx                       # grid x
    yh = (j + 0.5) * dy
    yg = j * dy

    def field(xp, yp):
        tr = np.exp(-((yp[:, None] - yc) / wy) ** 2)
        ph0 = 0.25 * math.pi       # the carrier an eighth of a period on
        inc = profile(xp)[None, :] * np.cos(xp - ph0)[None, :]
        refl = -profile(2 * xs - xp)[None, :] * np.cos(2 * xs - xp - ph0)[None, :]
        vac = xp[None, :] < xs
        inside = np.exp(-np.clip(xp - xs, 0, None) * wp)[None, :]
        e = np.where(vac, inc + refl, (inc + refl) * inside)
        b = np.where(vac, inc - refl, (inc - refl) * inside)
        return a0 * tr * e, a0 * tr * b

    Ey, _ = field(xg, yh)            # Ey at (i, j+1/2)
    _, Bz = field(xh, yh)            # Bz at (i+1/2, j+1/2)
    z = np.zeros((ny, nx), dtype=np.float32)
    return {"Ex": z, "Ey": Ey.astype(np.float32), "Ez": z, "Bx": z, "By": z,
            "Bz": Bz.astype(np.float32), "dx": dx, "dy": dy, "x0": 0.0, "y0": 0.0,
            "xs": xs}


def c3(n=30_000_000, seed=3, gamma0=4000.0, nx=4096, ny=2048, grid=None):
    """e- at gamma0 = 4000 moving along +x, uniform in the vacuum part of the box,
    unpolarised spins, counting-sorted by 32x32-cell tiles; dt = T0/64."""
    rng = np.random.default_rng(seed)
    g = grid if grid is not None else c3_grid(nx, ny, seed=seed)
    dx, dy = g["dx"], g["dy"]
    x = rng.uniform(2 * dx, g["xs"] - 2 * dx, n)
    y = rng.uniform(2 * dy, (ny - 2) * dy, n)
    tile = (np.floor(y / (32 * dy)).astype(np.int64) * (nx // 32) + np.floor(x / (32 * dx)).astype(np.int64))
    order = np.argsort(tile, kind="stable")
    x, y = x[order], y[order]
    s = _sphere(rng, n)
    e = {"x": x, "y": y, "z": np.zeros(n), "px": np.full(n, math.sqrt(gamma0 ** 2 - 1)),
         "py": np.zeros(n), "pz": np.zeros(n), "s1": s[:, 0], "s2": s[:, 1], "s3": s[:, 2],
         "w": np.ones(n), "id": _ids(n)}
    return {"e": e, "pos": empty(), "ph": empty(True), "grid": g,
            "field": {"kind": "grid2d"}, "dt": T0 / 64.0, "t0": 0.0, "steps": 200,
            "seed": seed, "next_id": n, "name": f"c3_grid_{nx}x{ny}_n{n}"}


# ---------------------------------------------------------------------------------
# Config 4: batched uneven ensembles
# ---------------------------------------------------------------------------------
def c4(n_ens=64, seed=4, cap_each=None):
    """64 independent collisions: sizes floor(10^U(3,6)), a0 ~ U(10,200), gamma0 ~ U(500,2e4),
    polarisation alternating LP/CP, spins cycling unpolarised / +-y / longitudinal;
    every fourth ensemble is a gamma beam (omega = gamma0, random pure Stokes)."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n_ens):
        n = int(math.floor(10 ** rng.uniform(3, 6)))
        if cap_each:
            n = min(n, cap_each)
        a0 = rng.uniform(10, 200)
        g0 = rng.uniform(500, 2e4)
        circ = k % 2
        sub = c2(n=n, seed=seed * 1000 + k, gamma0=g0, a0=a0)
        sub["field"]["circular"] = circ
        e = sub["e"]
        mode = k % 4
        if mode == 1:
            e["s1"][:], e["s2"][:], e["s3"][:] = 0.0, 1.0, 0.0
        elif mode == 2:
            e["s1"][:], e["s2"][:], e["s3"][:] = 0.0, -1.0, 0.0
        elif mode == 3:
            e["s1"][:], e["s2"][:], e["s3"][:] = 0.0, 0.0, 1.0
        if k % 4 == 3:   # gamma beam instead of electrons
            xi = _sphere(rng, n)
            ph = {"x": e["x"], "y": e["y"], "z": e["z"], "px": np.zeros(n), "py": np.zeros(n),
                  "pz": np.full(n, g0), "s1": xi[:, 0], "s2": xi[:, 1], "s3": xi[:, 2],
                  "theta": np.zeros(n), "w": np.ones(n), "id": _ids(n)}
            sub["ph"] = ph
            sub["e"] = empty()
        sub["name"] = f"c4_ens{k}"
        out.append(sub)
    return out


# ---------------------------------------------------------------------------------
# Matter (Sec. III E): an electron beam through a solid slab, no laser field -- the
# paper's bremsstrahlung test (1 GeV and 100 MeV electrons onto 5 mm of Au or Al, the
# field updater off).  Densities of the solid from its mass density and molar mass.
# ---------------------------------------------------------------------------------
LENGTH_UNIT_CM = 1e-4 / TWO_PI     # 1/k0 for lambda = 1 um
SOLIDS = {"Au": (79, 19.32, 196.966570), "Al": (13, 2.699, 26.9815385), "Cu": (29, 8.96, 63.546),
          "W": (74, 19.3, 183.84), "Pb": (82, 11.35, 207.2)}


def medium(name="Au", thickness_mm=5.0, k_min=1.0, axis=2):
    """The slab 0 <= x[axis] < thickness of solid `name`: atoms per (1/k0)^3; photons below
    k_min (m c^2) are not produced."""
    Z, rho, A = SOLIDS[name]
    n = rho * 6.02214076e23 / A * LENGTH_UNIT_CM ** 3
    return {"Z": Z, "n": n, "k_min": k_min, "axis": axis, "lo": 0.0, "hi": thickness_mm * 0.1 / LENGTH_UNIT_CM}


def slab(n=1_000_000, seed=5, gamma0=2000.0, spread=0.0, name="Au", thickness_mm=5.0, k_min=1.0, dt_um=5.0,
         depth_mm=0.0):
    """n electrons (gamma0 = 2000 is 1 GeV) along +z at depth `depth_mm` inside the slab
    (transverse Gaussian rms 10 um, spins along +y), no field; dt such that c dt = dt_um
    micrometres; crossing the 5 mm slab takes 1000 steps at 5 um."""
    rng = np.random.default_rng(seed)
    g = gamma0 * (1.0 + spread * rng.normal(size=n)) if spread > 0 else np.full(n, gamma0)
    pz = np.sqrt(np.maximum(g * g - 1.0, 0.0))
    sig = 10e-4 / LENGTH_UNIT_CM
    e = {"x": rng.normal(size=n) * sig, "y": rng.normal(size=n) * sig, "z": np.full(n, depth_mm * 0.1 / LENGTH_UNIT_CM),
         "px": np.zeros(n), "py": np.zeros(n), "pz": pz,
         "s1": np.zeros(n), "s2": np.ones(n), "s3": np.zeros(n), "w": np.ones(n), "id": _ids(n)}
    return {"e": e, "pos": empty(), "ph": empty(True), "field": {"kind": "none"},
            "dt": dt_um * 1e-4 / LENGTH_UNIT_CM, "t0": 0.0, "seed": seed, "next_id": n,
            "medium": medium(name, thickness_mm, k_min), "name": f"slab_{name}_{thickness_mm:g}mm_g{gamma0:g}_n{n}"}


# ---------------------------------------------------------------------------------
# Sharding: a small mixed population (e-, e+, polarised photons) in a strong crossed field
# where pairs and emissions happen every step, and its split over ranks
# ---------------------------------------------------------------------------------
def crossed(ne=400, npos=200, nph=600, E0=200.0, seed=1, dt=0.3):
    """e- and e+ at gamma ~ 4000 along +z with random spins, photons of ~1.5 GeV with random
    partial polarisation, in the uniform crossed field E = E0 x, B = -E0 y."""
    rng = np.random.default_rng(seed)

    def lep(n, first):
        s = _sphere(rng, n)
        p = rng.normal(size=(n, 3)) * 30 + np.array([0, 0, 4000.0])
        return {"x": rng.normal(size=n), "y": rng.normal(size=n), "z": rng.uniform(0, 50, n),
                "px": p[:, 0], "py": p[:, 1], "pz": p[:, 2], "s1": s[:, 0], "s2": s[:, 1], "s3": s[:, 2],
                "w": rng.uniform(0.5, 2, n), "id": _ids(n, first)}
    e, pos = lep(ne, 0), lep(npos, ne)
    k = rng.normal(size=(nph, 3)) * 50 + np.array([0, 0, 3000.0])
    xi = _sphere(rng, nph) * rng.uniform(0, 1, (nph, 1))
    first = ne + npos
    ph = {"x": rng.normal(size=nph), "y": rng.normal(size=nph), "z": rng.uniform(0, 50, nph), "px": k[:, 0],
          "py": k[:, 1], "pz": k[:, 2], "s1": xi[:, 0], "s2": xi[:, 1], "s3": xi[:, 2],
          "theta": rng.uniform(-3, 3, nph), "w": np.ones(nph), "id": _ids(nph, first)}
    return {"e": e, "pos": pos, "ph": ph, "field": {"kind": "uniform", "E": (E0, 0, 0), "B": (0, -E0, 0)},
            "dt": dt, "seed": seed + 4, "next_id": first + nph, "name": f"crossed_E{E0:g}_{ne}_{npos}_{nph}"}


def shard(wl, rank, world):
    """Rank `rank` of `world` takes a contiguous part of every species (the ranks' parts in
    rank order are the whole population in its order); fields, clock and id counter are
    every rank's."""
    out = dict(wl)
    for sp in ("e", "pos", "ph"):
        n = len(wl[sp]["id"])
        lo, hi = n * rank // world, n * (rank + 1) // world
        out[sp] = {k: v[lo:hi] for k, v in wl[sp].items()}
    return out
