"""qed_sort_cells: the stable cell sort of a particle set on a 2D grid, through the C ABI.

The expected order is computed here with numpy's stable argsort of the same key (32x32-cell
tile, then row-major cell inside the tile; outside a bounded grid last; a periodic grid
wraps): every array of the set must come out permuted exactly so, bit for bit.  Sizes span
one and many chunks of the sort, and 0 and 1 particles; electrons and photons (which carry
the basis angle); both precisions.  Sorting must not change the physics: a push-only run
of the sorted set equals that of the unsorted one particle by particle."""
import numpy as np
import pytest

import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2306_11288_gb300 as q  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    q.build()
    c = q.qed_init_tables()
    yield c
    torch.cuda.synchronize()


def _grid(nx, ny, periodic):
    g = {k: torch.zeros((ny, nx), dtype=torch.float32, device="cuda") for k in ("Ex", "Ey", "Ez", "Bx", "By", "Bz")}
    g.update({"dx": 0.3, "dy": 0.25, "x0": -1.0, "y0": 2.0, "periodic": periodic})
    return g


def _key(x, y, g, nx, ny):
    # the documented cell: floor((x - x0) * (1/dx)), each operation rounded in double
    ci = np.floor((x - g["x0"]) * (1.0 / g["dx"])).astype(np.int64)
    cj = np.floor((y - g["y0"]) * (1.0 / g["dy"])).astype(np.int64)
    if g["periodic"]:
        ci %= nx
        cj %= ny
    inside = (ci >= 0) & (ci < nx) & (cj >= 0) & (cj < ny)
    tx = (nx + 31) // 32
    ty = (ny + 31) // 32
    k = ((cj // 32) * tx + ci // 32) * 1024 + (cj % 32) * 32 + (ci % 32)
    return np.where(inside, k, tx * ty * 1024)


def _set(n, rng, photon, g, nx, ny):
    def frac():   # mostly in the box or just outside; a fifth one or more periods away
        u = rng.uniform(-0.1, 1.1, n)
        far = rng.uniform(size=n) < 0.2
        u[far] = rng.uniform(-2.6, 3.1, int(far.sum()))
        return u
    d = {"x": g["x0"] + frac() * nx * g["dx"], "y": g["y0"] + frac() * ny * g["dy"],
         "z": rng.normal(size=n), "px": rng.normal(size=n), "py": rng.normal(size=n), "pz": rng.normal(size=n),
         "s1": rng.normal(size=n), "s2": rng.normal(size=n), "s3": rng.normal(size=n), "w": rng.uniform(0.5, 2, n),
         "id": rng.permutation(n).astype(np.uint64) + 1000}
    if photon:
        d["theta"] = rng.uniform(-3, 3, n)
    return d


@pytest.mark.parametrize("prec", [q.QED_PREC_MIXED, q.QED_PREC_F64])
@pytest.mark.parametrize("periodic", [0, 1])
@pytest.mark.parametrize("n", [0, 1, 3001, 200_003])
def test_sort_order_is_the_stable_cell_order(ctx, prec, periodic, n):
    nx, ny = 300, 200   # not multiples of the 32-cell tile
    g = _grid(nx, ny, periodic)
    f = q.fields_from_spec({"kind": "grid2d"}, g)
    rng = np.random.default_rng(n + 7 * periodic)
    for species, photon in ((q.QED_ELECTRON, False), (q.QED_PHOTON, True)):
        d = _set(n, rng, photon, g, nx, ny)
        sp = q.Species(ctx, species, max(n, 16), prec).load(d)
        q.qed_sort_cells(ctx, sp.handle, f)
        got = sp.to_dict()
        sp.close()
        order = np.argsort(_key(d["x"], d["y"], g, nx, ny), kind="stable")
        for k, v in d.items():
            want = v[order]
            if k != "id" and prec == q.QED_PREC_MIXED and k not in ("x", "y", "z"):
                want = want.astype(np.float32).astype(np.float64)
            assert np.array_equal(got[k], want), (species, k)


def test_sorted_set_pushes_like_the_unsorted_one(ctx):
    g = workloads.c3_grid(nx=256, ny=128, a0=150.0)
    wl = workloads.c3(n=30000, seed=21, nx=256, ny=128, grid=g)
    rng = np.random.default_rng(3)
    perm = rng.permutation(len(wl["e"]["id"]))
    wl = dict(wl, e={k: v[perm] for k, v in wl["e"].items()})   # tile order lost
    out = []
    for sort in (False, True):
        sim = q.Simulation(wl, prec=q.QED_PREC_MIXED, ctx=ctx)
        if sort:
            q.qed_sort_cells(sim.ctx, sim.e.handle, sim.fields)
        sim.run(10, q.QED_F_SPIN)
        st = sim.state()["e"]
        o = np.argsort(st["id"])
        out.append({k: v[o] for k, v in st.items()})
        sim.close()
    for k in out[0]:
        assert np.array_equal(out[0][k], out[1][k]), k


def test_sort_validation(ctx):
    sp = q.Species(ctx, q.QED_ELECTRON, 16, q.QED_PREC_F64)
    with pytest.raises(q.QedError, match="grid"):
        q.qed_sort_cells(ctx, sp.handle, q.fields_from_spec({"kind": "uniform"}))
    sp.close()
