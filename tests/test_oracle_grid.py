"""Pins of the oracle's grid gather (config 3: TSC weights of Sec. II E on the 2D Yee
staggering of Sec. II B): the shape is a partition of unity and reproduces linear fields
exactly at the particle position for every staggered component (which fixes the half-cell
offsets), the gather of a smooth field converges at second order in the cell size, a
periodic grid wraps, and nodes outside a bounded grid contribute nothing."""
import math

import numpy as np
import pytest

import oracle

COMPS = ("Ex", "Ey", "Ez", "Bx", "By", "Bz")
# node of component c at (x0 + (i + sx/2) dx, y0 + (j + sy/2) dy)
STAGGER = {"Ex": (1, 0), "Ey": (0, 1), "Ez": (0, 0), "Bx": (0, 1), "By": (1, 0), "Bz": (1, 1)}


def _grid(fn, nx, ny, dx, dy, x0, y0, periodic=0):
    g = {"dx": dx, "dy": dy, "x0": x0, "y0": y0, "periodic": periodic}
    for c in COMPS:
        sx, sy = STAGGER[c]
        X = x0 + (np.arange(nx) + 0.5 * sx) * dx
        Y = y0 + (np.arange(ny) + 0.5 * sy) * dy
        g[c] = fn(c, X[None, :], Y[:, None]).astype(np.float32)
    return g


def _gather(g, x, y):
    f = oracle.make_fields(kind=oracle.FIELD_GRID2D, grid=g)
    E, B = oracle.field(f, x, y, 0.0, 0.0)
    return dict(zip(COMPS, list(E) + list(B)))


def _interior_points(rng, nx, ny, dx, dy, x0, y0, n=40):
    return [(x0 + rng.uniform(3, nx - 4) * dx, y0 + rng.uniform(3, ny - 4) * dy) for _ in range(n)]


def test_uniform_field_is_reproduced():
    nx, ny, dx, dy, x0, y0 = 40, 30, 0.3, 0.25, -1.0, 2.0
    vals = {c: 0.5 + k for k, c in enumerate(COMPS)}
    g = _grid(lambda c, X, Y: vals[c] + 0 * X + 0 * Y, nx, ny, dx, dy, x0, y0)
    for x, y in _interior_points(np.random.default_rng(1), nx, ny, dx, dy, x0, y0):
        got = _gather(g, x, y)
        for c in COMPS:
            assert got[c] == pytest.approx(vals[c], rel=1e-14)


def test_linear_fields_are_exact_at_the_particle_for_every_stagger():
    nx, ny, dx, dy, x0, y0 = 40, 30, 0.3, 0.25, -1.0, 2.0
    coef = {c: (0.3 + 0.1 * k, 0.7 - 0.2 * k, -0.4 + 0.15 * k) for k, c in enumerate(COMPS)}
    g = _grid(lambda c, X, Y: coef[c][0] + coef[c][1] * X + coef[c][2] * Y, nx, ny, dx, dy, x0, y0)
    for x, y in _interior_points(np.random.default_rng(2), nx, ny, dx, dy, x0, y0):
        got = _gather(g, x, y)
        for c in COMPS:
            a, b, d = coef[c]
            # float32 nodes: values of order 10 carry ~1e-6 absolute rounding
            assert got[c] == pytest.approx(a + b * x + d * y, abs=5e-6), c
            # a half-cell error in the stagger would move it by b dx / 2 or d dy / 2
            assert abs(got[c] - (a + b * (x + 0.5 * dx) + d * y)) > 1e-3 or abs(b) < 1e-9


def test_smooth_field_converges_at_second_order():
    kx, ky = 2 * math.pi / 7.0, 2 * math.pi / 5.0
    fn = lambda c, X, Y: np.sin(kx * X + 0.3) * np.cos(ky * Y - 0.2)
    rng = np.random.default_rng(3)
    pts = [(rng.uniform(2.0, 5.0), rng.uniform(2.0, 4.0)) for _ in range(30)]
    errs = []
    for n in (1, 2, 4):
        dx, dy = 0.2 / n, 0.2 / n
        nx, ny = int(8.0 / dx), int(7.0 / dy)
        g = _grid(fn, nx, ny, dx, dy, 0.0, 0.0)
        e = 0.0
        for x, y in pts:
            got = _gather(g, x, y)
            e = max(e, abs(got["Ez"] - math.sin(kx * x + 0.3) * math.cos(ky * y - 0.2)))
        errs.append(e)
    assert errs[0] / errs[1] == pytest.approx(4.0, rel=0.2)
    assert errs[1] / errs[2] == pytest.approx(4.0, rel=0.2)


def test_periodic_wrap_and_bounded_edge():
    nx, ny, dx, dy, x0, y0 = 32, 24, 0.5, 0.5, 0.0, 0.0
    rng = np.random.default_rng(4)
    base = {c: rng.normal(size=(ny, nx)).astype(np.float32) for c in COMPS}
    gp = dict(base, dx=dx, dy=dy, x0=x0, y0=y0, periodic=1)
    # a periodic grid gathers at x and at x + nx dx alike, and near its edge as the
    # interior gather of the grid rolled by half its size
    shift_i, shift_j = nx // 2, ny // 2
    gr = {c: np.roll(np.roll(base[c], shift_i, axis=1), shift_j, axis=0) for c in COMPS}
    gr.update(dx=dx, dy=dy, x0=x0, y0=y0, periodic=1)
    for x, y in [(0.1, 0.2), (nx * dx - 0.1, 3.0), (5.0, ny * dy - 0.05), (0.02, ny * dy - 0.3)]:
        a = _gather(gp, x, y)
        b = _gather(gp, x + nx * dx, y - ny * dy)
        r = _gather(gr, x + shift_i * dx, y + shift_j * dy)
        for c in COMPS:
            assert a[c] == pytest.approx(b[c], abs=1e-12)
            assert a[c] == pytest.approx(r[c], abs=1e-12)
    # bounded: a field living only outside a margin is not seen from deep inside, and
    # positions beyond the grid gather only the nodes inside it
    gb = dict({c: np.ones((ny, nx), dtype=np.float32) for c in COMPS}, dx=dx, dy=dy, x0=x0, y0=y0, periodic=0)
    far = _gather(gb, -10.0, -10.0)
    assert all(v == 0.0 for v in far.values())
    edge = _gather(gb, -0.5 * dx + 1e-9, 6.0)   # Ez: only the 2 inner of its 3 x-nodes exist
    assert 0.0 < edge["Ez"] < 1.0
