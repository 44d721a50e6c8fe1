"""The seeded synthetic inputs (workloads/) follow the recipes the paper's configurations
set (Secs. III-V and the benchmark configurations): distributions, geometry and field
parameters, determinism under a seed, and no method arithmetic in the generator."""
import math

import numpy as np
import pytest

import workloads

UM = 2 * math.pi      # 1 um in units of 1/k0 (lambda = 1 um)


def test_c1_recipe():
    w = workloads.c1(n=1000)
    e = w["e"]
    g = np.sqrt(1 + e["px"] ** 2 + e["py"] ** 2 + e["pz"] ** 2)
    assert np.allclose(g, 2000.0) and np.all(e["pz"] > 0)
    assert np.all(e["s2"] == 1.0) and np.all(e["s1"] == 0.0) and np.all(e["s3"] == 0.0)
    f = w["field"]
    assert f["kind"] == "plane" and f["circular"] == 0 and f["a0"] == 20.0
    assert f["len"] == pytest.approx(4 * 2 * math.pi)
    assert np.all(w["t0"] + e["z"] < f["phi0"])          # outside the pulse at the start
    assert w["dt"] == pytest.approx(math.pi / 100)


def test_c2_recipe():
    n = 200_000
    w = workloads.c2(n=n)
    e = w["e"]
    g = np.sqrt(1 + e["pz"] ** 2)
    assert g.mean() == pytest.approx(2.0e4, rel=2e-3)
    assert g.std() / g.mean() == pytest.approx(0.05, rel=0.02)
    for k in ("x", "y"):
        assert e[k].mean() == pytest.approx(0.0, abs=0.02 * UM)
        assert e[k].std() == pytest.approx(UM, rel=0.01)
    f = w["field"]
    assert e["z"].mean() == pytest.approx(-0.5 * f["len"], abs=0.02 * UM)
    assert e["z"].std() == pytest.approx(UM, rel=0.01)
    s = np.stack([e["s1"], e["s2"], e["s3"]], 1)
    assert np.allclose(np.linalg.norm(s, axis=1), 1.0)
    assert np.abs(s.mean(0)).max() < 0.01                # uniform on the sphere
    assert np.abs((s ** 2).mean(0) - 1 / 3).max() < 0.01
    assert f["kind"] == "gauss" and f["circular"] == 1 and f["a0"] == 100.0
    assert f["w0"] == pytest.approx(3 * UM) and f["len"] == pytest.approx(10 * 2 * math.pi)
    assert w["dt"] == pytest.approx(math.pi / 100)


def test_c3_recipe():
    nx, ny = 512, 256
    w = workloads.c3(n=100_000, nx=nx, ny=ny)
    g, e = w["grid"], w["e"]
    assert g["dx"] == pytest.approx(2 * math.pi / 32) and g["dy"] == g["dx"]
    for k in ("Ex", "Ey", "Ez", "Bx", "By", "Bz"):
        assert g[k].shape == (ny, nx) and g[k].dtype == np.float32
    for k in ("Ex", "Ez", "Bx", "By"):
        assert not g[k].any()
    # the standing wave in front of the slab carries both E and B (neither vanishes)
    assert 0.5 * 150 < np.abs(g["Ey"]).max() <= 2 * 150 + 1e-3
    assert 0.5 * 150 < np.abs(g["Bz"]).max() <= 2 * 150 + 1e-3
    assert np.all(e["x"] < g["xs"]) and np.all(e["x"] > 0) and np.all(e["y"] > 0)
    assert np.allclose(np.sqrt(1 + e["px"] ** 2), 4000.0)
    tile = np.floor(e["y"] / (32 * g["dy"])) * (nx // 32) + np.floor(e["x"] / (32 * g["dx"]))
    assert np.all(np.diff(tile) >= 0)                   # counting-sorted by 32 x 32 tiles
    assert w["dt"] == pytest.approx(2 * math.pi / 64)


def test_c4_recipe():
    ws = workloads.c4(cap_each=2000)
    assert len(ws) == 64
    circ = [w["field"]["circular"] for w in ws]
    assert circ == [k % 2 for k in range(64)]
    for k, w in enumerate(ws):
        assert 10 <= w["field"]["a0"] <= 200
        if k % 4 == 3:
            assert len(w["e"]["id"]) == 0
            ph = w["ph"]
            xi = np.stack([ph["s1"], ph["s2"], ph["s3"]], 1)
            assert np.allclose(np.linalg.norm(xi, axis=1), 1.0)
            assert 500 <= ph["pz"][0] <= 2e4
        else:
            e = w["e"]
            assert 1 <= len(e["id"]) <= 2000
    sizes = [int(math.floor(10 ** u)) for u in np.random.default_rng(4).uniform(3, 6, 1)]
    assert 1000 <= sizes[0] < 1_000_000


def test_seeded_and_independent():
    a, b, c = workloads.c2(n=1000, seed=5), workloads.c2(n=1000, seed=5), workloads.c2(n=1000, seed=6)
    for k in a["e"]:
        assert np.array_equal(a["e"][k], b["e"][k])
    assert not np.array_equal(a["e"]["x"], c["e"]["x"])
