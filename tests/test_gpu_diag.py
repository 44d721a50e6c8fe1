"""qed_diag (spectra, detector maps of the Stokes parameters in a detection basis, mean
spin, yields) through the C ABI against the oracle's read-out of the same particle arrays.

Both sides see identical inputs (the oracle reads back what the device holds), so bin
counts must agree exactly and sums to FP64 rounding of the summation order (1e-12 of the
set's total weight)."""
import math

import numpy as np
import pytest

import oracle.diag as OD
import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2306_11288_gb300 as q  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    q.build()
    return q.qed_init_tables()


def _photons(m, seed):
    rng = np.random.default_rng(seed)
    k = rng.normal(size=(m, 3)) * 40.0
    k[: m // 2, 2] += np.exp(rng.uniform(0, 8, m // 2))   # beam-like half with a wide spectrum
    xi = rng.normal(size=(m, 3))
    xi *= rng.uniform(0, 1, (m, 1)) / np.linalg.norm(xi, axis=1)[:, None]
    return {"x": rng.uniform(-3, 3, m), "y": rng.uniform(-2, 2, m), "z": rng.normal(size=m),
            "px": k[:, 0], "py": k[:, 1], "pz": k[:, 2], "s1": xi[:, 0], "s2": xi[:, 1], "s3": xi[:, 2],
            "theta": rng.uniform(-math.pi, math.pi, m), "w": rng.uniform(0.5, 2.0, m),
            "id": np.arange(m, dtype=np.uint64)}


def _leptons(m, seed):
    rng = np.random.default_rng(seed)
    s = rng.normal(size=(m, 3))
    s /= np.linalg.norm(s, axis=1)[:, None]
    p = rng.normal(size=(m, 3)) * 20 + np.array([0, 0, 1.0]) * np.exp(rng.uniform(0, 9, m))[:, None]
    return {"x": rng.uniform(-3, 3, m), "y": rng.uniform(-2, 2, m), "z": rng.normal(size=m),
            "px": p[:, 0], "py": p[:, 1], "pz": p[:, 2], "s1": s[:, 0], "s2": s[:, 1], "s3": s[:, 2],
            "w": rng.uniform(0.5, 2.0, m), "id": np.arange(m, dtype=np.uint64)}


def _compare(g, o):
    scale = max(abs(o["total"][0]), 1.0)
    assert np.array_equal(g["bins"][..., 4], o["bins"][..., 4])
    assert g["total"][4] == o["total"][4]
    assert np.abs(g["bins"][..., :4] - o["bins"][..., :4]).max() <= 1e-12 * scale
    assert np.abs(g["total"][:4] - o["total"][:4]).max() <= 1e-12 * scale
    assert abs(g["below"] - o["below"]) <= 1e-12 * scale and abs(g["above"] - o["above"]) <= 1e-12 * scale


SPECS = [
    dict(kind=q.QED_DIAG_SPECTRUM, nx=64, ny=1, lo_x=1.0, hi_x=3e3),
    dict(kind=q.QED_DIAG_DETECTOR, nx=32, ny=16, lo_x=-2.5, hi_x=2.5, lo_y=-1.5, hi_y=1.5),
    dict(kind=q.QED_DIAG_DETECTOR, nx=8, ny=8, lo_x=-2.5, hi_x=2.5, lo_y=-1.5, hi_y=1.5, ref=(0.2, 1.0, 0.3)),
    dict(kind=q.QED_DIAG_SPECTRUM, nx=1024, ny=1, lo_x=0.5, hi_x=1e4),
]


@pytest.mark.parametrize("prec", [q.QED_PREC_F64, q.QED_PREC_MIXED])
@pytest.mark.parametrize("photon", [True, False])
def test_diag_matches_oracle_readout(ctx, prec, photon):
    m = 70_001
    d = _photons(m, 3) if photon else _leptons(m, 4)
    sp = q.Species(ctx, q.QED_PHOTON if photon else q.QED_ELECTRON, m + 5, prec).load(d)
    host = sp.to_dict()          # what the device holds (float-rounded on the mixed path)
    for s in SPECS:
        g = q.diag(sp, q.diag_spec(**s))
        o = OD.diag(host, s["kind"], s["nx"], s["ny"], s.get("lo_x"), s.get("hi_x"), s.get("lo_y", 0.0),
                    s.get("hi_y", 1.0), s.get("ref", (0.0, 0.0, 0.0)), photon=photon)
        _compare(g, o)
    sp.close()


def test_diag_after_a_run_and_edge_cases(ctx):
    wl = workloads.c1(n=3000, seed=17)
    sim = q.Simulation(wl, prec=q.QED_PREC_MIXED, ctx=ctx)
    sim.run(300, q.QED_F_NCS | q.QED_F_SPIN | q.QED_F_VB)
    st = sim.state()
    assert len(st["ph"]["id"]) > 1000
    for sp, host, photon in ((sim.ph, st["ph"], True), (sim.e, st["e"], False)):
        for s in SPECS[:2]:
            g = q.diag(sp, q.diag_spec(**s))
            o = OD.diag(host, s["kind"], s["nx"], s["ny"], s.get("lo_x"), s.get("hi_x"), s.get("lo_y", 0.0),
                        s.get("hi_y", 1.0), photon=photon)
            _compare(g, o)
    # the positron set is empty: zero yield
    g = q.diag(sim.pos, q.diag_spec(q.QED_DIAG_SPECTRUM, 4, 1, 1.0, 10.0))
    assert not g["bins"].any() and not g["total"].any()
    with pytest.raises(q.QedError):
        q.diag(sim.e, q.diag_spec(q.QED_DIAG_SPECTRUM, 1025, 1, 1.0, 10.0))
    with pytest.raises(q.QedError):
        q.diag(sim.e, q.diag_spec(q.QED_DIAG_SPECTRUM, 8, 1, 0.0, 10.0))
    with pytest.raises(q.QedError):
        q.diag(sim.e, q.diag_spec(q.QED_DIAG_SPECTRUM, 8, 2, 1.0, 10.0))
    sim.close()
