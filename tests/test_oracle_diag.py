"""Pins of the end-of-run observables oracle (oracle/diag.py) against what the paper and
geometry fix, independently of its own rotation formula:

* Stokes parameters of a linearly polarised photon are (sin 2a, 0, cos 2a) with a the angle
  of its polarisation vector from the first basis vector (the definition of xi in Sec. III D);
  computing a geometrically in the detection plane must agree with the rotated Stokes vector,
  for photons in arbitrary directions and with arbitrary stored bases.
* Circular polarisation (xi2) and the degree of linear polarisation do not depend on the basis.
* Hand-counted spectra and detector maps, including under/overflow and empty sets."""
import math

import numpy as np

from oracle import diag as D


def _basis_vectors(n, theta):
    e1, e2 = D.canonical_frame(n)
    p1 = np.cos(theta)[:, None] * e1 + np.sin(theta)[:, None] * e2
    p2 = np.cross(n, p1)
    return p1, p2


def test_linear_polarisation_angle_matches_geometry():
    rng = np.random.default_rng(1)
    m = 500
    k = rng.normal(size=(m, 3))
    k[: m // 2, 2] += 20.0           # half of them beam-like, the rest in every direction
    om = rng.uniform(1, 1e3, m)
    k = k / np.linalg.norm(k, axis=1)[:, None] * om[:, None]
    n = k / om[:, None]
    theta = rng.uniform(-math.pi, math.pi, m)
    alpha = rng.uniform(-math.pi, math.pi, m)     # polarisation angle in the stored basis
    xi = np.stack([np.sin(2 * alpha), np.zeros(m), np.cos(2 * alpha)], 1)
    for ref in ((1.0, 0.0, 0.0), (0.3, -0.8, 0.1)):
        out = D.detector_stokes(k, theta, xi, ref)
        # the polarisation vector and its angle from d1 in the detection plane
        p1, p2 = _basis_vectors(n, theta)
        eps = np.cos(alpha)[:, None] * p1 + np.sin(alpha)[:, None] * p2
        r = np.asarray(ref)
        d1 = r[None, :] - (n @ r)[:, None] * n
        d1 /= np.linalg.norm(d1, axis=1)[:, None]
        d2 = np.cross(n, d1)
        a_det = np.arctan2(np.einsum("ij,ij->i", eps, d2), np.einsum("ij,ij->i", eps, d1))
        want = np.stack([np.sin(2 * a_det), np.zeros(m), np.cos(2 * a_det)], 1)
        assert np.abs(out - want).max() < 1e-12


def test_photon_along_z_closed_form():
    # n = z: the canonical e1 is x, so a photon polarised along its basis vector at angle t0
    # from x reads (sin 2 t0, 0, cos 2 t0) in the (x, y) detector
    t0 = np.array([0.0, 0.3, -1.1, math.pi / 4])
    k = np.tile([0.0, 0.0, 5.0], (4, 1))
    xi = np.tile([0.0, 0.0, 1.0], (4, 1))
    out = D.detector_stokes(k, t0, xi)
    assert np.allclose(out, np.stack([np.sin(2 * t0), np.zeros(4), np.cos(2 * t0)], 1), atol=1e-15)


def test_circular_part_and_linear_degree_invariant():
    rng = np.random.default_rng(2)
    m = 300
    k = rng.normal(size=(m, 3)) * 3
    xi = rng.normal(size=(m, 3))
    xi *= rng.uniform(0, 1, (m, 1)) / np.linalg.norm(xi, axis=1)[:, None]
    out = D.detector_stokes(k, rng.uniform(-3, 3, m), xi, (0.0, 1.0, 0.0))
    assert np.array_equal(out[:, 1], xi[:, 1])
    assert np.allclose(np.hypot(out[:, 0], out[:, 2]), np.hypot(xi[:, 0], xi[:, 2]), atol=1e-14)


def _set(px, py, pz, w, s=None, x=None, y=None, theta=None):
    n = len(px)
    s = np.zeros((n, 3)) if s is None else np.asarray(s, dtype=float)
    d = {"px": np.asarray(px, float), "py": np.asarray(py, float), "pz": np.asarray(pz, float),
         "s1": s[:, 0], "s2": s[:, 1], "s3": s[:, 2], "w": np.asarray(w, float),
         "x": np.zeros(n) if x is None else np.asarray(x, float), "y": np.zeros(n) if y is None else np.asarray(y, float),
         "z": np.zeros(n), "id": np.arange(n, dtype=np.uint64)}
    d["theta"] = np.zeros(n) if theta is None else np.asarray(theta, float)
    return d


def test_photon_spectrum_hand_counted():
    # bins uniform in ln(omega) over [1, 100): edges 1, 10, 100
    d = _set([0, 0, 0, 0, 0], [0, 0, 0, 0, 0], [0.5, 2.0, 9.99, 10.5, 500.0], [1, 2, 3, 4, 5],
             s=[[0, 0, 1]] * 5)
    r = D.diag(d, D.SPECTRUM, 2, 1, 1.0, 100.0, photon=True)
    b = r["bins"][0]
    assert b[0, 0] == 5.0 and b[0, 4] == 2 and b[1, 0] == 4.0 and b[1, 4] == 1
    # along z with theta = 0 the stored basis is the (x, y) detector basis: xi3 unchanged
    assert b[0, 3] == 5.0 and b[1, 3] == 4.0
    assert r["below"] == 1.0 and r["above"] == 5.0
    assert np.array_equal(r["total"], [15.0, 0.0, 0.0, 15.0, 5.0])


def test_lepton_spectrum_mean_spin():
    # gamma = sqrt(1 + p^2): p = 0 -> 1 (first bin of [1, 4)), p = sqrt(8) -> 3
    d = _set([0, 0, 0], [0, 0, 0], [0.0, math.sqrt(8.0), 100.0], [1.0, 3.0, 1.0],
             s=[[0, 1, 0], [0, -1, 0], [1, 0, 0]])
    r = D.diag(d, D.SPECTRUM, 2, 1, 1.0, 4.0)
    b = r["bins"][0]
    assert b[0, 0] == 1.0 and b[0, 2] == 1.0         # gamma 1 in [1, 2)
    assert b[1, 0] == 3.0 and b[1, 2] == -3.0        # gamma 3 in [2, 4)
    assert r["above"] == 1.0 and r["below"] == 0.0


def test_detector_map_and_empty_set():
    d = _set([0, 0, 0], [0, 0, 0], [5, 5, 5], [1, 1, 1], s=[[1, 0, 0]] * 3, x=[0.1, 1.5, 9.0], y=[0.1, 0.6, 0.1])
    r = D.diag(d, D.DETECTOR, 2, 2, 0.0, 2.0, 0.0, 1.0, photon=True)
    assert r["bins"][0, 0, 4] == 1 and r["bins"][1, 1, 4] == 1 and r["above"] == 1.0
    e = _set([], [], [], [])
    r = D.diag(e, D.SPECTRUM, 4, 1, 1.0, 10.0, photon=True)
    assert not r["bins"].any() and not r["total"].any()
