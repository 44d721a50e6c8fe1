"""Pins of the oracle's bremsstrahlung and Bethe-Heitler pair creation in matter (paper
Sec. III E): Tsai's cross-sections with his screening functions phi1,2 (gamma), psi1,2
(eps) for Z >= 5 and the Coulomb correction f(Z), the cumulative tables, and the direct
Monte Carlo sampling the paper describes (P = 1 - exp(-n sigma v dt), energy fraction from
r sigma(E) = sigma(y, E)).

* Complete screening (gamma = eps = 0): the radiation length that the screening
  functions and f(Z) imply, A / (4 alpha r0^2 N_A {Z^2 (phi1(0)/4 - ln Z / 3 - f) +
  Z (psi1(0)/4 - 2 ln Z / 3)}), reproduces the published radiation lengths of Al, Fe,
  Cu, W, Au and Pb (Particle Data Group tables, which use this form for Z >= 5) to 0.3 %.
* No screening (gamma, eps -> infinity): the brace must become the unscreened Bethe-Heitler
  amplitude, phi1 - 4/3 ln Z = psi1 - 8/3 ln Z = 4 ln(2 E E'/(m k)) - 2 (with gamma = 100 m k
  Z^-1/3/(E E')), and phi1 - phi2, psi1 - psi2 -> 0.
* Pair creation at high energy: sigma -> (7/9) A - (2/27)(Z^2 + Z) in units of alpha r0^2
  (the integral of 1 - 4/3 x(1-x) is 7/9; the second term of the brace, 1/42 of the first
  for complete screening, enters with the pair's sign).
* The tables against scipy quadrature of the braces, at nodes and between them.
* One Monte Carlo step of many leptons (photons) in the medium: the event fraction is
  1 - exp(-n sigma v dt) (binomial), the sampled y (x) follows the cross-section (KS against
  scipy's cumulative), and energy is conserved (E' + omega = E, E+ + E- = k).
"""
import math

import numpy as np
import pytest

import oracle

sp = pytest.importorskip("scipy.special")
si = pytest.importorskip("scipy.integrate")

ALPHA = 7.2973525693e-3
R0_CM = 2.8179403262e-13
NA = 6.02214076e23
R0N = 2.8179403262e-9 * 2 * math.pi       # r0 in units of 1 um / (2 pi)


def _x0(Z, A):
    s = oracle.screening(0.0, 0.0)
    f = oracle.coulomb_f(Z)
    lz = math.log(Z)
    brace = Z * Z * (s[0] / 4 - lz / 3 - f) + Z * (s[2] / 4 - 2 * lz / 3)
    return A / (4 * ALPHA * R0_CM ** 2 * NA * brace)


@pytest.mark.parametrize("Z,A,x0", [(13, 26.9815385, 24.01), (26, 55.845, 13.84), (29, 63.546, 12.86),
                                    (74, 183.84, 6.76), (79, 196.966570, 6.46), (82, 207.2, 6.37)])
def test_complete_screening_gives_published_radiation_lengths(Z, A, x0):
    assert abs(_x0(Z, A) / x0 - 1) < 3e-3


def test_complete_screening_differences_and_the_brace():
    s = oracle.screening(0.0, 0.0)
    assert abs(s[0] - s[1] - 2 / 3) < 1e-12 and abs(s[2] - s[3] - 2 / 3) < 1e-12
    # the brace at complete screening (very high energy): (4/3 - 4/3 y + y^2) A0 + (2/3)(1 - y)(2/3)(Z^2 + Z)
    Z = 29
    lz, f = math.log(Z), oracle.coulomb_f(Z)
    A0 = Z * Z * (s[0] - 4 / 3 * lz - 4 * f) + Z * (s[2] - 8 / 3 * lz)
    for y in (0.05, 0.3, 0.8):
        want = (4 / 3 - 4 / 3 * y + y * y) * A0 + (2 / 3) * (1 - y) * (2 / 3) * (Z * Z + Z)
        got = oracle.brems_D(Z, 1e13, y)
        assert abs(got / want - 1) < 1e-6, (y, got, want)
    for x in (0.1, 0.5, 0.9):
        want = (1 - 4 / 3 * x * (1 - x)) * A0 - (2 / 3) * x * (1 - x) * (2 / 3) * (Z * Z + Z)
        assert abs(oracle.pair_D(Z, 1e13, x) / want - 1) < 1e-6


@pytest.mark.parametrize("g", [300.0, 3e3, 3e4])
def test_no_screening_limit_is_bethe_heitler(g):
    # with gamma = 100 m k Z^-1/3 / (E E'): 4 ln(2 E E'/(m k)) - 2 - 4/3 ln Z = 4 ln(200/gamma) - 2
    s = oracle.screening(g, g)
    want = 4 * math.log(200 / g) - 2
    assert abs(s[0] - want) < 2e-3 and abs(s[2] - want) < 2e-3
    assert abs(s[0] - s[1]) < 1e-4 and abs(s[2] - s[3]) < 1e-4


def _med(Z=79, rho=19.32, A=196.966570, kmin=1.0):
    n = rho * NA / A * (1e-4 / (2 * math.pi)) ** 3     # atoms per (1 um / 2 pi)^3
    return dict(Z=Z, n=n, k_min=kmin, axis=2, lo=-1e300, hi=1e300)


def test_pair_cross_section_at_high_energy():
    orc = oracle.Oracle()
    for Z in (13, 79):
        orc.set_medium(_med(Z=Z))
        s = oracle.screening(0.0, 0.0)
        lz, f = math.log(Z), oracle.coulomb_f(Z)
        A0 = Z * Z * (s[0] - 4 / 3 * lz - 4 * f) + Z * (s[2] - 8 / 3 * lz)
        want = 7 / 9 * A0 - 2 / 27 * (Z * Z + Z)
        got = orc.medium_sigma(1, 2e6)
        assert abs(got / want - 1) < 2e-3, (Z, got, want)


def _brems_sigma_quad(Z, E, kmin):
    lo, hi = math.log(kmin / E), math.log(1 - 1 / E)
    return si.quad(lambda t: oracle.brems_D(Z, E, math.exp(t)), lo, hi, limit=400, epsrel=1e-11)[0]


def _pair_sigma_quad(Z, k):
    return si.quad(lambda x: oracle.pair_D(Z, k, x), 1 / k, 1 - 1 / k, limit=400, epsrel=1e-11)[0]


def test_tables_against_quadrature():
    orc = oracle.Oracle()
    orc.set_medium(_med(Z=29, rho=8.96, A=63.546, kmin=0.5))
    h = (math.log(2e6) - math.log(2)) / 255
    # at the nodes: the rows' 8-point Gauss-Legendre panels (uniform in the logit of the
    # energy fraction) against scipy's adaptive quadrature
    for i in (3, 60, 140, 250):
        E = math.exp(math.log(2) + i * h)
        assert abs(orc.medium_sigma(0, E) / _brems_sigma_quad(29, E, 0.5) - 1) < 1e-10
        if i >= 60:                     # (near threshold the high-energy brace is negative: sigma = 0)
            assert abs(orc.medium_sigma(1, E) / _pair_sigma_quad(29, E) - 1) < 1e-10
    assert orc.medium_sigma(1, 2.37) == 0.0 and _pair_sigma_quad(29, 2.37) == 0.0
    for E in (7.31, 311.7, 52003.0):    # between nodes: linear in ln E
        assert abs(orc.medium_sigma(0, E) / _brems_sigma_quad(29, E, 0.5) - 1) < 2e-3
        assert abs(orc.medium_sigma(1, E) / _pair_sigma_quad(29, E) - 1) < 2e-3


def _slab_run(orc, species, n, energy, target_p):
    """one step of n identical particles along +z inside the medium, dt for probability p"""
    which = 0 if species == "e" else 1
    sig = orc.medium_sigma(which, energy)
    m = orc._medium
    v = math.sqrt(1 - 1 / energy ** 2) if species == "e" else 1.0
    dt = -math.log(1 - target_p) / (m["n"] * ALPHA * R0N ** 2 * sig * v)
    pz = math.sqrt(energy ** 2 - 1) if species == "e" else energy
    one = {"x": np.zeros(n), "y": np.zeros(n), "z": np.zeros(n), "px": np.zeros(n), "py": np.zeros(n),
           "pz": np.full(n, pz), "s1": np.zeros(n), "s2": np.zeros(n), "s3": np.zeros(n), "w": np.ones(n),
           "id": np.arange(n, dtype=np.uint64)}
    empty = {k: v[:0] for k, v in one.items()}
    wl = {"e": empty, "pos": empty, "ph": dict(empty, theta=np.zeros(0)), "field": {"kind": "none"}, "dt": dt,
          "seed": 31, "next_id": n, "medium": m}
    if species == "e":
        wl["e"] = one
    else:
        wl["ph"] = dict(one, theta=np.zeros(n))
    sim = oracle.Sim(orc, wl, cap_e=2 * n, cap_p=2 * n, cap_ph=2 * n)
    stats = sim.run(1, oracle.F_BREMS if species == "e" else oracle.F_BH)
    return sim.state(), stats, 1 - math.exp(-m["n"] * ALPHA * R0N ** 2 * sig * v * dt)


def _ks(samples, cdf):
    xs = np.sort(samples)
    emp = np.arange(1, len(xs) + 1) / len(xs)
    return np.abs(emp - cdf(xs)).max()


def test_bremsstrahlung_step_statistics():
    orc = oracle.Oracle()
    med = _med()
    orc.set_medium(med)
    orc._medium = med
    E, N = 2000.0, 100_000
    st, stats, P = _slab_run(orc, "e", N, E, 0.5)
    k = stats["n_brems_e"]
    assert abs(k - P * N) < 5 * math.sqrt(N * P * (1 - P))
    ph, el = st["ph"], st["e"]
    assert len(ph["id"]) == k
    om = np.linalg.norm(np.stack([ph["px"], ph["py"], ph["pz"]], 1), axis=1)
    assert np.all(ph["px"] == 0) and np.all(ph["s1"] == 0) and np.all(ph["s3"] == 0)
    # energy conservation: the k-th photon (id N + k) comes from the k-th emitting electron
    oe, op = np.argsort(el["id"]), np.argsort(ph["id"])
    ge = np.sqrt(1 + el["px"][oe] ** 2 + el["py"][oe] ** 2 + el["pz"][oe] ** 2)
    emit = ge < E * (1 - 1e-13)
    assert emit.sum() == k
    assert np.allclose(ge[emit] + om[op], E, rtol=1e-12)
    # the photon energy fraction against the cross-section
    y = om / E
    lo, hi = math.log(1.0 / E), math.log(1 - 1 / E)
    ts = np.linspace(lo, hi, 2001)
    dens = np.array([oracle.brems_D(79, E, math.exp(t)) for t in ts])
    cum = np.concatenate([[0], np.cumsum(0.5 * (dens[1:] + dens[:-1]) * np.diff(ts))])
    cum /= cum[-1]
    d = _ks(np.log(y), lambda v: np.interp(v, ts, cum))
    assert d < 1.8 / math.sqrt(len(y)) + 2e-3


def test_bethe_heitler_step_statistics():
    orc = oracle.Oracle()
    med = _med(Z=13, rho=2.699, A=26.9815385)
    orc.set_medium(med)
    orc._medium = med
    k, N = 4000.0, 100_000
    st, stats, P = _slab_run(orc, "ph", N, k, 0.4)
    kk = stats["n_bh"]
    assert abs(kk - P * N) < 5 * math.sqrt(N * P * (1 - P))
    e, p = st["e"], st["pos"]
    assert len(e["id"]) == kk and len(p["id"]) == kk and len(st["ph"]["id"]) == N - kk
    ep = np.sqrt(1 + p["px"] ** 2 + p["py"] ** 2 + p["pz"] ** 2)
    em = np.sqrt(1 + e["px"] ** 2 + e["py"] ** 2 + e["pz"] ** 2)
    assert np.allclose(ep + em, k, rtol=1e-12)
    assert np.all(p["s1"] == 0) and np.all(e["s3"] == 0)
    x = ep / k
    xs = np.linspace(1 / k, 1 - 1 / k, 4001)
    dens = np.array([oracle.pair_D(13, k, v) for v in xs])
    cum = np.concatenate([[0], np.cumsum(0.5 * (dens[1:] + dens[:-1]) * np.diff(xs))])
    cum /= cum[-1]
    d = _ks(x, lambda v: np.interp(v, xs, cum))
    assert d < 1.8 / math.sqrt(len(x)) + 2e-3
    # the spectrum is symmetric in x <-> 1 - x
    assert abs(np.mean(x) - 0.5) < 5 * np.std(x) / math.sqrt(len(x))


def test_medium_slab_bounds():
    """Particles outside the slab (x^n outside [lo, hi) along the axis) are not affected."""
    orc = oracle.Oracle()
    med = dict(_med(), axis=2, lo=0.0, hi=1.0)
    orc.set_medium(med)
    orc._medium = med
    n = 2000
    E = 2000.0
    one = {"x": np.zeros(n), "y": np.zeros(n), "z": np.where(np.arange(n) % 2 == 0, 0.5, 1.5),
           "px": np.zeros(n), "py": np.zeros(n), "pz": np.full(n, math.sqrt(E * E - 1)), "s1": np.zeros(n),
           "s2": np.zeros(n), "s3": np.zeros(n), "w": np.ones(n), "id": np.arange(n, dtype=np.uint64)}
    empty = {k: v[:0] for k, v in one.items()}
    sig = orc.medium_sigma(0, E)
    dt = math.log(2) / (med["n"] * ALPHA * R0N ** 2 * sig)
    sim = oracle.Sim(orc, {"e": one, "pos": empty, "ph": dict(empty, theta=np.zeros(0)), "field": {"kind": "none"},
                           "dt": dt, "seed": 3, "next_id": n, "medium": med}, cap_ph=n)
    sim.run(1, oracle.F_BREMS)
    el = sim.state()["e"]
    o = np.argsort(el["id"])
    pz = el["pz"][o]
    assert np.all(pz[1::2] == math.sqrt(E * E - 1))   # outside: untouched
    assert np.any(pz[0::2] < math.sqrt(E * E - 1))    # inside: some emitted
