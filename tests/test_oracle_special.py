"""Pins of the oracle's building blocks against things fixed outside it:
published Philox known-answer vectors, library special functions (scipy, mpmath),
DLMF closed forms, and the constants the paper prints."""
import math
import os

import numpy as np
import pytest
from scipy import integrate, special

import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    rows = []
    for line in open(os.path.join(GOLD, name)):
        line = line.split("#")[0].strip()
        if line:
            rows.append(line.split())
    return rows


def test_philox_known_answers():
    rows = _golden("philox4x32_10_kat.txt")
    assert len(rows) == 3
    for r in rows:
        v = [int(h, 16) for h in r]
        assert oracle.philox(v[0:4], v[4:6]) == v[6:10]


def test_uniform_construction():
    # two 53-bit uniforms from one block: ((a>>5) 2^26 + (b>>6)) 2^-53
    seed, pid, step, ctr = 0x123456789ABCDEF, 987654321012, 77, 2
    w = oracle.philox([pid & 0xFFFFFFFF, pid >> 32, step, ctr], [seed & 0xFFFFFFFF, seed >> 32])
    exp0 = ((w[0] >> 5) * 2**26 + (w[1] >> 6)) / 2**53
    exp1 = ((w[2] >> 5) * 2**26 + (w[3] >> 6)) / 2**53
    u = oracle.uniforms(seed, pid, step, ctr)
    assert u[0] == exp0 and u[1] == exp1
    # statistical sanity: mean and variance of many uniforms
    us = np.array([oracle.uniforms(1, i, 0, 0) for i in range(20000)]).ravel()
    assert 0.0 <= us.min() and us.max() < 1.0
    assert abs(us.mean() - 0.5) < 5 * math.sqrt(1 / 12 / us.size)
    assert abs(us.var() - 1 / 12) < 0.003


@pytest.mark.parametrize("x", np.logspace(-10, 3, 27))
def test_besselk_vs_scipy(x):
    k = oracle.besselk_scaled(x)
    assert k[0] == pytest.approx(special.kve(1 / 3, x), rel=2e-13)
    assert k[1] == pytest.approx(special.kve(2 / 3, x), rel=2e-13)


@pytest.mark.parametrize("x", [1e-6, 1e-3, 0.05, 0.7, 3.0, 20.0, 150.0])
def test_intk_vs_quadrature(x):
    ik = oracle.besselk_scaled(x)[2] * math.exp(-x)
    ref, err = integrate.quad(lambda t: special.kv(1 / 3, t), x, np.inf, epsabs=0, epsrel=1e-13, limit=400)
    assert ik == pytest.approx(ref, rel=1e-10)


def test_bessel_closed_forms():
    # int_0^inf K_{1/3} = pi/sqrt(3)  (IntK13(0+))
    assert oracle.besselk_scaled(1e-14)[2] == pytest.approx(math.pi / math.sqrt(3), rel=1e-9)
    # small-x leading term Gamma(nu)/2 (2/x)^nu
    x = 1e-9
    k = oracle.besselk_scaled(x)
    assert k[1] == pytest.approx(0.5 * math.gamma(2 / 3) * (2 / x) ** (2 / 3), rel=1e-5)
    # large-x sqrt(pi/2x)(1 + (4nu^2-1)/(8x))
    x = 400.0
    for j, nu in ((0, 1 / 3), (1, 2 / 3)):
        asym = math.sqrt(math.pi / (2 * x)) * (1 + (4 * nu * nu - 1) / (8 * x) +
                                              (4 * nu * nu - 1) * (4 * nu * nu - 9) / (2 * (8 * x) ** 2))
        assert oracle.besselk_scaled(x)[j] == pytest.approx(asym, rel=1e-7)
    # recurrence K_{nu+1} - K_{nu-1} = (2 nu / x) K_nu with nu = 1/3: K_{4/3} - K_{2/3} = (2/(3x)) K_{1/3}
    for x in (0.01, 0.5, 4.0):
        k = oracle.besselk_scaled(x)
        assert special.kve(4 / 3, x) - k[1] == pytest.approx(2 / (3 * x) * k[0], rel=1e-11)


def test_ktable_offgrid(orc):
    rng = np.random.default_rng(3)
    xs = np.exp(rng.uniform(np.log(1e-6), np.log(3e4), 400))
    for x in xs:
        t = orc.ktable(x)
        ref = np.array([special.kve(1 / 3, x), special.kve(2 / 3, x), 0.0])
        ref[2] = oracle.besselk_scaled(x)[2]
        assert np.allclose(t, ref, rtol=3e-9, atol=0), (x, t, ref)


def test_scorer_gi_prime_vs_mpmath():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 30
    for y in (0.05, 0.3, 1.0, 2.5, 7.0, 20.0, 80.0):
        ref = float(mp.diff(mp.scorergi, y))
        assert oracle.scorer_gi_prime(y) == pytest.approx(ref, rel=1e-11, abs=1e-15)
    # large-argument limit pi y^2 Gi'(y) -> -1
    y = 3000.0
    assert math.pi * y * y * oracle.scorer_gi_prime(y) == pytest.approx(-1.0, rel=1e-6)


def test_vb_low_field_constants(orc):
    rows = {r[0]: (float(r[1]), float(r[2])) for r in _golden("paper_values.txt")}
    m = orc.vb_m(1.0001e-3)
    assert m[0] == pytest.approx(rows["vb_M_parallel_low"][0], rel=2e-6)
    assert m[1] == pytest.approx(rows["vb_M_perp_low"][0], rel=2e-6)
    # below the table the constants are used exactly
    assert list(orc.vb_m(1e-5)) == [4.0, 7.0]


def test_vb_table_vs_direct_mpmath(orc):
    """M at one chi_gamma by an independent mpmath quadrature of Eq. eqnn's real part."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 20
    chig = 2.0

    def integrand(v, par):
        x = 4 / ((1 - v * v) * chig)
        y = x ** (mp.mpf(2) / 3)
        g = mp.pi * x ** (mp.mpf(4) / 3) * mp.diff(mp.scorergi, y)
        w = (1 + v * v / 3) / 2 if par else (1 - v * v / 3)
        return (1 - v * v) * w * g

    mpar = float(-mp.mpf(45) / 4 * mp.quad(lambda v: integrand(v, True), [0, 0.5, 0.9, 1]))
    mperp = float(-mp.mpf(45) / 4 * mp.quad(lambda v: integrand(v, False), [0, 0.5, 0.9, 1]))
    m = orc.vb_m(chig)
    assert m[0] == pytest.approx(mpar, rel=1e-7)
    assert m[1] == pytest.approx(mperp, rel=1e-7)


def test_paper_printed_constants():
    rows = {r[0]: (float(r[1]), float(r[2])) for r in _golden("paper_values.txt")}
    xil = 2.42631023867e-6
    v, tol = rows["a_sch"]
    assert 1 / xil == pytest.approx(v, rel=tol)
    v, tol = rows["sokolov_ternov_degree"]
    assert 8 / (5 * math.sqrt(3)) == pytest.approx(v, abs=tol)
    # R = (2/3) alpha gamma chi with chi ~ 2 gamma a0 xi_L (head-on) -> coefficient of a0 gamma^2
    alpha = 7.2973525693e-3
    v, tol = rows["rr_ratio_coeff"]
    assert (2 / 3) * alpha * 2 * xil == pytest.approx(v, rel=tol)


def test_vb_large_chi_vs_direct_mpmath(orc):
    """At large chi_gamma the upsilon integrand has a boundary layer next to 1; an
    independent mpmath quadrature with graded break points pins the table there."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 20
    chig = 300.0

    def integrand(v, par):
        om = 1 - v * v
        if om <= 0:
            return mp.mpf(0)
        x = 4 / (om * chig)
        y = x ** (mp.mpf(2) / 3)
        g = mp.pi * x ** (mp.mpf(4) / 3) * mp.diff(mp.scorergi, y)
        w = (1 + v * v / 3) / 2 if par else (1 - v * v / 3)
        return om * w * g

    pts = [mp.mpf(0), mp.mpf("0.5"), mp.mpf("0.9"), mp.mpf("0.99"), mp.mpf("0.999"), mp.mpf("0.9999"),
           mp.mpf("0.99999"), mp.mpf(1)]
    mpar = float(-mp.mpf(45) / 4 * mp.quad(lambda v: integrand(v, True), pts))
    mperp = float(-mp.mpf(45) / 4 * mp.quad(lambda v: integrand(v, False), pts))
    m = orc.vb_m(chig)
    assert m[0] == pytest.approx(mpar, rel=1e-6)
    assert m[1] == pytest.approx(mperp, rel=1e-6)
