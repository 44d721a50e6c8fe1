"""Pins of the oracle's rate tables, samplers and rate algebra (Secs. III C, III D):
independent scipy quadratures, the reductions the paper states between its
equations, positivity, the classical-power limit and the Laplace asymptote."""
import math

import numpy as np
import pytest
from scipy import integrate, special

ALPHA = 7.2973525693e-3
XIL = 2.42631023867e-6


def _intk13(x):
    return integrate.quad(lambda t: special.kv(1 / 3, t), x, np.inf, epsabs=0, epsrel=1e-12, limit=400)[0]


def _ncs_AB(chi):
    """A, B of the u-integrated Eq. Wspin2 by scipy, with the IntK term integrated
    by parts: int IntK(u')/(1+u)^2 du = pi/sqrt3 - (2/3chi) int K13(u')/(1+u) du."""
    c = 2 / (3 * chi)
    kw = dict(epsabs=0, epsrel=1e-12, limit=500)
    brk = [0, 1.5 * chi, 15 * chi, 150 * chi]
    def q(f):
        s = 0.0
        for a, b in zip(brk[:-1], brk[1:]):
            s += integrate.quad(f, a, b, **kw)[0]
        return s + integrate.quad(f, brk[-1], np.inf, **kw)[0]
    k23 = q(lambda u: (2 + 2 * u + u * u) * special.kv(2 / 3, c * u) / (1 + u) ** 3)
    k13 = q(lambda u: special.kv(1 / 3, c * u) / (1 + u))
    A = k23 - (math.pi / math.sqrt(3) - c * k13)
    B = q(lambda u: u * special.kv(1 / 3, c * u) / (1 + u) ** 3)
    return A, B


@pytest.mark.parametrize("chi", [1.3e-4, 3.7e-3, 0.071, 0.93, 11.0, 420.0])
def test_ncs_rate_table_vs_scipy(orc, chi):
    A, B = _ncs_AB(chi)
    t = orc.ncs_rates(chi)
    assert t[0] == pytest.approx(A, rel=1e-8)
    assert t[1] == pytest.approx(B, rel=1e-8)


def test_ncs_rate_small_chi_closed_form(orc):
    # chi -> 0: A -> (3chi/2)(2 int K23 - int IntK13) = (3chi/2)(2pi - pi/3) = 5 pi chi/2,
    # B -> (3chi/2)^2 int x K13 = (9 chi^2/4)(pi/3)
    chi = 1.0e-4
    A, B = orc.ncs_rates(chi)
    assert A == pytest.approx(2.5 * math.pi * chi, rel=2e-3)
    assert B == pytest.approx(0.75 * math.pi * chi * chi, rel=2e-3)


def _ncs_cdf(chi, comp, U):
    """CDF in u of component comp (0: a-b, 1: a+b) by scipy."""
    c = 2 / (3 * chi)
    sg = -1.0 if comp == 0 else 1.0
    kw = dict(epsabs=0, epsrel=1e-12, limit=500)
    def part(U):
        brk = [x for x in [0, 1.5 * chi, 15 * chi, 150 * chi] if x < U] + [U]
        s23 = s13a = s13b = 0.0
        for a, b in zip(brk[:-1], brk[1:]):
            s23 += integrate.quad(lambda u: (2 + 2 * u + u * u) * special.kv(2 / 3, c * u) / (1 + u) ** 3, a, b, **kw)[0]
            s13a += integrate.quad(lambda u: special.kv(1 / 3, c * u) / (1 + u), a, b, **kw)[0]
            s13b += integrate.quad(lambda u: u * special.kv(1 / 3, c * u) / (1 + u) ** 3, a, b, **kw)[0]
        ik = math.pi / math.sqrt(3) - _intk13(c * U) / (1 + U) - c * s13a
        return s23 - ik + sg * s13b
    A, B = _ncs_AB(chi)
    return part(U) / (A + sg * B)


@pytest.mark.parametrize("chi,comp,t", [(0.05, 0, -3.0), (0.05, 1, 0.0), (0.8, 0, 2.5),
                                         (0.8, 1, -12.0), (7.0, 0, 1.0), (7.0, 1, -0.5)])
def test_ncs_inverse_cdf(orc, chi, comp, t):
    u = math.exp(orc.ncs_invcdf(comp, chi, t))
    lev = 1 / (1 + math.exp(-t))
    F = _ncs_cdf(chi, comp, u)
    if t <= 0:
        assert F == pytest.approx(lev, rel=2e-6)
    else:
        assert 1 - F == pytest.approx(1 - lev, rel=2e-5)


def test_ncs_inverse_cdf_tails(orc):
    # deep lower tail: CDF ~ u^{1/3}: ln u is 3 t + const
    chi = 0.3
    y1, y2 = orc.ncs_invcdf(1, chi, -36.0), orc.ncs_invcdf(1, chi, -30.0)
    assert (y2 - y1) / 6.0 == pytest.approx(3.0, rel=1e-6)
    # monotone in level
    ts = np.linspace(-38, 38, 2001)
    ys = np.array([orc.ncs_invcdf(0, chi, t) for t in ts])
    assert np.all(np.diff(ys) > 0)


def _t0t3(chig):
    kw = dict(epsabs=0, epsrel=1e-11, limit=400)
    def rho(d):
        return 2 / (3 * chig * d * (1 - d))
    # symmetric: 2 x integral over (0, 1/2]; scaled by exp(8/(3chig))
    r0 = 8 / (3 * chig)
    f3 = lambda d: special.kve(2 / 3, rho(d)) * math.exp(-(rho(d) - r0))
    f0 = lambda d: (_intk13(rho(d)) * math.exp(r0) + (d / (1 - d) + (1 - d) / d) *
                    special.kve(2 / 3, rho(d)) * math.exp(-(rho(d) - r0)))
    T3 = 2 * integrate.quad(f3, 0, 0.5, **kw)[0]
    T0 = 2 * integrate.quad(f0, 0, 0.5, **kw)[0]
    return T0 * math.exp(-r0), T3 * math.exp(-r0)


@pytest.mark.parametrize("chig", [0.03, 0.4, 2.2, 35.0])
def test_nbw_rate_table_vs_scipy(orc, chig):
    T0, T3 = _t0t3(chig)
    t = orc.nbw_rates(chig)
    assert t[0] == pytest.approx(T0, rel=1e-7)
    assert t[1] == pytest.approx(T3, rel=1e-7)


def test_nbw_laplace_asymptote(orc):
    # small chi_gamma: unpolarised rate alpha/(xi_L omega) (9/(16 sqrt6)) chi e^{-8/(3chi)}
    for chig, tol in ((0.012, 0.004), (0.02, 0.006)):
        T0 = orc.nbw_rates(chig)[0]
        rate = T0 / (math.sqrt(3) * math.pi)
        asym = 9 / (16 * math.sqrt(6)) * chig * math.exp(-8 / (3 * chig))
        assert rate / asym == pytest.approx(1.0, abs=tol)


@pytest.mark.parametrize("chig,comp,t", [(0.05, 0, -5.0), (0.05, 1, -0.2), (3.0, 0, -20.0), (3.0, 1, -1.0)])
def test_nbw_inverse_cdf(orc, chig, comp, t):
    d = math.exp(orc.nbw_invcdf(comp, chig, t))
    lam = math.exp(t)
    sg = -1.0 if comp == 0 else 1.0
    r0 = 8 / (3 * chig)
    def dens(x):
        rho = 2 / (3 * chig * x * (1 - x))
        k23 = special.kve(2 / 3, rho) * math.exp(-(rho - r0))
        ik = _intk13(rho) * math.exp(r0)
        return ik + (x / (1 - x) + (1 - x) / x) * k23 + sg * k23
    kw = dict(epsabs=0, epsrel=1e-11, limit=400)
    num = integrate.quad(dens, 0, d, **kw)[0]
    den = integrate.quad(dens, 0, 0.5, **kw)[0]
    assert num / den == pytest.approx(lam, rel=2e-5)


def _rand_unit(rng, k=1):
    v = rng.normal(size=(k, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def test_ncs_F_reductions_and_positivity(orc):
    """Eq. NCSW summed over photon states -> Eq. Wspin (= F0); summed over S_f ->
    Eq. Wspin2 (8 W_R {...}); averaged over S_i -> the unpolarised rate; F0 >= |F|."""
    rng = np.random.default_rng(11)
    n = np.array([0.0, 0.0, 1.0])
    a = np.array([1.0, 0.0, 0.0])
    z = np.cross(n, a)
    worst = 1e9
    for _ in range(400):
        u = math.exp(rng.uniform(-6, 3))
        chi = math.exp(rng.uniform(-5, 4))
        Si, Sf, ax = _rand_unit(rng, 3)
        k13, k23, ik = orc.ktable(2 * u / (3 * chi))
        Fp = orc.ncs_F(u, chi, n, a, Si, ax)
        Fm = orc.ncs_F(u, chi, n, a, Si, -ax)
        w2 = 8 * (-(1 + u) * ik + (2 + 2 * u + u * u) * k23 - u * np.dot(Si, z) * k13)
        assert Fp[0] + Fm[0] == pytest.approx(w2, rel=1e-11, abs=1e-12 * abs(k23))
        Fq = orc.ncs_F(u, chi, n, a, -Si, ax)
        Fr = orc.ncs_F(u, chi, n, a, -Si, -ax)
        unpol = 0.5 * (Fp[0] + Fm[0] + Fq[0] + Fr[0])
        assert unpol == pytest.approx(8 * (-(1 + u) * ik + (2 + 2 * u + u * u) * k23), rel=1e-11)
        F = orc.ncs_F(u, chi, n, a, Si, Sf)
        margin = (F[0] - np.linalg.norm(F[1:])) / F[0]
        worst = min(worst, margin)
    assert worst > -1e-12


def test_ncs_unpolarised_photon_is_linear_along_a(orc):
    """Unpolarised electron, summed final spin: xi3 = (1+u)K23/[(2+2u+u^2)K23 - (1+u)IntK] > 0."""
    n, a = np.array([0, 0, 1.0]), np.array([1.0, 0, 0])
    for u in (1e-3, 0.1, 2.0):
        chi = 1.0
        k13, k23, ik = orc.ktable(2 * u / (3 * chi))
        F = np.zeros(4)
        for Si in (np.eye(3)[1], -np.eye(3)[1]):
            for Sf in (np.eye(3)[1], -np.eye(3)[1]):
                F += orc.ncs_F(u, chi, n, a, Si, Sf)
        xi3 = F[3] / F[0]
        assert xi3 == pytest.approx((1 + u) * k23 / ((2 + 2 * u + u * u) * k23 - (1 + u) * ik), rel=1e-10)
        assert xi3 > 0 and abs(F[1]) < 1e-12 * F[0] and abs(F[2]) < 1e-12 * F[0]


def test_nbw_G_reductions_and_positivity(orc):
    """Eq. BW summed over S- -> Eq. BWposAxis (C + S+.D); over S+ -> Eq. BWeleAxis
    (C + S-.D'); both -> Eq. BWprob's bracket; G0 >= |(G1,G2,G3)| for unit states."""
    rng = np.random.default_rng(5)
    ap, bp, vp = np.eye(3)
    worst = 1e9
    for _ in range(400):
        delta = rng.uniform(0.02, 0.98)
        om = math.exp(rng.uniform(1, 9))
        chig = math.exp(rng.uniform(-3, 4))
        Sp, Sm, ax = _rand_unit(rng, 3)
        xi = _rand_unit(rng)[0] * rng.uniform(0, 1)
        ep, em = delta * om, (1 - delta) * om
        rho = 2 / (3 * chig * delta * (1 - delta))
        k13, k23, ik = orc.ktable(rho)
        sum2 = (em * em + ep * ep) / (em * ep)
        dif2 = (ep * ep - em * em) / (em * ep)
        Cc = ik + sum2 * k23 - xi[2] * k23
        D = (-(om / ep - xi[2] * om / em) * k13 * bp - xi[0] * (om / em) * k13 * ap +
             xi[1] * (dif2 * k23 + (om / ep) * ik) * vp)
        Dp = ((om / em - xi[2] * om / ep) * k13 * bp + xi[0] * (om / ep) * k13 * ap -
              xi[1] * (dif2 * k23 - (om / em) * ik) * vp)
        def rate(a1, a2):
            G = orc.nbw_G(delta, om, chig, ap, bp, vp, a1, a2)
            return G[0] + np.dot(xi, G[1:])
        s_minus = rate(Sp, ax) + rate(Sp, -ax)
        assert s_minus == pytest.approx(2 * (Cc + np.dot(Sp, D)), rel=1e-10, abs=1e-12 * Cc)
        s_plus = rate(ax, Sm) + rate(-ax, Sm)
        assert s_plus == pytest.approx(2 * (Cc + np.dot(Sm, Dp)), rel=1e-10, abs=1e-12 * Cc)
        both = s_minus + rate(-Sp, ax) + rate(-Sp, -ax)
        assert both == pytest.approx(4 * Cc, rel=1e-10)
        xi_pure = xi / np.linalg.norm(xi)
        G = orc.nbw_G(delta, om, chig, ap, bp, vp, Sp, Sm)
        worst = min(worst, (G[0] - np.linalg.norm(G[1:])) / abs(G[0]))
        assert G[0] + np.dot(xi_pure, G[1:]) >= -1e-12 * abs(G[0])
    assert worst > -1e-9


def _mean_fraction(orc, chi, s):
    """E[r] of the sampler at spin projection s, by quadrature over the level t."""
    A, B = orc.ncs_rates(chi)
    ts = np.linspace(-38, 38, 6001)
    lev = 1 / (1 + np.exp(-ts))
    dl = lev * (1 - lev)
    er = []
    for comp in (0, 1):
        u = np.exp([orc.ncs_invcdf(comp, chi, t) for t in ts])
        er.append(np.trapezoid(u / (1 + u) * dl, ts))
    w0 = 0.5 * (1 + s) * (A - B)
    w1 = 0.5 * (1 - s) * (A + B)
    return (w0 * er[0] + w1 * er[1]) / (w0 + w1), A, B


@pytest.mark.parametrize("chi", [1e-4, 1e-3])
def test_ncs_power_classical_limit(orc, chi):
    """Radiated power W gamma E[r] -> (2/3) alpha chi^2 / xi_L (Sec. III A) with the known
    quantum correction 1 - (55 sqrt3/16) chi + 48 chi^2 (independent of gamma: the 1/gamma
    in W_R is required)."""
    gamma = 3000.0
    er, A, B = _mean_fraction(orc, chi, 0.0)
    P = ALPHA / (math.sqrt(3) * math.pi * XIL * gamma) * A * gamma * er
    Pcl = 2 / 3 * ALPHA * chi * chi / XIL
    assert P / Pcl == pytest.approx(1 - 55 * math.sqrt(3) / 16 * chi + 48 * chi * chi, abs=3e-5)


@pytest.mark.parametrize("chi", [0.01, 0.1, 1.0])
def test_ncs_power_vs_paper_q_fits(orc, chi):
    """q(chi) = I_QED/I_C against the two fits printed in Sec. III A (each is a fit, so
    a few per cent)."""
    er, A, B = _mean_fraction(orc, chi, 0.0)
    q = ALPHA / (math.sqrt(3) * math.pi * XIL) * A * er / (2 / 3 * ALPHA * chi * chi / XIL)
    fit1 = (1 + 4.8 * (1 + chi) * math.log(1 + 1.7 * chi) + 2.44 * chi * chi) ** (-2 / 3)
    fit2 = (1 + 8.93 * chi + 2.41 * chi * chi) ** (-2 / 3)
    assert q == pytest.approx(fit1, rel=0.03)
    assert q == pytest.approx(fit2, rel=0.04)


def _ncs_ccdf(chi, comp, U):
    """Mass above u of component comp, integrated from u upwards (no 1 - CDF)."""
    c = 2 / (3 * chi)
    sg = -1.0 if comp == 0 else 1.0
    kw = dict(epsabs=0, epsrel=1e-12, limit=500)
    def dens(u):
        x = c * u
        return ((2 + 2 * u + u * u) * special.kv(2 / 3, x) - (1 + u) * _intk13(x) + sg * u * special.kv(1 / 3, x)) / (1 + u) ** 3
    brk = [U, U * 1.2, U * 1.5, U * 2, U * 4, np.inf]
    s = sum(integrate.quad(dens, a, b, **kw)[0] for a, b in zip(brk[:-1], brk[1:]))
    A, B = _ncs_AB(chi)
    return s / (A + sg * B)


@pytest.mark.parametrize("i,comp,j", [(200, 0, 470), (150, 1, 505), (100, 0, 480), (30, 1, 511)])
def test_ncs_inverse_cdf_far_upper_tail_nodes(orc, i, comp, j):
    """At table nodes the upper tail (1 - level down to 3e-17) is exact to quadrature."""
    hx = (math.log(1e3) - math.log(1e-4)) / 255
    chi = math.exp(math.log(1e-4) + i * hx)
    t = -38 + j * 76 / 511
    u = math.exp(orc.ncs_invcdf(comp, chi, t))
    assert _ncs_ccdf(chi, comp, u) == pytest.approx(1 / (1 + math.exp(t)), rel=1e-9)


@pytest.mark.parametrize("chi,comp,t", [(0.8, 0, 30.0), (0.05, 1, 35.0), (2.0, 0, 37.5)])
def test_ncs_inverse_cdf_far_upper_tail_offgrid(orc, chi, comp, t):
    u = math.exp(orc.ncs_invcdf(comp, chi, t))
    assert _ncs_ccdf(chi, comp, u) == pytest.approx(1 / (1 + math.exp(t)), rel=1e-6)


@pytest.mark.parametrize("chig,comp,t", [(0.0105, 0, -36.0), (0.3, 1, -33.0), (150.0, 0, -37.0)])
def test_nbw_inverse_cdf_deep_tail(orc, chig, comp, t):
    d = math.exp(orc.nbw_invcdf(comp, chig, t))
    sg = -1.0 if comp == 0 else 1.0
    r0 = 8 / (3 * chig)
    def dens(x):
        rho = 2 / (3 * chig * x * (1 - x))
        k23 = special.kve(2 / 3, rho) * math.exp(-(rho - r0))
        ik = _intk13(rho) * math.exp(r0)
        return ik + (x / (1 - x) + (1 - x) / x) * k23 + sg * k23
    kw = dict(epsabs=0, epsrel=1e-11, limit=400)
    num = integrate.quad(dens, 0, d, **kw)[0]
    den = sum(integrate.quad(dens, a, b, **kw)[0] for a, b in ((0, 0.4), (0.4, 0.5)))
    assert num / den == pytest.approx(math.exp(t), rel=1e-5)
