"""Pins of the oracle's radiative pusher: the Landau-Lifshitz force and its quantum
correction q(chi) (Sec. III A), and the radiative T-BMT term with psi1..psi3 (Sec. III B,
Eq. spin1).

* q and psi1..3 against independent scipy quadratures of their defining integrals, and
  against their small-chi closed forms from the Mellin transform of K_nu (DLMF 10.43.19);
  q against the two fits printed in Sec. III A.
* One LL step radiates the classical (Larmor) power (2/3) alpha chi^2 / xi_L of Sec. III A,
  as a drag along -beta for both charges; one modified-LL step radiates q(chi) times it.
* The radiative T-BMT in a uniform magnetic field relaxes the spin component along B to
  the Sokolov-Ternov equilibrium -+8/(5 sqrt3) at the rate (5 sqrt3/8) alpha chi^3/(xi_L
  gamma) (closed forms of the chi -> 0 limit).
* The paper's statement (Sec. III C) that the mean of the Monte Carlo emission follows the
  modified LL + radiative T-BMT dynamics: one step of many electrons, mean momentum and
  spin change of the stochastic step against the deterministic one."""
import math

import numpy as np
import pytest
from scipy import integrate, special

import oracle
import workloads

ALPHA = 7.2973525693e-3
XIL = 2.42631023867e-6
F_RAD = oracle.F_MLL | oracle.F_MBMT


def _quad(f, chi):
    kw = dict(epsabs=0, epsrel=1e-12, limit=500)
    brk = [0, 0.15 * chi, 1.5 * chi, 15 * chi, 150 * chi]
    s = sum(integrate.quad(f, a, b, **kw)[0] for a, b in zip(brk[:-1], brk[1:]))
    return s + integrate.quad(f, brk[-1], np.inf, **kw)[0]


def _psi_scipy(chi):
    """psi1, psi2, psi3 of Eq. spin1's legend by scipy; the IntK term by parts:
    int u^2/(1+u)^3 IntK13(u') du = (2/3chi) int G(u) K13(u') du with
    G(u) = int_0^u t^2/(1+t)^3 dt = ln(1+u) - u(3u+2)/(2(1+u)^2)."""
    c = 2 / (3 * chi)
    upp = lambda u: u * u / (1 + u) ** 3
    p1 = _quad(lambda u: upp(u) * special.kv(2 / 3, c * u), chi)
    p3 = _quad(lambda u: upp(u) * special.kv(1 / 3, c * u), chi)
    G = lambda u: math.log1p(u) - u * (3 * u + 2) / (2 * (1 + u) ** 2)
    pi = c * _quad(lambda u: G(u) * special.kv(1 / 3, c * u), chi)
    return p1, pi - p1, p3


def _q_scipy(chi):
    """q = I_QED/I_C (Sec. III A): the spin-averaged power of Eq. Wspin2 (photon energy
    gamma u/(1+u)) over (2/3) alpha chi^2/xi_L; IntK by parts with
    int_0^u t/(1+t)^3 dt = u^2/(2(1+u)^2)."""
    c = 2 / (3 * chi)
    a = _quad(lambda u: u * (2 + 2 * u + u * u) * special.kv(2 / 3, c * u) / (1 + u) ** 4, chi)
    b = c * _quad(lambda u: u * u / (2 * (1 + u) ** 2) * special.kv(1 / 3, c * u), chi)
    return math.sqrt(3) / (2 * math.pi * chi * chi) * (a - b)


def _mellin(mu, nu):
    """int_0^inf x^(mu-1) K_nu(x) dx (DLMF 10.43.19)"""
    return 2 ** (mu - 2) * special.gamma((mu - nu) / 2) * special.gamma((mu + nu) / 2)


@pytest.mark.parametrize("chi", [3.3e-4, 0.052, 0.71, 4.2, 63.0])
def test_rr_functions_vs_scipy(orc, chi):
    q, p1, p2, p3 = orc.rr_funcs(chi)
    s1, s2, s3 = _psi_scipy(chi)
    # off the nodes: 4-point Lagrange in ln chi (spacing 0.0315) of psi/chi^3, which falls
    # as chi^(-7/3) at large chi: interpolation errors up to a few 1e-7
    assert q == pytest.approx(_q_scipy(chi), rel=1e-6)
    assert p1 == pytest.approx(s1, rel=1e-6)
    assert p3 == pytest.approx(s3, rel=1e-6)
    assert p2 == pytest.approx(s2, rel=2e-6)


def test_rr_functions_small_chi_closed_forms(orc):
    """u^2/(1+u)^3 = u^2 - 3u^3 + O(u^4) and u' = 2u/(3chi): two terms of each psi from
    the Mellin transforms of K_nu; q = 1 - (55 sqrt3/16) chi + 48 chi^2 (known expansion)."""
    chi = 1e-4
    h = 1.5 * chi
    q, p1, p2, p3 = orc.rr_funcs(chi)
    e1 = h ** 3 * _mellin(3, 2 / 3) - 3 * h ** 4 * _mellin(4, 2 / 3)
    e3 = h ** 3 * _mellin(3, 1 / 3) - 3 * h ** 4 * _mellin(4, 1 / 3)
    # int x^m IntK(x) dx = M(m+2, nu)/(m+1)
    ei = h ** 3 * _mellin(4, 1 / 3) / 3 - 3 * h ** 4 * _mellin(5, 1 / 3) / 4
    assert p1 == pytest.approx(e1, rel=2e-6)
    assert p3 == pytest.approx(e3, rel=2e-6)
    assert p2 == pytest.approx(ei - e1, rel=2e-6)
    # the leading ratio is the Sokolov-Ternov degree 8/(5 sqrt3)
    assert _mellin(3, 1 / 3) / _mellin(3, 2 / 3) == pytest.approx(8 / (5 * math.sqrt(3)), rel=1e-12)
    for c in (1e-4, 1e-3):
        assert orc.rr_funcs(c)[0] == pytest.approx(1 - 55 * math.sqrt(3) / 16 * c + 48 * c * c, abs=2e-6)


@pytest.mark.parametrize("chi", [0.01, 0.1, 1.0])
def test_q_vs_paper_fits(orc, chi):
    q = orc.rr_funcs(chi)[0]
    fit1 = (1 + 4.8 * (1 + chi) * math.log(1 + 1.7 * chi) + 2.44 * chi * chi) ** (-2 / 3)
    fit2 = (1 + 8.93 * chi + 2.41 * chi * chi) ** (-2 / 3)
    assert q == pytest.approx(fit1, rel=0.03)
    assert q == pytest.approx(fit2, rel=0.04)


def _beam(n, p, s=(0, 1, 0)):
    d = {k: np.zeros(n) for k in ("x", "y", "z")}
    d.update({k: np.full(n, float(v)) for k, v in zip(("px", "py", "pz"), p)})
    d.update({k: np.full(n, float(v)) for k, v in zip(("s1", "s2", "s3"), s)})
    d["w"] = np.ones(n)
    d["id"] = np.arange(n, dtype=np.uint64)
    return d


def _wl(e=None, pos=None, field=None, dt=0.01, seed=1):
    e = e if e is not None else workloads.empty()
    pos = pos if pos is not None else workloads.empty()
    return {"e": e, "pos": pos, "ph": workloads.empty(True), "field": field, "dt": dt, "seed": seed,
            "next_id": len(e["id"]) + len(pos["id"])}


@pytest.mark.parametrize("species", ["e", "pos"])
@pytest.mark.parametrize("flag,chi", [(oracle.F_LL, 1e-3), (oracle.F_LL, 0.3), (oracle.F_MLL, 0.5)])
def test_one_step_radiates_larmor_power(orc, species, flag, chi):
    """Head-on with a crossed field (E = E0 x, B = E0 y, the electron along -z): the
    Lorentz force does no work to first order, so gamma falls by the radiated power:
    (2/3) alpha chi^2/xi_L for LL (Sec. III A, ultrarelativistic limit, corrections
    O(1/gamma^2)) and q(chi) times it for the modified LL, q from scipy."""
    gamma = 1.0e4
    E0 = chi / (2 * gamma * XIL)
    pz = -math.sqrt(gamma * gamma - 1)
    dt = 0.05
    beam = _beam(1, (0, 0, pz))
    wl = _wl(**{species: beam}, field={"kind": "uniform", "E": (E0, 0, 0), "B": (0, E0, 0)}, dt=dt)
    sim = oracle.Sim(orc, wl)
    sim.run(1, flag)
    st = sim.state()[species]
    p1 = np.array([st["px"][0], st["py"][0], st["pz"][0]])
    dg = (math.sqrt(1 + p1 @ p1) - gamma) / dt
    qf = 1.0 if flag == oracle.F_LL else _q_scipy(chi)
    assert dg == pytest.approx(-qf * 2 / 3 * ALPHA * chi * chi / XIL, rel=2e-5)
    assert p1[2] > pz   # a drag: |pz| decreases


@pytest.mark.parametrize("species,sign", [("e", -1.0), ("pos", 1.0)])
def test_radiative_tbmt_sokolov_ternov_buildup(orc, species, sign):
    """Uniform B along x, longitudinal initial spin: precession leaves S.B alone and the
    radiative term drives it exponentially to sign * psi3/psi1 (e- antiparallel, e+
    parallel to B) at the rate P psi1, P = alpha/(sqrt3 pi gamma xi_L) -- the
    Sokolov-Ternov build-up, whose chi -> 0 limits 8/(5 sqrt3) and (5 sqrt3/8) alpha
    chi^3/(xi_L gamma) follow from the Mellin forms above.  chi = 0.05, gamma = 1e4 (one
    e-fold in about 5 gyrations), 200 steps per gyration; psi from scipy."""
    gamma, chi = 1.0e4, 0.05
    B0 = chi / (XIL * gamma)
    p1, p2, p3 = _psi_scipy(chi)
    rate = ALPHA / (math.sqrt(3) * math.pi * gamma * XIL) * p1
    seq = p3 / p1
    assert abs(seq - 8 / (5 * math.sqrt(3))) < 0.02   # close to the chi -> 0 degree
    dt = 2 * math.pi * gamma / B0 / 200
    pz = math.sqrt(gamma * gamma - 1)
    beam = _beam(1, (0, 0, pz), s=(0, 0, 1))
    sim = oracle.Sim(orc, _wl(**{species: beam}, field={"kind": "uniform", "B": (B0, 0, 0)}, dt=dt))
    nstep = 0
    for k in range(4):
        sim.run(300, oracle.F_SPIN | oracle.F_MBMT)
        nstep += 300
        sx = sim.state()[species]["s1"][0]
        expect = sign * seq * (1 - math.exp(-nstep * dt * rate))
        assert sx == pytest.approx(expect, abs=2e-3 * seq), (nstep, sx, expect)
    assert abs(sim.state()[species]["s1"][0]) > 0.5 * seq


def test_mc_mean_follows_mll_and_radiative_tbmt(orc):
    """Sec. III C: the Monte Carlo emission (recoil and spin) averaged over many electrons
    follows the modified LL force and the radiative T-BMT term.  One step at chi = 1 of
    300k identical electrons (no precession): the mean momentum change and the mean spin
    change of the stochastic step agree with the deterministic step within statistics."""
    gamma, chi = 1.0e4, 1.0
    B0 = chi / (XIL * gamma)
    pz = math.sqrt(gamma * gamma - 1)
    dt = 1.0
    # S.zeta = 0 (zeta = +x here): the MC energy loss has a spin term (B of Eq. Wspin2)
    # that the spin-averaged modified LL force does not carry
    S0 = np.array([0.0, -0.6, 0.8])
    field = {"kind": "uniform", "B": (B0, 0, 0)}
    N = 300_000
    mc = oracle.Sim(orc, _wl(e=_beam(N, (0, 0, pz), s=S0), field=field, dt=dt, seed=5))
    mc.run(1, oracle.F_NCS | oracle.F_DROP_PHOTONS)
    m = mc.state()["e"]
    det = oracle.Sim(orc, _wl(e=_beam(1, (0, 0, pz), s=S0), field=field, dt=dt))
    det.run(1, F_RAD)
    d = det.state()["e"]
    # the Lorentz part of the step is the same Boris push in both
    lor = oracle.Sim(orc, _wl(e=_beam(1, (0, 0, pz), s=S0), field=field, dt=dt))
    lor.run(1, 0)
    l = lor.state()["e"]
    P_mc = np.stack([m["px"], m["py"], m["pz"]], 1)
    P_l = np.array([l["px"][0], l["py"][0], l["pz"][0]])
    P_d = np.array([d["px"][0], d["py"][0], d["pz"][0]])
    # along the momentum: the radiated energy.  Across it the two differ at O(theta), the
    # Lorentz rotation of one step: the Monte Carlo recoils along the end-of-step
    # direction, the force acts along the time-centred one.
    nl = P_l / np.linalg.norm(P_l)
    theta = math.hypot(P_l[0], P_l[1]) / abs(P_l[2])
    along = (P_mc - P_l) @ nl
    dpl_det = (P_d - P_l) @ nl
    assert abs(along.mean() - dpl_det) < 5 * along.std() / math.sqrt(N) + 1e-3 * abs(dpl_det)
    assert dpl_det < 0
    perp_mc = (P_mc - P_l).mean(0) - along.mean() * nl
    perp_det = (P_d - P_l) - dpl_det * nl
    assert np.linalg.norm(perp_mc - perp_det) < 1.5 * theta * abs(dpl_det)
    S_mc = np.stack([m["s1"], m["s2"], m["s3"]], 1)
    ds_mc = (S_mc - S0).mean(0)
    err_s = (S_mc - S0).std(0) / math.sqrt(N)
    ds_det = np.array([d["s1"][0], d["s2"][0], d["s3"][0]]) - S0
    assert np.all(np.abs(ds_mc - ds_det) < 5 * err_s + 2e-3 * np.abs(ds_det).max()), (ds_mc, ds_det, err_s)
