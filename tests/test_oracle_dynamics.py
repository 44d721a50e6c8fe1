"""Dynamical pins of the oracle step: Boris and T-BMT closed forms (Secs. II A,
III B), plane-wave invariants (Sec. III A closed form), the radiative T-BMT drift of
the spin Monte Carlo (Eq. spin1), Stokes frame changes (Eq. rotation), VB phase
(Eq. rotation2), NBW pair statistics (Sec. III D) and the id/compaction rules."""
import math

import numpy as np
import pytest
from scipy import integrate, special

import oracle
import workloads

ALPHA = 7.2973525693e-3
XIL = 2.42631023867e-6
AE = 1.15965218128e-3


def _beam(n, p, s=(0, 1, 0), x=(0, 0, 0), first=0):
    d = {k: np.full(n, float(v)) for k, v in zip(("x", "y", "z"), x)}
    d.update({k: np.full(n, float(v)) for k, v in zip(("px", "py", "pz"), p)})
    d.update({k: np.full(n, float(v)) for k, v in zip(("s1", "s2", "s3"), s)})
    d["w"] = np.ones(n)
    d["id"] = np.arange(first, first + n, dtype=np.uint64)
    return d


def _wl(e=None, pos=None, ph=None, field=None, dt=0.01, seed=1, next_id=None):
    e = e if e is not None else workloads.empty()
    pos = pos if pos is not None else workloads.empty()
    ph = ph if ph is not None else workloads.empty(True)
    nid = next_id if next_id is not None else len(e["id"]) + len(pos["id"]) + len(ph["id"])
    return {"e": e, "pos": pos, "ph": ph, "field": field, "dt": dt, "seed": seed, "next_id": nid}


def test_boris_pure_B(orc):
    """|p| conserved to rounding; gyro angle per step 2 atan(B dt/(2 gamma))."""
    B = 3.0
    sim = oracle.Sim(orc, _wl(e=_beam(1, (50.0, 0, 0)), field={"kind": "uniform", "B": (0, 0, B)}, dt=0.05))
    n = 4000
    sim.run(n, 0)
    st = sim.state()["e"]
    p = np.array([st["px"][0], st["py"][0], st["pz"][0]])
    g = math.sqrt(1 + 50.0 ** 2)
    assert np.linalg.norm(p) == pytest.approx(50.0, rel=1e-13)
    ang = n * 2 * math.atan(B * 0.05 / (2 * g))
    # electron (q = -1) rotates counter-clockwise about +B
    assert math.atan2(p[1], p[0]) % (2 * math.pi) == pytest.approx(ang % (2 * math.pi), abs=1e-9)


def test_tbmt_g_minus_2(orc):
    """Uniform B: the angle from p to S advances at |q|(g/2-1) B per unit time."""
    B = 2.0
    for q_species in ("e", "pos"):
        beam = _beam(1, (20.0, 0, 0), s=(1, 0, 0))
        wl = _wl(**{q_species: beam}, field={"kind": "uniform", "B": (0, 0, B)}, dt=0.02)
        sim = oracle.Sim(orc, wl)
        n = 20000
        sim.run(n, oracle.F_SPIN)
        st = sim.state()[q_species]
        p = np.array([st["px"][0], st["py"][0]])
        s = np.array([st["s1"][0], st["s2"][0], st["s3"][0]])
        assert np.linalg.norm(s) == pytest.approx(1.0, abs=1e-12)
        rel = math.atan2(p[0] * s[1] - p[1] * s[0], p @ s[:2])
        sign = 1.0 if q_species == "e" else -1.0
        expected = sign * AE * B * n * 0.02
        assert rel == pytest.approx(expected, rel=2e-4)


@pytest.mark.parametrize("dt", [math.pi / 100, math.pi / 200])
def test_plane_wave_invariants(orc, dt):
    """Lorentz motion in the config-1 plane wave: gamma + p_z (light-front) and
    p_x + q A_x(phi) are constant, and p returns to p0 after the pulse (Sec. III A,
    plane-wave solution).  Errors are second order in dt."""
    wl = workloads.c1(n=1)
    wl["dt"] = dt
    sim = oracle.Sim(orc, wl)
    g0 = 2000.0
    p0 = np.array([0, 0, math.sqrt(g0 * g0 - 1)])
    h0 = g0 + p0[2]
    worst_h = worst_px = 0.0
    steps = int(450 * (math.pi / 100) / dt)
    L = 8 * math.pi
    for k in range(steps):
        sim.run(1, 0)
        st = sim.state()["e"]
        p = np.array([st["px"][0], st["py"][0], st["pz"][0]])
        g = math.sqrt(1 + p @ p)
        worst_h = max(worst_h, abs(g + p[2] - h0) / h0)
        # p^{n+1/2} pairs with the phase at t^{n+1/2}, x^{n+1/2}
        t_half = (k + 0.5) * dt
        z_half = 0.5 * (st["z"][0] + (st["z"][0] - dt * p[2] / g))
        phi = t_half + z_half
        if 0 < phi < L:
            A = -integrate.quad(lambda f: 20 * math.sin(f / 8) ** 2 * math.cos(f), 0, phi)[0]
        else:
            A = 0.0
        worst_px = max(worst_px, abs(p[0] - A * 1.0 - p0[0]))
    scale = 20.0
    k2 = (dt / (math.pi / 100)) ** 2
    assert worst_h < 3e-6 * k2 + 1e-12
    assert worst_px < 0.03 * scale * k2
    st = sim.state()["e"]
    assert abs(st["px"][0]) < 1e-3 * scale * k2
    assert abs(st["pz"][0] - p0[2]) / p0[2] < 1e-6 * k2


def _psi(chi):
    c = 2 / (3 * chi)
    kw = dict(epsabs=0, epsrel=1e-11, limit=400)
    upp = lambda u: u * u / (1 + u) ** 3
    brk = [0, 1.5 * chi, 15 * chi, np.inf]
    def q(f):
        return sum(integrate.quad(f, a, b, **kw)[0] for a, b in zip(brk[:-1], brk[1:]))
    p1 = q(lambda u: upp(u) * special.kv(2 / 3, c * u))
    p3 = q(lambda u: upp(u) * special.kv(1 / 3, c * u))
    intk = lambda x: integrate.quad(lambda t: special.kv(1 / 3, t), x, np.inf, epsabs=0, epsrel=1e-11, limit=200)[0]
    p2 = q(lambda u: upp(u) * intk(c * u)) - p1
    return p1, p2, p3


def test_sokolov_ternov_limit_of_radiative_tbmt():
    """Equilibrium of Eq. spin1 for S along n_B: S = -psi3/psi1 -> -8/(5 sqrt3) (Sec. I's
    ~92.5%) as chi -> 0."""
    p1, p2, p3 = _psi(1e-4)
    assert -p3 / p1 == pytest.approx(-8 / (5 * math.sqrt(3)), rel=3e-4)


@pytest.mark.parametrize("S0", [(0.6, 0.0, 0.8), (0.0, 1.0, 0.0), (0.36, -0.48, 0.8)])
def test_spin_mc_mean_drift_is_radiative_tbmt(orc, S0):
    """One step, many electrons: the ensemble mean of S_new - S equals dt times the
    radiative T-BMT term -P[psi1 S + psi2 (S.n) n + psi3 n_B] (Eq. spin1), P =
    alpha/(sqrt3 pi gamma xi_L).  Precession is switched off to isolate it."""
    gamma = 1.0e4
    chi = 1.0
    B0 = chi / (XIL * gamma)
    N = 300_000
    dt = 1.6
    pz = math.sqrt(gamma * gamma - 1)
    S0 = np.array(S0) / np.linalg.norm(S0)
    wl = _wl(e=_beam(N, (0, 0, pz), s=S0), field={"kind": "uniform", "B": (B0, 0, 0)}, dt=dt, seed=7)
    sim = oracle.Sim(orc, wl)
    sim.run(1, oracle.F_NCS | oracle.F_NO_RECOIL)
    st = sim.state()["e"]
    S = np.stack([st["s1"], st["s2"], st["s3"]], 1)
    p = np.array([st["px"][0], st["py"][0], st["pz"][0]])
    g = math.sqrt(1 + p @ p)
    n = p / np.linalg.norm(p)
    Bv = np.array([B0, 0, 0])
    v = np.cross(p, Bv)                       # E = 0: v = p x B
    chi_now = XIL * np.linalg.norm(v)
    a = -v / np.linalg.norm(v)                # q = -1
    zeta = np.cross(n, a)
    p1, p2, p3 = _psi(chi_now)
    P = ALPHA / (math.sqrt(3) * math.pi * g * XIL)
    drift = -P * (p1 * S0 + p2 * (S0 @ n) * n + p3 * zeta)
    mean = (S - S0).mean(0) / dt
    err = (S - S0).std(0) / math.sqrt(N) / dt
    assert np.all(np.abs(mean - drift) < 5 * err + 1e-4 * np.abs(drift).max()), (mean, drift, err)


def _lab_density(xi, th, n):
    """Photon polarisation density matrix in lab coordinates from Stokes + basis angle."""
    a = n[2]; c = -n[0]
    m = math.sqrt(a * a + c * c)
    e1 = np.array([a, 0, c]) / m
    e2 = np.cross(n, e1)
    P1 = math.cos(th) * e1 + math.sin(th) * e2
    P2 = np.cross(n, P1)
    return 0.5 * ((1 + xi[2]) * np.outer(P1, P1) + (1 - xi[2]) * np.outer(P2, P2) +
                  (xi[0] - 1j * xi[1]) * np.outer(P1, P2) + (xi[0] + 1j * xi[1]) * np.outer(P2, P1))


def test_stokes_frame_change_is_a_pure_basis_change(orc):
    """ROT(psi) (Eq. rotation) with the basis update of the VB algorithm leaves the
    lab-frame polarisation state unchanged (photon below pair threshold, VB off)."""
    rng = np.random.default_rng(2)
    for _ in range(20):
        k = rng.normal(size=3); k /= np.linalg.norm(k)
        xi = rng.normal(size=3); xi *= rng.uniform(0.1, 1) / np.linalg.norm(xi)
        th = rng.uniform(-3, 3)
        ph = {"x": np.zeros(1), "y": np.zeros(1), "z": np.zeros(1), "px": [1.5 * k[0]], "py": [1.5 * k[1]],
              "pz": [1.5 * k[2]], "s1": [xi[0]], "s2": [xi[1]], "s3": [xi[2]], "theta": [th], "w": [1.0],
              "id": np.array([0], dtype=np.uint64)}
        E, B = rng.normal(size=3), rng.normal(size=3)
        sim = oracle.Sim(orc, _wl(ph=ph, field={"kind": "uniform", "E": E, "B": B}))
        sim.run(1, oracle.F_NBW)
        st = sim.state()["ph"]
        xi1 = np.array([st["s1"][0], st["s2"][0], st["s3"][0]])
        rho0 = _lab_density(xi, th, k)
        rho1 = _lab_density(xi1, st["theta"][0], k)
        assert np.allclose(rho0, rho1, atol=1e-13)
        # new basis P1' is along E_perp + n x B
        Er = E - k * (k @ E) + np.cross(k, B)
        a = k[2]; c = -k[0]; m = math.sqrt(a * a + c * c)
        e1 = np.array([a, 0, c]) / m; e2 = np.cross(k, e1)
        P1 = math.cos(st["theta"][0]) * e1 + math.sin(st["theta"][0]) * e2
        assert np.allclose(P1, Er / np.linalg.norm(Er), atol=1e-13)


def test_vb_phase_constant_crossed_field(orc):
    """Static crossed field E_y = -B_z (Fig. VB workload): after the first step the frame is
    fixed and (xi1, xi2) turn by dphi = (M_par - M_perp) alpha/(90 pi) xi_L omega |E_r|^2 dt
    per step (Eq. rotation2); xi3 in that frame is constant."""
    om = 1957.0
    E0 = 100.0
    dt = 0.05
    ph = {"x": np.zeros(1), "y": np.zeros(1), "z": np.zeros(1), "px": [om], "py": [0.0], "pz": [0.0],
          "s1": [1.0], "s2": [0.0], "s3": [0.0], "theta": [0.0], "w": [1.0], "id": np.array([0], np.uint64)}
    sim = oracle.Sim(orc, _wl(ph=ph, field={"kind": "uniform", "E": (0, E0, 0), "B": (0, 0, -E0)}, dt=dt))
    n = 3000
    sim.run(n, oracle.F_VB)
    st = sim.state()["ph"]
    er = 2 * E0
    chig = XIL * om * er
    M = orc.vb_m(chig)
    dphi = (M[0] - M[1]) * ALPHA / (90 * math.pi) * XIL * om * er * er * dt
    # initial basis: theta = 0 -> P1 = e1(n = x) = -z; field frame P1' = +y: psi = -pi/2
    xi0 = np.array([1.0, 0, 0])
    c2, s2 = math.cos(2 * -math.pi / 2), math.sin(2 * -math.pi / 2)
    xr = np.array([xi0[0] * c2 - xi0[2] * s2, xi0[1], xi0[0] * s2 + xi0[2] * c2])
    ang = n * dphi
    exp = np.array([math.cos(ang) * xr[0] - math.sin(ang) * xr[1], math.sin(ang) * xr[0] + math.cos(ang) * xr[1], xr[2]])
    got = np.array([st["s1"][0], st["s2"][0], st["s3"][0]])
    assert np.allclose(got, exp, atol=1e-10)
    assert abs(ang) > 1.0   # a visible rotation


def test_nbw_one_step_statistics(orc):
    """Photons at chi_gamma ~ 1 for one step: decay fraction = T dt (binomial), exact
    energy sharing, delta distribution = the xi3-resolved density (KS), and the positron
    spin mean along its SQA equals |D|/C (Eq. BWposAxis)."""
    om = 4000.0
    chig = 1.0
    E0 = chig / (XIL * om * 2)
    N = 200_000
    xi = np.array([0.3, -0.4, 0.5])
    ph = {"x": np.zeros(N), "y": np.zeros(N), "z": np.zeros(N), "px": np.full(N, om), "py": np.zeros(N),
          "pz": np.zeros(N), "s1": np.full(N, xi[0]), "s2": np.full(N, xi[1]), "s3": np.full(N, xi[2]),
          "theta": np.zeros(N), "w": np.ones(N), "id": np.arange(N, dtype=np.uint64)}
    T = orc.nbw_rates(chig)
    # xi3 in the pair frame: theta=0 basis P1 = -z; field frame P1' = +y (psi = -pi/2)
    xi3p = -xi[2]
    rate = ALPHA / (math.sqrt(3) * math.pi * XIL * om) * (T[0] - xi3p * T[1])
    dt = 0.3 / rate
    sim = oracle.Sim(orc, _wl(ph=ph, field={"kind": "uniform", "E": (0, E0, 0), "B": (0, 0, -E0)}, dt=dt),
                     cap_e=N + 10, cap_p=N + 10)
    stats = sim.run(1, oracle.F_NBW)
    k = stats["n_nbw"]
    assert abs(k - 0.3 * N) < 5 * math.sqrt(N * 0.3 * 0.7)
    st = sim.state()
    e, p = st["e"], st["pos"]
    assert len(e["id"]) == k and len(p["id"]) == k
    ep = np.sqrt(1 + p["px"] ** 2 + p["py"] ** 2 + p["pz"] ** 2)
    em = np.sqrt(1 + e["px"] ** 2 + e["py"] ** 2 + e["pz"] ** 2)
    assert np.allclose(ep + em, om, rtol=1e-12)
    delta = np.sort(ep / om)
    # exact CDF of delta for this xi3'
    r0 = 8 / (3 * chig)
    def dens(d):
        rho = 2 / (3 * chig * d * (1 - d))
        k23 = special.kve(2 / 3, rho) * math.exp(-(rho - r0))
        ik = integrate.quad(lambda t: special.kv(1 / 3, t), rho, np.inf, epsabs=0, epsrel=1e-10)[0] * math.exp(r0)
        return ik + (d / (1 - d) + (1 - d) / d) * k23 - xi3p * k23
    grid = np.linspace(1e-4, 1 - 1e-4, 801)
    f = np.array([dens(d) for d in grid])
    cdf = np.concatenate([[0], np.cumsum(0.5 * (f[1:] + f[:-1]) * np.diff(grid))])
    cdf /= cdf[-1]
    emp = np.searchsorted(delta, grid) / len(delta)
    assert np.abs(emp - cdf).max() < 1.8 / math.sqrt(len(delta))
    # positron spin: mean projection on its SQA D/|D| equals |D|/C
    Sp = np.stack([p["s1"], p["s2"], p["s3"]], 1)
    P1, P2, nv = np.array([0, 1.0, 0]), np.array([0, 0, 1.0]), np.array([1.0, 0, 0])
    # Stokes in the pair frame: basis P1 = -z -> P1' = +y is psi = pi/2, so
    # ROT(psi) flips xi1 and xi3
    xq = np.array([-xi[0], xi[1], -xi[2]])
    resid = []
    for i in range(0, k, 7):
        d = ep[i] / om
        epp, emm = ep[i], em[i]
        k13, k23, ik = orc.ktable(2 / (3 * chig * d * (1 - d)))
        dif2 = (epp * epp - emm * emm) / (epp * emm)
        C = ik + (emm * emm + epp * epp) / (emm * epp) * k23 - xq[2] * k23
        D = (-(om / epp - xq[2] * om / emm) * k13 * P2 - xq[0] * (om / emm) * k13 * P1 +
             xq[1] * (dif2 * k23 + (om / epp) * ik) * nv)
        resid.append(Sp[i] @ D / np.linalg.norm(D) - np.linalg.norm(D) / C)
    resid = np.array(resid)
    assert abs(resid.mean()) < 5 * resid.std() / math.sqrt(len(resid))


def test_step_ids_and_compaction(orc):
    """Id rule: NBW pairs first (photon order; e- then e+), then NCS photons (e- order,
    then e+ order); decayed photon slots are refilled from the tail of the array."""
    wl = workloads.c2(n=400, seed=9, a0=100.0, gamma0=2e4)
    sim = oracle.Sim(orc, wl)
    sim.t = 9.5 * math.pi          # near the pulse centre at the focus
    sim.step_no = 950
    # move the beam to the collision point at t = 9.5 pi
    sim.e.arr["z"][: sim.e.n] += 9.5 * math.pi
    flags = oracle.F_NCS | oracle.F_NBW | oracle.F_VB | oracle.F_SPIN
    seen_nbw = 0
    for _ in range(60):
        before = sim.state()
        nid0 = before["next_id"]
        s = sim.run(1, flags)
        after = sim.state()
        nn = s["n_nbw"]
        seen_nbw += nn
        ne0, np0 = len(before["e"]["id"]), len(before["pos"]["id"])
        assert list(after["e"]["id"][:ne0]) == list(before["e"]["id"])
        assert list(after["e"]["id"][ne0:]) == [nid0 + 2 * k for k in range(nn)]
        assert list(after["pos"]["id"][np0:]) == [nid0 + 2 * k + 1 for k in range(nn)]
        nph0 = len(before["ph"]["id"])
        nph_surv = nph0 - nn
        surv = after["ph"]["id"][:nph_surv]
        assert set(surv) <= set(before["ph"]["id"]) and len(set(surv)) == nph_surv
        # removal rule: slots below the new count keep their photon unless it decayed, in
        # which case they hold the next surviving photon from the tail (index order)
        gone = sorted(set(before["ph"]["id"]) - set(surv))
        pos = {int(v): k for k, v in enumerate(before["ph"]["id"])}
        holes = sorted(pos[int(g)] for g in gone)
        tail = [k for k in range(nph_surv, nph0) if k not in set(holes)]
        expect = list(before["ph"]["id"][:nph_surv])
        for h, src in zip([h for h in holes if h < nph_surv], tail):
            expect[h] = before["ph"]["id"][src]
        assert list(surv) == expect
        new = after["ph"]["id"][nph_surv:]
        assert list(new) == [nid0 + 2 * nn + j for j in range(s["n_ncs_e"] + s["n_ncs_p"])]
        assert after["next_id"] == nid0 + 2 * nn + len(new)
    assert len(sim.state()["ph"]["id"]) > 100


def test_helicity_transfer_sign(orc):
    """Longitudinally polarised electrons give circularly polarised photons whose xi2 flips
    with the electron helicity (Sec. V, CP gamma photons)."""
    res = []
    for sz in (1.0, -1.0):
        wl = workloads.c1(n=3000, seed=5)
        wl["e"]["s2"][:] = 0.0
        wl["e"]["s3"][:] = sz
        sim = oracle.Sim(orc, wl)
        sim.run(450, oracle.F_NCS)
        ph = sim.state()["ph"]
        hard = ph["pz"] > 0.3 * 2000
        res.append(ph["s2"][hard].mean())
    assert res[0] * res[1] < 0 and abs(res[0]) > 0.2 and abs(res[1]) > 0.2


def test_unpolarised_beam_gives_linear_polarisation(orc):
    """Unpolarised electrons in an LP wave: photon xi3 > 0 in the (a, n x a) basis
    (Sec. V, LP gamma photons; degree of order 50-60%)."""
    wl = workloads.c1(n=3000, seed=6)
    rng = np.random.default_rng(1)
    s = rng.normal(size=(3000, 3)); s /= np.linalg.norm(s, axis=1, keepdims=True)
    wl["e"]["s1"][:], wl["e"]["s2"][:], wl["e"]["s3"][:] = s.T
    sim = oracle.Sim(orc, wl)
    sim.run(450, oracle.F_NCS | oracle.F_SPIN)
    ph = sim.state()["ph"]
    assert len(ph["id"]) > 3000
    m = ph["s3"].mean()
    assert 0.3 < m < 0.8
