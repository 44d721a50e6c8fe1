"""Pin of the oracle's emission collapse (paper Sec. III C, Eqs. NCSW, F0-F3 and the
Monte Carlo procedure that follows them): final spin along the SQA of F0 with
P(+) = (1 + |g|/c0)/2, then the photon pure state +-F/|F| with P(+) = (1 + |F|/F0)/2.

Whatever the collapse rules, their means are fixed by the rates.  With F0 = c0 + g.S_f
and F = f + H S_f (both affine in S_f, Eqs. F0-F3):

* E[S_f | u] = g / c0 (spin summed over the two outcomes +-g/|g|);
* E[xi | u, S_f] = F(S_f)/F0(S_f), so E[xi | u] = f / c0 (F summed over S_f = +-g/|g|);
* E[xi sigma | u] = (F(g_hat) - F(-g_hat)) / (2 c0), with S_f = sigma g_hat,

and in a bin of u each is the ratio of the u-integrals weighted by the emission density
W_R F0(S_f = 0) ~ c0/(1+u)^3.  A wrong sign of a term of F1 (the one checked only by
positivity before), a wrong collapse probability (P(+) = |F|/F0 makes E[xi | S_f] =
(2|F|/F0 - 1) F_hat) or a transposed frame vector moves these means by O(0.1); the
sampling error per bin here is below 0.01.

The rates on this side are a second transcription of Eqs. F0-F3, in numpy with
scipy.special.kv and scipy quadrature for IntK_1/3: nothing of the oracle's C code.
Electrons: one state (gamma ~ 4000, chi_e ~ 1 in a uniform magnetic field), 2e5 of them
stepped once with the emission probability near 1/2 (dt chosen from the oracle's rate),
for two initial spins with components along a, zeta and n.
"""
import math

import numpy as np
import pytest

import oracle

sp = pytest.importorskip("scipy.special")
si = pytest.importorskip("scipy.integrate")

XI_L = 2.42631023867e-6
ALPHA = 7.2973525693e-3


_IK = {}


def _intk13(x):
    """IntK_1/3(x) = int_x^inf K_1/3: scipy quadrature between the nodes of a log grid
    (summed from the top), cubic spline in (ln x, ln IntK) between them."""
    if "f" not in _IK:
        from scipy.interpolate import CubicSpline
        xs = np.geomspace(1e-6, 300.0, 4000)
        pieces = [si.quad(lambda t: sp.kv(1 / 3, t), xs[i], xs[i + 1], limit=200)[0] for i in range(len(xs) - 1)]
        tail = si.quad(lambda t: sp.kv(1 / 3, t), xs[-1], np.inf)[0]
        vals = tail + np.concatenate([np.cumsum(pieces[::-1])[::-1], [0.0]])
        _IK["f"] = CubicSpline(np.log(xs), np.log(vals))
    return np.exp(_IK["f"](np.log(x)))


def _F(u, chi, n, a, Si, Sf):
    """F0..F3 of Eqs. F0-F3 (the paper's expressions, term by term) at an array u, for
    the final spin Sf of shape [3] or [3, len(u)] (zero drops every S_f term).  Returns an
    array [4, len(u)]."""
    x = 2 * u / (3 * chi)
    k13, k23, ik = sp.kv(1 / 3, x), sp.kv(2 / 3, x), _intk13(x)
    z = np.cross(n, a)
    Sf = np.asarray(Sf, dtype=np.float64)
    Sf = Sf[:, None] * np.ones_like(u) if Sf.ndim == 1 else Sf
    Sif = Si @ Sf
    si_z, sf_z = Si @ z, z @ Sf
    si_a, sf_a = Si @ a, a @ Sf
    si_n, sf_n = Si @ n, n @ Sf
    sfxsi = np.cross(Sf.T, Si).T                     # [3, nu]
    n_sfxsi, a_sfxsi = n @ sfxsi, a @ sfxsi
    u2 = u * u
    F0 = (-(2 + u) ** 2 * (ik - 2 * k23) * (1 + Sif) + u2 * (1 - Sif) * (ik + 2 * k23) + 2 * u2 * Sif * ik
          - (4 * u + 2 * u2) * (sf_z + si_z) * k13 - 2 * u2 * (sf_z - si_z) * k13
          - 4 * u2 * (ik - k23) * si_n * sf_n)
    F1 = (-2 * u2 * ik * (si_a * sf_z + sf_a * si_z) + 4 * u * (si_a * (1 + u) + sf_a) * k13
          + 2 * u * (2 + u) * n_sfxsi * k23)
    F2 = (-(2 * u2 * (si_n * sf_z + sf_n * si_z) + 2 * u * (2 + u) * a_sfxsi) * k13
          - 4 * u * (si_n + sf_n * (1 + u)) * ik + 4 * u * (2 + u) * (si_n + sf_n) * k23)
    F3 = (4 * (1 + u + (1 + u + u2 / 2) * Sif - u2 / 2 * si_n * sf_n) * k23
          + 2 * u2 * (si_z * sf_z - si_a * sf_a) * ik - 4 * u * ((1 + u) * si_z + sf_z) * k13)
    return np.stack([F0, F1, F2, F3])


def _c0_g(u, chi, n, a, Si):
    """c0 = F0(S_f = 0) and g = dF0/dS_f (F0 is affine in S_f): [len(u)], [3, len(u)]"""
    c0 = _F(u, chi, n, a, Si, np.zeros(3))[0]
    g = np.stack([_F(u, chi, n, a, Si, e)[0] - c0 for e in np.eye(3)])
    return c0, g


def _bin_means(u_lo, u_hi, chi, n, a, Si, nodes=64):
    """Bin averages (weight c0/(1+u)^3) of E[S_f], E[xi] and E[xi sigma] over [u_lo, u_hi]:
    Gauss-Legendre in ln u."""
    x, w = np.polynomial.legendre.leggauss(nodes)
    s = 0.5 * (math.log(u_hi) - math.log(u_lo)) * x + 0.5 * (math.log(u_hi) + math.log(u_lo))
    u = np.exp(s)
    wt = w * u / (1 + u) ** 3                               # du = u ds
    c0, g = _c0_g(u, chi, n, a, Si)
    f = _F(u, chi, n, a, Si, np.zeros(3))[1:]
    gh = g / np.linalg.norm(g, axis=0)
    Fp, Fm = _F(u, chi, n, a, Si, gh)[1:], _F(u, chi, n, a, Si, -gh)[1:]
    norm = (wt * c0).sum()
    return (wt * g).sum(1) / norm, (wt * f).sum(1) / norm, (wt * 0.5 * (Fp - Fm)).sum(1) / norm


@pytest.mark.parametrize("spin", [(0.3, 0.5, 0.8), (-0.7, 0.2, -0.4)])
def test_emission_collapse_means_match_eqs_F0_F3(orc, spin):
    p0, B0 = 4000.0, 1.0 / (XI_L * 4000.0)        # chi_e ~ 1 in B = B0 x
    bvec = np.array([B0, 0.0, 0.0])
    field = {"kind": "uniform", "E": (0.0, 0.0, 0.0), "B": tuple(bvec)}
    # initial frame (p along z): n = z, a = -(p x B)/|p x B| (electron), zeta = n x a
    n0 = np.array([0.0, 0.0, 1.0])
    a0 = -np.cross(n0, bvec) / B0
    Si = spin[0] * a0 + spin[1] * np.cross(n0, a0) + spin[2] * n0
    Si /= np.linalg.norm(Si)
    # dt for an emission probability ~ 1/2 (from the oracle's rate at the initial state)
    chi0 = XI_L * p0 * B0
    A, Bv = orc.ncs_rates(chi0)
    W = ALPHA / (math.sqrt(3) * math.pi * XI_L * math.sqrt(1 + p0 * p0)) * (A - (Si @ np.cross(n0, a0)) * Bv)
    dt = 0.5 / W
    N = 200_000
    e = {"x": np.zeros(N), "y": np.zeros(N), "z": np.zeros(N), "px": np.zeros(N), "py": np.zeros(N),
         "pz": np.full(N, p0), "s1": np.full(N, Si[0]), "s2": np.full(N, Si[1]), "s3": np.full(N, Si[2]),
         "w": np.ones(N), "id": np.arange(N, dtype=np.uint64)}
    empty = {k: v[:0] for k, v in e.items()}
    sim = oracle.Sim(orc, {"e": e, "pos": empty, "ph": dict(empty, theta=np.zeros(0)), "field": field, "dt": dt,
                           "seed": 77, "next_id": N}, cap_ph=N)
    sim.run(1, oracle.F_NCS)                      # no T-BMT: S_i is the spin at the decision
    out = sim.state()
    el, ph = out["e"], out["ph"]
    # every electron was pushed alike, so all share one emission probability P: the
    # emitters are the len(ph) electrons with the smallest decision draws (step 0, draw 0)
    r0 = np.array([oracle.uniforms(77, i, 0, 0)[0] for i in range(N)])
    emit = np.zeros(N, dtype=bool)
    emit[np.argsort(r0)[:len(ph["id"])]] = True
    assert r0[emit].max() < r0[~emit].min() and 0.3 < emit.mean() < 0.7
    # the frame at p^{n+1/2}: from a non-emitter
    pn = np.array([el["px"][~emit][0], el["py"][~emit][0], el["pz"][~emit][0]])
    g1 = math.sqrt(1 + pn @ pn)
    n = pn / np.linalg.norm(pn)
    v = np.cross(pn, bvec)
    a = -v / np.linalg.norm(v)
    chi = XI_L * np.linalg.norm(v)
    # k-th photon (id N + k) <- k-th emitting electron in array order
    order = np.argsort(ph["id"])
    assert np.array_equal(ph["id"][order], N + np.arange(emit.sum(), dtype=np.uint64))
    k = np.stack([ph["px"], ph["py"], ph["pz"]], 1)[order]
    xi = np.stack([ph["s1"], ph["s2"], ph["s3"]], 1)[order]
    Sf = np.stack([el["s1"], el["s2"], el["s3"]], 1)[emit]
    om = np.linalg.norm(k, axis=1)
    u = om / (g1 - om)
    assert np.allclose(np.linalg.norm(xi, axis=1), 1.0, atol=1e-12)   # pure states
    edges = np.geomspace(0.02, 20.0, 7)
    checked = 0
    for lo, hi in zip(edges[:-1], edges[1:]):
        m = (u >= lo) & (u < hi)
        cnt = int(m.sum())
        if cnt < 2000:
            continue
        e_sf, e_xi, e_xis = _bin_means(lo, hi, chi, n, a, Si)
        # per photon: sigma = S_f . g_hat(u), g_hat from this side's transcription of F0
        _, g = _c0_g(u[m], chi, n, a, Si)
        gh = (g / np.linalg.norm(g, axis=0)).T
        sig = np.einsum("ij,ij->i", Sf[m], gh)
        assert np.allclose(np.abs(sig), 1.0, atol=1e-6)              # S_f = +-g_hat
        for name, samp, pred in (("S_f", Sf[m], e_sf), ("xi", xi[m], e_xi),
                                 ("xi sigma", xi[m] * sig[:, None], e_xis)):
            mean = samp.mean(0)
            se = samp.std(0, ddof=1) / math.sqrt(cnt) + 1e-12
            pull = (mean - pred) / se
            assert np.all(np.abs(pull) < 4.0), (name, lo, hi, mean, pred, pull)
            checked += 3
    assert checked >= 27
