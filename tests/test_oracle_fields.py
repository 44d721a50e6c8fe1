"""Pins of the oracle's analytic focused field (config 2: first-order paraxial Gaussian beam
along -z, Sec. II D's laser input).  The field is checked against what the mathematics of
a paraxial beam fixes, not against its own formula:

- with the temporal envelope made flat, E = Re[v(x, y, z) exp(i(t + z))], and the complex
  amplitude v (read from the field at t and t + pi/2) satisfies the paraxial wave equation
  of a wave moving along -z, lap_perp v + 2i dv/dz = 0 (finite differences);
- at the focus the phase front is flat and |v| = a0 exp(-r^2 / w0^2);
- the transverse power, integral |v|^2 dx dy = pi w0^2 a0^2 / 2, is the same at every z;
- circular polarisation keeps |E_perp| = |v| at all times, and B = k x E with k = -z."""
import math

import numpy as np
import pytest

import oracle

W0 = 6.0 * math.pi          # config 2: w0 = 3 um in units of 1/k0
ZR = 0.5 * W0 * W0          # Rayleigh length k0 w0^2 / 2
A0 = 3.0
L_FLAT = 1.0e8              # envelope length: sin^2 is flat to 1e-11 near its middle
PHI_C = 10.0                # the middle of the envelope sits at phase t + z = PHI_C


def _fields(circular=0, zf=0.0):
    return oracle.make_fields(kind=oracle.FIELD_GAUSS, circular=circular, a0=A0, phi0=PHI_C - 0.5 * L_FLAT,
                              length=L_FLAT, w0=W0, zf=zf)


def _v(f, x, y, z):
    """complex amplitude v with E_x = Re[v exp(i(t + z))], at a time placing t + z near PHI_C"""
    t = PHI_C - z
    e0 = oracle.field(f, x, y, z, t)[0][0]
    e1 = oracle.field(f, x, y, z, t + 0.5 * math.pi)[0][0]
    return (e0 - 1j * e1) * np.exp(-1j * (t + z))


@pytest.mark.parametrize("zeta", [0.0, 0.5 * ZR, -2.0 * ZR, 3.0 * ZR])
def test_paraxial_wave_equation(zeta):
    f = _fields(zf=0.0)
    z = -zeta                   # zeta = zf - z: distance travelled past the focus
    h, hz = 0.05, 0.5
    for x, y in [(0.0, 0.0), (0.7 * W0, 0.0), (0.3 * W0, -0.9 * W0), (1.2 * W0, 0.8 * W0)]:
        v = _v(f, x, y, z)
        lap = (_v(f, x + h, y, z) + _v(f, x - h, y, z) + _v(f, x, y + h, z) + _v(f, x, y - h, z) - 4 * v) / h ** 2
        dz = (_v(f, x, y, z + hz) - _v(f, x, y, z - hz)) / (2 * hz)
        res = lap + 2j * dz
        scale = abs(v) * 4.0 / W0 ** 2 + 1e-300
        assert abs(res) / scale < 1e-3, (zeta, x, y, abs(res) / scale)
        # the wrong propagation direction (+z) leaves an O(1) residual
        assert abs(lap - 2j * dz) / scale > 0.1


def test_focus_is_flat_and_gaussian():
    f = _fields(zf=0.0)
    for r in [0.0, 0.2 * W0, 0.8 * W0, 1.5 * W0]:
        v = _v(f, r / math.sqrt(2), r / math.sqrt(2), 0.0)
        assert abs(v.imag) < 1e-9 * A0
        assert v.real == pytest.approx(A0 * math.exp(-r * r / W0 ** 2), rel=1e-9, abs=1e-12)


@pytest.mark.parametrize("zeta", [0.0, 0.7 * ZR, 2.5 * ZR])
def test_transverse_power_is_conserved(zeta):
    f = _fields(zf=0.0)
    w = W0 * math.sqrt(1.0 + (zeta / ZR) ** 2)
    xs = np.linspace(-4.5 * w, 4.5 * w, 241)
    t = PHI_C + zeta
    I = np.zeros((len(xs), len(xs)))
    for a, x in enumerate(xs):
        for b, y in enumerate(xs):
            e0 = oracle.field(f, x, y, -zeta, t)[0][0]
            e1 = oracle.field(f, x, y, -zeta, t + 0.5 * math.pi)[0][0]
            I[a, b] = e0 * e0 + e1 * e1
    trap = getattr(np, "trapezoid", None) or np.trapz   # numpy 2 renamed it
    P = trap(trap(I, xs, axis=1), xs)
    assert P == pytest.approx(0.5 * math.pi * W0 ** 2 * A0 ** 2, rel=1e-6)


def test_circular_polarisation_and_b_equals_k_cross_e():
    f = _fields(circular=1, zf=0.0)
    x, y, z = 0.4 * W0, -0.2 * W0, -0.3 * ZR
    mags = []
    for t in np.linspace(PHI_C - z - 3.0, PHI_C - z + 3.0, 13):
        E, B = oracle.field(f, x, y, z, t)
        assert E[2] == 0.0 and B[2] == 0.0
        assert np.allclose(B, np.cross([0.0, 0.0, -1.0], E), rtol=0, atol=1e-14)
        mags.append(math.hypot(E[0], E[1]))
    assert np.ptp(mags) < 1e-12 * max(mags)
    assert mags[0] == pytest.approx(abs(_v(_fields(zf=0.0), x, y, z)), rel=1e-12)
