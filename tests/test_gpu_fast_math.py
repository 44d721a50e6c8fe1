"""The mixed path's fast FP32 helpers on the device, one by one, against FP64 references
and against CUDA's own atan2f.

The FP32 step trades the accurate library functions for hardware approximations and a
fitted odd polynomial for the arctangent (the emission azimuth and the photon's
polarisation angle).  The bounds here are what the step's 2e-5 per-particle tolerance
is budgeted on:

* atan01 (degree-15 odd polynomial on [0, 1]): absolute error <= 1.5e-7 (the fit's 4e-8
  plus FP32 rounding of the Horner chain and of the result near pi/4);
* f_atan, f_atan2: absolute error <= 6e-7 over every quadrant and 40 decades of
  magnitude (the reciprocal's 2 ulp and the pi/2 and pi reflections add to atan01's),
  within 8e-7 of atan2f, the same sign and quadrant, and the exact special values
  (axes, signed zeros); a zero vector gives +0, the path's convention;
* f_exp, f_log, f_sincos, f_rcp, f_rsqrt: the documented accuracy of the hardware
  approximations they call, plus the explicit reduction of f_sincos to [-pi, pi].
"""
import ctypes as C
import math
import os
import shutil
import subprocess

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ULP = 2.0 ** -23          # FP32 relative spacing just above a power of two


@pytest.fixture(scope="module")
def probe(tmp_path_factory):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    so = str(tmp_path_factory.mktemp("fastmath") / "libfast_math_probe.so")
    r = subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "-shared",
                        "-Xcompiler", "-fPIC", "-o", so, os.path.join(HERE, "fast_math_probe.cu")],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    L = C.CDLL(so)
    L.fast_math_eval.argtypes = [C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_uint64]
    L.fast_math_eval.restype = C.c_int

    def ev(which, x, y=None):
        xd = torch.from_numpy(np.ascontiguousarray(x, np.float32)).cuda()
        yd = torch.from_numpy(np.ascontiguousarray(x if y is None else y, np.float32)).cuda()
        out = torch.empty_like(xd)
        assert L.fast_math_eval(which, xd.data_ptr(), yd.data_ptr(), out.data_ptr(), xd.numel()) == 0
        return out.cpu().numpy().astype(np.float64)
    return ev


def test_atan01_on_unit_interval(probe):
    t = np.concatenate([np.linspace(0, 1, 2 ** 22 + 1), [1e-30, 1e-10, 1e-5, np.nextafter(1, 0)]]).astype(np.float32)
    got = probe(0, t)
    err = np.abs(got - np.arctan(t.astype(np.float64)))
    assert err.max() <= 1.5e-7, (err.max(), t[err.argmax()])
    assert got[0] == 0.0                                   # odd polynomial: atan01(0) = 0 exactly
    assert abs(got[2 ** 22] - math.pi / 4) <= 1.5e-7
    assert np.all(np.diff(got[: 2 ** 22 + 1]) >= 0)        # monotone on the grid


def test_f_atan_full_line(probe):
    rng = np.random.default_rng(5)
    x = np.concatenate([np.linspace(-4, 4, 400_001), 10 ** rng.uniform(-20, 20, 200_000),
                        -(10 ** rng.uniform(-20, 20, 200_000)), [0.0, -0.0, 1.0, -1.0]]).astype(np.float32)
    got = probe(1, x)
    err = np.abs(got - np.arctan(x.astype(np.float64)))
    assert err.max() <= 6e-7, (err.max(), x[err.argmax()])
    assert np.array_equal(np.signbit(got[x != 0]), np.signbit(x[x != 0]))


def _atan2_inputs():
    rng = np.random.default_rng(7)
    n = 1_000_000
    ang = rng.uniform(-math.pi, math.pi, n)
    mag = 10 ** rng.uniform(-20, 20, n)
    y, x = mag * np.sin(ang), mag * np.cos(ang)
    # near the quadrant boundaries and the diagonal, where the reflections switch
    k = 200_000
    y[:k] = rng.uniform(-1, 1, k)
    x[:k] = y[:k] * (1 + rng.choice([-1, 1], k) * 10 ** rng.uniform(-7, -1, k)) * rng.choice([-1, 1], k)
    x[k:2 * k] = rng.uniform(-1, 1, k) * 10 ** rng.uniform(-9, -1, k)
    y[k:2 * k] = rng.choice([-1.0, 1.0], k)
    return y.astype(np.float32), x.astype(np.float32)


def test_f_atan2_all_quadrants(probe):
    y, x = _atan2_inputs()
    got = probe(2, y, x)
    ref = np.arctan2(y.astype(np.float64), x.astype(np.float64))
    err = np.abs(got - ref)
    assert err.max() <= 6e-7, (err.max(), y[err.argmax()], x[err.argmax()])
    cuda = probe(3, y, x)
    assert np.abs(got - cuda).max() <= 8e-7
    nz = y != 0
    assert np.array_equal(np.signbit(got[nz]), np.signbit(cuda[nz]))
    assert np.all(np.abs(got) <= np.float32(math.pi))


def test_f_atan2_special_values(probe):
    pi, h = np.float32(math.pi), np.float32(math.pi / 2)
    cases = [  # (y, x, expected)
        (0.0, 1.0, 0.0), (-0.0, 1.0, -0.0), (0.0, -1.0, pi), (-0.0, -1.0, -pi),
        (1.0, 0.0, h), (-1.0, 0.0, -h), (1.0, -0.0, h), (-1.0, -0.0, -h),
        (1.0, 1.0, None), (-1.0, -1.0, None), (3e-30, -2e-30, None), (1e30, 1e30, None),
        (0.0, 0.0, 0.0), (-0.0, -0.0, 0.0),           # zero vector: +0, the path's convention
    ]
    y = np.array([c[0] for c in cases], np.float32)
    x = np.array([c[1] for c in cases], np.float32)
    got = probe(2, y, x)
    for (yy, xx, want), g in zip(cases, got):
        if want is None:
            assert abs(g - math.atan2(yy, xx)) <= 6e-7, (yy, xx, g)
        else:
            assert g == want and np.signbit(g) == np.signbit(want), (yy, xx, g)
    cuda = probe(3, y[:12], x[:12])
    assert np.abs(got[:12] - cuda).max() <= 8e-7


def test_exp_log_rcp_rsqrt(probe):
    rng = np.random.default_rng(11)
    x = rng.uniform(-30, 30, 500_000).astype(np.float32)
    got = probe(4, x)
    ref = np.exp(x.astype(np.float64))
    # documented: at most 2 + floor(1.173 |x|) ulp; an ulp is at most 2^-23 of the value
    assert np.all(np.abs(got - ref) <= (2 + np.floor(1.173 * np.abs(x)) + 0.5) * ULP * ref)
    x = np.concatenate([rng.uniform(0.5, 2, 250_000), 10 ** rng.uniform(-30, 30, 250_000)]).astype(np.float32)
    got, ref = probe(5, x), np.log(x.astype(np.float64))
    inside = (x >= 0.5) & (x <= 2)
    assert np.abs(got - ref)[inside].max() <= 2 ** -21.41
    assert np.all(np.abs(got - ref)[~inside] <= 3.5 * ULP * np.abs(ref[~inside]))
    x = (rng.choice([-1, 1], 500_000) * 10 ** rng.uniform(-30, 30, 500_000)).astype(np.float32)
    for which, ref in ((8, 1.0 / x.astype(np.float64)), (9, None)):
        if which == 9:
            x = np.abs(x)
            ref = 1.0 / np.sqrt(x.astype(np.float64))
        got = probe(which, x)
        assert np.all(np.abs(got - ref) <= 2.5 * ULP * np.abs(ref)), which


def test_sincos_with_reduction(probe):
    rng = np.random.default_rng(13)
    x = np.concatenate([rng.uniform(-math.pi, math.pi, 300_000), rng.uniform(-1e3, 1e3, 300_000),
                        [0.0, math.pi, -math.pi, 2 * math.pi, 1e3]]).astype(np.float32)
    xd = x.astype(np.float64)
    s, c = probe(6, x), probe(7, x)
    # the hardware pair's 2^-21.41 on [-pi, pi], plus the reduction: the two-part 2 pi
    # leaves k * 1e-10 (k <= 160 here) and one FP32 rounding of the reduced argument
    bound = 2 ** -21.41 + 2.5e-7
    assert np.abs(s - np.sin(xd)).max() <= bound
    assert np.abs(c - np.cos(xd)).max() <= bound
    assert np.abs(s * s + c * c - 1).max() <= 4 * bound
