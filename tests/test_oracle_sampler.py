"""Pins of the learned-sampler references in oracle/sampler.py.

* The one-uniform mixture inverse draws the same distribution as the table sampler's own
  two-uniform draw (component, then level) -- the spin mixture of Eq. Wspin2 -- checked by a
  two-sample Kolmogorov-Smirnov test at several chi_e and spin projections, including the
  pure components s = +-1.
* The mixture inverse is monotone in r and, at s = +1 (only the "+" component), equals the
  component's own inverse CDF.
* BF16 rounding is round-to-nearest-even on the float32 bit pattern (hand-checked values),
  and the numpy network with zero hidden weights reduces to its closed form."""
import math

import numpy as np
import pytest
from scipy import stats

import oracle.sampler as SM


def test_mixture_inverse_matches_two_uniform_draw(orc):
    rng = np.random.default_rng(3)
    for chi, s in ((0.01, 0.0), (1.0, 0.7), (5.0, -0.9), (0.3, 1.0), (0.3, -1.0)):
        n = 600
        one = np.array([SM.mixture_inverse(orc, chi, s, r, iters=40) for r in rng.uniform(size=n)])
        two = np.array([SM.two_uniform_sample(orc, chi, s, a, b) for a, b in rng.uniform(size=(n, 2))])
        assert stats.ks_2samp(one, two).pvalue > 1e-3, (chi, s)


def test_mixture_inverse_monotone_and_pure_component(orc):
    rs = np.linspace(0.01, 0.99, 25)
    ys = [SM.mixture_inverse(orc, 0.5, 0.3, r) for r in rs]
    assert np.all(np.diff(ys) > 0)
    for r in (0.05, 0.5, 0.93):
        t = float(SM.logit_clamped(r))
        assert abs(SM.mixture_inverse(orc, 2.0, 1.0, r) - orc.ncs_invcdf(0, 2.0, t)) < 1e-9


def test_bf16_round_to_nearest_even():
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, 1.0 + 2 ** -9, 1.0 + 2 ** -8 + 2 ** -12, -2.5],
                 dtype=np.float32)
    want = np.array([1.0, 1.0, 1.0 + 2 ** -6, 1.0, 1.0 + 2 ** -7, -2.5], dtype=np.float32)
    assert np.array_equal(SM.bf16_round(x), want)


def test_forward_closed_form_with_zero_hidden_weights():
    p = np.zeros(SM.N_PARAMS, dtype=np.float32)
    w1, b1, w2, b2, w3, b3 = SM.unpack(p)
    # only biases: z2 = b2, y = w3 . gelu(b2) + b3
    p[SM.H * 3 + SM.H + SM.H * SM.H: SM.H * 3 + SM.H + SM.H * SM.H + SM.H] = 0.5       # b2
    p[-SM.H - 1:-1] = 0.25                                                              # w3
    p[-1] = -0.1                                                                        # b3
    lnchi, s, r = np.array([math.log(0.2)]), np.array([0.3]), np.array([0.4])
    y = 0.25 * SM.H * SM.gelu(0.5) + float(np.float32(-0.1))
    t = math.log(0.4 / 0.6)
    want = math.log(0.2) - 3 * math.log1p(math.exp(-t)) + 8 * y
    assert abs(SM.forward(p, lnchi, s, r)[0] - want) < 1e-12
