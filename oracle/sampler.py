"""Oracle side of the learned photon-energy sampler (test infrastructure: only tests, the
smoke check and the benchmark's CPU legs use this package).

* ``mixture_inverse``: the distribution the table sampler draws the NCS energy from, written
  as one map of one uniform.  At spin projection s = S.zeta the photon spectrum of Eq. Wspin2
  is the mixture of its two spin components (weights w+- = (1 +- s)(A -+ B)/2, A and B the
  integrated rates); its CDF is F(y) = [w+ F+(y) + w- F-(y)] / (w+ + w-) in y = ln u, with
  F+-(y) the level at which the oracle's own component inverse CDF reaches y.  F is
  inverted by bisection.  Built on the oracle's tables only.
* ``forward``: the network the library evaluates (3 -> 64 -> 64 -> 1, GELU with the tanh
  form), in numpy, with the library's BF16 rounding of the hidden activations and weights
  of the 64 x 64 layer (round to nearest even), and its input features / output transform.
"""
from __future__ import annotations

import math

import numpy as np

LNCHI_LO, LNCHI_HI = math.log(1e-3), math.log(10.0)
T_LO, T_HI = -38.0, 38.0
H = 64
N_PARAMS = H * 3 + H + H * H + H + H + 1


def logit_clamped(r):
    t = np.log(r) - np.log1p(-np.asarray(r, dtype=np.float64))
    return np.clip(t, T_LO, T_HI)


def mixture_inverse(orc, chi: float, s: float, r: float, iters: int = 60) -> float:
    A, B = orc.ncs_rates(chi)
    wp, wm = 0.5 * (1 + s) * (A - B), 0.5 * (1 - s) * (A + B)
    t_r = float(logit_clamped(r))
    r = 1.0 / (1.0 + math.exp(-t_r))

    def level(c, y):
        lo, hi = T_LO, T_HI
        if orc.ncs_invcdf(c, chi, lo) >= y:
            return 0.0
        if orc.ncs_invcdf(c, chi, hi) <= y:
            return 1.0
        for _ in range(iters):
            m = 0.5 * (lo + hi)
            if orc.ncs_invcdf(c, chi, m) < y:
                lo = m
            else:
                hi = m
        return 1.0 / (1.0 + math.exp(-0.5 * (lo + hi)))

    ylo = min(orc.ncs_invcdf(0, chi, T_LO), orc.ncs_invcdf(1, chi, T_LO))
    yhi = max(orc.ncs_invcdf(0, chi, T_HI), orc.ncs_invcdf(1, chi, T_HI))
    for _ in range(iters):
        y = 0.5 * (ylo + yhi)
        if (wp * level(0, y) + wm * level(1, y)) / (wp + wm) < r:
            ylo = y
        else:
            yhi = y
    return 0.5 * (ylo + yhi)


def two_uniform_sample(orc, chi: float, s: float, um0: float, um1: float) -> float:
    """The table sampler's own draw (component by one uniform, level by the other)."""
    A, B = orc.ncs_rates(chi)
    comp = 0 if um0 * (A - s * B) < 0.5 * (1 + s) * (A - B) else 1
    return orc.ncs_invcdf(comp, chi, float(logit_clamped(um1)))


def bf16_round(x: np.ndarray) -> np.ndarray:
    """float32 -> nearest BF16 (ties to even), returned as float32."""
    b = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


def gelu(x):
    c = math.sqrt(2.0 / math.pi)
    return 0.5 * x * (1.0 + np.tanh(c * (x + 0.044715 * x ** 3)))


def unpack(p: np.ndarray):
    p = np.asarray(p, dtype=np.float32)
    o = 0
    w1 = p[o:o + H * 3].reshape(H, 3); o += H * 3
    b1 = p[o:o + H]; o += H
    w2 = p[o:o + H * H].reshape(H, H); o += H * H
    b2 = p[o:o + H]; o += H
    w3 = p[o:o + H]; o += H
    b3 = p[o]
    return w1, b1, w2, b2, w3, b3


def features(lnchi, s, t):
    x0 = (2.0 * lnchi - (LNCHI_LO + LNCHI_HI)) / (LNCHI_HI - LNCHI_LO)
    return np.stack([x0, s, t * 0.125], 1)


def base(lnchi, t):
    return lnchi - 3.0 * np.where(t < -20.0, -t, np.log1p(np.exp(-np.minimum(t, 700.0))))


def forward(p: np.ndarray, lnchi, s, r) -> np.ndarray:
    """ln u of the network for rows (ln chi_e, s, r)."""
    w1, b1, w2, b2, w3, b3 = unpack(p)
    lnchi = np.asarray(lnchi, dtype=np.float64)
    t = logit_clamped(np.asarray(r, dtype=np.float64))
    x = features(lnchi, np.asarray(s, dtype=np.float64), t).astype(np.float32)
    h1 = bf16_round(gelu(x.astype(np.float64) @ w1.T.astype(np.float64) + b1).astype(np.float32))
    z2 = h1.astype(np.float64) @ bf16_round(w2).T.astype(np.float64) + b2
    y = gelu(z2) @ w3.astype(np.float64) + b3
    return base(lnchi, t) + 8.0 * y
