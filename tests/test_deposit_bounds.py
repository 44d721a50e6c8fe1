"""The bounds the fixed-point deposition window relies on (Sec. II C's Esirkepov terms with
the TSC shape of Sec. II E), checked numerically on random moves of less than one cell:

- the cumulative sum over nodes of the shape differences S1 - S0 (the charge a move carries
  through each face) never exceeds the move |X1 - X0| in magnitude;
- the averaged shape product of the Jz term, S0x S0y + dSx S0y / 2 + S0x dSy / 2 +
  dSx dSy / 3, lies in [0, 1].

They bound each lepton's Jx, Jy and Jz terms by |cx dX|, |cy dY| and |cz|, which sets the
window's integer scale so that 256 terms per cell cannot overflow 32 bits."""
import numpy as np


def _tsc5(X, base):
    """TSC weights of position X (cell units) on the five nodes base-2 .. base+2"""
    nodes = base + np.arange(-2, 3)
    d = np.abs(X - nodes)
    return np.where(d <= 0.5, 0.75 - d * d, np.where(d <= 1.5, 0.5 * (1.5 - d) ** 2, 0.0))


def test_face_flux_is_bounded_by_the_move():
    rng = np.random.default_rng(0)
    worst = 0.0
    for _ in range(20000):
        X0 = rng.uniform(-50, 50)
        dX = rng.uniform(-1, 1) * rng.choice([1.0, 1e-3, 1e-6])
        base = int(np.floor(X0 + 0.5))
        s0, s1 = _tsc5(X0, base), _tsc5(X0 + dX, base)
        if abs(int(np.floor(X0 + dX + 0.5)) - base) > 1:
            continue
        assert abs(s0.sum() - 1) < 1e-12 and abs(s1.sum() - 1) < 1e-12
        flux = np.cumsum(s1 - s0)
        worst = max(worst, np.abs(flux).max() / abs(dX) if dX else 0.0)
        assert np.abs(flux).max() <= abs(dX) * (1 + 1e-9) + 1e-15
    assert worst > 0.7          # the bound is nearly reached (a shape peak crossing a face)


def test_jz_weight_is_in_unit_interval():
    rng = np.random.default_rng(1)
    for _ in range(20000):
        X0, Y0 = rng.uniform(-50, 50, 2)
        dX, dY = rng.uniform(-1, 1, 2)
        bx, by = int(np.floor(X0 + 0.5)), int(np.floor(Y0 + 0.5))
        s0x, s1x = _tsc5(X0, bx), _tsc5(X0 + dX, bx)
        s0y, s1y = _tsc5(Y0, by), _tsc5(Y0 + dY, by)
        dsx, dsy = s1x - s0x, s1y - s0y
        wz = (np.outer(s0y, s0x) + 0.5 * np.outer(s0y, dsx) + 0.5 * np.outer(dsy, s0x)
              + np.outer(dsy, dsx) / 3.0)
        assert wz.min() >= -1e-12 and wz.max() <= 1.0 + 1e-12
        assert abs(wz.sum() - 1.0) < 1e-12     # the averaged shape keeps unit charge
