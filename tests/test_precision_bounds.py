"""The constants of tests/precision_bounds.py, recomputed (no GPU)."""
import math

import numpy as np

import precision_bounds as PB


def test_lid_deviation_constants():
    # 2 U_W max|c| e^{-c^2} / pi and 2 U_W max c^2 e^{-c^2} / pi per unit U_W,
    # and the shear weight max c_x^2 |c_y| e^{-c^2}, maximised on a fine grid
    c = np.linspace(0.0, 6.0, 60001)
    assert abs(2 * (c * np.exp(-c * c)).max() / math.pi - 0.273) < 5e-4
    assert abs(2 * (c * c * np.exp(-c * c)).max() / math.pi - 0.234) < 5e-4
    x = np.linspace(0.0, 3.0, 1501)
    X, Y = np.meshgrid(x, x)
    assert abs((X * X * Y * np.exp(-X * X - Y * Y)).max() - 0.1578) < 2e-4
    md, mcd = PB.cavity_max_d(0.0456, 0.05, 1e-3)
    assert md > 0.273 * 0.0456 and mcd > 0.234 * 0.0456


def test_spread_and_f32():
    assert PB.spread(1, 0.05) == 1.0                       # one step: nothing spread yet
    assert PB.spread(10 ** 5, 0.05) < PB.spread(10 ** 5, 0.01)  # faster streaming spreads more
    b = PB.f32(2000)
    assert b["n"] == (6 * 2000 + 1) * 2.0 ** -24 and b["theta"] == 2 * b["n"]
