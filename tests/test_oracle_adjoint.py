"""Pins of the oracle's reverse pass against central finite differences of
the oracle's own forward run (h = 1e-6), on tiny cavities.

With the effective-parameter correction off the reverse pass is the exact
derivative of the forward map; with it on, the reverse pass linearises the
map p(q) by the identity, which is exact up to the quadrature residual of
the velocity grid, so that case uses a well-resolved grid."""
import math

import numpy as np
import pytest

from paper_0903_4044_gb300 import workloads as W

H = 1e-6


def _cavity(orc, n=4, nv=8, scale=1.0, uw=0.3, cons=0, vbox=4.0, ny=None):
    ny = ny or n - 1
    L = 2.0 * scale
    return orc.make_config(dim=2, nx=n, ny=ny, lx=L, ly=L * ny / n, nvx=nv, nvy=nv, vx=(-vbox, vbox),
                           vy=(-vbox, vbox), cfl=0.7, conservative=cons,
                           bc_kind=(1, 1, 1, 1),
                           bc_state=((1, 0, 0, 1), (1, 0, 0.1, 1.2), (1, -0.2, 0, 0.9), (1, uw, 0, 1.1)))


def _state(orc, cfg, seed):
    prob = orc.Problem(cfg)
    xi = W.perturbation(seed, prob.ncell, prob.nv)
    g, h = orc.init_uniform(prob, (1.0, 0.05, -0.03, 1.0), xi, 0.2)
    return prob, g, h


def _J(orc, cfg, g, h, steps):
    prob = orc.Problem(cfg)
    g1, h1, _ = orc.step(prob, g, h, steps)
    return orc.lid_shear(prob, g1, h1)


@pytest.mark.parametrize("cons,nv,vbox,steps", [(0, 8, 4.0, 6), (1, 24, 6.0, 4)])
def test_adjoint_matches_finite_differences(orc, cons, nv, vbox, steps):
    cfg = _cavity(orc, nv=nv, cons=cons, vbox=vbox)
    prob, g, h = _state(orc, cfg, 3)
    J, dlnL, dUW, dg, dh = orc.adjoint_lid_shear(prob, g, h, steps)
    assert J == pytest.approx(_J(orc, cfg, g, h, steps), rel=1e-14)
    tol = 1e-6
    # lid speed
    fd = (_J(orc, _cavity(orc, nv=nv, cons=cons, vbox=vbox, uw=0.3 + H), g, h, steps)
          - _J(orc, _cavity(orc, nv=nv, cons=cons, vbox=vbox, uw=0.3 - H), g, h, steps)) / (2 * H)
    assert dUW == pytest.approx(fd, rel=tol, abs=1e-9)
    # domain scale (Kn = 1/L): lengths and the Courant-derived time step
    fd = (_J(orc, _cavity(orc, nv=nv, cons=cons, vbox=vbox, scale=math.exp(H)), g, h, steps)
          - _J(orc, _cavity(orc, nv=nv, cons=cons, vbox=vbox, scale=math.exp(-H)), g, h, steps)) / (2 * H)
    assert dlnL == pytest.approx(fd, rel=tol, abs=1e-9)
    # initial state entries, g and h, interior and wall cells
    for cell, j in [(0, 3), (5, nv * nv // 2 + 1), (prob.ncell - 1, 2), (prob.ncell - 2, nv * nv - 3)]:
        for arr, grad in ((g, dg), (h, dh)):
            a = arr.copy()
            a[cell, j] += H
            jp = _J(orc, cfg, a if arr is g else g, a if arr is h else h, steps)
            a[cell, j] -= 2 * H
            jm = _J(orc, cfg, a if arr is g else g, a if arr is h else h, steps)
            fd = (jp - jm) / (2 * H)
            assert grad[cell, j] == pytest.approx(fd, rel=1e-5, abs=1e-9)


def test_adjoint_directional_derivative(orc):
    # one random direction over the whole initial state
    cfg = _cavity(orc, n=5, nv=8)
    prob, g, h = _state(orc, cfg, 8)
    steps = 5
    J, _, _, dg, dh = orc.adjoint_lid_shear(prob, g, h, steps)
    vg = W.uniform_pm1(41, g.size).reshape(g.shape)
    vh = W.uniform_pm1(42, h.size).reshape(h.shape)
    fd = (_J(orc, cfg, g + H * vg, h + H * vh, steps) - _J(orc, cfg, g - H * vg, h - H * vh, steps)) / (2 * H)
    assert float((dg * vg).sum() + (dh * vh).sum()) == pytest.approx(fd, rel=1e-6)
