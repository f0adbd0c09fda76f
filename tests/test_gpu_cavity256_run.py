"""The 256^2-cell, 48^2-velocity cavity (Kn 0.05, lid Mach 0.05) against the
oracle's stored fields after 2000 of its 20000 steps
(tests/golden/cavity256_2000steps_*.txt, written by gen_cavity256.py, which
calls only the oracle): n, U, theta on 3136 sampled cells (every
wall-adjacent layer and a 5-cell lattice), the lid's wall fluxes per face
cell, the lid-integrated shear J and the total mass.

FP64: the per-step rounding of the two paths differs at about 1e-16 and the
scheme does not amplify it, so every field agrees to 1e-12 (velocities
relative to the lid speed U_W, the rest relative to the field's scale).

Reduced precisions: the bounds of tests/precision_bounds.py (storage
precision only, stated before the run) for N = 2000 steps, nv = 2304
velocities per cell, dv = (10/48)^2, 65536 cells of side dx = 20/256, dt =
0.00399, lid speed U_W = 0.0456 (Mach 0.05), perturbation amplitude 1e-3:
FP32 n and mass 7.2e-4, theta 1.4e-3, U 1.4e-2 of U_W; BF16 n 3.3e-3, theta
5.5e-3, U 8.6e-2 of U_W, mass 1.2e-4.  The lid shear (tau >= 0.01 on the
lid) gets the n bound times sum |c_x c_y| F / tau <= (1/pi) / 0.01 in FP32;
in BF16 the sum of the stochastic errors of the nv/2 incident velocities,
6 spread sqrt(nv / 2) 2^-8 max|c_x c_y d| dv / tau with max|c_x c_y d| <=
2 U_W max(c_x^2 |c_y| e^{-c^2}) / pi + Mach^2 = 7.1e-3 (0.12), and J,
averaged over 256 lid cells whose errors are correlated over about 10, that
over sqrt(25.6) (2.4e-2).
"""
import math
import os

import numpy as np
import pytest

import precision_bounds as PB
from paper_0903_4044_gb300 import bgk as B
from paper_0903_4044_gb300 import build, solver
from paper_0903_4044_gb300 import workloads as W

pytestmark = pytest.mark.gpu

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
STEPS = 2000
NV, DV, DX, DT, CELLS = 48 * 48, (10.0 / 48) ** 2, 20.0 / 256, 0.5 * (20.0 / 256) / (2 * 4.8958333333333333), 65536
UW, MACH, AMP = 0.05 * (5.0 / 6.0) ** 0.5, 0.05, 1e-3
TAU_MIN = 0.01
_F = PB.f32(STEPS)
_B = PB.bf16(STEPS, NV, DV, CELLS, DX, DT, UW, MACH, AMP)
_K = 6 * PB.spread(STEPS, PB.MEAN_SPEED_2D * DT / DX)
_TAU16 = _K * (NV / 2) ** 0.5 * 2.0 ** -8 * (2 * UW * 0.1578 / math.pi + MACH ** 2) * DV / TAU_MIN
BOUNDS = {
    "f64": dict(n=1e-12, u=1e-12, theta=1e-12, shear=1e-12, J=1e-12, mass=1e-13),
    "f32": dict(n=_F["n"], u=_F["u"] / UW, theta=_F["theta"], shear=_F["n"] / math.pi / TAU_MIN,
                J=_F["n"] / math.pi / TAU_MIN, mass=_F["mass"]),
    "bf16": dict(n=_B["n"], u=_B["u"] / UW, theta=_B["theta"], shear=_TAU16, J=_TAU16 / 25.6 ** 0.5,
                 mass=_B["mass"]),
}


def _golden():
    rows = np.loadtxt(os.path.join(HERE, f"cavity256_{STEPS}steps_moments.txt"))
    lidf = os.path.join(HERE, f"cavity256_{STEPS}steps_lid.txt")
    lid = np.loadtxt(lidf)
    meta = {}
    with open(lidf) as f:
        for line in f:
            if line.startswith("# J ") or line.startswith("# mass "):
                k, v = line[2:].split()
                meta[k] = float(v)
    return rows, lid, meta


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    B.lib()


def test_bounds_are_the_stated_numbers():
    # the docstring's figures, recomputed from the formulas
    f, b = BOUNDS["f32"], BOUNDS["bf16"]
    assert f["n"] == pytest.approx(7.2e-4, rel=2e-2) and f["u"] == pytest.approx(1.4e-2, rel=2e-2)
    assert b["n"] == pytest.approx(3.3e-3, rel=3e-2) and b["theta"] == pytest.approx(5.5e-3, rel=3e-2)
    assert b["u"] == pytest.approx(8.6e-2, rel=3e-2) and b["mass"] == pytest.approx(1.2e-4, rel=5e-2)
    assert b["shear"] == pytest.approx(0.12, rel=5e-2) and b["J"] == pytest.approx(2.4e-2, rel=5e-2)


@pytest.mark.parametrize("prec", ["f64", "f32", "bf16"])
def test_cavity256_prefix_against_oracle(prec):
    rows, lid, meta = _golden()
    w = W.CAVITY_256
    n = w["n"]
    s = solver.make_cavity(w, xi=W.perturbation(w["seed"], n * n, NV), precision=solver.PRECISIONS[prec])
    s.step(STEPS)
    mom = s.moments().reshape(n, n, 4)
    fl = s.wall_fluxes(B.BGK_FACE_YHI)
    J = s.lid_shear()
    dx = s.info.dx
    s.close()
    ix, iy = rows[:, 0].astype(int), rows[:, 1].astype(int)
    got, want = mom[iy, ix], rows[:, 2:6]
    b = BOUNDS[prec]
    err = {
        "n": np.abs(got[:, 0] - want[:, 0]).max() / np.abs(want[:, 0]).max(),
        "u": np.abs(got[:, 1:3] - want[:, 1:3]).max() / UW,
        "theta": np.abs(got[:, 3] - want[:, 3]).max() / np.abs(want[:, 3]).max(),
        "shear": np.abs(fl[:, 1] - lid[:, 2]).max() / np.abs(lid[:, 2]).max(),
        "J": abs(J - meta["J"]) / abs(meta["J"]),
        "mass": abs(mom[:, :, 0].sum() * dx * dx - meta["mass"]) / meta["mass"],
    }
    print(prec, {k: f"{v:.2e}" for k, v in err.items()})
    for k, v in err.items():
        assert v <= b[k], (prec, k, v, b[k])
    if prec == "f64":
        # the other wall fluxes of the lid per face cell, relative to the
        # size of the one-sided fluxes (the normal momentum flux, about 0.5;
        # the net mass flux itself is zero to rounding)
        scale = np.abs(lid[:, 3]).max()
        for col in (1, 3, 4):
            assert np.abs(fl[:, col - 1] - lid[:, col]).max() <= 1e-12 * scale, col
