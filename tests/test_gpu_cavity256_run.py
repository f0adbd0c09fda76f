"""The 256^2-cell, 48^2-velocity cavity (Kn 0.05, lid Mach 0.05) against the
oracle's stored fields after 2000 of its 20000 steps
(tests/golden/cavity256_2000steps_*.txt, written by gen_cavity256.py, which
calls only the oracle): n, U, theta on 3136 sampled cells (every
wall-adjacent layer and a 5-cell lattice), the lid's wall fluxes per face
cell, the lid-integrated shear J and the total mass.

FP64: the per-step rounding of the two paths differs at about 1e-16 and the
scheme does not amplify it, so every field agrees to 1e-12 (velocities
relative to the lid speed U_W, the rest relative to the field's scale).

Reduced precisions: bounds from the storage precision, stated before the
run (N = 2000 steps, nv = 2304 velocities per cell, dv = (10/48)^2, 65536
cells of side dx = 20/256, lid speed U_W = 0.0456, lid shear tau >= 0.01):
  FP32 rounds every stored value to 2^-24 relative each step.  With every
  rounding of the same sign (no cancellation at all), a moment drifts by at
  most eps = N 2^-24 = 1.19e-4 of its sum of absolute terms: n and the total
  mass by eps, U by eps <|c|> / U_W = eps (sqrt(pi)/2) / U_W (2.3e-3 of U_W),
  theta = (2/3)(E/n - U^2) by 2 eps, the lid shear by eps sum |c_x c_y| F /
  tau <= eps (1/pi) / 0.01 (3.8e-3).
  BF16 stores d = f - M_abs with stochastic rounding: a store errs by at most
  one ulp, 2^-7 |d|, with zero mean and standard deviation at most half an
  ulp, independently across velocities.  The lid drives deviations
  2 |c| U_W M(c) <= 0.0125 (and 2 c^2 U_W M <= 0.0107 in c d), the seeded
  perturbation 3.2e-4, density and temperature changes of order Mach^2 less
  than 8e-4: max|d| <= 0.015, max|c d| <= 0.0123.  One step thus adds to a
  cell's n an error of standard deviation s_n = sqrt(nv) 2^-8 max|d| dv
  (1.2e-4), to its n U one of s_u = sqrt(nv) 2^-8 max|c d| dv.  Streaming
  carries each step's errors away at about 0.05 cells per step (the mean
  speed times dt / dx), so after k steps they are spread over about
  0.0079 k^2 cells; summing the variances, sum_k 1 / max(1, 0.0079 k^2) =
  21.9, a cell's accumulated error has a standard deviation at most
  sqrt(21.9) s = 4.7 s.  The bounds are six of those: n 28 s_n (3.4e-3), U
  28 s_u / U_W (6.2e-2 of U_W), theta (2/3)(1 + 1.5) x the n bound (5.7e-3),
  the lid shear per cell 28 sqrt(nv / 2) 2^-8 max|c_x c_y d| dv / tau with
  max|c_x c_y d| <= 0.0075 (0.12), J (256 lid cells, errors correlated over
  about 10) that over sqrt(25.6) (2.4e-2), and the total mass, whose errors
  do not spread out, 6 sqrt(N cells) s_n dx^2 / 400 (1.3e-4).
"""
import os

import numpy as np
import pytest

from paper_0903_4044_gb300 import bgk as B
from paper_0903_4044_gb300 import build, solver
from paper_0903_4044_gb300 import workloads as W

pytestmark = pytest.mark.gpu

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
STEPS = 2000
N_, NV, DV, DX, CELLS = 2000, 48 * 48, (10.0 / 48) ** 2, 20.0 / 256, 256 * 256
EPS32 = N_ * 2.0 ** -24
UW = 0.05 * (5.0 / 6.0) ** 0.5
TAU_MIN = 0.01
S_N = NV ** 0.5 * 2.0 ** -8 * 0.015 * DV
S_U = NV ** 0.5 * 2.0 ** -8 * 0.0123 * DV
S_TAU = (NV / 2) ** 0.5 * 2.0 ** -8 * 0.0075 * DV
SPREAD = sum(1.0 / max(1.0, 0.0079 * k * k) for k in range(1, N_ + 1)) ** 0.5   # 4.7
BOUNDS = {
    "f64": dict(n=1e-12, u=1e-12, theta=1e-12, shear=1e-12, J=1e-12, mass=1e-13),
    "f32": dict(n=EPS32, u=EPS32 * np.sqrt(np.pi) / 2 / UW, theta=2 * EPS32, shear=EPS32 / np.pi / TAU_MIN,
                J=EPS32 / np.pi / TAU_MIN, mass=EPS32),
    "bf16": dict(n=6 * SPREAD * S_N, u=6 * SPREAD * S_U / UW, theta=(2 / 3) * 2.5 * 6 * SPREAD * S_N,
                 shear=6 * SPREAD * S_TAU / TAU_MIN, J=6 * SPREAD * S_TAU / TAU_MIN / 25.6 ** 0.5,
                 mass=6 * (N_ * CELLS) ** 0.5 * S_N * DX * DX / 400.0),
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
    # the docstring's figures, recomputed from the formulas above
    assert EPS32 == pytest.approx(1.19e-4, rel=1e-2)
    assert BOUNDS["f32"]["u"] == pytest.approx(2.3e-3, rel=2e-2)
    assert SPREAD == pytest.approx(4.7, rel=1e-2)
    assert BOUNDS["bf16"]["n"] == pytest.approx(3.4e-3, rel=2e-2)
    assert BOUNDS["bf16"]["u"] == pytest.approx(6.2e-2, rel=2e-2)
    assert BOUNDS["bf16"]["theta"] == pytest.approx(5.7e-3, rel=2e-2)
    assert BOUNDS["bf16"]["J"] == pytest.approx(2.4e-2, rel=2e-2)
    assert BOUNDS["bf16"]["mass"] == pytest.approx(1.3e-4, rel=2e-2)


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
        # the other wall fluxes of the lid per face cell
        for col in (1, 3, 4):
            scale = max(np.abs(lid[:, col]).max(), 1e-3)
            assert np.abs(fl[:, col - 1] - lid[:, col]).max() <= 1e-12 * scale
