"""Seeded synthetic inputs and raw workload parameters.

This module is shared by the CUDA path's callers and by the CPU oracle's
tests, so it holds none of the method's arithmetic: only primary parameters
(grid sizes, boxes, Mach and Knudsen numbers, step counts) and the random
perturbation drawn from a seed.  Derived values (time step, domain length,
lid speed, Rankine-Hugoniot states, Maxwellians) are computed separately by
each side.

Random numbers: SplitMix64 (Steele, Lea, Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), used counter-style: output k
(k = 0, 1, ...) of seed s mixes s + (k+1)*0x9E3779B97F4A7C15.  xi in [-1, 1)
is the top 53 bits scaled by 2**-52, minus 1.
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, start: int = 0) -> np.ndarray:
    """Outputs start .. start+count-1 of the SplitMix64 stream of ``seed`` (uint64)."""
    k = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed % (1 << 64)) + k * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform_pm1(seed: int, count: int, start: int = 0) -> np.ndarray:
    """count float64 values in [-1, 1) from the SplitMix64 stream."""
    z = splitmix64(seed, count, start) >> np.uint64(11)
    return z.astype(np.float64) * (2.0 ** -52) - 1.0


def perturbation(seed: int, ncell: int, nv: int) -> np.ndarray:
    """xi for every (cell, velocity, function) in the state layout
    [cell][v][g|h], flattened: length ncell*nv*2."""
    return uniform_pm1(seed, ncell * nv * 2)


# Raw parameters of the benchmark problems.  Velocity boxes are in units of
# sqrt(2 R T0); lengths in mean free paths; omega is the viscosity exponent.
SHOCK_M2 = dict(
    name="shock_m2_nx200_nv64_f64", kind="shock", mach=2.0, nx=200, length=40.0,
    nvx=64, vx=(-8.0, 8.0), omega=0.5, cfl=0.5, steps=4000,
)
CAVITY_64 = dict(
    name="cavity_kn0.1_ma0.1_64x64_v32x32_f64", kind="cavity", kn=0.1, lid_mach=0.1,
    n=64, nv=32, vbox=(-5.0, 5.0), omega=0.5, cfl=0.5, steps=5000, seed=0, amp=1e-3,
)
CAVITY_256 = dict(
    name="cavity_kn0.05_ma0.05_256x256_v48x48", kind="cavity", kn=0.05, lid_mach=0.05,
    n=256, nv=48, vbox=(-5.0, 5.0), omega=0.5, cfl=0.5, steps=20000, seed=0, amp=1e-3,
)
CAVITY_128 = dict(
    name="cavity_kn0.1_ma0.1_128x128_v32x32", kind="cavity", kn=0.1, lid_mach=0.1,
    n=128, nv=32, vbox=(-5.0, 5.0), omega=0.5, cfl=0.5, steps=2000, seed=0, amp=1e-3,
)

# The shock as the paper computed it (Sec. 4.1): full velocity grid, no Chu
# reduction, omega 0.74, domain 70 mean free paths, dt 0.05.
SHOCK3V_M15 = dict(
    name="shock3v_m1.5_nx512_v16x16x16", kind="shock3v", mach=1.5, nx=512, length=70.0,
    nv=(16, 16, 16), vx=(-5.0, 7.0), vt=(-6.0, 6.0), omega=0.74, dt=0.05, steps=400,
)
SHOCK3V_M3 = dict(
    name="shock3v_m3_nx2048_v30x30x30", kind="shock3v", mach=3.0, nx=2048, length=70.0,
    nv=(30, 30, 30), vx=(-10.0, 12.0), vt=(-11.0, 11.0), omega=0.74, dt=0.05, steps=100,
)

WORKLOADS = {w["name"]: w for w in (SHOCK_M2, CAVITY_64, CAVITY_256, CAVITY_128, SHOCK3V_M15, SHOCK3V_M3)}


def scaled(w: dict, **over) -> dict:
    """A copy of a workload with some raw parameters replaced (smaller test cases)."""
    d = dict(w)
    d.update(over)
    return d


def batch_instances(seed: int = 0, cavities: int = 64, shocks: int = 16) -> list[dict]:
    """Raw parameters of the batched workload: `cavities` lid-driven cavities
    with side cells from {32, 64, 96, 128, 192}, velocity grids from
    {24, 32, 40, 48}^2 on [-5, 5]^2, Kn log-uniform in [0.01, 1] and lid Mach
    log-uniform in [0.02, 0.3]; then `shocks` normal shocks with
    Mach uniform in [1.2, 5], cells uniform in [100, 800] on 40 mean free
    paths, and a velocity box [-V, V] with V = 4 + 3 Mach cut into
    8 round(V / 1.2) cells (about 0.3 thermal speeds each); every instance
    holds an FP32 state."""
    u = (uniform_pm1(seed, 4 * cavities + 2 * shocks) + 1.0) * 0.5  # [0, 1)
    out = []
    sides, grids = (32, 64, 96, 128, 192), (24, 32, 40, 48)
    for i in range(cavities):
        a, b, c, d = u[4 * i: 4 * i + 4]
        out.append(dict(
            name=f"batch_cavity_{i}", kind="cavity", n=sides[int(a * 5)], nv=grids[int(b * 4)],
            kn=float(10.0 ** (-2.0 + 2.0 * c)),
            lid_mach=float(10.0 ** (np.log10(0.02) + (np.log10(0.3) - np.log10(0.02)) * d)),
            vbox=(-5.0, 5.0), omega=0.5, cfl=0.5, seed=seed + 1 + i, amp=1e-3, precision="f32"))
    base = 4 * cavities
    for k in range(shocks):
        a, b = u[base + 2 * k: base + 2 * k + 2]
        mach = float(1.2 + 3.8 * a)
        v = 4.0 + 3.0 * mach
        out.append(dict(
            name=f"batch_shock_{k}", kind="shock", mach=mach, nx=min(800, int(100 + 701 * b)),
            length=40.0, nvx=8 * int(round(v / 1.2)), vx=(-v, v), omega=0.5, cfl=0.5, precision="f32"))
    return out
