"""Write the oracle's moments after the full 64x64-cell, 32x32-velocity cavity run.

Calls only ``oracle/`` (and the seeded input generator): Kn = 0.1, lid Mach
0.1, diffuse walls at theta = 1, CFL 0.5, initial resting Maxwellian times
(1 + 1e-3 xi) with xi from SplitMix64 seed 0, 5000 steps, exact exponential
relaxation with the conservative effective-parameter Maxwellian.

Output: cavity64_moments.txt, one line per cell (cell = iy*64 + ix):
n ux uy theta of the final state, 17 significant digits.

Run from the repository root:  python tests/golden/gen_cavity64.py
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_0903_4044_gb300 import workloads as W  # noqa: E402


def main() -> None:
    w = W.CAVITY_64
    prob, _, _ = oracle.cavity_problem(**w)
    xi = W.perturbation(w["seed"], prob.ncell, prob.nv)
    prob, g, h = oracle.cavity_problem(**w, xi=xi)
    t0 = time.time()
    g1, h1, _ = oracle.step(prob, g, h, w["steps"])
    mom = oracle.state_moments(prob, g1, h1)
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "cavity64_moments.txt")
    header = (f"oracle moments (n ux uy theta) after {w['steps']} steps of {w['name']}, "
              f"dt={prob.cfg.dt!r}; {time.time() - t0:.0f} s on {oracle.threads()} threads")
    np.savetxt(out, mom, fmt="%.17g", header=header)
    print(header)


if __name__ == "__main__":
    main()
