"""Write the oracle's fields after a prefix of the 256x256-cell, 48x48-velocity cavity run.

Calls only ``oracle/`` (and the seeded input generator): Kn = 0.05, lid Mach
0.05, diffuse walls at theta = 1, CFL 0.5, initial resting Maxwellian times
(1 + 1e-3 xi) with xi from SplitMix64 seed 0, exact exponential relaxation
with the conservative effective-parameter Maxwellian.  The full run is 20000
steps; the oracle does about 5e7 (8 x86 cores) to 3e8 (16 Grace cores)
updates/s, i.e. 0.5-3 s per step of 1.5e8 updates, so the stored values are
those after a stated prefix (default 2000 steps, about 2 h on 8 cores).

Outputs (N = number of steps):
- cavity256_<N>steps_moments.txt: one line per sampled cell,
  ``ix iy n ux uy theta`` of the final state, 17 significant digits.  The
  sampled rows and columns are 0, 1, 2, 5, 10, ..., 250, 253, 254, 255 (56
  per axis, 3136 cells): every wall-adjacent layer and a 5-cell lattice.
- cavity256_<N>steps_lid.txt: the lid's wall fluxes per face cell
  (``ix mass shear normal energy``), with the lid-integrated shear J and the
  total mass sum(g) dV dx dy in the header.

Run from the repository root:  python tests/golden/gen_cavity256.py [N]
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_0903_4044_gb300 import workloads as W  # noqa: E402

SAMPLE = sorted({0, 1, 2, 253, 254, 255} | set(range(5, 251, 5)))


def main(steps: int) -> None:
    w = W.CAVITY_256
    prob, _, _ = oracle.cavity_problem(**w)
    xi = W.perturbation(w["seed"], prob.ncell, prob.nv)
    prob, g, h = oracle.cavity_problem(**w, xi=xi)
    t0 = time.time()
    g1, h1, _ = oracle.step(prob, g, h, steps)
    secs = time.time() - t0
    n = w["n"]
    mom = oracle.state_moments(prob, g1, h1).reshape(n, n, 4)
    rows = [(ix, iy, *mom[iy, ix]) for iy in SAMPLE for ix in SAMPLE]
    here = os.path.dirname(os.path.abspath(__file__))
    tag = f"cavity256_{steps}steps"
    header = (f"oracle state moments after {steps} of the {w['steps']} steps of {w['name']}, "
              f"dt={prob.cfg.dt!r}; {secs:.0f} s on {oracle.threads()} threads\n"
              "ix iy n ux uy theta")
    np.savetxt(os.path.join(here, tag + "_moments.txt"), np.array(rows),
               fmt=["%d", "%d"] + ["%.17g"] * 4, header=header)
    fl = oracle.wall_fluxes(prob, g1, h1, oracle.YHI)
    J = oracle.lid_shear(prob, g1, h1)
    side = prob.meta["side"]
    mass = float(g1.sum()) * oracle.dv(prob.cfg) * (side / n) ** 2
    lid = np.column_stack([np.arange(n), *fl])
    np.savetxt(os.path.join(here, tag + "_lid.txt"), lid, fmt=["%d"] + ["%.17g"] * 4,
               header=(f"oracle lid (y = L) wall fluxes per face cell after {steps} steps of "
                       f"{w['name']}\nJ {J!r}\nmass {mass!r}\nix mass shear normal energy"))
    print(f"{tag}: {secs:.0f} s, J = {J!r}, mass = {mass!r}")


if __name__ == "__main__":
    main(int(sys.argv[1]) if len(sys.argv) > 1 else 2000)
