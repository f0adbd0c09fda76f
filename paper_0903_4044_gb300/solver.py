"""A small object wrapper over the C ABI plus builders for the paper's two problems.

The builders turn raw workload parameters (``workloads.py``) into a
``bgk_config``: the 1D normal shock of Sec. 4.1 (domain [-L/2, L/2],
Rankine-Hugoniot end states as inflow boundary values, step initial profile)
and the lid-driven cavity of Sec. 5.1 (side 1/Kn mean free paths, isothermal
diffuse walls, lid speed U_W = Ma sqrt(gamma/2) along +x, perturbed resting
Maxwellian initial state).
"""
from __future__ import annotations

import math

import numpy as np

from . import bgk as B

GAMMA = 5.0 / 3.0  # monatomic gas


class Solver:
    """Owns one ``bgk_solver`` handle; frees it on close()/context exit."""

    def __init__(self, cfg: B.bgk_config):
        self.cfg = cfg
        self.h = B.bgk_create(cfg)
        self.info = B.bgk_get_info(self.h)
        self.ncell = int(self.info.ncell)
        self.nv = int(self.info.nv)

    # lifetime
    def close(self) -> None:
        if self.h:
            B.bgk_destroy(self.h)
            self.h = 0

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # state
    def init_step(self, x_split, left, right) -> None:
        B.bgk_init_maxwellian_step(self.h, x_split, left, right)

    def init_uniform(self, state, xi=None, amplitude=0.0) -> None:
        B.bgk_init_uniform(self.h, state, xi, amplitude)

    def set_state(self, f) -> None:
        B.bgk_set_state(self.h, f)

    def get_state(self, out=None):
        if out is None:
            out = np.empty((self.ncell, self.nv, 2))
        B.bgk_get_state(self.h, out)
        return out

    # stepping and outputs
    def step(self, n: int) -> None:
        B.bgk_step(self.h, n)

    def sync(self) -> None:
        B.bgk_sync(self.h)

    def moments(self, which: int = 0, out=None):
        if out is None:
            out = np.empty((self.ncell, 4))
        B.bgk_moments(self.h, out, which)
        return out

    def wall_fluxes(self, face: int, out=None):
        n = (self.cfg.ny if face in (B.BGK_FACE_XLO, B.BGK_FACE_XHI) else self.cfg.nx)
        if out is None:
            out = np.empty((n, 4))
        B.bgk_wall_fluxes(self.h, face, out)
        return out

    def lid_shear(self) -> float:
        """Lid-integrated shear of the current state (bgk_lid_shear)."""
        return B.bgk_lid_shear(self.h)

    @property
    def dt(self) -> float:
        return self.info.dt


def shock_config(*, mach, nx, length, nvx, vx, omega, cfl, conservative=1, relax_exact=1,
                 precision=B.BGK_F64, tile_cells=0, stream=None, **_ignored):
    """(cfg, up, down) for the Sec. 4.1 normal shock."""
    up, down = B.bgk_rankine_hugoniot(mach, GAMMA)
    bc = [(B.BGK_BC_INFLOW, *up), (B.BGK_BC_INFLOW, *down)]
    cfg = B.make_config(dim=1, nx=nx, ny=1, x0=-0.5 * length, lx=length, nvx=nvx, nvy=1, vx=vx,
                        omega=omega, cfl=cfl, conservative=conservative, relax_exact=relax_exact,
                        precision=precision, tile_cells=tile_cells, bc=bc, stream=stream)
    return cfg, up, down


def cavity_config(*, kn, lid_mach=None, n, nv, vbox, omega, cfl, conservative=1, relax_exact=1,
                  precision=B.BGK_F64, wall="diffuse", tile_cells=0, stream=None, lid_speed=None,
                  **_ignored):
    """cfg for the Sec. 5.1 lid-driven cavity (lid at y = L moving along +x);
    ``lid_speed`` (units of sqrt(2 R T0)) overrides the one derived from Mach."""
    side = 1.0 / kn
    uw = lid_mach * math.sqrt(GAMMA / 2.0) if lid_speed is None else lid_speed
    kind = B.BGK_BC_DIFFUSE if wall == "diffuse" else B.BGK_BC_SPECULAR
    rest = (kind, 1.0, 0.0, 0.0, 1.0)
    lid = (kind, 1.0, uw, 0.0, 1.0)
    return B.make_config(dim=2, nx=n, ny=n, lx=side, ly=side, nvx=nv, nvy=nv, vx=vbox, vy=vbox,
                         omega=omega, cfl=cfl, conservative=conservative, relax_exact=relax_exact,
                         precision=precision, tile_cells=tile_cells, bc=[rest, rest, rest, lid],
                         stream=stream)


def make_shock(w: dict, stream=None, **over) -> Solver:
    """Solver for a shock workload, initialised with the step profile at x = 0."""
    cfg, up, down = shock_config(**{**w, **over}, stream=stream)
    s = Solver(cfg)
    s.init_step(0.0, up, down)
    s.up, s.down = up, down
    return s


def make_cavity(w: dict, xi=None, stream=None, **over) -> Solver:
    """Solver for a cavity workload, initialised to the resting Maxwellian
    times (1 + amp*xi) (xi in the state layout, host array or CUDA tensor)."""
    p = {**w, **over}
    s = Solver(cavity_config(**p, stream=stream))
    s.init_uniform((1.0, 0.0, 0.0, 1.0), xi, p.get("amp", 0.0) if xi is not None else 0.0)
    return s


PRECISIONS = {"f64": B.BGK_F64, "f32": B.BGK_F32, "bf16": B.BGK_BF16_DEV}


def instance_config(w: dict, stream=None):
    """bgk_config of one raw workload entry (cavity or shock), with its precision."""
    prec = PRECISIONS[w.get("precision", "f64")] if isinstance(w.get("precision"), str) else w.get("precision", 0)
    p = {**w, "precision": prec}
    if w["kind"] == "shock":
        return shock_config(**p, stream=stream)[0]
    return cavity_config(**p, stream=stream)


class Batch:
    """Owns a bgk_batch of instances built from raw workload entries and
    initialised like make_shock / make_cavity (cavities perturbed from their
    own seeds)."""

    def __init__(self, ws: list[dict], stream=None, perturb=True):
        from . import workloads as W

        self.ws = ws
        self.cfgs = [instance_config(w, stream) for w in ws]
        self.h = B.bgk_batch_create(self.cfgs, stream)
        self.solvers = []
        for i, w in enumerate(ws):
            s = Solver.__new__(Solver)
            s.cfg = self.cfgs[i]
            s.h = B.bgk_batch_solver(self.h, i)
            s.info = B.bgk_get_info(s.h)
            s.ncell, s.nv = int(s.info.ncell), int(s.info.nv)
            s.close = lambda: None          # owned by the batch
            if w["kind"] == "shock":
                up, down = B.bgk_rankine_hugoniot(w["mach"], GAMMA)
                s.init_step(0.0, up, down)
            else:
                xi = W.perturbation(w.get("seed", 0), s.ncell, s.nv) if perturb else None
                s.init_uniform((1.0, 0.0, 0.0, 1.0), xi, w.get("amp", 0.0) if perturb else 0.0)
            self.solvers.append(s)

    def step(self, n: int) -> None:
        B.bgk_batch_step(self.h, n)

    def sync(self) -> None:
        B.bgk_batch_sync(self.h)

    def autotune(self, trial_steps: int = 4) -> None:
        B.bgk_batch_autotune(self.h, trial_steps)
        for s in self.solvers:
            s.info = B.bgk_get_info(s.h)

    def set_persistent(self, enable: bool = True, timeout_s: float = 5.0) -> None:
        """One cooperative launch per step() call (FP32 instances only)."""
        B.bgk_batch_set_persistent(self.h, enable, timeout_s)
        for s in self.solvers:
            s.info = B.bgk_get_info(s.h)

    def points(self) -> int:
        return sum(s.ncell * s.nv for s in self.solvers)

    def close(self) -> None:
        if self.h:
            B.bgk_batch_destroy(self.h)
            self.h = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Solver3v:
    """Owns one ``bgk3v_solver`` (full 3D velocity grid, one spatial dimension)."""

    def __init__(self, cfg: B.bgk3v_config):
        self.cfg = cfg
        self.h = B.bgk3v_create(cfg)
        self.info = B.bgk3v_get_info(self.h)
        self.ncell = int(self.info.ncell)
        self.nv = int(self.info.nv)

    def close(self) -> None:
        if self.h:
            B.bgk3v_destroy(self.h)
            self.h = 0

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init_step(self, x_split, left, right) -> None:
        B.bgk3v_init_step(self.h, x_split, left, right)

    def set_state(self, f) -> None:
        B.bgk3v_set_state(self.h, f)

    def get_state(self, out=None):
        if out is None:
            out = np.empty((self.ncell, self.nv))
        B.bgk3v_get_state(self.h, out)
        return out

    def step(self, n: int) -> None:
        B.bgk3v_step(self.h, n)

    def sync(self) -> None:
        B.bgk3v_sync(self.h)

    def moments(self, which: int = 0, out=None):
        if out is None:
            out = np.empty((self.ncell, 5))
        B.bgk3v_moments(self.h, out, which)
        return out

    @property
    def dt(self) -> float:
        return self.info.dt


def shock3v_config(*, mach, nx, length, nv, vx, vt, omega, dt, conservative=1, relax_exact=1, stream=None,
                   **_ignored):
    """(cfg, up, down) for the Sec. 4.1 shock on the full velocity grid
    nv = (N_vx, N_vy, N_vz) over vx x vt x vt with a fixed time step."""
    up4, down4 = B.bgk_rankine_hugoniot(mach, GAMMA)
    up = (up4[0], up4[1], 0.0, 0.0, up4[3])
    down = (down4[0], down4[1], 0.0, 0.0, down4[3])
    cfg = B.make_config3v(nx=nx, x0=-0.5 * length, lx=length, nv=nv, vmin=(vx[0], vt[0], vt[0]),
                          vmax=(vx[1], vt[1], vt[1]), omega=omega, dt=dt, conservative=conservative,
                          relax_exact=relax_exact, inflow=(up, down), stream=stream)
    return cfg, up, down


def make_shock3v(w: dict, stream=None, **over) -> Solver3v:
    cfg, up, down = shock3v_config(**{**w, **over}, stream=stream)
    s = Solver3v(cfg)
    s.init_step(0.0, up, down)
    s.up, s.down = up, down
    return s
