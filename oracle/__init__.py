"""Plain FP64 CPU oracle of the BGK phase-space step (ctypes wrapper).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline legs of ``bench.py`` may import this package.  It shares no code
with ``paper_0903_4044_gb300``: the arithmetic lives in ``bgk_oracle.c``, which
restates the paper (Frezzotti, Ghiroldi, Gibelli, "Solving Kinetic Equations on
GPUs I") section by section, and the few workload derivations below (domain
length from Kn, lid speed from the Mach number, time step from the Courant
number) are written here again on purpose.

Layout of the oracle's state: ``g`` and ``h`` are float64 arrays of shape
``(ncell, nv)`` with ``cell = iy*nx + ix`` and ``v = jy*nvx + jx``.

Every function is pinned by ``tests/test_oracle_pins.py`` against closed
forms, invariants and brute-force sums; see that file for which pin covers
which function.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bgk_oracle.c")
_SRCS = [_SRC, os.path.join(_HERE, "bgk_oracle3v.c")]
_HDRS = [os.path.join(_HERE, "bgk_oracle.h"), os.path.join(_HERE, "bgk_oracle3v.h")]
_LIB_PATH = os.path.join(_HERE, "liboracle.so")

BC_INFLOW, BC_DIFFUSE, BC_SPECULAR = 0, 1, 2
XLO, XHI, YLO, YHI = 0, 1, 2, 3
GAMMA = 5.0 / 3.0  # monatomic gas (Sec. 4.1)


def build(force: bool = False) -> str:
    """Compile the oracle's C sources into ``liboracle.so`` (gcc, OpenMP, no FMA contraction)."""
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= max(
        os.path.getmtime(f) for f in _SRCS + _HDRS
    ):
        return _LIB_PATH
    cmd = [
        "gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
        "-ffp-contract=off", "-fno-fast-math", "-Wall",
        *_SRCS, "-o", _LIB_PATH + ".tmp", "-lm",
    ]
    subprocess.run(cmd, check=True)
    os.replace(_LIB_PATH + ".tmp", _LIB_PATH)
    return _LIB_PATH


class OrcConfig(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("x0", ctypes.c_double), ("lx", ctypes.c_double),
        ("y0", ctypes.c_double), ("ly", ctypes.c_double),
        ("nvx", ctypes.c_int), ("nvy", ctypes.c_int),
        ("vx_min", ctypes.c_double), ("vx_max", ctypes.c_double),
        ("vy_min", ctypes.c_double), ("vy_max", ctypes.c_double),
        ("omega", ctypes.c_double), ("dt", ctypes.c_double),
        ("conservative", ctypes.c_int), ("relax_exact", ctypes.c_int),
        ("bc_kind", ctypes.c_int * 4), ("bc_state", (ctypes.c_double * 4) * 4),
    ]


class Orc3Config(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("x0", ctypes.c_double), ("lx", ctypes.c_double),
        ("nvx", ctypes.c_int), ("nvy", ctypes.c_int), ("nvz", ctypes.c_int),
        ("vmin", ctypes.c_double * 3), ("vmax", ctypes.c_double * 3),
        ("omega", ctypes.c_double), ("dt", ctypes.c_double),
        ("conservative", ctypes.c_int), ("relax_exact", ctypes.c_int),
        ("inflow", (ctypes.c_double * 5) * 2),
    ]


_lib = None
_D = ctypes.POINTER(ctypes.c_double)
_C = ctypes.POINTER(OrcConfig)


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        L.orc_nv.argtypes = [_C]
        L.orc_ncell.argtypes = [_C]
        L.orc_cx.argtypes = [_C, ctypes.c_int]
        L.orc_cx.restype = ctypes.c_double
        L.orc_cy.argtypes = [_C, ctypes.c_int]
        L.orc_cy.restype = ctypes.c_double
        L.orc_dv.argtypes = [_C]
        L.orc_dv.restype = ctypes.c_double
        L.orc_dt_from_cfl.argtypes = [_C, ctypes.c_double]
        L.orc_dt_from_cfl.restype = ctypes.c_double
        L.orc_maxwellian.argtypes = [_C, _D, _D, _D]
        L.orc_moments.argtypes = [_C, _D, _D, _D]
        L.orc_effective_params.argtypes = [_C, _D, _D]
        L.orc_rankine_hugoniot.argtypes = [ctypes.c_double, ctypes.c_double, _D, _D]
        L.orc_init_step.argtypes = [_C, ctypes.c_double, _D, _D, _D, _D]
        L.orc_init_uniform.argtypes = [_C, _D, _D, ctypes.c_double, _D, _D]
        L.orc_stream.argtypes = [_C, _D, _D, _D, _D]
        L.orc_relax.argtypes = [_C, _D, _D, _D]
        L.orc_step.argtypes = [_C, _D, _D, ctypes.c_long, _D]
        L.orc_set_threads.argtypes = [ctypes.c_int]
        L.orc_set_threads.restype = None
        L.orc_wall_fluxes.argtypes = [_C, _D, _D, ctypes.c_int, _D, _D, _D, _D]
        L.orc_threads.argtypes = []
        L.orc_lid_shear.argtypes = [_C, _D, _D]
        L.orc_lid_shear.restype = ctypes.c_double
        L.orc_adjoint_lid_shear.argtypes = [_C, _D, _D, ctypes.c_long, _D, _D, _D]
        C3 = ctypes.POINTER(Orc3Config)
        L.orc3_nv.argtypes = [C3]
        L.orc3_c.argtypes = [C3, ctypes.c_int, ctypes.c_int]
        L.orc3_c.restype = ctypes.c_double
        L.orc3_dv.argtypes = [C3]
        L.orc3_dv.restype = ctypes.c_double
        L.orc3_dt_from_cfl.argtypes = [C3, ctypes.c_double]
        L.orc3_dt_from_cfl.restype = ctypes.c_double
        L.orc3_maxwellian.argtypes = [C3, _D, _D]
        L.orc3_moments.argtypes = [C3, _D, _D]
        L.orc3_effective_params.argtypes = [C3, _D, _D]
        L.orc3_init_step.argtypes = [C3, ctypes.c_double, _D, _D, _D]
        L.orc3_stream.argtypes = [C3, _D, _D]
        L.orc3_relax.argtypes = [C3, _D, _D]
        L.orc3_step.argtypes = [C3, _D, ctypes.c_long, _D]
        _lib = L
    return _lib


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_D)


def _vec(x) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x, dtype=np.float64))


@dataclass
class Problem:
    """A configured problem: the oracle's config plus its derived workload values."""

    cfg: OrcConfig
    steps: int = 0
    meta: dict = field(default_factory=dict)

    @property
    def nv(self) -> int:
        return lib().orc_nv(ctypes.byref(self.cfg))

    @property
    def ncell(self) -> int:
        return lib().orc_ncell(ctypes.byref(self.cfg))

    def zeros(self) -> tuple[np.ndarray, np.ndarray]:
        return np.zeros((self.ncell, self.nv)), np.zeros((self.ncell, self.nv))


def make_config(*, dim, nx, ny=1, x0=0.0, lx=1.0, y0=0.0, ly=1.0, nvx, nvy=1,
                vx=(-1.0, 1.0), vy=(-1.0, 1.0), omega=0.5, dt=0.0, cfl=None,
                conservative=1, relax_exact=1, bc_kind=(0, 0, 0, 0),
                bc_state=((1, 0, 0, 1),) * 4) -> OrcConfig:
    c = OrcConfig()
    c.dim, c.nx, c.ny = dim, nx, (ny if dim == 2 else 1)
    c.x0, c.lx, c.y0, c.ly = x0, lx, y0, ly
    c.nvx, c.nvy = nvx, (nvy if dim == 2 else 1)
    c.vx_min, c.vx_max = vx
    c.vy_min, c.vy_max = vy
    c.omega, c.dt = omega, dt
    c.conservative, c.relax_exact = conservative, relax_exact
    for k in range(4):
        c.bc_kind[k] = bc_kind[k]
        for m in range(4):
            c.bc_state[k][m] = float(bc_state[k][m])
    if cfl is not None:
        c.dt = lib().orc_dt_from_cfl(ctypes.byref(c), cfl)
    return c


# --- grids ---------------------------------------------------------------
def velocities(cfg: OrcConfig) -> tuple[np.ndarray, np.ndarray]:
    """(cx, cy) per velocity index v = jy*nvx + jx."""
    L = lib()
    nv = L.orc_nv(ctypes.byref(cfg))
    cx = np.array([L.orc_cx(ctypes.byref(cfg), v % cfg.nvx) for v in range(nv)])
    cy = np.array([L.orc_cy(ctypes.byref(cfg), v // cfg.nvx) for v in range(nv)])
    return cx, cy


def dv(cfg: OrcConfig) -> float:
    return lib().orc_dv(ctypes.byref(cfg))


# --- per-cell functions --------------------------------------------------
def maxwellian(cfg: OrcConfig, p) -> tuple[np.ndarray, np.ndarray]:
    nv = lib().orc_nv(ctypes.byref(cfg))
    G, H = np.zeros(nv), np.zeros(nv)
    lib().orc_maxwellian(ctypes.byref(cfg), _p(_vec(p)), _p(G), _p(H))
    return G, H


def moments(cfg: OrcConfig, g: np.ndarray, h: np.ndarray) -> np.ndarray:
    """Moments (n, ux, uy, theta) of every cell: shape (ncell, 4)."""
    g2 = np.ascontiguousarray(np.atleast_2d(g), dtype=np.float64)
    h2 = np.ascontiguousarray(np.atleast_2d(h), dtype=np.float64)
    out = np.zeros((g2.shape[0], 4))
    for k in range(g2.shape[0]):
        o = np.zeros(4)
        lib().orc_moments(ctypes.byref(cfg), _p(np.ascontiguousarray(g2[k])),
                          _p(np.ascontiguousarray(h2[k])), _p(o))
        out[k] = o
    return out


def effective_params(cfg: OrcConfig, q) -> tuple[np.ndarray, int]:
    out = np.zeros(4)
    it = lib().orc_effective_params(ctypes.byref(cfg), _p(_vec(q)), _p(out))
    return out, it


def rankine_hugoniot(mach: float, gamma: float = GAMMA) -> tuple[np.ndarray, np.ndarray]:
    up, down = np.zeros(4), np.zeros(4)
    lib().orc_rankine_hugoniot(mach, gamma, _p(up), _p(down))
    return up, down


# --- whole-grid functions ------------------------------------------------
def init_step(prob: Problem, x_split, left, right):
    g, h = prob.zeros()
    lib().orc_init_step(ctypes.byref(prob.cfg), x_split, _p(_vec(left)), _p(_vec(right)), _p(g), _p(h))
    return g, h


def init_uniform(prob: Problem, state, xi=None, amp=0.0):
    g, h = prob.zeros()
    xp = _p(_vec(xi)) if xi is not None else None
    lib().orc_init_uniform(ctypes.byref(prob.cfg), _p(_vec(state)), xp, amp, _p(g), _p(h))
    return g, h


def stream(prob: Problem, g, h):
    gt, ht = prob.zeros()
    rc = lib().orc_stream(ctypes.byref(prob.cfg), _p(g), _p(h), _p(gt), _p(ht))
    if rc != 0:
        raise RuntimeError("oracle streaming failed")
    return gt, ht


def relax(prob: Problem, g, h):
    """Collision sub-step on copies; returns (g', h', moments of the input)."""
    g2, h2 = g.copy(), h.copy()
    mom = np.zeros((prob.ncell, 4))
    rc = lib().orc_relax(ctypes.byref(prob.cfg), _p(g2), _p(h2), _p(mom))
    if rc != 0:
        raise RuntimeError("oracle relaxation met a non-physical state")
    return g2, h2, mom


def step(prob: Problem, g, h, nsteps: int):
    """nsteps full steps on copies; returns (g, h, moments of the last f~)."""
    g2, h2 = g.copy(), h.copy()
    mom = np.zeros((prob.ncell, 4))
    rc = lib().orc_step(ctypes.byref(prob.cfg), _p(g2), _p(h2), nsteps, _p(mom))
    if rc != 0:
        raise RuntimeError("oracle step failed")
    return g2, h2, mom


def state_moments(prob: Problem, g, h) -> np.ndarray:
    return moments(prob.cfg, g, h)


def wall_fluxes(prob: Problem, g, h, face: int):
    nf = prob.cfg.ny if face in (XLO, XHI) else prob.cfg.nx
    if prob.cfg.dim == 1 and face in (XLO, XHI):
        nf = 1
    out = [np.zeros(nf) for _ in range(4)]
    rc = lib().orc_wall_fluxes(ctypes.byref(prob.cfg), _p(g), _p(h), face, *[_p(o) for o in out])
    if rc != 0:
        raise RuntimeError("oracle wall fluxes failed")
    return out


def lid_shear(prob: Problem, g, h) -> float:
    """Objective of the adjoint: lid-integrated shear of the state."""
    return lib().orc_lid_shear(ctypes.byref(prob.cfg), _p(g), _p(h))


def adjoint_lid_shear(prob: Problem, g, h, nsteps: int):
    """CPU reverse pass: (J, dJ/dlnL, dJ/dU_W, dJ/dg0, dJ/dh0) after nsteps."""
    dg, dh = prob.zeros()
    out = np.zeros(3)
    rc = lib().orc_adjoint_lid_shear(ctypes.byref(prob.cfg), _p(np.ascontiguousarray(g)),
                                     _p(np.ascontiguousarray(h)), nsteps, _p(dg), _p(dh), _p(out))
    if rc != 0:
        raise RuntimeError("oracle adjoint failed")
    return out[0], out[1], out[2], dg, dh


def threads() -> int:
    return lib().orc_threads()


def set_threads(n: int) -> None:
    """Threads of the oracle's OpenMP loops from now on."""
    lib().orc_set_threads(int(n))


# --- the two problems of the paper, from raw workload parameters ---------
def shock_problem(*, mach, nx, length, nvx, vx, omega, cfl, steps, conservative=1,
                  relax_exact=1, **_ignored) -> tuple[Problem, np.ndarray, np.ndarray]:
    """Sec. 4.1: domain [-L/2, L/2], Rankine-Hugoniot end states held as inflow
    boundary values, initial step profile at x = 0.  Returns (problem, g0, h0)."""
    up, down = rankine_hugoniot(mach)
    cfg = make_config(dim=1, nx=nx, x0=-0.5 * length, lx=length, nvx=nvx, vx=vx,
                      omega=omega, cfl=cfl, conservative=conservative,
                      relax_exact=relax_exact, bc_kind=(BC_INFLOW, BC_INFLOW, 0, 0),
                      bc_state=(up, down, up, up))
    prob = Problem(cfg, steps, {"up": up, "down": down})
    g, h = init_step(prob, 0.0, up, down)
    return prob, g, h


def cavity_problem(*, kn, lid_mach, n, nv, vbox, omega, cfl, steps, xi=None, amp=0.0,
                   conservative=1, relax_exact=1, wall="diffuse",
                   **_ignored) -> tuple[Problem, np.ndarray, np.ndarray]:
    """Sec. 5.1: square cavity of side 1/Kn mean free paths, isothermal walls at
    theta = 1, lid (y = L) moving along +x at U_W = Ma sqrt(gamma/2).  The
    initial state is the resting Maxwellian (n = 1, theta = 1) times
    (1 + amp*xi).  Returns (problem, g0, h0)."""
    side = 1.0 / kn
    uw = lid_mach * math.sqrt(GAMMA / 2.0)
    kind = BC_DIFFUSE if wall == "diffuse" else BC_SPECULAR
    rest = (1.0, 0.0, 0.0, 1.0)
    lid = (1.0, uw, 0.0, 1.0)
    cfg = make_config(dim=2, nx=n, ny=n, lx=side, ly=side, nvx=nv, nvy=nv, vx=vbox, vy=vbox,
                      omega=omega, cfl=cfl, conservative=conservative,
                      relax_exact=relax_exact, bc_kind=(kind,) * 4,
                      bc_state=(rest, rest, rest, lid))
    prob = Problem(cfg, steps, {"uw": uw, "side": side})
    g, h = init_uniform(prob, rest, xi, amp)
    return prob, g, h



# --- full 3D velocity grid, one spatial dimension (bgk_oracle3v.c) -------
@dataclass
class Problem3v:
    """A configured full-velocity-grid problem: the oracle's config and derived values."""

    cfg: Orc3Config
    steps: int = 0
    meta: dict = field(default_factory=dict)

    @property
    def nv(self) -> int:
        return lib().orc3_nv(ctypes.byref(self.cfg))

    @property
    def ncell(self) -> int:
        return self.cfg.nx

    def zeros(self) -> np.ndarray:
        return np.zeros((self.ncell, self.nv))


def make_config3v(*, nx, x0=0.0, lx=1.0, nv=(8, 8, 8), vmin=(-1.0, -1.0, -1.0), vmax=(1.0, 1.0, 1.0),
                  omega=0.5, dt=0.0, cfl=None, conservative=1, relax_exact=1,
                  inflow=((1, 0, 0, 0, 1), (1, 0, 0, 0, 1))) -> Orc3Config:
    c = Orc3Config()
    c.nx, c.x0, c.lx = nx, x0, lx
    c.nvx, c.nvy, c.nvz = nv
    for k in range(3):
        c.vmin[k], c.vmax[k] = vmin[k], vmax[k]
    c.omega, c.conservative, c.relax_exact = omega, conservative, relax_exact
    for s in range(2):
        for k in range(5):
            c.inflow[s][k] = inflow[s][k]
    c.dt = dt if cfl is None else lib().orc3_dt_from_cfl(ctypes.byref(c), cfl)
    return c


def velocities3v(prob: Problem3v):
    L, c = lib(), ctypes.byref(prob.cfg)
    n = (prob.cfg.nvx, prob.cfg.nvy, prob.cfg.nvz)
    return [np.array([L.orc3_c(c, a, j) for j in range(n[a])]) for a in range(3)]


def maxwellian3v(prob: Problem3v, p) -> np.ndarray:
    out = np.zeros(prob.nv)
    lib().orc3_maxwellian(ctypes.byref(prob.cfg), _p(_vec(p)), _p(out))
    return out


def moments3v(prob: Problem3v, f) -> np.ndarray:
    out = np.zeros(5)
    lib().orc3_moments(ctypes.byref(prob.cfg), _p(np.ascontiguousarray(f, dtype=np.float64)), _p(out))
    return out


def state_moments3v(prob: Problem3v, f) -> np.ndarray:
    return np.array([moments3v(prob, f[i]) for i in range(prob.ncell)])


def effective_params3v(prob: Problem3v, q):
    out = np.zeros(5)
    it = lib().orc3_effective_params(ctypes.byref(prob.cfg), _p(_vec(q)), _p(out))
    return it, out


def init_step3v(prob: Problem3v, x_split, left, right) -> np.ndarray:
    f = prob.zeros()
    lib().orc3_init_step(ctypes.byref(prob.cfg), x_split, _p(_vec(left)), _p(_vec(right)), _p(f))
    return f


def stream3v(prob: Problem3v, f) -> np.ndarray:
    ft = prob.zeros()
    lib().orc3_stream(ctypes.byref(prob.cfg), _p(np.ascontiguousarray(f)), _p(ft))
    return ft


def relax3v(prob: Problem3v, f):
    f = np.array(f, dtype=np.float64, copy=True)
    mom = np.zeros((prob.ncell, 5))
    if lib().orc3_relax(ctypes.byref(prob.cfg), _p(f), _p(mom)) != 0:
        raise RuntimeError("oracle relaxation failed")
    return f, mom


def step3v(prob: Problem3v, f, nsteps: int):
    f = np.array(f, dtype=np.float64, copy=True)
    mom = np.zeros((prob.ncell, 5))
    if lib().orc3_step(ctypes.byref(prob.cfg), _p(f), nsteps, _p(mom)) != 0:
        raise RuntimeError("oracle step failed")
    return f, mom


def shock3v_problem(*, mach, nx, length, nv, vx, vt, omega, dt, steps=0, conservative=1, relax_exact=1,
                    **_ignored) -> tuple[Problem3v, np.ndarray]:
    """Sec. 4.1 as the paper computed it: domain [-L/2, L/2], full velocity grid
    nv = (N_vx, N_vy, N_vz) on vx x vt x vt, fixed time step, Rankine-Hugoniot
    inflow states, step profile at x = 0.  Returns (problem, f0)."""
    up, down = rankine_hugoniot(mach)
    u5 = (up[0], up[1], 0.0, 0.0, up[3])
    d5 = (down[0], down[1], 0.0, 0.0, down[3])
    cfg = make_config3v(nx=nx, x0=-0.5 * length, lx=length, nv=nv, vmin=(vx[0], vt[0], vt[0]),
                        vmax=(vx[1], vt[1], vt[1]), omega=omega, dt=dt, conservative=conservative,
                        relax_exact=relax_exact, inflow=(u5, d5))
    prob = Problem3v(cfg, steps, {"up": u5, "down": d5})
    return prob, init_step3v(prob, 0.0, u5, d5)
