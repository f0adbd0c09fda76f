"""ctypes binding of libbgk.so (include/bgk.h): argument marshalling only.

Every step of the method runs in the library's CUDA kernels; this module
converts Python values to the C structs, passes pointers (numpy host arrays
or torch CUDA tensors) and raises :class:`BgkError` on a non-OK status.  The
functions keep the C names.  There is no CPU fallback: if ``libbgk.so`` is
missing or cannot load, :func:`lib` raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libbgk.so")

BGK_OK, BGK_ERR_INVALID_ARG, BGK_ERR_UNSUPPORTED, BGK_ERR_OOM = 0, 1, 2, 3
BGK_ERR_CUDA, BGK_ERR_NUMERIC, BGK_ERR_TIMEOUT = 4, 5, 6
BGK_F64, BGK_F32, BGK_BF16_DEV = 0, 1, 2
BGK_BC_INFLOW, BGK_BC_DIFFUSE, BGK_BC_SPECULAR = 0, 1, 2
BGK_FACE_XLO, BGK_FACE_XHI, BGK_FACE_YLO, BGK_FACE_YHI = 0, 1, 2, 3

# Names of every entry point declared in include/bgk.h.
EXPORTS = (
    "bgk_create", "bgk_destroy", "bgk_get_info", "bgk_init_maxwellian_step", "bgk_init_uniform",
    "bgk_set_state", "bgk_get_state", "bgk_step", "bgk_moments", "bgk_wall_fluxes", "bgk_sync",
    "bgk_rankine_hugoniot", "bgk_last_error", "bgk_status_string", "bgk_abi_version",
    "bgk_step_noalloc", "bgk_batch_create", "bgk_batch_solver", "bgk_batch_step", "bgk_batch_sync",
    "bgk_batch_destroy", "bgk_autotune", "bgk_batch_autotune", "bgk_adjoint_lid_shear",
    "bgk3v_create", "bgk3v_destroy", "bgk3v_get_info", "bgk3v_init_step", "bgk3v_set_state",
    "bgk3v_get_state", "bgk3v_step", "bgk3v_moments", "bgk3v_sync", "bgk_batch_set_persistent",
    "bgk_lid_shear",
)


class BgkError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        super().__init__(f"{where}: status {status}: {message}")
        self.status = status


class bgk_bc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("reserved", ctypes.c_int32), ("n", ctypes.c_double),
                ("ux", ctypes.c_double), ("uy", ctypes.c_double), ("theta", ctypes.c_double)]


class bgk_config(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int32), ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
        ("nvx", ctypes.c_int32), ("nvy", ctypes.c_int32), ("conservative", ctypes.c_int32),
        ("relax_exact", ctypes.c_int32), ("precision", ctypes.c_int32),
        ("tile_cells", ctypes.c_int32), ("reserved0", ctypes.c_int32),
        ("x0", ctypes.c_double), ("lx", ctypes.c_double), ("y0", ctypes.c_double), ("ly", ctypes.c_double),
        ("vx_min", ctypes.c_double), ("vx_max", ctypes.c_double),
        ("vy_min", ctypes.c_double), ("vy_max", ctypes.c_double),
        ("omega", ctypes.c_double), ("dt", ctypes.c_double), ("cfl", ctypes.c_double),
        ("bc", bgk_bc * 4), ("cuda_stream", ctypes.c_void_p),
    ]


class bgk_info(ctypes.Structure):
    _fields_ = [
        ("dt", ctypes.c_double), ("dx", ctypes.c_double), ("dy", ctypes.c_double),
        ("dcx", ctypes.c_double), ("dcy", ctypes.c_double), ("dv", ctypes.c_double),
        ("max_courant", ctypes.c_double), ("ncell", ctypes.c_int64), ("nv", ctypes.c_int64),
        ("state_doubles", ctypes.c_int64), ("steps_done", ctypes.c_int64),
        ("device_bytes", ctypes.c_int64), ("precision", ctypes.c_int32), ("tile_cells", ctypes.c_int32),
    ]


_lib = None
class bgk3v_config(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("nvx", ctypes.c_int32), ("nvy", ctypes.c_int32),
                ("nvz", ctypes.c_int32), ("conservative", ctypes.c_int32), ("relax_exact", ctypes.c_int32),
                ("reserved0", ctypes.c_int32), ("reserved1", ctypes.c_int32),
                ("x0", ctypes.c_double), ("lx", ctypes.c_double),
                ("vmin", ctypes.c_double * 3), ("vmax", ctypes.c_double * 3),
                ("omega", ctypes.c_double), ("dt", ctypes.c_double), ("cfl", ctypes.c_double),
                ("inflow", (ctypes.c_double * 5) * 2), ("cuda_stream", ctypes.c_void_p)]


class bgk3v_info(ctypes.Structure):
    _fields_ = [("dt", ctypes.c_double), ("dx", ctypes.c_double), ("dv", ctypes.c_double),
                ("max_courant", ctypes.c_double), ("ncell", ctypes.c_int64), ("nv", ctypes.c_int64),
                ("steps_done", ctypes.c_int64), ("device_bytes", ctypes.c_int64)]


_P = ctypes.c_void_p
_D4 = ctypes.c_double * 4
_D5 = ctypes.c_double * 5


def lib() -> ctypes.CDLL:
    """Load libbgk.so (built by ``paper_0903_4044_gb300.build``); raise if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run __graft_entry__.build() (no CPU fallback exists)")
        L = ctypes.CDLL(LIB_PATH)
        sig = {
            "bgk_create": ([ctypes.POINTER(bgk_config), ctypes.POINTER(_P)], ctypes.c_int),
            "bgk_destroy": ([_P], ctypes.c_int),
            "bgk_get_info": ([_P, ctypes.POINTER(bgk_info)], ctypes.c_int),
            "bgk_init_maxwellian_step": ([_P, ctypes.c_double, _D4, _D4], ctypes.c_int),
            "bgk_init_uniform": ([_P, _D4, _P, ctypes.c_int, ctypes.c_double], ctypes.c_int),
            "bgk_set_state": ([_P, _P, ctypes.c_int], ctypes.c_int),
            "bgk_get_state": ([_P, _P, ctypes.c_int], ctypes.c_int),
            "bgk_step": ([_P, ctypes.c_int64], ctypes.c_int),
            "bgk_moments": ([_P, ctypes.c_int, _P, ctypes.c_int], ctypes.c_int),
            "bgk_wall_fluxes": ([_P, ctypes.c_int, _P, ctypes.c_int], ctypes.c_int),
            "bgk_sync": ([_P], ctypes.c_int),
            "bgk_lid_shear": ([_P, ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
            "bgk_rankine_hugoniot": ([ctypes.c_double, ctypes.c_double, _D4, _D4], ctypes.c_int),
            "bgk_last_error": ([], ctypes.c_char_p),
            "bgk_status_string": ([ctypes.c_int], ctypes.c_char_p),
            "bgk_abi_version": ([], ctypes.c_int),
            "bgk_step_noalloc": ([ctypes.POINTER(bgk_config), _P, _P, _P], ctypes.c_int),
            "bgk_batch_create": ([ctypes.POINTER(bgk_config), ctypes.c_int, _P, ctypes.POINTER(_P)], ctypes.c_int),
            "bgk_batch_solver": ([_P, ctypes.c_int, ctypes.POINTER(_P)], ctypes.c_int),
            "bgk_batch_step": ([_P, ctypes.c_int64], ctypes.c_int),
            "bgk_batch_sync": ([_P], ctypes.c_int),
            "bgk_batch_destroy": ([_P], ctypes.c_int),
            "bgk_autotune": ([_P, ctypes.c_int, ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
            "bgk_batch_autotune": ([_P, ctypes.c_int], ctypes.c_int),
            "bgk_adjoint_lid_shear": ([_P, ctypes.c_int64, ctypes.c_int, _P, ctypes.c_int, _D4], ctypes.c_int),
            "bgk3v_create": ([ctypes.POINTER(bgk3v_config), ctypes.POINTER(_P)], ctypes.c_int),
            "bgk3v_destroy": ([_P], ctypes.c_int),
            "bgk3v_get_info": ([_P, ctypes.POINTER(bgk3v_info)], ctypes.c_int),
            "bgk3v_init_step": ([_P, ctypes.c_double, _D5, _D5], ctypes.c_int),
            "bgk3v_set_state": ([_P, _P, ctypes.c_int], ctypes.c_int),
            "bgk3v_get_state": ([_P, _P, ctypes.c_int], ctypes.c_int),
            "bgk3v_step": ([_P, ctypes.c_int64], ctypes.c_int),
            "bgk3v_moments": ([_P, ctypes.c_int, _P, ctypes.c_int], ctypes.c_int),
            "bgk3v_sync": ([_P], ctypes.c_int),
            "bgk_batch_set_persistent": ([_P, ctypes.c_int, ctypes.c_double], ctypes.c_int),
        }
        for name, (args, res) in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


def _check(status: int, where: str) -> None:
    if status != BGK_OK:
        msg = lib().bgk_last_error().decode(errors="replace")
        raise BgkError(status, where, msg)


def _ptr(a) -> tuple[int, int]:
    """(address, on_device) of a C-contiguous float64 numpy array or torch tensor."""
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
            raise ValueError("host arrays must be C-contiguous float64")
        return a.ctypes.data, 0
    import torch

    if isinstance(a, torch.Tensor):
        if a.dtype != torch.float64 or not a.is_contiguous():
            raise ValueError("tensors must be contiguous float64")
        return a.data_ptr(), int(a.is_cuda)
    raise TypeError(f"unsupported buffer type {type(a)}")


# --- configuration ---------------------------------------------------------
def make_config(*, dim, nx, ny=1, x0=0.0, lx=1.0, y0=0.0, ly=1.0, nvx, nvy=1, vx=(-1.0, 1.0),
                vy=(-1.0, 1.0), omega=0.5, dt=0.0, cfl=0.0, conservative=1, relax_exact=1,
                precision=BGK_F64, tile_cells=0, bc=None, stream=None) -> bgk_config:
    """Fill a bgk_config.  ``bc`` is a sequence of up to four (kind, n, ux, uy, theta)."""
    c = bgk_config()
    c.dim, c.nx, c.ny, c.nvx, c.nvy = dim, nx, ny, nvx, nvy
    c.conservative, c.relax_exact, c.precision = conservative, relax_exact, precision
    c.tile_cells = tile_cells
    c.x0, c.lx, c.y0, c.ly = x0, lx, y0, ly
    c.vx_min, c.vx_max = vx
    c.vy_min, c.vy_max = vy
    c.omega, c.dt, c.cfl = omega, dt, cfl
    for k, b in enumerate(bc or ()):
        c.bc[k].kind = int(b[0])
        c.bc[k].n, c.bc[k].ux, c.bc[k].uy, c.bc[k].theta = (float(x) for x in b[1:5])
    c.cuda_stream = stream
    return c


# --- entry points (C names) -------------------------------------------------
def bgk_create(cfg: bgk_config) -> int:
    h = _P()
    _check(lib().bgk_create(ctypes.byref(cfg), ctypes.byref(h)), "bgk_create")
    return h.value


def bgk_destroy(h: int) -> None:
    _check(lib().bgk_destroy(h), "bgk_destroy")


def bgk_get_info(h: int) -> bgk_info:
    out = bgk_info()
    _check(lib().bgk_get_info(h, ctypes.byref(out)), "bgk_get_info")
    return out


def bgk_init_maxwellian_step(h: int, x_split: float, left, right) -> None:
    _check(lib().bgk_init_maxwellian_step(h, x_split, _D4(*left), _D4(*right)), "bgk_init_maxwellian_step")


def bgk_init_uniform(h: int, state, xi=None, amplitude: float = 0.0) -> None:
    addr, dev = _ptr(xi) if xi is not None else (None, 0)
    _check(lib().bgk_init_uniform(h, _D4(*state), addr, dev, amplitude), "bgk_init_uniform")


def bgk_set_state(h: int, f) -> None:
    addr, dev = _ptr(f)
    _check(lib().bgk_set_state(h, addr, dev), "bgk_set_state")


def bgk_get_state(h: int, out) -> None:
    addr, dev = _ptr(out)
    _check(lib().bgk_get_state(h, addr, dev), "bgk_get_state")


def bgk_step(h: int, nsteps: int) -> None:
    _check(lib().bgk_step(h, nsteps), "bgk_step")


def bgk_moments(h: int, out, which: int = 0) -> None:
    addr, dev = _ptr(out)
    _check(lib().bgk_moments(h, which, addr, dev), "bgk_moments")


def bgk_wall_fluxes(h: int, face: int, out) -> None:
    addr, dev = _ptr(out)
    _check(lib().bgk_wall_fluxes(h, face, addr, dev), "bgk_wall_fluxes")


def bgk_lid_shear(h: int) -> float:
    J = ctypes.c_double()
    _check(lib().bgk_lid_shear(h, ctypes.byref(J)), "bgk_lid_shear")
    return J.value


def bgk_sync(h: int) -> None:
    _check(lib().bgk_sync(h), "bgk_sync")


def bgk_rankine_hugoniot(mach: float, gamma: float = 5.0 / 3.0):
    up, down = _D4(), _D4()
    _check(lib().bgk_rankine_hugoniot(mach, gamma, up, down), "bgk_rankine_hugoniot")
    return np.array(up[:]), np.array(down[:])


def bgk_status_string(st: int) -> str:
    return lib().bgk_status_string(st).decode()


def bgk_abi_version() -> int:
    return lib().bgk_abi_version()


def bgk_step_noalloc(cfg: bgk_config, f_in, f_out, mom_out) -> None:
    """One step f_in -> f_out (device tensors) with no device allocation by the
    library, for callers that must not have it call cudaMalloc; see bgk.h."""
    a, da = _ptr(f_in)
    b, db = _ptr(f_out)
    m, dm = _ptr(mom_out)
    if not (da and db and dm):
        raise ValueError("bgk_step_noalloc takes device buffers only")
    # the C call cannot see buffer sizes: check them here
    ncell = cfg.nx * (cfg.ny if cfg.dim == 2 else 1)
    nv = cfg.nvx * (cfg.nvy if cfg.dim == 2 else 1)
    if not (f_in.numel() == f_out.numel() == ncell * nv * 2 and mom_out.numel() >= ncell * 4):
        raise ValueError(f"bgk_step_noalloc: f_in and f_out need {ncell * nv * 2} doubles, "
                         f"mom_out at least {ncell * 4}")
    _check(lib().bgk_step_noalloc(ctypes.byref(cfg), a, b, m), "bgk_step_noalloc")


def bgk_batch_create(cfgs, stream=None) -> int:
    arr = (bgk_config * len(cfgs))(*cfgs)
    h = _P()
    _check(lib().bgk_batch_create(arr, len(cfgs), stream, ctypes.byref(h)), "bgk_batch_create")
    return h.value


def bgk_batch_solver(b: int, index: int) -> int:
    h = _P()
    _check(lib().bgk_batch_solver(b, index, ctypes.byref(h)), "bgk_batch_solver")
    return h.value


def bgk_batch_step(b: int, nsteps: int) -> None:
    _check(lib().bgk_batch_step(b, nsteps), "bgk_batch_step")


def bgk_batch_sync(b: int) -> None:
    _check(lib().bgk_batch_sync(b), "bgk_batch_sync")


def bgk_batch_destroy(b: int) -> None:
    _check(lib().bgk_batch_destroy(b), "bgk_batch_destroy")


def bgk_autotune(h: int, trial_steps: int) -> int:
    t = ctypes.c_int(0)
    _check(lib().bgk_autotune(h, trial_steps, ctypes.byref(t)), "bgk_autotune")
    return t.value


def bgk_batch_autotune(b: int, trial_steps: int) -> None:
    _check(lib().bgk_batch_autotune(b, trial_steps), "bgk_batch_autotune")


def bgk_adjoint_lid_shear(h: int, nsteps: int, checkpoint_every: int, grad_out=None):
    """(J, dJ/dlnL, dJ/dU_W); dJ/df0 into grad_out (host array or CUDA tensor) if given."""
    out = _D4()
    addr, dev = _ptr(grad_out) if grad_out is not None else (None, 0)
    _check(lib().bgk_adjoint_lid_shear(h, nsteps, checkpoint_every, addr, dev, out), "bgk_adjoint_lid_shear")
    return out[0], out[1], out[2]


# --- full 3D velocity grid, one spatial dimension -------------------------
def make_config3v(*, nx, x0=0.0, lx=1.0, nv=(8, 8, 8), vmin=(-1.0, -1.0, -1.0), vmax=(1.0, 1.0, 1.0),
                  omega=0.5, dt=0.0, cfl=0.0, conservative=1, relax_exact=1,
                  inflow=((1, 0, 0, 0, 1), (1, 0, 0, 0, 1)), stream=None) -> bgk3v_config:
    """Fill a bgk3v_config; inflow = ((n, ux, uy, uz, theta) at XLO, at XHI)."""
    c = bgk3v_config()
    c.nx = nx
    c.nvx, c.nvy, c.nvz = nv
    c.conservative, c.relax_exact = conservative, relax_exact
    c.x0, c.lx = x0, lx
    for k in range(3):
        c.vmin[k], c.vmax[k] = vmin[k], vmax[k]
    c.omega, c.dt, c.cfl = omega, dt, cfl
    for e in range(2):
        for k in range(5):
            c.inflow[e][k] = inflow[e][k]
    c.cuda_stream = stream
    return c


def bgk3v_create(cfg: bgk3v_config) -> int:
    h = _P()
    _check(lib().bgk3v_create(ctypes.byref(cfg), ctypes.byref(h)), "bgk3v_create")
    return h.value


def bgk3v_destroy(h: int) -> None:
    _check(lib().bgk3v_destroy(h), "bgk3v_destroy")


def bgk3v_get_info(h: int) -> bgk3v_info:
    info = bgk3v_info()
    _check(lib().bgk3v_get_info(h, ctypes.byref(info)), "bgk3v_get_info")
    return info


def bgk3v_init_step(h: int, x_split: float, left, right) -> None:
    _check(lib().bgk3v_init_step(h, x_split, _D5(*left), _D5(*right)), "bgk3v_init_step")


def bgk3v_set_state(h: int, f) -> None:
    addr, dev = _ptr(f)
    _check(lib().bgk3v_set_state(h, addr, dev), "bgk3v_set_state")


def bgk3v_get_state(h: int, out) -> None:
    addr, dev = _ptr(out)
    _check(lib().bgk3v_get_state(h, addr, dev), "bgk3v_get_state")


def bgk3v_step(h: int, nsteps: int) -> None:
    _check(lib().bgk3v_step(h, nsteps), "bgk3v_step")


def bgk3v_moments(h: int, out, which: int = 0) -> None:
    addr, dev = _ptr(out)
    _check(lib().bgk3v_moments(h, which, addr, dev), "bgk3v_moments")


def bgk3v_sync(h: int) -> None:
    _check(lib().bgk3v_sync(h), "bgk3v_sync")


def bgk_batch_set_persistent(b: int, enable: bool = True, timeout_s: float = 5.0) -> None:
    _check(lib().bgk_batch_set_persistent(b, int(enable), timeout_s), "bgk_batch_set_persistent")
