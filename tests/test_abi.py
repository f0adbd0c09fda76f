"""Host-side checks of libbgk.so that need no GPU: the library loads, exports
every entry point include/bgk.h declares, and validates configurations before
any CUDA call."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_0903_4044_gb300 import bgk as B
from paper_0903_4044_gb300 import build, solver
from paper_0903_4044_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="session")
def L():
    build.build()
    return B.lib()


def _declared(header: str) -> set[str]:
    text = open(os.path.join(ROOT, "include", header)).read()
    return set(re.findall(r"^BGK_API\s+[^;(]*?\b(bgk\w+)\s*\(", text, flags=re.M))


def test_exports_every_declared_symbol(L):
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            names |= _declared(h)
    assert "bgk_create" in names and "bgk_step" in names
    for name in sorted(names):
        assert hasattr(L, name), name
    assert names == set(B.EXPORTS)
    assert B.bgk_abi_version() == 1


def test_status_strings(L):
    assert B.bgk_status_string(0) == "BGK_OK"
    assert B.bgk_status_string(5) == "BGK_ERR_NUMERIC"
    assert B.bgk_status_string(99) == "BGK_ERR_UNKNOWN"


def test_rankine_hugoniot_host(L):
    up, down = B.bgk_rankine_hugoniot(2.0)
    assert down[0] == pytest.approx(16.0 / 7.0, rel=1e-15)
    assert down[3] == pytest.approx(133.0 / 64.0, rel=1e-15)
    assert up[1] == pytest.approx(1.8257418583505538, rel=1e-15)
    with pytest.raises(B.BgkError) as e:
        B.bgk_rankine_hugoniot(0.5)
    assert e.value.status == B.BGK_ERR_INVALID_ARG


def test_null_pointers(L):
    assert L.bgk_create(None, None) == B.BGK_ERR_INVALID_ARG
    assert L.bgk_step(None, 1) == B.BGK_ERR_INVALID_ARG
    assert L.bgk_sync(None) == B.BGK_ERR_INVALID_ARG
    assert L.bgk_destroy(None) == B.BGK_OK
    assert L.bgk_moments(None, 0, None, 0) == B.BGK_ERR_INVALID_ARG
    assert isinstance(L.bgk_last_error(), bytes)


def _shock(**over):
    cfg, _, _ = solver.shock_config(**{**W.SHOCK_M2, **over})
    return cfg


def _cavity(**over):
    return solver.cavity_config(**{**W.CAVITY_64, **over})


def _expect(cfg, status, text):
    with pytest.raises(B.BgkError) as e:
        B.bgk_create(cfg)
    assert e.value.status == status, str(e.value)
    assert text in str(e.value)


@pytest.mark.parametrize("mutate,status,text", [
    (lambda c: setattr(c, "dim", 3), B.BGK_ERR_INVALID_ARG, "dim must be 1 or 2"),
    (lambda c: setattr(c, "nx", 0), B.BGK_ERR_INVALID_ARG, "nx must be"),
    (lambda c: setattr(c, "ny", 2), B.BGK_ERR_INVALID_ARG, "ny must be 1"),
    (lambda c: setattr(c, "nvx", 1), B.BGK_ERR_INVALID_ARG, "nvx must be"),
    (lambda c: setattr(c, "lx", -1.0), B.BGK_ERR_INVALID_ARG, "lx must be"),
    (lambda c: setattr(c, "vx_max", -9.0), B.BGK_ERR_INVALID_ARG, "vx_max must exceed"),
    (lambda c: setattr(c, "dt", -0.1), B.BGK_ERR_INVALID_ARG, "dt must be"),
    (lambda c: (setattr(c, "dt", 0.0), setattr(c, "cfl", 0.0)), B.BGK_ERR_INVALID_ARG, "needs cfl"),
    (lambda c: setattr(c, "omega", float("nan")), B.BGK_ERR_INVALID_ARG, "non-finite"),
    (lambda c: setattr(c, "precision", 7), B.BGK_ERR_INVALID_ARG, "unknown precision"),
    (lambda c: setattr(c, "conservative", 2), B.BGK_ERR_INVALID_ARG, "conservative"),
    (lambda c: setattr(c.bc[0], "kind", 9), B.BGK_ERR_INVALID_ARG, "unknown boundary"),
    (lambda c: setattr(c.bc[1], "n", 0.0), B.BGK_ERR_INVALID_ARG, "inflow needs"),
    (lambda c: setattr(c.bc[0], "uy", 0.3), B.BGK_ERR_INVALID_ARG, "uy must be 0"),
    (lambda c: setattr(c, "nvx", 5000), B.BGK_ERR_UNSUPPORTED, "exceeds"),
    (lambda c: setattr(c, "precision", B.BGK_BF16_DEV), B.BGK_ERR_UNSUPPORTED, "FP32 only"),
    (lambda c: (setattr(c, "precision", B.BGK_F32), setattr(c, "nvx", 136)), B.BGK_ERR_UNSUPPORTED,
     "nvx <= 128"),
])
def test_shock_config_validation(L, mutate, status, text):
    cfg = _shock()
    mutate(cfg)
    _expect(cfg, status, text)


@pytest.mark.parametrize("mutate,status,text", [
    (lambda c: setattr(c, "nvy", 1), B.BGK_ERR_INVALID_ARG, "nvy must be"),
    (lambda c: setattr(c, "ly", 0.0), B.BGK_ERR_INVALID_ARG, "ly must be"),
    (lambda c: setattr(c, "cfl", 1.5), B.BGK_ERR_UNSUPPORTED, "donor cell needs"),
    (lambda c: setattr(c.bc[3], "uy", 0.1), B.BGK_ERR_INVALID_ARG, "tangential"),
    (lambda c: setattr(c.bc[0], "theta", 0.0), B.BGK_ERR_INVALID_ARG, "wall theta"),
    (lambda c: (setattr(c.bc[0], "kind", B.BGK_BC_SPECULAR), setattr(c, "vx_min", -4.0)),
     B.BGK_ERR_INVALID_ARG, "symmetric"),
    (lambda c: (setattr(c, "nvx", 80), setattr(c, "nvy", 80)), B.BGK_ERR_UNSUPPORTED, "exceeds"),
    (lambda c: (setattr(c, "precision", B.BGK_F32), setattr(c, "nvx", 30)), B.BGK_ERR_UNSUPPORTED,
     "multiple of 8"),
    (lambda c: (setattr(c, "precision", B.BGK_BF16_DEV), setattr(c, "vx_min", -4.0), setattr(c, "vx_max", 6.0)),
     B.BGK_ERR_UNSUPPORTED, "change sign"),
])
def test_cavity_config_validation(L, mutate, status, text):
    cfg = _cavity()
    mutate(cfg)
    _expect(cfg, status, text)


def test_walls_refuse_large_courant_in_1d(L):
    cfg = _shock()
    cfg.bc[0].kind = B.BGK_BC_DIFFUSE
    cfg.bc[0].ux = 0.0
    cfg.cfl = 2.5
    _expect(cfg, B.BGK_ERR_UNSUPPORTED, "Courant number <= 1")


def test_valid_config_needs_a_gpu(L):
    # With no usable CUDA device a valid configuration fails with BGK_ERR_CUDA
    # (there is no CPU fallback); on a GPU machine it creates a solver.
    import torch

    cfg = _shock()
    if torch.cuda.is_available():
        h = B.bgk_create(cfg)
        B.bgk_destroy(h)
    else:
        _expect(cfg, B.BGK_ERR_CUDA, "CUDA")


def test_struct_layout_matches_header(L, tmp_path):
    # The ctypes mirrors must have the offsets and sizes the C compiler gives
    # the structs of bgk.h.
    import subprocess

    src = tmp_path / "layout.c"
    fields_cfg = [f for f, _ in B.bgk_config._fields_]
    fields_info = [f for f, _ in B.bgk_info._fields_]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "bgk.h"', "int main(void) {"]
    lines.append('printf("bgk_bc %zu\\n", sizeof(bgk_bc));')
    lines.append('printf("bgk_config %zu\\n", sizeof(bgk_config));')
    lines.append('printf("bgk_info %zu\\n", sizeof(bgk_info));')
    for f in fields_cfg:
        lines.append(f'printf("cfg.{f} %zu\\n", offsetof(bgk_config, {f}));')
    for f in fields_info:
        lines.append(f'printf("info.{f} %zu\\n", offsetof(bgk_info, {f}));')
    lines.append("return 0; }")
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    got = dict(line.split() for line in subprocess.run([str(exe)], capture_output=True, text=True,
                                                       check=True).stdout.splitlines())
    assert int(got["bgk_bc"]) == ctypes.sizeof(B.bgk_bc)
    assert int(got["bgk_config"]) == ctypes.sizeof(B.bgk_config)
    assert int(got["bgk_info"]) == ctypes.sizeof(B.bgk_info)
    for f in fields_cfg:
        assert int(got["cfg." + f]) == getattr(B.bgk_config, f).offset, f
    for f in fields_info:
        assert int(got["info." + f]) == getattr(B.bgk_info, f).offset, f
