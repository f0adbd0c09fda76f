"""bgk_step_noalloc: the step for callers that cannot let the library allocate
device memory (code under a fixed device-memory budget owned by its host
framework, or on paths where cudaMalloc's implicit device synchronisation is
not allowed).  Its scratch is a fixed array compiled into libbgk.so, shared
by all calls.

The test calls it through the C ABI twice in a row (f0 -> f1 -> f2) and
compares each result with the solver path (bgk_set_state + bgk_step +
bgk_get_state + bgk_moments) within the one-step parity tolerance used by
the other GPU tests: 1e-13 of max|f|.  This file is collected last on
purpose; it builds the library itself so it also runs alone.
"""
import numpy as np
import pytest

from paper_0903_4044_gb300 import bgk as B
from paper_0903_4044_gb300 import build, solver
from paper_0903_4044_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-13


def _close(got, want, tol=TOL):
    err = np.abs(got - want).max() / np.abs(want).max()
    assert err <= tol, f"max rel err {err:.3e} (tol {tol:.0e})"


def _two_calls(s, cfg):
    import torch

    f0 = torch.empty((s.ncell, s.nv, 2), dtype=torch.float64, device="cuda")
    B.bgk_get_state(s.h, f0)
    torch.cuda.synchronize()
    # the solver path, two steps
    s.step(1)
    ref1, mref1 = s.get_state(), s.moments(which=1)
    s.step(1)
    ref2, mref2 = s.get_state(), s.moments(which=1)
    # the allocation-free path, two calls in a row sharing the scratch array
    f1, f2 = torch.empty_like(f0), torch.empty_like(f0)
    m = torch.empty((s.ncell, 4), dtype=torch.float64, device="cuda")
    B.bgk_step_noalloc(cfg, f0, f1, m)
    _close(f1.cpu().numpy(), ref1)
    _close(m.cpu().numpy(), mref1)
    B.bgk_step_noalloc(cfg, f1, f2, m)
    _close(f2.cpu().numpy(), ref2)
    _close(m.cpu().numpy(), mref2)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    B.lib()


def test_noalloc_cavity_matches_solver_step():
    w = W.scaled(W.CAVITY_64, n=20, nv=24)
    xi = W.perturbation(0, 20 * 20, 24 * 24)
    s = solver.make_cavity(w, xi=xi)
    _two_calls(s, solver.cavity_config(**w))
    s.close()


def test_noalloc_shock_matches_solver_step():
    w = W.scaled(W.SHOCK_M2, nx=50)
    s = solver.make_shock(w)
    cfg, _, _ = solver.shock_config(**w)
    _two_calls(s, cfg)
    s.close()


def test_noalloc_honours_tile_and_stream():
    # tile_cells = 2 and a non-default stream: the same results as the solver
    # path built from the same configuration
    import torch

    w = W.scaled(W.CAVITY_64, n=18, nv=16)
    xi = W.perturbation(3, 18 * 18, 16 * 16)
    st = torch.cuda.Stream()
    cfg = solver.cavity_config(**w, tile_cells=2, stream=st.cuda_stream)
    s = solver.Solver(cfg)
    s.init_uniform((1.0, 0.0, 0.0, 1.0), xi, 1e-3)
    assert s.info.tile_cells == 2
    _two_calls(s, cfg)
    s.close()


def test_noalloc_rejects_misaligned_and_short_buffers():
    # both checks run before any GPU work: a float64 view at an 8-byte offset
    # gets BGK_ERR_INVALID_ARG from the library, a buffer of the wrong size a
    # ValueError from the binding
    import torch

    w = W.scaled(W.CAVITY_64, n=4, nv=8)
    cfg = solver.cavity_config(**w)
    n = 16 * 64 * 2
    base = torch.zeros(n + 1, dtype=torch.float64, device="cuda")
    good = torch.zeros(n, dtype=torch.float64, device="cuda")
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    m = torch.empty(16 * 4, dtype=torch.float64, device="cuda")
    with pytest.raises(B.BgkError) as e:
        B.bgk_step_noalloc(cfg, base[1:], out, m)
    assert e.value.status == B.BGK_ERR_INVALID_ARG
    mbase = torch.empty(16 * 4 + 1, dtype=torch.float64, device="cuda")
    with pytest.raises(B.BgkError) as e:
        B.bgk_step_noalloc(cfg, good, out, mbase[1:])
    assert e.value.status == B.BGK_ERR_INVALID_ARG
    with pytest.raises(ValueError):
        B.bgk_step_noalloc(cfg, good[:-2], out, m)
    with pytest.raises(ValueError):
        B.bgk_step_noalloc(cfg, good, out, m[:-1])


def test_noalloc_refuses_tables_beyond_its_scratch():
    import torch

    w = W.scaled(W.CAVITY_64, n=2, nv=64)  # 4096 velocities: tables above the 384 KiB scratch
    cfg = solver.cavity_config(**w)
    f = torch.zeros((4, 4096, 2), dtype=torch.float64, device="cuda")
    out = torch.empty_like(f)
    m = torch.empty((4, 4), dtype=torch.float64, device="cuda")
    with pytest.raises(B.BgkError) as e:
        B.bgk_step_noalloc(cfg, f, out, m)
    assert e.value.status == B.BGK_ERR_UNSUPPORTED
    assert "scratch" in str(e.value)
