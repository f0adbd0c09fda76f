"""Parity of the full-velocity-grid step (bgk3v_* through the C ABI) with the
FP64 oracle of bgk_oracle3v.c.  Each side derives its own grids, time step,
shifts and Rankine-Hugoniot states from the raw workload parameters.

Tolerances (FP64): one step element by element 1e-13 of max|f|; moments
after a run 1e-12 relative (velocities relative to max(|U|, 1)); states
after a run 1e-11 of max|f| (rounding of differently ordered sums grows
slowly with the number of steps)."""
import numpy as np
import pytest

import oracle
from paper_0903_4044_gb300 import build, solver
from paper_0903_4044_gb300 import bgk as B
from paper_0903_4044_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    oracle.build()
    B.lib()


def _pair(w):
    s = solver.make_shock3v(w)
    prob, f = oracle.shock3v_problem(**w)
    return s, prob, f


def _assert_state(gpu, ref, tol):
    err = np.abs(gpu - ref).max() / np.abs(ref).max()
    assert err <= tol, f"max rel err {err:.3e} (tol {tol:.0e})"


def _assert_moments(m_gpu, m_orc, tol=1e-12):
    en = np.abs(m_gpu[:, 0] - m_orc[:, 0]) / np.abs(m_orc[:, 0])
    et = np.abs(m_gpu[:, 4] - m_orc[:, 4]) / np.abs(m_orc[:, 4])
    eu = np.abs(m_gpu[:, 1:4] - m_orc[:, 1:4]).max(axis=1) / np.maximum(np.abs(m_orc[:, 1:4]).max(axis=1), 1.0)
    worst = max(en.max(), et.max(), eu.max())
    assert worst <= tol, f"n {en.max():.3e} U {eu.max():.3e} theta {et.max():.3e}"


M15 = W.scaled(W.SHOCK3V_M15, nx=64)


def test_grid_and_initial_state_agree():
    s, prob, f = _pair(M15)
    assert s.dt == prob.cfg.dt == 0.05
    assert s.nv == prob.nv == 4096
    _assert_state(s.get_state(), f, 1e-15)
    s.close()


def test_one_step_elementwise():
    s, prob, f = _pair(M15)
    s.step(1)
    f1, mom = oracle.step3v(prob, f, 1)
    _assert_state(s.get_state(), f1, 1e-13)
    _assert_moments(s.moments(which=1), mom, tol=1e-14)
    s.close()


def test_run_matches_oracle():
    w = W.scaled(W.SHOCK3V_M15, nx=128)
    s, prob, f = _pair(w)
    s.step(60)
    f1, _ = oracle.step3v(prob, f, 60)
    _assert_moments(s.moments(), oracle.state_moments3v(prob, f1))
    _assert_state(s.get_state(), f1, 1e-11)
    s.close()


def test_mach3_on_30_cubed():
    w = W.scaled(W.SHOCK3V_M3, nx=40)
    s, prob, f = _pair(w)
    s.step(6)
    f1, mom = oracle.step3v(prob, f, 6)
    _assert_moments(s.moments(which=1), mom)
    _assert_state(s.get_state(), f1, 1e-12)
    s.close()


def test_large_courant_numbers():
    # 2048 cells on 70 mean free paths: C = c_x dt/dx reaches 10 (shifts of 0..10)
    w = W.scaled(W.SHOCK3V_M15, nx=2048)
    s, prob, f = _pair(w)
    assert s.info.max_courant > 9.0
    s.step(2)
    f1, mom = oracle.step3v(prob, f, 2)
    _assert_moments(s.moments(which=1), mom)
    _assert_state(s.get_state(), f1, 1e-12)
    s.close()


@pytest.mark.parametrize("exact,cons", [(0, 1), (1, 0), (0, 0)])
def test_variants(exact, cons):
    w = W.scaled(W.SHOCK3V_M15, nx=48, nv=(12, 10, 8), vx=(-5.0, 7.0), vt=(-5.0, 5.0))
    s = solver.make_shock3v(w, relax_exact=exact, conservative=cons)
    prob, f = oracle.shock3v_problem(**w, relax_exact=exact, conservative=cons)
    s.step(20)
    f1, _ = oracle.step3v(prob, f, 20)
    _assert_moments(s.moments(), oracle.state_moments3v(prob, f1))
    s.close()


def test_full_size_sampled_cells():
    # The 2048-cell, 30^3-velocity workload, one step from the step profile,
    # checked at sampled cells against oracle runs on sub-domains holding
    # every source cell of the sample (|C| <= 17 here).
    w = W.SHOCK3V_M3
    s = solver.make_shock3v(w)
    s.step(1)
    got = s.get_state()
    reach = int(np.ceil(s.info.max_courant)) + 2
    dx = w["length"] / w["nx"]
    for i in (5, w["nx"] // 2 - 1, w["nx"] // 2, w["nx"] - 3):
        lo, hi = max(0, i - reach), min(w["nx"], i + reach + 1)
        sub = dict(w, nx=hi - lo, length=(hi - lo) * dx)
        prob, _ = oracle.shock3v_problem(**sub)
        # sub-domain [x(lo), x(hi)) with the full problem's initial step at x = 0
        prob.cfg.x0 = -0.5 * w["length"] + lo * dx
        f0 = oracle.init_step3v(prob, 0.0, prob.meta["up"], prob.meta["down"])
        f1, _ = oracle.step3v(prob, f0, 1)
        ref = f1[i - lo]
        err = np.abs(got[i] - ref).max() / np.abs(ref).max()
        assert err <= 1e-13, f"cell {i}: {err:.3e}"
    s.close()


def test_rejections():
    base = dict(W.SHOCK3V_M15)
    cfg, _, _ = solver.shock3v_config(**base)
    cfg.nvz = 300
    with pytest.raises(B.BgkError) as e:
        solver.Solver3v(cfg)
    assert e.value.status == B.BGK_ERR_UNSUPPORTED
    cfg, _, _ = solver.shock3v_config(**base)
    cfg.inflow[0][4] = -1.0
    with pytest.raises(B.BgkError) as e:
        solver.Solver3v(cfg)
    assert e.value.status == B.BGK_ERR_INVALID_ARG
