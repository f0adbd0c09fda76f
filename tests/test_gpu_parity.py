"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Same seeded inputs on both sides; each side derives its own grids, time step
and boundary states from the raw workload parameters.  Tolerances (FP64):
  * one step, element by element: |gpu - oracle| <= 1e-13 * max|f|
    (a handful of roundings of differently ordered sums and of CUDA's exp);
  * and every element relative to its own size, the Maxwellian tails down to
    1e-41 of the peak included: |gpu - oracle| <= 1e-12 |oracle| (every
    value is a positive combination of positive values, each operation
    rounds relative to its result, and the Gaussian factors' recurrence adds
    at most one rounding per velocity: 48 x 1.1e-16 = 5e-15 a step;
    measured up to 1.5e-13, after 4000 shock steps 6e-14);
  * macroscopic fields after a full run: 1e-12 relative (velocities relative
    to the larger of |U| and the lid / thermal scale).
"""
import os

import numpy as np
import pytest

import oracle
from paper_0903_4044_gb300 import bgk as B
from paper_0903_4044_gb300 import build, solver
from paper_0903_4044_gb300 import workloads as W

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
TOL_STEP = 1e-13
TOL_RUN = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    oracle.build()
    B.lib()


def split(state):
    return np.ascontiguousarray(state[..., 0]), np.ascontiguousarray(state[..., 1])


TOL_ELEM = 1e-12


def assert_state_close(gpu_state, g, h, tol=TOL_STEP):
    gg, hh = split(gpu_state)
    scale_g, scale_h = np.abs(g).max(), np.abs(h).max()
    eg = np.abs(gg - g).max() / scale_g
    eh = np.abs(hh - h).max() / scale_h
    assert eg <= tol and eh <= tol, f"max rel err g {eg:.3e} h {eh:.3e} (tol {tol:.0e})"
    # each element against its own magnitude (tails included); an exact
    # zero of the oracle must be an exact zero here
    for name, a, b in (("g", gg, g), ("h", hh, h)):
        err = np.abs(a - b)
        bad = err > TOL_ELEM * np.abs(b)
        assert not bad.any(), (
            f"{name}: {bad.sum()} elements off by more than {TOL_ELEM:.0e} of their size, worst "
            f"{(err[bad] / np.maximum(np.abs(b[bad]), 1e-300)).max():.3e}")


def assert_moments_close(m_gpu, m_orc, vscale, tol=TOL_RUN):
    en = np.abs(m_gpu[:, 0] - m_orc[:, 0]) / np.abs(m_orc[:, 0])
    et = np.abs(m_gpu[:, 3] - m_orc[:, 3]) / np.abs(m_orc[:, 3])
    eu = np.abs(m_gpu[:, 1:3] - m_orc[:, 1:3]).max(axis=1) / np.maximum(np.abs(m_orc[:, 1:3]).max(axis=1), vscale)
    worst = max(en.max(), et.max(), eu.max())
    assert worst <= tol, f"n {en.max():.3e} U {eu.max():.3e} theta {et.max():.3e} (tol {tol:.0e})"


def cavity_pair(w, seed=None, **over):
    """(gpu solver, oracle problem, g0, h0) for a cavity workload."""
    w = {**w, **over}
    prob0, _, _ = oracle.cavity_problem(**w)
    xi = W.perturbation(w.get("seed", 0) if seed is None else seed, prob0.ncell, prob0.nv)
    prob, g, h = oracle.cavity_problem(**w, xi=xi)
    s = solver.make_cavity(w, xi=xi)
    return s, prob, g, h


# ---------------------------------------------------------------------------
# Set-up: grids, time step and initial states agree
# ---------------------------------------------------------------------------
def test_initial_states_and_dt_agree():
    s = solver.make_shock(W.SHOCK_M2)
    prob, g, h = oracle.shock_problem(**W.SHOCK_M2)
    assert s.dt == prob.cfg.dt
    assert_state_close(s.get_state(), g, h, tol=1e-15)
    s.close()
    s, prob, g, h = cavity_pair(W.CAVITY_64)
    assert s.dt == prob.cfg.dt
    assert_state_close(s.get_state(), g, h, tol=1e-15)
    s.close()


# ---------------------------------------------------------------------------
# 1D normal shock (Mach 2, 200 cells, 64 velocities)
# ---------------------------------------------------------------------------
def test_shock_one_step_elementwise():
    s = solver.make_shock(W.SHOCK_M2)
    prob, g, h = oracle.shock_problem(**W.SHOCK_M2)
    s.step(1)
    g1, h1, mom = oracle.step(prob, g, h, 1)
    assert_state_close(s.get_state(), g1, h1)
    assert_moments_close(s.moments(which=1), mom, vscale=1.0, tol=1e-14)
    s.close()


def test_shock_full_run_matches_oracle():
    # Sec. 4.1 shock, 4000 steps (the graph-replayed chunks and the tail).
    s = solver.make_shock(W.SHOCK_M2)
    prob, g, h = oracle.shock_problem(**W.SHOCK_M2)
    s.step(W.SHOCK_M2["steps"])
    g1, h1, _ = oracle.step(prob, g, h, W.SHOCK_M2["steps"])
    m_orc = oracle.state_moments(prob, g1, h1)
    assert_moments_close(s.moments(), m_orc, vscale=1.0)
    assert_state_close(s.get_state(), g1, h1, tol=1e-11)
    s.close()


@pytest.mark.parametrize("cfl,exact,cons", [(2.6, 1, 1), (0.9, 0, 1), (0.5, 1, 0), (1.0, 1, 1)])
def test_shock_variants(cfl, exact, cons):
    # integer Courant shift (cfl 2.6: shifts of 0..2 cells), Euler
    # relaxation, no conservative correction, Courant number exactly 1.
    w = W.scaled(W.SHOCK_M2, nx=77, nvx=40, cfl=cfl, relax_exact=exact, conservative=cons)
    s = solver.make_shock(w)
    prob, g, h = oracle.shock_problem(**w)
    s.step(37)
    g1, h1, _ = oracle.step(prob, g, h, 37)
    assert_state_close(s.get_state(), g1, h1, tol=1e-12)
    s.close()


# ---------------------------------------------------------------------------
# 2D lid-driven cavity
# ---------------------------------------------------------------------------
def test_cavity_small_ragged_multi_step():
    # 23 x 23 cells, 20 x 20 velocities = 400 per cell: one CTA of 256
    # threads covers a cell in two passes with a ragged tail.  Graph chunks
    # (64 steps) and single launches both run (150 = 2*64 + 22).
    w = W.scaled(W.CAVITY_64, n=23, nv=20, steps=150)
    s, prob, g, h = cavity_pair(w)
    s.step(150)
    g1, h1, mom = oracle.step(prob, g, h, 150)
    assert_state_close(s.get_state(), g1, h1, tol=1e-12)
    assert_moments_close(s.moments(which=1), mom, vscale=0.09)
    s.close()


def test_cavity_nonsquare_grids():
    # nx != ny and nvx != nvy need explicit configs on both sides.
    uw = 0.1 * np.sqrt(5.0 / 6.0)
    bc = [(1, 1, 0, 0, 1)] * 3 + [(1, 1, uw, 0, 1)]
    cfg = B.make_config(dim=2, nx=13, ny=7, lx=6.5, ly=3.5, nvx=22, nvy=14, vx=(-5, 5), vy=(-4.5, 4.5),
                        omega=0.74, cfl=0.7, bc=bc)
    oc = oracle.make_config(dim=2, nx=13, ny=7, lx=6.5, ly=3.5, nvx=22, nvy=14, vx=(-5, 5), vy=(-4.5, 4.5),
                            omega=0.74, cfl=0.7, bc_kind=(1, 1, 1, 1),
                            bc_state=((1, 0, 0, 1), (1, 0, 0, 1), (1, 0, 0, 1), (1, uw, 0, 1)))
    prob = oracle.Problem(oc)
    xi = W.perturbation(5, prob.ncell, prob.nv)
    g, h = oracle.init_uniform(prob, (1.0, 0.0, 0.0, 1.0), xi, 1e-2)
    s = solver.Solver(cfg)
    s.init_uniform((1.0, 0.0, 0.0, 1.0), xi, 1e-2)
    assert s.dt == oc.dt
    s.step(90)
    g1, h1, _ = oracle.step(prob, g, h, 90)
    assert_state_close(s.get_state(), g1, h1, tol=1e-12)
    for face in range(4):
        want = np.stack(oracle.wall_fluxes(prob, g1, h1, face), axis=1)
        got = s.wall_fluxes(face)
        np.testing.assert_allclose(got, want, rtol=1e-11, atol=1e-13 * np.abs(want).max())
    s.close()


@pytest.mark.parametrize("variant", ["specular", "euler", "nonconservative", "inflow"])
def test_cavity_variants(variant):
    w = W.scaled(W.CAVITY_64, n=12, nv=16, steps=40)
    if variant == "specular":
        w["wall"] = "specular"
    elif variant == "euler":
        w["relax_exact"] = 0
    elif variant == "nonconservative":
        w["conservative"] = 0
    if variant != "inflow":
        s, prob, g, h = cavity_pair(w)
    else:
        # 2D channel: inflow on x faces, diffuse walls on y faces
        inl, outl = (1.0, 0.3, 0.0, 1.0), (0.9, 0.3, 0.0, 1.1)
        cfg = B.make_config(dim=2, nx=12, ny=9, lx=6, ly=4, nvx=16, nvy=16, vx=(-5, 5), vy=(-5, 5),
                            cfl=0.5, bc=[(0, *inl), (0, *outl), (1, 1, 0.2, 0, 1), (1, 1, -0.1, 0, 1.2)])
        oc = oracle.make_config(dim=2, nx=12, ny=9, lx=6, ly=4, nvx=16, nvy=16, vx=(-5, 5), vy=(-5, 5),
                                cfl=0.5, bc_kind=(0, 0, 1, 1),
                                bc_state=(inl, outl, (1, 0.2, 0, 1), (1, -0.1, 0, 1.2)))
        prob = oracle.Problem(oc)
        xi = W.perturbation(9, prob.ncell, prob.nv)
        g, h = oracle.init_uniform(prob, (1.0, 0.3, 0.0, 1.0), xi, 1e-3)
        s = solver.Solver(cfg)
        s.init_uniform((1.0, 0.3, 0.0, 1.0), xi, 1e-3)
    s.step(40)
    g1, h1, _ = oracle.step(prob, g, h, 40)
    assert_state_close(s.get_state(), g1, h1, tol=1e-12)
    s.close()


def test_cavity64_one_step_full_size():
    # Full 64x64 x 32x32 size in the benchmark's launch configuration.
    s, prob, g, h = cavity_pair(W.CAVITY_64)
    s.step(1)
    g1, h1, mom = oracle.step(prob, g, h, 1)
    assert_state_close(s.get_state(), g1, h1)
    assert_moments_close(s.moments(which=1), mom, vscale=0.09, tol=1e-13)
    for face in range(4):
        want = np.stack(oracle.wall_fluxes(prob, g1, h1, face), axis=1)
        np.testing.assert_allclose(s.wall_fluxes(face), want, rtol=1e-11, atol=1e-13 * np.abs(want).max())
    s.close()


def test_cavity64_full_run_matches_golden():
    # 5000 steps of the 64x64 cavity against the oracle's stored result
    # (tests/golden/gen_cavity64.py).
    path = os.path.join(GOLDEN, "cavity64_moments.txt")
    want = np.loadtxt(path)
    s, prob, g, h = cavity_pair(W.CAVITY_64)
    s.step(W.CAVITY_64["steps"])
    got = s.moments()
    uw = 0.1 * np.sqrt(5.0 / 6.0)
    assert_moments_close(got, want, vscale=uw)
    # mass conserved by the diffuse walls and the conservative collision step
    n0 = oracle.state_moments(prob, g, h)[:, 0].sum()
    assert got[:, 0].sum() == pytest.approx(n0, rel=1e-12)
    s.close()


def test_cavity256_one_step_full_size():
    # The 256x256 x 48x48 grid (2304 velocities: 9 passes of 256 threads per
    # cell), one step from the perturbed rest state, whole state compared.
    w = W.scaled(W.CAVITY_256)
    s, prob, g, h = cavity_pair(w)
    s.step(1)
    g1, h1, _ = oracle.step(prob, g, h, 1)
    assert_state_close(s.get_state(), g1, h1)
    s.close()


@pytest.mark.parametrize("tile", [4, 8])
def test_f64_ragged_grid_48_columns(tile):
    # 130 x 121 cells (3933 CTAs of 4 cells, the last one with 2; or 1967 of
    # 8, the last one with 2) with 48 x 48 velocities (the row mapping of the
    # interior cells); three steps, whole state and the post-streaming moments
    w = W.scaled(W.CAVITY_256, n=130, tile_cells=tile)
    prob0, _, _ = oracle.cavity_problem(**w)
    cfg = solver.cavity_config(**w)
    cfg.ny = 121
    cfg.ly = cfg.ly * 121 / 130
    oc = oracle.make_config(dim=2, nx=130, ny=121, lx=cfg.lx, ly=cfg.ly, nvx=48, nvy=48, vx=(-5, 5), vy=(-5, 5),
                            cfl=0.5, bc_kind=(1, 1, 1, 1), bc_state=prob0.cfg.bc_state)
    prob = oracle.Problem(oc)
    xi = W.perturbation(4, prob.ncell, prob.nv)
    g, h = oracle.init_uniform(prob, (1.0, 0.0, 0.0, 1.0), xi, 1e-3)
    s = solver.Solver(cfg)
    s.init_uniform((1.0, 0.0, 0.0, 1.0), xi, 1e-3)
    assert s.info.tile_cells == tile
    s.step(3)
    g1, h1, mom = oracle.step(prob, g, h, 3)
    assert_state_close(s.get_state(), g1, h1)
    assert_moments_close(s.moments(which=1), mom, vscale=0.05)
    s.close()


# ---------------------------------------------------------------------------
# Edge cases and invariants
# ---------------------------------------------------------------------------
def _wall_box(nx, ny, nvx, nvy, cons):
    bc = [(1, 1, 0, 0, 1)] * 3 + [(1, 1, 0.05, 0, 1)]
    kw = dict(dim=2, nx=nx, ny=ny, lx=nx * 0.5, ly=ny * 0.5, nvx=nvx, nvy=nvy, vx=(-4, 4), vy=(-4, 4),
              cfl=0.6, conservative=cons)
    cfg = B.make_config(**kw, bc=bc)
    oc = oracle.make_config(**kw, bc_kind=(1, 1, 1, 1),
                            bc_state=((1, 0, 0, 1),) * 3 + ((1, 0.05, 0, 1),))
    prob = oracle.Problem(oc)
    xi = W.perturbation(3, prob.ncell, prob.nv)
    g, h = oracle.init_uniform(prob, (1.0, 0.0, 0.0, 1.0), xi, 1e-2)
    s = solver.Solver(cfg)
    s.init_uniform((1.0, 0.0, 0.0, 1.0), xi, 1e-2)
    return s, prob, g, h


@pytest.mark.parametrize("nx,ny,nvx,nvy,cons", [(1, 5, 12, 10, 1), (7, 1, 10, 12, 1), (1, 1, 2, 2, 0),
                                                (3, 2, 64, 64, 1)])
def test_degenerate_and_maximum_grids(nx, ny, nvx, nvy, cons):
    # a single cell row/column (cells touching opposite walls), a single
    # cell with the smallest velocity grid, and the largest velocity set one
    # CTA takes (4096).
    s, prob, g, h = _wall_box(nx, ny, nvx, nvy, cons)
    s.step(5)
    g1, h1, _ = oracle.step(prob, g, h, 5)
    assert_state_close(s.get_state(), g1, h1, tol=1e-12)
    s.close()


def test_too_coarse_grid_fails_on_both_sides():
    # On a 6 x 4 velocity grid the discrete Maxwellian is too far from the
    # continuous one for the effective-parameter iteration to converge: the
    # oracle refuses, and the GPU reports BGK_ERR_NUMERIC instead of a state.
    s, prob, g, h = _wall_box(1, 5, 6, 4, 1)
    with pytest.raises(RuntimeError):
        oracle.step(prob, g, h, 1)
    s.step(1)
    with pytest.raises(B.BgkError) as e:
        s.sync()
    assert e.value.status == B.BGK_ERR_NUMERIC
    s.close()


def test_equilibrium_is_fixed_point_on_gpu():
    w = W.scaled(W.CAVITY_64, n=16, nv=16, lid_mach=0.0)
    s = solver.make_cavity(w)
    f0 = s.get_state()
    s.step(100)
    f1 = s.get_state()
    np.testing.assert_allclose(f1, f0, rtol=5e-14, atol=1e-30)
    s.close()


def test_zero_steps_and_determinism():
    s1, prob, g, h = cavity_pair(W.scaled(W.CAVITY_64, n=16, nv=16))
    f0 = s1.get_state()
    s1.step(0)
    assert np.array_equal(s1.get_state(), f0)
    s1.step(70)
    s2 = solver.make_cavity(W.scaled(W.CAVITY_64, n=16, nv=16),
                            xi=W.perturbation(0, prob.ncell, prob.nv))
    s2.step(70)
    assert np.array_equal(s1.get_state(), s2.get_state())
    s1.close()
    s2.close()


def test_state_roundtrip_and_device_buffers():
    import torch

    s = solver.make_shock(W.SHOCK_M2)
    st = s.get_state()
    d = torch.empty(st.shape, dtype=torch.float64, device="cuda")
    B.bgk_get_state(s.h, d)
    torch.cuda.synchronize()
    assert np.array_equal(d.cpu().numpy(), st)
    d.mul_(1.0)
    B.bgk_set_state(s.h, d)
    s.step(3)
    m = torch.empty((s.ncell, 4), dtype=torch.float64, device="cuda")
    B.bgk_moments(s.h, m, 1)
    host = s.moments(which=1)
    assert np.array_equal(m.cpu().numpy(), host)
    s.close()


def test_user_stream():
    import torch

    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        s = solver.make_shock(W.SHOCK_M2, stream=st.cuda_stream)
        s.step(130)
        m = s.moments()
    prob, g, h = oracle.shock_problem(**W.SHOCK_M2)
    g1, h1, _ = oracle.step(prob, g, h, 130)
    assert_moments_close(m, oracle.state_moments(prob, g1, h1), vscale=1.0)
    s.close()


def test_numeric_failure_is_reported_not_faulted():
    # A negative-density cell is a host-made failure: the kernel flags it and
    # the next synchronising call returns BGK_ERR_NUMERIC; the context lives on.
    s = solver.make_shock(W.SHOCK_M2)
    f = s.get_state()
    f[10] *= -1.0
    s.set_state(f)
    s.step(1)
    with pytest.raises(B.BgkError) as e:
        s.sync()
    assert e.value.status == B.BGK_ERR_NUMERIC
    s.init_step(0.0, s.up, s.down)   # resets the flag
    s.step(2)
    s.sync()
    s.close()


@pytest.mark.parametrize("tile", [1, 2, 4, 8])
def test_every_tile_matches_oracle(tile):
    # The cells-per-CTA knob changes only how work is spread over lanes.
    w = W.scaled(W.CAVITY_64, n=13, nv=24, steps=20)
    prob0, _, _ = oracle.cavity_problem(**w)
    xi = W.perturbation(0, prob0.ncell, prob0.nv)
    prob, g, h = oracle.cavity_problem(**w, xi=xi)
    s = solver.make_cavity(w, xi=xi, tile_cells=tile)
    assert s.info.tile_cells == tile
    s.step(20)
    g1, h1, mom = oracle.step(prob, g, h, 20)
    assert_state_close(s.get_state(), g1, h1, tol=1e-12)
    assert_moments_close(s.moments(which=1), mom, vscale=0.09)
    s.close()
    ws = W.scaled(W.SHOCK_M2, nx=29)
    s = solver.make_shock(ws, tile_cells=tile)
    prob, g, h = oracle.shock_problem(**ws)
    s.step(20)
    g1, h1, _ = oracle.step(prob, g, h, 20)
    assert_state_close(s.get_state(), g1, h1, tol=1e-12)
    s.close()
