"""Pins of the full-velocity-grid oracle (bgk_oracle3v.c) against what the
paper and the mathematics fix, and against the Chu-reduced oracle (itself
pinned in test_oracle_pins.py).  Sizes keep the whole file to seconds."""
import math

import numpy as np
import pytest

import oracle


def _prob(nx=1, lx=1.0, nv=(12, 12, 12), box=6.0, omega=0.74, dt=0.05, cons=1, exact=1, inflow=None):
    inflow = inflow or ((1, 0, 0, 0, 1), (1, 0, 0, 0, 1))
    cfg = oracle.make_config3v(nx=nx, x0=0.0, lx=lx, nv=nv, vmin=(-box,) * 3, vmax=(box,) * 3, omega=omega,
                               dt=dt, conservative=cons, relax_exact=exact, inflow=inflow)
    return oracle.Problem3v(cfg)


def test_maxwellian_moments_on_a_fine_grid():
    # the discrete moments of Phi approach its parameters (closed-form
    # integrals) on a wide, fine grid
    prob = _prob(nv=(40, 40, 40), box=8.0)
    p = (1.3, 0.4, -0.25, 0.1, 1.2)
    m = oracle.moments3v(prob, oracle.maxwellian3v(prob, p))
    assert np.allclose(m, p, rtol=0, atol=1e-10)


def test_maxwellian_reduces_to_the_chu_functions():
    # sum over (c_y, c_z) of Phi dc_y dc_z = G of the 1D Chu reduction and
    # sum of (c_y^2 + c_z^2) Phi dc_y dc_z = H = theta G (Sec. 4.1 with Chu)
    prob = _prob(nv=(10, 48, 48), box=8.0)
    p = (0.9, 0.3, 0.0, 0.0, 1.4)
    phi = oracle.maxwellian3v(prob, p).reshape(48, 48, 10)  # [jz][jy][jx]
    cx, cy, cz = oracle.velocities3v(prob)
    dcy, dcz = cy[1] - cy[0], cz[1] - cz[0]
    g = phi.sum(axis=(0, 1)) * dcy * dcz
    t2 = (cy[None, :, None] ** 2 + cz[:, None, None] ** 2)
    h = (t2 * phi).sum(axis=(0, 1)) * dcy * dcz
    cfg1 = oracle.make_config(dim=1, nx=1, nvx=10, vx=(-8.0, 8.0), omega=0.5, dt=0.01)
    G, H = oracle.maxwellian(cfg1, (0.9, 0.3, 0.0, 1.4))
    assert np.allclose(g, G, rtol=1e-12, atol=0)
    assert np.allclose(h, H, rtol=1e-11, atol=0)


def test_moments_scale_and_translate():
    # n scales with f; shifting f by one velocity cell along an axis adds
    # that cell width to the velocity component and leaves theta alone
    prob = _prob(nv=(12, 10, 8), box=6.0)
    rng = np.random.default_rng(3)
    f = np.zeros((8, 10, 12))
    f[2:6, 2:8, 2:10] = rng.random((4, 6, 8))
    m = oracle.moments3v(prob, f.ravel())
    assert oracle.moments3v(prob, 2.5 * f.ravel()) == pytest.approx(np.array([2.5, 1, 1, 1, 1]) * m, rel=1e-13)
    cx, cy, cz = oracle.velocities3v(prob)
    for axis, dc in ((2, cx[1] - cx[0]), (1, cy[1] - cy[0]), (0, cz[1] - cz[0])):
        ms = oracle.moments3v(prob, np.roll(f, 1, axis=axis).ravel())
        k = {2: 1, 1: 2, 0: 3}[axis]
        expect = m.copy()
        expect[k] += dc
        assert ms == pytest.approx(expect, rel=1e-12, abs=1e-13)


def test_effective_parameters_reproduce_the_moments():
    # coarse grid: the discrete Maxwellian of q misses q; the effective one hits it
    prob = _prob(nv=(7, 7, 7), box=4.0)
    q = (1.1, 0.35, -0.2, 0.05, 0.9)
    naive = oracle.moments3v(prob, oracle.maxwellian3v(prob, q))
    assert np.abs(naive - q).max() > 1e-3
    it, p = oracle.effective_params3v(prob, q)
    assert it > 0
    assert oracle.moments3v(prob, oracle.maxwellian3v(prob, p)) == pytest.approx(q, rel=1e-13, abs=1e-14)


@pytest.mark.parametrize("cons", [1, 0])
def test_relaxation_conserves_when_conservative(cons):
    # homogeneous cell (no streaming effect: huge cell), bi-Maxwellian start
    prob = _prob(nx=1, lx=1e15, nv=(8, 8, 8), box=5.0, cons=cons, dt=0.3)
    f = 0.5 * oracle.maxwellian3v(prob, (1.0, 0.8, 0.0, 0.0, 0.7)) + 0.5 * oracle.maxwellian3v(
        prob, (1.0, -0.8, 0.1, 0.0, 1.1))
    m0 = oracle.moments3v(prob, f)
    f1, _ = oracle.relax3v(prob, f[None, :])
    m1 = oracle.moments3v(prob, f1[0])
    n0, n1 = m0[0], m1[0]
    mom0, mom1 = n0 * m0[1:4], n1 * m1[1:4]
    e0 = n0 * (1.5 * m0[4] + (m0[1:4] ** 2).sum())
    e1 = n1 * (1.5 * m1[4] + (m1[1:4] ** 2).sum())
    err = max(abs(n1 - n0), np.abs(mom1 - mom0).max(), abs(e1 - e0))
    if cons:
        assert err < 1e-13
    else:
        assert err > 1e-7


def test_homogeneous_relaxation_decays_at_nu():
    # Eq. (relaxation) on a homogeneous state: f - Phi decays as exp(-nu t),
    # nu = n theta^(1 - omega) of the (conserved) moments
    prob = _prob(nx=1, lx=1e15, nv=(14, 14, 14), box=6.0, dt=0.1, omega=0.74)
    f0 = 0.5 * oracle.maxwellian3v(prob, (1.2, 0.6, 0.0, 0.0, 0.8)) + 0.5 * oracle.maxwellian3v(
        prob, (1.2, -0.6, 0.0, 0.0, 1.3))
    q = oracle.moments3v(prob, f0)
    _, p = oracle.effective_params3v(prob, q)
    phi = oracle.maxwellian3v(prob, p)
    nu = q[0] * q[4] ** (1 - 0.74)
    f, _ = oracle.step3v(prob, f0[None, :], 7)
    expect = phi + math.exp(-nu * 0.7) * (f0 - phi)
    assert np.abs(f[0] - expect).max() < 1e-12 * np.abs(f0).max()


def test_integer_courant_streaming_is_an_exact_shift():
    # c_x = +-0.5, +-1.5, ... and dt/dx = 2: every Courant number is an odd
    # integer, so Eq. (exact) moves each velocity by whole cells
    nvx = 6
    # (different inflow states at the two ends: sources beyond each end
    # must read that end's Maxwellian)
    left, right = (1, 0, 0, 0, 1), (1.3, 0.2, 0, 0, 0.8)
    cfg = oracle.make_config3v(nx=20, lx=20.0, nv=(nvx, 2, 2), vmin=(-3.0, -1.0, -1.0), vmax=(3.0, 1.0, 1.0),
                               dt=2.0, inflow=(left, right))
    prob = oracle.Problem3v(cfg)
    rng = np.random.default_rng(5)
    f = rng.random((20, prob.nv))
    ft = oracle.stream3v(prob, f)
    cx = oracle.velocities3v(prob)[0]
    gl, gr = oracle.maxwellian3v(prob, left), oracle.maxwellian3v(prob, right)
    for j in range(prob.nv):
        s = int(round(cx[j % nvx] * 2.0))
        for i in range(20):
            src = i - s
            want = gl[j] if src < 0 else gr[j] if src >= 20 else f[src, j]
            assert ft[i, j] == want


@pytest.mark.parametrize("nt,tol_g,tol_h", [(24, 1e-10, 1e-9), (16, 1e-6, 2e-6)])
def test_reduces_to_the_chu_oracle_on_the_shock(nt, tol_g, tol_h):
    # Integrating the full-grid shock run over (c_y, c_z) gives the
    # Chu-reduced (g, h) run of the 1D oracle, up to the quadrature error of
    # the transverse grid.  With 24 cells on [-6, 6] (spacing 0.5) that
    # error is ~exp(-pi^2 theta / 0.25) and the runs agree to round-off;
    # with the paper's 16 cells (spacing 0.75) the discrete transverse
    # second moment is off by ~1e-6 relative and so is the agreement.
    mach, nx, L, dt, steps = 1.5, 24, 70.0, 0.05, 30
    prob, f = oracle.shock3v_problem(mach=mach, nx=nx, length=L, nv=(16, nt, nt), vx=(-5.0, 7.0),
                                     vt=(-6.0, 6.0), omega=0.74, dt=dt)
    f1, _ = oracle.step3v(prob, f, steps)
    cx, cy, cz = oracle.velocities3v(prob)
    dcy, dcz = cy[1] - cy[0], cz[1] - cz[0]
    F = f1.reshape(nx, nt, nt, 16)  # [cell][jz][jy][jx]
    g3 = F.sum(axis=(1, 2)) * dcy * dcz
    t2 = cy[None, None, :, None] ** 2 + cz[None, :, None, None] ** 2
    h3 = (t2 * F).sum(axis=(1, 2)) * dcy * dcz

    up, down = oracle.rankine_hugoniot(mach)
    cfg1 = oracle.make_config(dim=1, nx=nx, x0=-0.5 * L, lx=L, nvx=16, vx=(-5.0, 7.0), omega=0.74, dt=dt,
                              bc_kind=(oracle.BC_INFLOW, oracle.BC_INFLOW, 0, 0), bc_state=(up, down, up, up))
    p1 = oracle.Problem(cfg1)
    g, h = oracle.init_step(p1, 0.0, up, down)
    g1, h1, _ = oracle.step(p1, g, h, steps)
    assert np.abs(g3 - g1).max() < tol_g * np.abs(g1).max()
    assert np.abs(h3 - h1).max() < tol_h * np.abs(h1).max()
    # the shock is actually moving the state (not a trivial comparison)
    assert np.abs(g1 - g).max() > 1e-3 * np.abs(g).max()
