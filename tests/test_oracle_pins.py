"""Pins of the CPU oracle against what the paper and mathematics fix.

Each test names the oracle function(s) it pins and the fact it checks.  None
of them re-derives an oracle formula and compares it with itself: they use
closed forms, conservation laws, exactness properties of the scheme,
brute-force sums over a full 3D velocity grid, and literal values computed by
hand from the paper's equations.
"""
import math

import numpy as np
import pytest

from paper_0903_4044_gb300 import workloads as W


# --------------------------------------------------------------------------
# Seeded inputs
# --------------------------------------------------------------------------
def test_splitmix64_published_first_output():
    # SplitMix64 (Steele, Lea, Flood 2014) from state 0: the first output of
    # the reference generator is 0xE220A8397B1DCDAF.
    assert int(W.splitmix64(0, 1)[0]) == 0xE220A8397B1DCDAF
    xi = W.uniform_pm1(7, 100000)
    assert xi.min() >= -1.0 and xi.max() < 1.0
    assert abs(xi.mean()) < 0.01
    # counter-based: a window of the stream equals the same slice of the whole
    assert np.array_equal(W.uniform_pm1(3, 10, start=5), W.uniform_pm1(3, 15)[5:])


# --------------------------------------------------------------------------
# Grids and time step (Sec. 2.1 grid; Courant rule)
# --------------------------------------------------------------------------
def test_grid_literals(orc):
    # 64 cells on [-8, 8]: centres -7.875 ... 7.875, dV = 0.25
    c = orc.make_config(dim=1, nx=200, x0=-20, lx=40, nvx=64, vx=(-8, 8), cfl=0.5)
    cx, _ = orc.velocities(c)
    assert cx[0] == -7.875 and cx[-1] == 7.875 and not np.any(cx == 0)
    assert orc.dv(c) == 0.25
    # dt = 0.5 * 0.2 / 7.875
    assert c.dt == pytest.approx(0.012698412698412698, rel=1e-15)
    # 2D: dx = 10/64, max|c| = 4.84375 -> dt = 0.5 / (2 * 4.84375 * 6.4) = 1/124
    c2 = orc.make_config(dim=2, nx=64, ny=64, lx=10, ly=10, nvx=32, nvy=32, vx=(-5, 5),
                         vy=(-5, 5), cfl=0.5)
    assert c2.dt == pytest.approx(1.0 / 124.0, rel=1e-15)
    assert orc.dv(c2) == pytest.approx(0.3125 ** 2, rel=1e-15)


# --------------------------------------------------------------------------
# Eq. (RH)
# --------------------------------------------------------------------------
def test_rankine_hugoniot_literals_mach2(orc):
    # Eq. (RH) at M = 2 by hand: n+/n- = 16/7, T+/T- = 19*7/64 = 133/64,
    # V- = 2 sqrt(5/6) in units of sqrt(2RT-), V+ = V- * 7/16.
    up, down = orc.rankine_hugoniot(2.0)
    assert up[0] == 1.0 and up[3] == 1.0
    assert up[1] == pytest.approx(1.8257418583505538, rel=1e-15)
    assert down[0] == pytest.approx(16.0 / 7.0, rel=1e-15)
    assert down[3] == pytest.approx(133.0 / 64.0, rel=1e-15)
    assert down[1] == pytest.approx(1.8257418583505538 * 7.0 / 16.0, rel=1e-15)


@pytest.mark.parametrize("mach", [1.2, 1.5, 2.0, 3.0, 5.0])
def test_rankine_hugoniot_conserves_fluxes(orc, mach):
    # Independent of Eq. (RH): the Euler fluxes of mass, momentum and energy
    # of a monatomic gas are continuous across the shock.  In units of
    # sqrt(2RT0): pressure p = n theta / 2, energy flux n u (u^2 + 5 theta / 2).
    up, down = orc.rankine_hugoniot(mach)

    def fluxes(s):
        n, u, th = s[0], s[1], s[3]
        return np.array([n * u, n * u * u + 0.5 * n * th, n * u * (u * u + 2.5 * th)])

    np.testing.assert_allclose(fluxes(up), fluxes(down), rtol=1e-14)
    # and the Mach number definition: u = M sqrt(gamma theta / 2)
    assert up[1] == pytest.approx(mach * math.sqrt(5.0 / 6.0), rel=1e-15)


# --------------------------------------------------------------------------
# Eq. (Maxw) reduced, pinned against the full 3D Maxwellian summed over the
# unresolved components, and its moments against their closed forms.
# --------------------------------------------------------------------------
def _maxwell3d(c3, n, u, th):
    cx, cy, cz = c3
    d2 = (cx - u[0]) ** 2 + (cy - u[1]) ** 2 + (cz - u[2]) ** 2
    return n / (math.pi * th) ** 1.5 * np.exp(-d2 / th)


@pytest.mark.parametrize("p", [(1.0, 0.3, 0.0, 1.0), (2.2, -0.7, 0.0, 2.1), (0.4, 1.2, 0.0, 0.6)])
def test_maxwellian_1d_matches_3d_reduction(orc, p):
    c = orc.make_config(dim=1, nx=1, nvx=40, vx=(-6, 6))
    G, H = orc.maxwellian(c, p)
    cx, _ = orc.velocities(c)
    # reduce the 3D Maxwellian over (cy, cz) numerically on a fine grid
    t = np.linspace(-9, 9, 361)
    dt_ = t[1] - t[0]
    CX, CY, CZ = np.meshgrid(cx, t, t, indexing="ij")
    f = _maxwell3d((CX, CY, CZ), p[0], (p[1], 0, 0), p[3])
    g = f.sum(axis=(1, 2)) * dt_ * dt_
    h = ((CY ** 2 + CZ ** 2) * f).sum(axis=(1, 2)) * dt_ * dt_
    np.testing.assert_allclose(G, g, rtol=1e-10, atol=1e-300)
    np.testing.assert_allclose(H, h, rtol=1e-10, atol=1e-300)


def test_maxwellian_2d_matches_3d_reduction(orc):
    p = (1.3, 0.4, -0.25, 1.4)
    c = orc.make_config(dim=2, nx=1, ny=1, nvx=12, nvy=10, vx=(-5, 5), vy=(-4, 6))
    G, H = orc.maxwellian(c, p)
    cx, cy = orc.velocities(c)
    t = np.linspace(-10, 10, 801)
    dt_ = t[1] - t[0]
    f = _maxwell3d((cx[:, None], cy[:, None], t[None, :]), p[0], (p[1], p[2], 0), p[3])
    g = f.sum(axis=1) * dt_
    h = (t[None, :] ** 2 * f).sum(axis=1) * dt_
    np.testing.assert_allclose(G, g, rtol=1e-10)
    np.testing.assert_allclose(H, h, rtol=1e-10)


@pytest.mark.parametrize("dim", [1, 2])
def test_discrete_maxwellian_moments_converge(orc, dim):
    # On a fine velocity grid the midpoint quadrature of a Gaussian is
    # spectrally accurate: the moments of Phi(n, U, theta) return n, U, theta.
    p = (1.7, 0.35, -0.2 if dim == 2 else 0.0, 1.3)
    c = orc.make_config(dim=dim, nx=1, ny=1, nvx=96, nvy=96, vx=(-9, 9), vy=(-9, 9))
    G, H = orc.maxwellian(c, p)
    m = orc.moments(c, G, H)[0]
    np.testing.assert_allclose(m, p, rtol=1e-12, atol=1e-13)


# --------------------------------------------------------------------------
# Eq. (macroscopic) on reduced (g, h) == Eq. (macroscopic) on a full 3D grid
# (brute force), for an arbitrary non-equilibrium f.
# --------------------------------------------------------------------------
def _sym_random(shape, axes, seed):
    r = 0.5 + W.uniform_pm1(seed, int(np.prod(shape))).reshape(shape) * 0.4
    for ax in axes:
        r = 0.5 * (r + np.flip(r, axis=ax))
    return r


def _moments3d(f, cx, cy, cz, d3v):
    CX, CY, CZ = np.meshgrid(cx, cy, cz, indexing="ij")
    n = f.sum() * d3v
    V = np.array([(CX * f).sum(), (CY * f).sum(), (CZ * f).sum()]) * d3v / n
    T = ((((CX - V[0]) ** 2 + (CY - V[1]) ** 2 + (CZ - V[2]) ** 2) * f).sum() * d3v) / (1.5 * n)
    return n, V, T


def test_moments_1d_equal_3d_brute_force(orc):
    c = orc.make_config(dim=1, nx=1, nvx=7, vx=(-2.5, 4.5))
    cx, _ = orc.velocities(c)
    t = (np.arange(6) - 2.5) * 0.8  # symmetric (cy, cz) grid, dc = 0.8
    f = _sym_random((7, 6, 6), axes=(1, 2), seed=11)
    n, V, T = _moments3d(f, cx, t, t, orc.dv(c) * 0.64)
    g = f.sum(axis=(1, 2)) * 0.64
    h = ((t[None, :, None] ** 2 + t[None, None, :] ** 2) * f).sum(axis=(1, 2)) * 0.64
    m = orc.moments(c, g, h)[0]
    np.testing.assert_allclose(m, [n, V[0], 0.0, T], rtol=1e-13, atol=1e-15)


def test_moments_2d_equal_3d_brute_force(orc):
    c = orc.make_config(dim=2, nx=1, ny=1, nvx=5, nvy=4, vx=(-2, 3), vy=(-1.5, 2.5))
    cxv, cyv = orc.velocities(c)
    cx, cy = cxv[:5], cyv[::5]
    t = (np.arange(4) - 1.5) * 0.9
    f = _sym_random((5, 4, 4), axes=(2,), seed=12)
    n, V, T = _moments3d(f, cx, cy, t, orc.dv(c) * 0.9)
    g = (f.sum(axis=2) * 0.9).T.reshape(-1)                    # v = jy*nvx + jx
    h = ((t[None, None, :] ** 2 * f).sum(axis=2) * 0.9).T.reshape(-1)
    m = orc.moments(c, g, h)[0]
    np.testing.assert_allclose(m, [n, V[0], V[1], T], rtol=1e-13, atol=1e-15)


# --------------------------------------------------------------------------
# Effective Maxwellian parameters: the discrete moments of Phi(p_eff) equal
# the target exactly even where the quadrature error is large.
# --------------------------------------------------------------------------
@pytest.mark.parametrize("dim", [1, 2])
def test_effective_params_reproduce_target(orc, dim):
    c = orc.make_config(dim=dim, nx=1, ny=1, nvx=9, nvy=8, vx=(-3.2, 3.6), vy=(-3.4, 3.0))
    q = np.array([1.1, 0.3, -0.15 if dim == 2 else 0.0, 0.9])
    p, it = orc.effective_params(c, q)
    assert it > 1
    assert np.max(np.abs(p - q)) > 1e-6   # the correction is not trivial here
    G, H = orc.maxwellian(c, p)
    cx, cy = orc.velocities(c)
    dv = orc.dv(c)
    # moments of the discrete Maxwellian by brute force
    n = G.sum() * dv
    ux, uy = (cx * G).sum() * dv / n, (cy * G).sum() * dv / n
    e = ((cx * cx + cy * cy) * G + H).sum() * dv
    th = (2.0 / 3.0) * (e / n - ux * ux - uy * uy)
    np.testing.assert_allclose([n, ux, uy, th], q, rtol=1e-13, atol=1e-14)


# --------------------------------------------------------------------------
# Collision sub-step: exact conservation with the correction; exponential
# relaxation of a homogeneous state (Eq. (relaxation)).
# --------------------------------------------------------------------------
def _bimaxwellian(orc, c, a, b, wa=0.6):
    Ga, Ha = orc.maxwellian(c, a)
    Gb, Hb = orc.maxwellian(c, b)
    return wa * Ga + (1 - wa) * Gb, wa * Ha + (1 - wa) * Hb


def _conserved(orc, c, g, h):
    cx, cy = orc.velocities(c)
    dv = orc.dv(c)
    return np.array([g.sum(), (cx * g).sum(), (cy * g).sum(),
                     ((cx * cx + cy * cy) * g + h).sum()]) * dv


@pytest.mark.parametrize("dim", [1, 2])
def test_collision_conserves_mass_momentum_energy(orc, dim):
    c = orc.make_config(dim=dim, nx=3, ny=1, nvx=10, nvy=10, vx=(-4, 4.4), vy=(-4.2, 4),
                        dt=0.3, conservative=1)
    prob = orc.Problem(c)
    g, h = prob.zeros()
    for k in range(prob.ncell):
        g[k], h[k] = _bimaxwellian(orc, c, (1.0, 0.8, 0.1, 0.7), (0.5 + k, -0.6, -0.3, 1.6))
    g1, h1, _ = orc.relax(prob, g, h)
    for k in range(prob.ncell):
        before, after = _conserved(orc, c, g[k], h[k]), _conserved(orc, c, g1[k], h1[k])
        np.testing.assert_allclose(after, before, rtol=0, atol=2e-15 * np.abs(before).max())
    # without the correction the coarse grid visibly breaks conservation
    c.conservative = 0
    g2, h2, _ = orc.relax(orc.Problem(c), g, h)
    err = np.abs(_conserved(orc, c, g2[0], h2[0]) - _conserved(orc, c, g[0], h[0])).max()
    assert err > 1e-8


@pytest.mark.parametrize("dim,exact", [(1, 1), (2, 1), (1, 0), (2, 0)])
def test_homogeneous_relaxation_is_exponential(orc, dim, exact):
    # A homogeneous state keeps n, U, theta, so nu and Phi stay fixed and
    # f_k - Phi = r^k (f_0 - Phi) with r = exp(-nu dt) (Eq. (relaxation)) or
    # r = 1 - nu dt (Euler).  nu = n theta^(1-omega) uses the closed-form
    # moments of the bi-Maxwellian mixture (fine grid: quadrature error ~1e-15).
    omega, dt = 0.74, 0.05
    c = orc.make_config(dim=dim, nx=1, ny=1, nvx=72, nvy=72, vx=(-9, 9), vy=(-9, 9),
                        dt=dt, omega=omega, relax_exact=exact)
    a, b, wa = (1.0, 0.9, 0.2, 0.8), (1.0, -0.5, -0.3, 1.9), 0.6
    if dim == 1:
        a, b = (1.0, 0.9, 0.0, 0.8), (1.0, -0.5, 0.0, 1.9)
    g, h = _bimaxwellian(orc, c, a, b, wa)
    n = 1.0
    U = wa * np.array(a[1:3]) + (1 - wa) * np.array(b[1:3])
    E = wa * (a[1] ** 2 + a[2] ** 2 + 1.5 * a[3]) + (1 - wa) * (b[1] ** 2 + b[2] ** 2 + 1.5 * b[3])
    theta = (E - U @ U) / 1.5
    nu = n * theta ** (1 - omega)
    r = math.exp(-nu * dt) if exact else 1.0 - nu * dt
    prob = orc.Problem(c)
    seq = [(g[None, :], h[None, :])]
    for _ in range(4):
        g1, h1, _ = orc.relax(prob, *seq[-1])
        seq.append((g1, h1))
    d1 = seq[2][0] - seq[1][0]
    d2 = seq[3][0] - seq[2][0]
    big = np.abs(d1) > 1e-3 * np.abs(d1).max()
    np.testing.assert_allclose(d2[big] / d1[big], r, rtol=1e-9)


# --------------------------------------------------------------------------
# Streaming sub-step
# --------------------------------------------------------------------------
def test_integer_courant_shift_is_exact(orc):
    # Courant numbers -3, -1, 1, 3: Eq. (exact) says f~_i = f_{i-C}; outside
    # the domain the inflow Maxwellians of Eq. (bc_shock) enter.
    left, right = (1.0, 0.5, 0.0, 1.0), (2.0, -0.2, 0.0, 1.5)
    c = orc.make_config(dim=1, nx=9, x0=0, lx=9, nvx=4, vx=(-4, 4), dt=1.0,
                        bc_kind=(0, 0, 0, 0), bc_state=(left, right, left, left))
    prob = orc.Problem(c)
    g = 1.0 + W.uniform_pm1(1, 36).reshape(9, 4)
    h = 2.0 + W.uniform_pm1(2, 36).reshape(9, 4)
    gt, ht = orc.stream(prob, g, h)
    Gl, Hl = orc.maxwellian(c, left)
    Gr, Hr = orc.maxwellian(c, right)
    cx, _ = orc.velocities(c)
    for j, C in enumerate(cx.astype(int)):
        for i in range(9):
            src = i - C
            if src < 0:
                exp_g, exp_h = Gl[j], Hl[j]
            elif src >= 9:
                exp_g, exp_h = Gr[j], Hr[j]
            else:
                exp_g, exp_h = g[src, j], h[src, j]
            assert gt[i, j] == exp_g and ht[i, j] == exp_h


@pytest.mark.parametrize("dt", [0.013, 0.37, 1.37])
def test_upwind_transports_linear_profiles_exactly_1d(orc, dt):
    # The donor-cell update (with the integer shift when |C| > 1) moves a
    # linear profile f = a + b x to a + b (x - c dt) at every cell whose
    # stencil lies inside the domain.
    c = orc.make_config(dim=1, nx=12, x0=-3, lx=6, nvx=6, vx=(-1.5, 1.5), dt=dt)
    prob = orc.Problem(c)
    cx, _ = orc.velocities(c)
    x = -3 + (np.arange(12) + 0.5) * 0.5
    a, b = 3.0 + 0.1 * np.arange(6), 0.2 - 0.05 * np.arange(6)
    g = a[None, :] + b[None, :] * x[:, None]
    h = 2 * a[None, :] - b[None, :] * x[:, None]
    gt, ht = orc.stream(prob, g, h)
    for j in range(6):
        C = cx[j] * dt / 0.5
        reach = int(abs(C)) + 1
        inner = range(reach, 12) if C > 0 else range(0, 12 - reach)
        for i in inner:
            assert gt[i, j] == pytest.approx(a[j] + b[j] * (x[i] - cx[j] * dt), rel=1e-14)
            assert ht[i, j] == pytest.approx(2 * a[j] - b[j] * (x[i] - cx[j] * dt), rel=1e-14)


def test_upwind_transports_linear_profiles_exactly_2d(orc):
    c = orc.make_config(dim=2, nx=7, ny=6, lx=7, ly=3, nvx=4, nvy=3, vx=(-2, 2), vy=(-1.5, 1.5),
                        cfl=0.8)
    prob = orc.Problem(c)
    cx, cy = orc.velocities(c)
    ix, iy = np.meshgrid(np.arange(7), np.arange(6), indexing="xy")
    x = ((ix + 0.5) * 1.0).reshape(-1)
    y = ((iy + 0.5) * 0.5).reshape(-1)
    g = 5.0 + 0.3 * x[:, None] - 0.2 * y[:, None] + 0.01 * np.arange(12)[None, :]
    h = 4.0 - 0.1 * x[:, None] + 0.4 * y[:, None] + 0 * g
    gt, ht = orc.stream(prob, g, h)
    for cell in range(42):
        i, k = cell % 7, cell // 7
        if i in (0, 6) or k in (0, 5):
            continue
        xs, ys = x[cell] - cx * c.dt, y[cell] - cy * c.dt
        np.testing.assert_allclose(gt[cell], 5.0 + 0.3 * xs - 0.2 * ys + 0.01 * np.arange(12), rtol=1e-14)
        np.testing.assert_allclose(ht[cell], 4.0 - 0.1 * xs + 0.4 * ys, rtol=1e-14)


def _random_state(prob, seed, base=1.0):
    g = base + 0.5 * W.uniform_pm1(seed, prob.ncell * prob.nv).reshape(prob.ncell, prob.nv)
    h = base + 0.5 * W.uniform_pm1(seed + 1, prob.ncell * prob.nv).reshape(prob.ncell, prob.nv)
    return g, h


@pytest.mark.parametrize("wall", [1, 2])
@pytest.mark.parametrize("dim", [1, 2])
def test_walls_conserve_mass_in_streaming(orc, wall, dim):
    # Diffuse walls (zero-net-mass-flux n_W below Eq. (bc_cavity)) and
    # specular walls: streaming changes no cell's mass except by interior
    # exchange, so the total is conserved to round-off for any state.
    c = orc.make_config(dim=dim, nx=6, ny=5, lx=3, ly=2, nvx=8, nvy=6, vx=(-3, 3), vy=(-2.5, 2.5),
                        cfl=0.9, bc_kind=(wall,) * 4,
                        bc_state=((1, 0, 0.1, 1), (1, 0, -0.2, 1.2), (1, 0.3, 0, 0.9), (1, -0.1, 0, 1.1)))
    prob = orc.Problem(c)
    g, h = _random_state(prob, 21)
    gt, ht = orc.stream(prob, g, h)
    assert gt.sum() == pytest.approx(g.sum(), rel=1e-14)
    for face in range(4 if dim == 2 else 2):
        mass, shear, normal, energy = orc.wall_fluxes(prob, g, h, face)
        scale = np.abs(normal).max()  # size of the one-sided fluxes
        np.testing.assert_allclose(mass, 0.0, atol=1e-14 * scale)
        if wall == 2:   # specular: no shear, no energy exchange
            np.testing.assert_allclose(shear, 0.0, atol=1e-14 * scale)
            np.testing.assert_allclose(energy, 0.0, atol=1e-13 * scale)


def test_wall_flux_equilibrium_pressure(orc):
    # Resting Maxwellian against resting walls at the same temperature: the
    # normal momentum flux is the pressure n theta / 2, shear and energy 0.
    c = orc.make_config(dim=2, nx=3, ny=3, lx=1, ly=1, nvx=48, nvy=48, vx=(-7, 7), vy=(-7, 7),
                        cfl=0.5, bc_kind=(1,) * 4, bc_state=((1, 0, 0, 1),) * 4)
    prob = orc.Problem(c)
    g, h = orc.init_uniform(prob, (1.0, 0.0, 0.0, 1.0))
    for face in range(4):
        mass, shear, normal, energy = orc.wall_fluxes(prob, g, h, face)
        np.testing.assert_allclose(normal, 0.5, rtol=1e-12)
        np.testing.assert_allclose(shear, 0.0, atol=1e-15)
        np.testing.assert_allclose(energy, 0.0, atol=1e-14)
        np.testing.assert_allclose(mass, 0.0, atol=1e-15)


_NC, _THC, _UW, _THW = 1.3, 0.8, 0.37, 1.45   # gas density, temperature; wall speed, temperature


def _moving_wall_fluxes(orc, face, nn, h_factor=None, thw=_THW):
    """orc_wall_fluxes (and orc_lid_shear on the lid face) for a resting
    Maxwellian gas (n_c, theta_c), written here from Eq. (Maxw) reduced to two
    velocity components, G = n/(pi theta) exp(-|c|^2/theta) and H = theta G/2
    unless ``h_factor`` replaces theta/2, against a diffuse wall of ``face``
    moving tangentially at U_W with temperature theta_W.  The velocity box is
    [-10, 10]^2 (Gaussian tails below 1e-40), with ``nn`` nodes along the
    wall normal and 64 along the tangent; 3 x 3 identical cells."""
    xface = face in (orc.XLO, orc.XHI)
    nvx, nvy = (nn, 64) if xface else (64, nn)
    wall = (1.0, 0.0, _UW, thw) if xface else (1.0, _UW, 0.0, thw)
    states = [(1.0, 0.0, 0.0, 1.0)] * 4
    states[face] = wall
    c = orc.make_config(dim=2, nx=3, ny=3, lx=1.5, ly=1.5, nvx=nvx, nvy=nvy, vx=(-10, 10),
                        vy=(-10, 10), dt=1e-3, bc_kind=(1,) * 4, bc_state=tuple(states))
    prob = orc.Problem(c)
    cx, cy = orc.velocities(c)
    G = _NC / (math.pi * _THC) * np.exp(-(cx ** 2 + cy ** 2) / _THC)
    H = (0.5 * _THC if h_factor is None else h_factor) * G
    g, h = np.tile(G, (prob.ncell, 1)), np.tile(H, (prob.ncell, 1))
    out = np.array(orc.wall_fluxes(prob, g, h, face))   # (mass, shear, normal, energy) x 3 face cells
    J = orc.lid_shear(prob, g, h) if face == orc.YHI else None
    return out, J


@pytest.mark.parametrize("face", [0, 1, 2, 3])
def test_wall_fluxes_moving_hot_wall_closed_form(orc, face):
    # Pins orc_wall_fluxes (mass, shear, normal momentum, energy) and
    # orc_lid_shear with non-zero closed forms: the zero-net-mass-flux diffuse
    # wall below Eq. (bc_cavity), moving tangentially at U_W with temperature
    # theta_W, facing a resting Maxwellian gas (n_c, theta_c).
    #
    # Per unit density, a resting reduced Maxwellian at temperature theta
    # carries, over the half-space of velocities moving one way along the
    # normal (1D half-range Gaussian integrals, the tangential factor being 1):
    #   int |c_n| G           = sqrt(theta) / (2 sqrt(pi))       (particle flux)
    #   int c_n^2 G           = theta / 4                        (half the pressure)
    #   int |c_n| c_n^2 G     = theta^(3/2) / (2 sqrt(pi))
    # and over the full tangential line int c_t G = U_t, int c_t^2 G = theta/2 + U_t^2;
    # the Chu function H = theta G / 2 adds theta/2 per particle to |c|^2.
    # Incident particle flux: Gamma = n_c sqrt(theta_c) / (2 sqrt(pi)).  The
    # wall density n_W makes the emitted flux equal it, so
    #   n_W = n_c sqrt(theta_c / theta_W),
    #   mass   = 0,
    #   shear  = sum c_t c_n F dV = U_W Gamma   (only emitted particles carry c_t),
    #   normal = sum c_n^2 F dV = (n_c theta_c + n_W theta_W) / 4,
    #   energy = sum c_n (|c|^2 g + h) dV
    #          = Gamma [theta_W + theta_W/2 + U_W^2 + theta_W/2]        (emitted)
    #          - Gamma [theta_c + theta_c/2 + theta_c/2]                 (incident)
    #          = Gamma (2 theta_W - 2 theta_c + U_W^2),
    #   lid shear J = L_x * shear (on the lid face).
    # The oracle's half-range sums are midpoint rules on [0, 10] whose error
    # expands in even powers of the node spacing (Euler-Maclaurin; the cut at
    # c_n = 0 falls on a cell edge), so three spacings extrapolated by
    # Richardson leave an O(h^6) error, measured at 3e-12 of the largest flux.
    F = {nn: _moving_wall_fluxes(orc, face, nn) for nn in (400, 800, 1600)}
    r1 = (4 * F[800][0] - F[400][0]) / 3
    r2 = (4 * F[1600][0] - F[800][0]) / 3
    ext = (16 * r2 - r1) / 15
    gam = _NC * math.sqrt(_THC) / (2 * math.sqrt(math.pi))
    closed = np.array([0.0, _UW * gam, _NC * (_THC + math.sqrt(_THC * _THW)) / 4,
                       gam * (2 * _THW - 2 * _THC + _UW ** 2)])
    scale = np.abs(closed).max()
    for k in range(4):
        np.testing.assert_allclose(ext[k], closed[k], rtol=0, atol=1e-11 * scale)
    # mass is zero exactly at every spacing, not only in the limit
    np.testing.assert_allclose(F[400][0][0], 0.0, atol=1e-14 * scale)
    if face == orc.YHI:
        Js = {nn: F[nn][1] for nn in F}
        j1 = (4 * Js[800] - Js[400]) / 3
        j2 = (4 * Js[1600] - Js[800]) / 3
        assert (16 * j2 - j1) / 15 == pytest.approx(1.5 * _UW * gam, rel=1e-11)


@pytest.mark.parametrize("face", [0, 3])
def test_wall_fluxes_exact_discrete_relations(orc, face):
    # Pins the same function at one spacing (64 nodes over [-10, 10]), where
    # the half-range sums are still about 1e-2 from their limits, through
    # relations that hold for the discrete sums exactly: at this spacing the
    # full-line sums of a Gaussian (the tangential factors, and the normal
    # pressure below) converge spectrally, to below 1e-30.
    # (1) Only incident particles carry the gas's h, with weight c_n < 0, so
    #     the energy flux changes by -(k1 - k0) Gamma_d when h = k G replaces
    #     h = k0 G; and the shear is U_W Gamma_d with the same discrete
    #     incident particle flux Gamma_d.  Hence
    #     (e(k1) - e(k0)) / shear = -(k1 - k0) / U_W.
    # (2) With theta_W = theta_c the half-range sums of both halves coincide,
    #     n_W = n_c, and energy = U_W^2 Gamma_d = U_W * shear, while the normal
    #     flux is the full-range pressure n_c theta_c / 2.
    out0, _ = _moving_wall_fluxes(orc, face, 64, h_factor=0.0)
    out1, _ = _moving_wall_fluxes(orc, face, 64, h_factor=0.7)
    shear = out0[1]
    np.testing.assert_allclose((out1[3] - out0[3]) / shear, -0.7 / _UW, rtol=1e-12)
    np.testing.assert_allclose(out1[1], shear, rtol=1e-14)
    iso, _ = _moving_wall_fluxes(orc, face, 64, thw=_THC)
    np.testing.assert_allclose(iso[3], _UW * iso[1], rtol=1e-12)
    np.testing.assert_allclose(iso[2], _NC * _THC / 2, rtol=1e-12)


# --------------------------------------------------------------------------
# Whole steps: invariants of the two problems of the paper
# --------------------------------------------------------------------------
def test_global_equilibrium_stays_fixed(orc):
    # Gas at rest in a resting isothermal box: Phi_W equals the gas's
    # distribution and, with the correction, the discrete Maxwellian is the
    # state itself, so no sub-step changes anything.
    w = W.scaled(W.CAVITY_64, n=10, nv=12, lid_mach=0.0, steps=0)
    prob, g, h = orc.cavity_problem(**w)
    g1, h1, _ = orc.step(prob, g, h, 30)
    np.testing.assert_allclose(g1, g, rtol=2e-14, atol=1e-30)
    np.testing.assert_allclose(h1, h, rtol=2e-14, atol=1e-30)
    # uniform flow through inflow boundaries (Mach 1: RH is the identity)
    w1 = W.scaled(W.SHOCK_M2, mach=1.0, nx=20)
    prob, g, h = orc.shock_problem(**w1)
    g1, h1, _ = orc.step(prob, g, h, 30)
    np.testing.assert_allclose(g1, g, rtol=2e-14, atol=1e-30)


def test_cavity_conserves_mass_and_lid_drives_flow(orc):
    w = W.scaled(W.CAVITY_64, n=12, nv=12, steps=0)
    prob, g, h = orc.cavity_problem(**w)
    xi = W.perturbation(0, prob.ncell, prob.nv)
    prob, g, h = orc.cavity_problem(**w, xi=xi)
    g1, h1, mom = orc.step(prob, g, h, 300)
    assert g1.sum() == pytest.approx(g.sum(), rel=1e-13)
    top = mom.reshape(12, 12, 4)[-1]
    assert np.all(top[:, 1] > 0)           # gas under the lid follows it
    bottom = mom.reshape(12, 12, 4)[1]
    assert np.mean(bottom[:, 1]) < 0       # return flow lower down


@pytest.mark.slow
def test_shock_reaches_rankine_hugoniot_states(orc):
    # Full 1D shock problem (Mach 2, 200 cells, 64 velocities, 4000 steps):
    # the ends sit at the Rankine-Hugoniot states and the mass flux n u is
    # uniform to the 1% left by the shock still settling at t = 50.8.
    prob, g, h = orc.shock_problem(**W.SHOCK_M2)
    g1, h1, mom = orc.step(prob, g, h, prob.steps)
    up, down = prob.meta["up"], prob.meta["down"]
    np.testing.assert_allclose(mom[0][[0, 1, 3]], up[[0, 1, 3]], rtol=2e-5)
    np.testing.assert_allclose(mom[-1][[0, 1, 3]], down[[0, 1, 3]], rtol=5e-4)
    flux = mom[:, 0] * mom[:, 1]
    assert np.ptp(flux) / flux.mean() < 2e-2
    np.testing.assert_allclose(flux[[0, -1]], up[0] * up[1], rtol=2e-4)
    # the profile is monotone from the upstream to the downstream density
    assert np.all(np.diff(mom[:, 0]) > -1e-4)
