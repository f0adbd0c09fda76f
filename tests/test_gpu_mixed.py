"""Reduced-precision forms (FP32 state; BF16 deviation from the absolute
Maxwellian) against the FP64 oracle.

One step, element by element: FP32 rounds a value at most six times per
step (four operations of the flux-form streaming, two of the relaxation)
plus once on the way in, each by 2^-24 of operands within the local max|f|:
7 2^-24 = 4.2e-7, so 2e-6 of max|f|.  BF16 keeps 8 significant bits of the
deviation d = f - M_abs: the initial rounding to nearest is at most 2^-8 |d|
and a stochastic rounding (used for the stored steps) at most 2^-7 |d|;
with the FP32 arithmetic on top, 1.2e-2 max|d| + 2e-6 max|f|.  Runs: the
moment and mass bounds of tests/precision_bounds.py (storage precision
only, see there), evaluated for each run's steps and grid.
"""
import numpy as np
import pytest

import oracle
import precision_bounds as PB
from paper_0903_4044_gb300 import bgk as B
from paper_0903_4044_gb300 import build, solver
from paper_0903_4044_gb300 import workloads as W

pytestmark = pytest.mark.gpu

PRECS = {"f32": B.BGK_F32, "bf16": B.BGK_BF16_DEV}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    oracle.build()
    B.lib()


def _pair(w, prec):
    prob0, _, _ = oracle.cavity_problem(**w)
    xi = W.perturbation(w.get("seed", 0), prob0.ncell, prob0.nv)
    prob, g, h = oracle.cavity_problem(**w, xi=xi)
    s = solver.make_cavity(w, xi=xi, precision=prec)
    return s, prob, g, h


def _mabs(prob):
    return oracle.maxwellian(prob.cfg, (1.0, 0.0, 0.0, 1.0))


def _check_state(name, st, prob, g, h):
    gg, hh = st[..., 0], st[..., 1]
    if name == "f32":
        eg = np.abs(gg - g).max() / np.abs(g).max()
        eh = np.abs(hh - h).max() / np.abs(h).max()
        assert eg < 2e-6 and eh < 2e-6, (eg, eh)
    else:
        Gm, Hm = _mabs(prob)
        dg, dh = g - Gm[None, :], h - Hm[None, :]
        tg = 1.2e-2 * np.abs(dg).max() + 2e-6 * np.abs(g).max()
        th = 1.2e-2 * np.abs(dh).max() + 2e-6 * np.abs(h).max()
        assert np.abs(gg - g).max() < tg and np.abs(hh - h).max() < th


def _moment_err(m, ref, uscale):
    en = np.abs(m[:, 0] - ref[:, 0]).max() / np.abs(ref[:, 0]).max()
    et = np.abs(m[:, 3] - ref[:, 3]).max() / np.abs(ref[:, 3]).max()
    eu = np.abs(m[:, 1:3] - ref[:, 1:3]).max() / uscale
    return en, eu, et


@pytest.mark.parametrize("name", ["f32", "bf16"])
def test_mixed_one_step_elementwise(name):
    w = W.scaled(W.CAVITY_64, n=20, nv=24, amp=1e-2)
    s, prob, g, h = _pair(w, PRECS[name])
    s.step(1)
    g1, h1, _ = oracle.step(prob, g, h, 1)
    _check_state(name, s.get_state(), prob, g1, h1)
    s.close()


def _bounds(name, s, w, steps):
    """precision_bounds for this solver's run (n and theta relative, U over U_W)."""
    uw = w["lid_mach"] * np.sqrt(5.0 / 6.0)
    if name == "f32":
        b = PB.f32(steps)
    else:
        ncell = s.ncell
        b = PB.bf16(steps, s.nv, s.info.dv, ncell, s.info.dx, s.info.dt, uw, w["lid_mach"], w["amp"])
    return {"n": b["n"], "u": b["u"] / uw, "theta": b["theta"], "mass": b["mass"]}, uw


@pytest.mark.parametrize("name", ["f32", "bf16"])
def test_mixed_run_moments(name):
    # 300 steps of a 24 x 24 cavity, 32 x 32 velocities, lid Mach 0.1
    w = W.scaled(W.CAVITY_64, n=24, nv=32)
    s, prob, g, h = _pair(w, PRECS[name])
    s.step(300)
    g1, h1, _ = oracle.step(prob, g, h, 300)
    ref = oracle.state_moments(prob, g1, h1)
    b, uw = _bounds(name, s, w, 300)
    en, eu, et = _moment_err(s.moments(), ref, uscale=uw)
    print(name, f"n {en:.2e} / {b['n']:.2e}  U {eu:.2e} / {b['u']:.2e}  theta {et:.2e} / {b['theta']:.2e}")
    assert en <= b["n"] and eu <= b["u"] and et <= b["theta"], (en, eu, et, b)
    s.close()


@pytest.mark.parametrize("name", ["f32", "bf16"])
def test_mixed_conserves_mass(name):
    # diffuse walls + conservative collision: mass changes only by rounding
    w = W.scaled(W.CAVITY_64, n=24, nv=32)
    s, prob, g, h = _pair(w, PRECS[name])
    n0 = s.moments()[:, 0].sum()
    s.step(1000)
    n1 = s.moments()[:, 0].sum()
    b, _ = _bounds(name, s, w, 1000)
    print(name, f"mass drift {abs(n1 - n0) / n0:.2e} / {b['mass']:.2e}")
    assert abs(n1 - n0) / n0 <= b["mass"], abs(n1 - n0) / n0
    s.close()


def test_bf16_stochastic_rounding_is_unbiased():
    # A homogeneous bi-Maxwellian (temperatures 1.3, 1.1, 1.2 along x, y, z)
    # between specular walls: streaming leaves it unchanged and the
    # relaxation, which conserves n, U and theta, damps the anisotropy
    # A = sum (c_x^2 - c_y^2) g dv by exactly b = exp(-nu dt) per step (the
    # discrete Maxwellian of a grid symmetric in c_x and c_y has none).  At
    # Kn 6 on 16 cells (dt = 1e-3) a step changes a deviation by about 1e-3 of
    # its distance to the Maxwellian, far below half a BF16 ulp of the
    # deviation: round-to-nearest storage would leave A where it started,
    # while unbiased stochastic rounding follows b^N on average.
    # Bound: each store adds a zero-mean error of standard deviation at most
    # 2^-8 |d| per value; A's error decays like A, so it settles at a standard
    # deviation of at most sigma_step / sqrt(2 (1 - b)) per cell,
    # sigma_step = sqrt(sum (c_x^2 - c_y^2)^2 (2^-8 max|d|)^2) dv, and the mean
    # over the cells at that over sqrt(cells); the test allows six of those,
    # plus the initial rounding to nearest, 2^-8 sum |c_x^2 - c_y^2| |d| dv, times b^N.
    n, nv, box = 16, 32, 5.5
    side = 1.0 / 6.0
    cfg = B.make_config(dim=2, nx=n, ny=n, lx=side, ly=side, nvx=nv, nvy=nv, vx=(-box, box), vy=(-box, box),
                        cfl=0.5, precision=B.BGK_BF16_DEV, bc=[(B.BGK_BC_SPECULAR, 1, 0, 0, 1)] * 4)
    s = solver.Solver(cfg)
    c = -box + (np.arange(nv) + 0.5) * (2 * box / nv)
    cx, cy = np.meshgrid(c, c)          # v = jy * nvx + jx
    cx, cy = cx.ravel(), cy.ravel()
    dv = (2 * box / nv) ** 2
    tx, ty, tz = 1.3, 1.1, 1.2
    g = np.exp(-cx ** 2 / tx - cy ** 2 / ty) / (np.pi * np.sqrt(tx * ty))
    f0 = np.stack([g, 0.5 * tz * g], axis=-1)[None].repeat(n * n, axis=0)
    s.set_state(np.ascontiguousarray(f0))
    w = cx ** 2 - cy ** 2
    A0 = float((w * g).sum() * dv)
    nden = g.sum() * dv
    theta = (2.0 / 3.0) * (((cx ** 2 + cy ** 2) * g + 0.5 * tz * g).sum() * dv) / nden
    b = np.exp(-nden * np.sqrt(theta) * s.info.dt)
    steps = int(round(1.0 / (1.0 - b)))          # nu t = 1
    s.step(steps)
    st = s.get_state()
    s.close()
    A = float(((st[..., 0] * w[None]).sum(axis=1) * dv).mean())
    mabs = np.exp(-(cx ** 2 + cy ** 2)) / np.pi
    geq = nden * np.exp(-(cx ** 2 + cy ** 2) / theta) / (np.pi * theta)
    dmax = np.maximum(np.abs(g - mabs), np.abs(geq - mabs))
    sigma = np.sqrt((w ** 2 * (2.0 ** -8 * dmax) ** 2).sum()) * dv / np.sqrt(2 * (1 - b)) / n
    bound = 6 * sigma + 2.0 ** -8 * (np.abs(w) * np.abs(g - mabs)).sum() * dv * b ** steps
    want = A0 * b ** steps
    print(f"A0 {A0:.4f} A {A:.5f} want {want:.5f} bound {bound:.5f}")
    assert abs(A - want) <= bound, (A, want, bound)
    assert abs(A0 - want) > 3 * bound          # round-to-nearest (A stuck near A0) would fail


@pytest.mark.parametrize("name", ["f32", "bf16"])
def test_mixed_variants_and_tiles(name):
    # specular walls, Euler relaxation, every tile size, non-square grids
    for tile in (1, 2, 4, 8):
        w = W.scaled(W.CAVITY_64, n=11, nv=16, amp=1e-2, tile_cells=tile, relax_exact=tile % 2,
                     wall="specular" if tile == 4 else "diffuse")
        s, prob, g, h = _pair(w, PRECS[name])
        assert s.info.tile_cells == tile
        s.step(3)
        g1, h1, _ = oracle.step(prob, g, h, 3)
        st = s.get_state()
        if name == "f32":
            assert np.abs(st[..., 0] - g1).max() / np.abs(g1).max() < 6e-6
        else:
            Gm, _ = _mabs(prob)
            assert np.abs(st[..., 0] - g1).max() < 3e-2 * np.abs(g1 - Gm).max() + 6e-6 * np.abs(g1).max()
        s.close()


@pytest.mark.parametrize("name", ["f32", "bf16"])
def test_mixed_tile1_large_velocity_grid(name):
    # 56 x 56 velocities: four groups of four per streaming thread of the
    # pipelined tile-1 kernel (the last ragged), fewer cells than CTAs
    w = W.scaled(W.CAVITY_64, n=6, nv=56, amp=1e-2, tile_cells=1)
    s, prob, g, h = _pair(w, PRECS[name])
    assert s.info.tile_cells == 1
    s.step(2)
    g1, h1, _ = oracle.step(prob, g, h, 2)
    st = s.get_state()
    if name == "f32":
        assert np.abs(st[..., 0] - g1).max() / np.abs(g1).max() < 4e-6
        assert np.abs(st[..., 1] - h1).max() / np.abs(h1).max() < 4e-6
    else:
        Gm, _ = _mabs(prob)
        assert np.abs(st[..., 0] - g1).max() < 3e-2 * np.abs(g1 - Gm).max() + 4e-6 * np.abs(g1).max()
    s.close()


def test_mixed_full_size_one_step():
    # The 256 x 256 x 48 x 48 grid in FP32 and BF16, one step, whole state.
    w = W.scaled(W.CAVITY_256)
    prob0, _, _ = oracle.cavity_problem(**w)
    xi = W.perturbation(0, prob0.ncell, prob0.nv)
    prob, g, h = oracle.cavity_problem(**w, xi=xi)
    g1, h1, _ = oracle.step(prob, g, h, 1)
    for name in ("f32", "bf16"):
        s = solver.make_cavity(w, xi=xi, precision=PRECS[name])
        s.step(1)
        _check_state(name, s.get_state(), prob, g1, h1)
        s.close()


@pytest.mark.parametrize("nv", [16, 24])
def test_mixed_state_roundtrip(nv):
    # 24 x 24 velocities: 144 groups of 4, the last chunk of the FP32
    # storage order holds 16 groups instead of 32
    import torch

    w = W.scaled(W.CAVITY_64, n=9, nv=nv, amp=1e-2)
    for name in ("f32", "bf16"):
        s, prob, g, h = _pair(w, PRECS[name])
        st = s.get_state()
        d = torch.empty(st.shape, dtype=torch.float64, device="cuda")
        B.bgk_get_state(s.h, d)
        torch.cuda.synchronize()
        assert np.array_equal(d.cpu().numpy(), st)
        B.bgk_set_state(s.h, d)        # device FP64 -> storage
        assert np.array_equal(s.get_state(), st)
        s.set_state(st)                 # host FP64 -> storage
        assert np.array_equal(s.get_state(), st)
        s.close()


# ---------------------------------------------------------------------------
# 1D (normal shock), FP32 state
# ---------------------------------------------------------------------------
def test_shock_f32_one_step_elementwise():
    w = W.SHOCK_M2
    s = solver.make_shock(w, precision=B.BGK_F32)
    prob, g, h = oracle.shock_problem(**w)
    s.step(1)
    g1, h1, _ = oracle.step(prob, g, h, 1)
    st = s.get_state()
    eg = np.abs(st[..., 0] - g1).max() / np.abs(g1).max()
    eh = np.abs(st[..., 1] - h1).max() / np.abs(h1).max()
    assert eg < 2e-6 and eh < 2e-6, (eg, eh)
    s.close()


@pytest.mark.parametrize("cfl", [0.5, 2.6])
def test_shock_f32_run(cfl):
    # The Mach 2 shock run in FP32 against the FP64 oracle.  The shock's
    # position is neutrally stable, so FP32 rounding makes it wander
    # (measured: 1e-3 cells after 4000 steps, errors 4e-8 after 10 steps and
    # 2e-6 after 1000); that wander dominates the field error at the shock
    # (5.5e-5 measured), the far field stays within 2e-5.  Bounds: shock
    # position 1e-2 cells, fields 2e-4 at the shock and 1e-4 elsewhere.
    w = W.scaled(W.SHOCK_M2, cfl=cfl, steps=4000 if cfl == 0.5 else 800)
    s = solver.make_shock(w, precision=B.BGK_F32)
    prob, g, h = oracle.shock_problem(**w)
    s.step(w["steps"])
    g1, h1, _ = oracle.step(prob, g, h, w["steps"])
    m_orc = oracle.state_moments(prob, g1, h1)
    m = s.moments()
    en = np.abs(m[:, 0] - m_orc[:, 0]) / m_orc[:, 0]
    eu = np.abs(m[:, 1] - m_orc[:, 1]) / np.abs(m_orc[:, 1]).max()
    et = np.abs(m[:, 3] - m_orc[:, 3]) / m_orc[:, 3]
    err = np.maximum(np.maximum(en, eu), et)
    assert err.max() < 2e-4, (en.max(), eu.max(), et.max())
    x = np.arange(len(err))
    mid = 0.5 * (m_orc[0, 0] + m_orc[-1, 0])
    shock = np.interp(mid, m_orc[:, 0], x)
    far = np.abs(x - shock) > 40
    assert err[far].max() < 1e-4, err[far].max()
    assert abs(np.interp(mid, m[:, 0], x) - shock) < 1e-2
    s.close()


def test_shock_reduced_precision_restrictions():
    cfg, _, _ = solver.shock_config(**W.SHOCK_M2, precision=B.BGK_BF16_DEV)
    with pytest.raises(B.BgkError) as e:
        solver.Solver(cfg)
    assert e.value.status == B.BGK_ERR_UNSUPPORTED


@pytest.mark.parametrize("name", ["f32", "bf16"])
def test_full_size_one_step(name):
    # the 256x256 x 48x48 cavity the benchmark times (automatic tile), one
    # step from the perturbed rest state, the whole state against the oracle
    s, prob, g, h = _pair(W.CAVITY_256, PRECS[name])
    s.step(1)
    g1, h1, _ = oracle.step(prob, g, h, 1)
    st = np.empty((s.ncell, s.nv, 2))
    B.bgk_get_state(s.h, st)
    _check_state(name, st, prob, g1, h1)
    s.close()
