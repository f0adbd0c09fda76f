"""The GPU reverse pass of the lid-integrated shear (through the C ABI).

Checks, in order of independence from the code under test:
  * against the oracle's CPU reverse pass on the same seeded states (both
    linearise the effective-parameter map by the identity, so they agree to
    rounding): J to 1e-12, dJ/d ln L and dJ/dU_W to 1e-10 relative, dJ/df0
    element by element to 1e-10 of its largest entry;
  * against central finite differences (h = 1e-6) of the GPU's own FP64
    forward run, for Kn, the lid speed and a direction over 1e4 seeded
    entries of f0.  The forward solves the effective parameters to 1e-13
    relative, so a difference quotient carries about 1e-13 / 1e-6 = 1e-7 of
    relative noise; the tolerance is 1e-5;
  * checkpoint spacing changes nothing (the recomputed states and the
    reverse sums are deterministic): bitwise equality;
  * the torch.autograd.Function passes the same numbers through backward.
"""
import math

import numpy as np
import pytest

import oracle
from paper_0903_4044_gb300 import adjoint as A
from paper_0903_4044_gb300 import bgk as B
from paper_0903_4044_gb300 import build, solver
from paper_0903_4044_gb300 import workloads as W

pytestmark = pytest.mark.gpu

H = 1e-6
TOL_FD = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    oracle.build()
    B.lib()


# walls: (kind, n, ux, uy, theta) for XLO, XHI, YLO, YHI
WALLS_DIFFUSE = ((1, 1, 0, 0, 1.0), (1, 1, 0, 0.1, 1.2), (1, 1, -0.2, 0, 0.9), (1, 1, 0.3, 0, 1.1))
WALLS_MIXED = ((2, 1, 0, 0, 1.0), (2, 1, 0, 0, 1.0), (1, 1, 0.05, 0, 0.95), (1, 1, 0.25, 0, 1.05))


def _pair(nx, ny, nv, vbox, walls, cons, cfl=0.7, scale=1.0, seed=3):
    """(gpu solver, oracle problem, g0, h0) for a rectangle with the given walls."""
    lx, ly = 2.0 * scale * nx / 4, 2.0 * scale * ny / 4
    kinds = tuple(w[0] for w in walls)
    states = tuple(tuple(w[1:]) for w in walls)
    ocfg = oracle.make_config(dim=2, nx=nx, ny=ny, lx=lx, ly=ly, nvx=nv, nvy=nv, vx=(-vbox, vbox),
                              vy=(-vbox, vbox), cfl=cfl, conservative=cons, bc_kind=kinds, bc_state=states)
    prob = oracle.Problem(ocfg)
    xi = W.perturbation(seed, prob.ncell, prob.nv)
    g, h = oracle.init_uniform(prob, (1.0, 0.05, -0.03, 1.0), xi, 0.2)
    gcfg = B.make_config(dim=2, nx=nx, ny=ny, lx=lx, ly=ly, nvx=nv, nvy=nv, vx=(-vbox, vbox), vy=(-vbox, vbox),
                         cfl=cfl, conservative=cons, bc=list(walls))
    s = solver.Solver(gcfg)
    s.set_state(np.ascontiguousarray(np.stack([g, h], axis=-1)))
    return s, prob, g, h


def _grad(s, nsteps, k):
    grad = np.zeros((s.ncell, s.nv, 2))
    J, dlnl, duw = B.bgk_adjoint_lid_shear(s.h, nsteps, k, grad)
    return J, dlnl, duw, grad


# ---------------------------------------------------------------------------
# against the oracle's reverse pass
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("walls,cons,nx,ny,nv,vbox,steps,k", [
    (WALLS_DIFFUSE, 0, 7, 5, 8, 4.0, 11, 4),
    (WALLS_DIFFUSE, 1, 9, 6, 20, 6.0, 13, 5),
    (WALLS_MIXED, 1, 6, 8, 16, 5.0, 9, 2),
])
def test_matches_oracle_reverse_pass(walls, cons, nx, ny, nv, vbox, steps, k):
    s, prob, g, h = _pair(nx, ny, nv, vbox, walls, cons)
    J, dlnl, duw, grad = _grad(s, steps, k)
    oJ, odlnl, oduw, odg, odh = oracle.adjoint_lid_shear(prob, g, h, steps)
    assert J == pytest.approx(oJ, rel=1e-12)
    assert dlnl == pytest.approx(odlnl, rel=1e-10)
    assert duw == pytest.approx(oduw, rel=1e-10)
    ref = np.stack([odg, odh], axis=-1)
    err = np.abs(grad - ref).max() / np.abs(ref).max()
    assert err <= 1e-10, f"dJ/df0 max rel err {err:.3e}"
    # the solver is left at the state after `steps`
    g1, h1, _ = oracle.step(prob, g, h, steps)
    st = s.get_state()
    assert np.abs(st[..., 0] - g1).max() <= 1e-13 * np.abs(g1).max()
    s.close()


def test_checkpoint_spacing_changes_nothing():
    outs = []
    for k in (1, 3, 17, 40, 0):   # 0: ceil(sqrt(17)) = 5 steps per checkpoint
        s, _, _, _ = _pair(8, 8, 12, 5.0, WALLS_DIFFUSE, 1)
        outs.append(_grad(s, 17, k))
        s.close()
    for o in outs[1:]:
        assert o[:3] == outs[0][:3]
        assert np.array_equal(o[3], outs[0][3])


def test_device_output_and_final_state():
    import torch

    s, prob, g, h = _pair(8, 7, 12, 5.0, WALLS_DIFFUSE, 1)
    dev = torch.zeros((s.ncell, s.nv, 2), dtype=torch.float64, device="cuda")
    J, dlnl, duw = B.bgk_adjoint_lid_shear(s.h, 9, 4, dev)
    host = np.zeros((s.ncell, s.nv, 2))
    s.set_state(np.ascontiguousarray(np.stack([g, h], axis=-1)))
    J2, dlnl2, duw2 = B.bgk_adjoint_lid_shear(s.h, 9, 4, host)
    assert (J, dlnl, duw) == (J2, dlnl2, duw2)
    assert np.array_equal(dev.cpu().numpy(), host)
    # the forward left behind equals plain stepping
    ref = solver.Solver(s.cfg)
    ref.set_state(np.ascontiguousarray(np.stack([g, h], axis=-1)))
    ref.step(9)
    assert np.array_equal(ref.get_state(), s.get_state())
    ref.close()
    s.close()


def test_rejections():
    s = solver.make_shock(W.scaled(W.SHOCK_M2, nx=20, nvx=16))
    with pytest.raises(B.BgkError) as e:
        B.bgk_adjoint_lid_shear(s.h, 4, 2, None)
    assert e.value.status == B.BGK_ERR_UNSUPPORTED
    s.close()
    w = W.scaled(W.CAVITY_64, n=8, nv=16)
    for over, code in (({"precision": B.BGK_F32}, B.BGK_ERR_UNSUPPORTED),
                       ({"wall": "specular"}, B.BGK_ERR_UNSUPPORTED)):
        s = solver.make_cavity(w, **over)
        with pytest.raises(B.BgkError) as e:
            B.bgk_adjoint_lid_shear(s.h, 4, 2, None)
        assert e.value.status == code
        s.close()
    s = solver.make_cavity(w)
    for n, k in ((0, 1), (4, -1)):
        with pytest.raises(B.BgkError) as e:
            B.bgk_adjoint_lid_shear(s.h, n, k, None)
        assert e.value.status == B.BGK_ERR_INVALID_ARG
    s.close()


# ---------------------------------------------------------------------------
# against finite differences of the GPU forward run
# ---------------------------------------------------------------------------
def _f0(w):
    import torch

    prob0, _, _ = oracle.cavity_problem(**w)
    s = solver.make_cavity(w, xi=W.perturbation(w.get("seed", 0), prob0.ncell, prob0.nv))
    f0 = torch.from_numpy(s.get_state()).cuda()
    s.close()
    return f0


def _lid_speed(w):
    return w["lid_mach"] * math.sqrt(solver.GAMMA / 2.0)


def _direction(ncell, nv, count, seed):
    """count seeded entries of the state (distinct), with values in [-1, 1)."""
    size = ncell * nv * 2
    u = (W.uniform_pm1(seed, 4 * count) + 1.0) * 0.5
    idx = np.unique((u * size).astype(np.int64))[:count]
    assert idx.size == count
    v = np.zeros(size)
    v[idx] = W.uniform_pm1(seed + 1, count)
    return v.reshape(ncell, nv, 2)


def _fd_checks(w, nsteps, k, entries):
    import torch

    spec = A.cavity_spec(w, nsteps, k)
    f0 = _f0(w)
    kn, uw = w["kn"], _lid_speed(w)
    grad = torch.empty_like(f0)
    J, dkn, duw = A.lid_shear_and_gradient(spec, f0, kn, uw, grad)
    assert J == pytest.approx(A.lid_shear(spec, f0, kn, uw), rel=1e-12)
    fd = (A.lid_shear(spec, f0, kn + H, uw) - A.lid_shear(spec, f0, kn - H, uw)) / (2 * H)
    assert dkn == pytest.approx(fd, rel=TOL_FD), (dkn, fd)
    fd = (A.lid_shear(spec, f0, kn, uw + H) - A.lid_shear(spec, f0, kn, uw - H)) / (2 * H)
    assert duw == pytest.approx(fd, rel=TOL_FD), (duw, fd)
    v = torch.from_numpy(_direction(f0.shape[0], f0.shape[1], entries, 11)).cuda()
    fd = (A.lid_shear(spec, f0 + H * v, kn, uw) - A.lid_shear(spec, f0 - H * v, kn, uw)) / (2 * H)
    ad = float((grad * v).sum())
    assert ad == pytest.approx(fd, rel=TOL_FD), (ad, fd)


def test_finite_differences_small_cavity():
    w = W.scaled(W.CAVITY_128, n=24, nv=24)
    _fd_checks(w, 60, 16, 2000)


def test_finite_differences_full_size():
    # 128 x 128 cells, 32 x 32 velocities, Kn 0.1, lid Mach 0.1, 2000 steps,
    # a checkpoint every 100 steps, 1e4 seeded entries of f0
    _fd_checks(W.CAVITY_128, W.CAVITY_128["steps"], 100, 10000)


def test_finite_differences_single_entries_full_size():
    # 20 individual entries of dJ/df0 at full size (128 x 128 cells, 32 x 32
    # velocities, 2000 steps, a checkpoint every 100): in ten cells (the lid's
    # corners and middle, the row below it, the interior, the three other
    # walls) the entry with the largest |dJ/df0| of the cell and one seeded
    # entry, g or h.  A central difference with h = 1e-6 carries the rounding
    # of the two forward runs: J is reproduced to about 1e-15 relative, so
    # the quotient has an absolute noise of about 1e-15 |J| / (2h); the bound
    # allows ten times that plus 1e-5 relative.
    import torch

    w = W.CAVITY_128
    spec = A.cavity_spec(w, w["steps"], 100)
    f0 = _f0(w)
    kn, uw = w["kn"], _lid_speed(w)
    grad = torch.empty_like(f0)
    J, _, _ = A.lid_shear_and_gradient(spec, f0, kn, uw, grad)
    g = grad.cpu().numpy()
    n, nv = w["n"], f0.shape[1]
    floor = 10 * 1e-15 * abs(J) / (2 * H)
    cells = [(64, 127), (0, 127), (127, 127), (64, 126), (30, 110), (64, 64), (10, 0), (127, 40), (0, 90),
             (90, 20)]
    u = (W.uniform_pm1(17, 2 * len(cells)) + 1.0) * 0.5
    checked = 0
    for i, (ix, iy) in enumerate(cells):
        c = iy * n + ix
        vmax, kmax = np.unravel_index(np.abs(g[c]).argmax(), g[c].shape)
        for v, k in ((int(vmax), int(kmax)), (int(u[2 * i] * nv), int(u[2 * i + 1] * 2))):
            e = torch.zeros_like(f0)
            e[c, v, k] = H
            fd = (A.lid_shear(spec, f0 + e, kn, uw) - A.lid_shear(spec, f0 - e, kn, uw)) / (2 * H)
            ad = g[c, v, k]
            assert abs(ad - fd) <= TOL_FD * abs(ad) + floor, ((ix, iy), v, k, ad, fd)
            checked += 1
    assert checked == 20


def test_lid_shear_matches_wall_fluxes():
    # bgk_lid_shear is dx times the sum of the lid's shear fluxes
    w = W.scaled(W.CAVITY_64, n=20, nv=24)
    s = solver.make_cavity(w, xi=W.perturbation(0, 400, 576))
    s.step(7)
    fl = s.wall_fluxes(B.BGK_FACE_YHI)
    dx = s.cfg.lx / s.cfg.nx
    assert s.lid_shear() == pytest.approx(dx * fl[:, 1].sum(), rel=1e-14)
    s.close()
    s = solver.make_shock(W.scaled(W.SHOCK_M2, nx=20))
    with pytest.raises(B.BgkError) as e:
        s.lid_shear()
    assert e.value.status == B.BGK_ERR_UNSUPPORTED
    s.close()


# ---------------------------------------------------------------------------
# torch.autograd.Function
# ---------------------------------------------------------------------------
def test_autograd_function():
    import torch

    w = W.scaled(W.CAVITY_128, n=16, nv=16)
    spec = A.cavity_spec(w, 30, 8)
    f0 = _f0(w).requires_grad_(True)
    kn = torch.tensor(w["kn"], dtype=torch.float64, requires_grad=True)
    uw = torch.tensor(_lid_speed(w), dtype=torch.float64, requires_grad=True)
    J = A.lid_shear_fn(f0, kn, uw, spec)
    (3.0 * J).backward()
    grad = torch.empty_like(f0)
    J0, dkn, duw = A.lid_shear_and_gradient(spec, f0.detach(), kn.item(), uw.item(), grad)
    assert float(J) == J0
    assert float(kn.grad) == pytest.approx(3.0 * dkn, rel=1e-15)
    assert float(uw.grad) == pytest.approx(3.0 * duw, rel=1e-15)
    assert torch.equal(f0.grad, 3.0 * grad)
    with torch.no_grad():
        J1 = A.lid_shear_fn(f0, kn, uw, spec)
    assert float(J1) == pytest.approx(J0, rel=1e-12)
