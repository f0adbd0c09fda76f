"""Batches of uneven instances in one graph launch, and the autotuner."""
import numpy as np
import pytest

import oracle
import precision_bounds as PB
from paper_0903_4044_gb300 import bgk as B
from paper_0903_4044_gb300 import build, solver
from paper_0903_4044_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    oracle.build()
    B.lib()


MIX = [
    W.scaled(W.CAVITY_64, name="c0", n=12, nv=16, precision="f64"),
    W.scaled(W.CAVITY_64, name="c1", n=17, nv=24, precision="f32", seed=5),
    W.scaled(W.SHOCK_M2, name="s0", nx=40, precision="f64"),
    W.scaled(W.SHOCK_M2, name="s1", nx=56, precision="f32"),
    W.scaled(W.CAVITY_64, name="c2", n=9, nv=32, precision="bf16", seed=7),
]


def _single(w):
    cfg = solver.instance_config(w)
    s = solver.Solver(cfg)
    if w["kind"] == "shock":
        up, down = B.bgk_rankine_hugoniot(w["mach"])
        s.init_step(0.0, up, down)
    else:
        s.init_uniform((1.0, 0.0, 0.0, 1.0), W.perturbation(w["seed"], s.ncell, s.nv), w["amp"])
    return s


def test_batch_equals_independent_solvers():
    # 70 steps = one 64-step graph + a 6-step graph; every instance must come
    # out bit for bit as when stepped alone.
    b = solver.Batch(MIX)
    b.step(70)
    b.sync()
    for w, sb in zip(MIX, b.solvers):
        s = _single(w)
        s.step(70)
        assert np.array_equal(sb.get_state(), s.get_state()), w["name"]
        assert np.array_equal(sb.moments(which=1), s.moments(which=1)), w["name"]
        s.close()
    b.close()


def test_batch_instance_error_names_instance():
    bad = [MIX[0], W.scaled(MIX[0], nv=90)]
    with pytest.raises(B.BgkError) as e:
        solver.Batch(bad)
    assert "instance 1" in str(e.value)


def test_autotune_restores_state_and_keeps_parity():
    w = W.scaled(W.CAVITY_64, n=20, nv=24)
    prob0, _, _ = oracle.cavity_problem(**w)
    xi = W.perturbation(0, prob0.ncell, prob0.nv)
    prob, g, h = oracle.cavity_problem(**w, xi=xi)
    s = solver.make_cavity(w, xi=xi)
    s.step(5)
    before = s.get_state()
    tile = B.bgk_autotune(s.h, 3)
    assert tile in (1, 2, 4, 8)
    assert B.bgk_get_info(s.h).tile_cells == tile
    assert np.array_equal(s.get_state(), before)      # trials leave no trace
    s.step(20)
    g1, h1, _ = oracle.step(prob, g, h, 25)
    st = s.get_state()
    assert np.abs(st[..., 0] - g1).max() / np.abs(g1).max() < 1e-12
    s.close()


def test_batch_autotune_then_step():
    b = solver.Batch(MIX)
    b.autotune(2)
    b.step(9)
    b.sync()
    # the FP64 cavity instance against the oracle
    w = MIX[0]
    prob0, _, _ = oracle.cavity_problem(**w)
    xi = W.perturbation(w["seed"], prob0.ncell, prob0.nv)
    prob, g, h = oracle.cavity_problem(**w, xi=xi)
    g1, h1, _ = oracle.step(prob, g, h, 9)
    st = b.solvers[0].get_state()
    assert np.abs(st[..., 0] - g1).max() / np.abs(g1).max() < 1e-12
    b.close()


# ---------------------------------------------------------------------------
# persistent mode: one cooperative launch per step() call
# ---------------------------------------------------------------------------
MIX32 = [
    W.scaled(W.CAVITY_64, name="p0", n=13, nv=48, precision="f32", seed=2),
    W.scaled(W.CAVITY_64, name="p1", n=21, nv=32, precision="f32", seed=3),
    W.scaled(W.SHOCK_M2, name="p2", nx=57, precision="f32"),
    W.scaled(W.CAVITY_64, name="p3", n=8, nv=24, precision="f32", seed=4),
    dict(W.SHOCK_M2, name="p4", mach=5.0, nx=90, nvx=128, vx=(-19.0, 19.0), precision="f32"),
    dict(W.SHOCK_M2, name="p5", mach=1.2, nx=33, nvx=48, vx=(-7.6, 7.6), precision="f32"),
]


def test_persistent_equals_independent_solvers():
    b = solver.Batch(MIX32)
    b.set_persistent(True)
    tiles = [int(s.info.tile_cells) for s in b.solvers]
    b.step(37)
    b.step(4)
    b.sync()
    for w, sb, t in zip(MIX32, b.solvers, tiles):
        s = _single(dict(w, tile_cells=t))
        s.step(41)
        assert np.array_equal(sb.get_state(), s.get_state()), w["name"]
        assert np.array_equal(sb.moments(which=1), s.moments(which=1)), w["name"]
        s.close()
    b.close()


def test_pipelined_tile1_equals_block():
    # tile 1 of a single solver runs the pipelined kernel (one cell per
    # iteration of a resident CTA, parameters on a ninth warp); the
    # persistent kernel runs the one-cell block: the states must agree bit
    # for bit (1, 3 and 4 velocity groups per thread, ragged ones included,
    # fewer cells than resident CTAs, and more)
    ws = [W.scaled(W.CAVITY_64, name="q0", n=13, nv=48, precision="f32", seed=5, tile_cells=1),
          W.scaled(W.CAVITY_64, name="q1", n=37, nv=32, precision="f32", seed=6, tile_cells=1),
          W.scaled(W.CAVITY_64, name="q2", n=5, nv=64, precision="f32", seed=7, tile_cells=1),
          W.scaled(W.CAVITY_64, name="q3", n=9, nv=24, precision="f32", seed=8, tile_cells=1,
                   wall="specular")]
    b = solver.Batch(ws)
    b.set_persistent(True)
    assert [int(s.info.tile_cells) for s in b.solvers] == [1] * len(ws)
    b.step(23)
    b.sync()
    for w, sb in zip(ws, b.solvers):
        s = _single(w)
        s.step(23)
        assert np.array_equal(sb.get_state(), s.get_state()), w["name"]
        assert np.array_equal(sb.moments(which=1), s.moments(which=1)), w["name"]
        s.close()
    b.close()


def test_persistent_against_oracle():
    # one FP32 cavity and one FP32 shock stepped 20 times inside a persistent
    # batch, against the FP64 oracle, within the FP32 bounds of
    # tests/precision_bounds.py: eps = (6 N + 1) 2^-24 of a moment's sum of
    # absolute terms, so n within eps, theta within 2 eps, U within eps times
    # the mean particle speed, at most <|c - U|> + |U| (<|c - U|> <= 2 at the
    # temperatures of these problems)
    nsteps = 20
    eps = PB.f32(nsteps)["n"]
    ws = [W.scaled(W.CAVITY_64, name="o0", n=16, nv=24, precision="f32", seed=9),
          W.scaled(W.SHOCK_M2, name="o1", nx=60, precision="f32")]
    b = solver.Batch(ws)
    b.set_persistent(True)
    b.step(nsteps)
    b.sync()
    for w, sb in zip(ws, b.solvers):
        if w["kind"] == "cavity":
            prob0, _, _ = oracle.cavity_problem(**w)
            xi = W.perturbation(w["seed"], prob0.ncell, prob0.nv)
            prob, g, h = oracle.cavity_problem(**w, xi=xi)
        else:
            prob, g, h = oracle.shock_problem(**w)
        g1, h1, _ = oracle.step(prob, g, h, nsteps)
        want = oracle.state_moments(prob, g1, h1)
        got = sb.moments()
        assert np.abs(got[:, 0] - want[:, 0]).max() / np.abs(want[:, 0]).max() <= eps, w["name"]
        assert np.abs(got[:, 3] - want[:, 3]).max() / np.abs(want[:, 3]).max() <= 2 * eps, w["name"]
        speed = 2.0 + np.abs(want[:, 1:3]).max()
        assert np.abs(got[:, 1:3] - want[:, 1:3]).max() <= eps * speed, w["name"]
    b.close()


def test_persistent_needs_fp32():
    b = solver.Batch(MIX[:2])
    with pytest.raises(B.BgkError) as e:
        b.set_persistent(True)
    assert e.value.status == B.BGK_ERR_UNSUPPORTED
    b.close()


def test_persistent_barrier_timeout_is_reported():
    # a wait limit far below one step's duration: the grid barrier gives up,
    # the launch ends, sync reports the timeout and the batch stays usable
    b = solver.Batch(MIX32[:3])
    b.set_persistent(True, timeout_s=1e-7)
    b.step(3)
    with pytest.raises(B.BgkError) as e:
        b.sync()
    assert e.value.status == B.BGK_ERR_TIMEOUT
    b.set_persistent(True, timeout_s=5.0)
    b.step(2)
    b.sync()
    b.close()


# ---------------------------------------------------------------------------
# the batched workload at full size (64 cavities + 16 shocks, FP32)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("persistent", [False, True])
def test_full_batch_sampled_instances(persistent):
    # the launch configuration the benchmark times: tiles from the autotuner,
    # then steps of the whole batch (graph branches or the persistent
    # kernel); sampled instances bit for bit as when stepped alone
    ws = W.batch_instances(0)
    b = solver.Batch(ws)
    b.autotune(2)
    if persistent:
        b.set_persistent(True)
    tiles = [int(s.info.tile_cells) for s in b.solvers]
    b.step(5)
    b.sync()
    for i in (0, 17, 40, 63, 64, 71, 79):
        s = _single(dict(ws[i], tile_cells=tiles[i]))
        s.step(5)
        assert np.array_equal(b.solvers[i].get_state(), s.get_state()), ws[i]["name"]
        s.close()
    b.close()
