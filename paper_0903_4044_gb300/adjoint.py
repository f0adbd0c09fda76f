"""Gradients of the lid-integrated shear of the Sec. 5.1 cavity.

J = sum over the lid cells of dx * tau_k, tau_k the shear flux through the
lid (the drag of Sec. 5.2 up to its normalisation), after ``nsteps`` FP64
split steps from an initial state f0.  ``bgk_adjoint_lid_shear`` runs the
steps forward with a checkpoint every ``checkpoint_every`` steps, then the
hand-written reverse pass (transposed donor-cell streaming, wall-density
coupling of the diffuse walls, relaxation differentiated through the moments
and the Maxwellian) segment by segment.  It returns J, dJ/d ln L (L scales
the cavity and, through the Courant rule, the time step: Kn = 1/L, so
dJ/dKn = -(dJ/d ln L) / Kn), dJ/dU_W and dJ/df0.
"""
from __future__ import annotations

import torch

from . import bgk as B
from . import solver as S


def cavity_spec(w: dict, nsteps: int | None = None, checkpoint_every: int = 100) -> dict:
    """Fixed (non-differentiated) parameters of a cavity workload."""
    keys = ("n", "nv", "vbox", "omega", "cfl", "conservative")
    spec = {k: w[k] for k in keys if k in w}
    spec["nsteps"] = int(nsteps if nsteps is not None else w["steps"])
    spec["checkpoint_every"] = int(checkpoint_every)
    return spec


def _solver(spec: dict, kn: float, lid_speed: float, stream: int) -> S.Solver:
    cfg = S.cavity_config(kn=kn, lid_speed=lid_speed, n=spec["n"], nv=spec["nv"], vbox=spec["vbox"],
                          omega=spec["omega"], cfl=spec["cfl"], conservative=spec.get("conservative", 1),
                          stream=stream)
    return S.Solver(cfg)


def lid_shear_and_gradient(spec: dict, f0: torch.Tensor, kn: float, lid_speed: float,
                           grad_out: torch.Tensor | None = None):
    """(J, dJ/dKn, dJ/dU_W); dJ/df0 into ``grad_out`` (CUDA float64, state layout)."""
    stream = torch.cuda.current_stream(f0.device).cuda_stream
    with torch.cuda.device(f0.device):
        s = _solver(spec, kn, lid_speed, stream)
        try:
            s.set_state(f0)
            J, dlnl, duw = B.bgk_adjoint_lid_shear(s.h, spec["nsteps"], spec["checkpoint_every"], grad_out)
        finally:
            s.close()
    return J, -dlnl / kn, duw


def lid_shear(spec: dict, f0: torch.Tensor, kn: float, lid_speed: float) -> float:
    """J alone: nsteps forward steps, then bgk_lid_shear."""
    stream = torch.cuda.current_stream(f0.device).cuda_stream
    with torch.cuda.device(f0.device):
        s = _solver(spec, kn, lid_speed, stream)
        try:
            s.set_state(f0)
            s.step(spec["nsteps"])
            return s.lid_shear()
        finally:
            s.close()


class LidShear(torch.autograd.Function):
    """J(f0, Kn, U_W) with gradients from the hand-written reverse pass.

    f0: CUDA float64 tensor (cells, velocities, 2) in the state layout;
    kn, lid_speed: 0-dim float64 tensors.  The reverse pass runs inside
    forward when any input needs a gradient (it needs the forward states
    anyway); backward only scales the stored derivatives."""

    @staticmethod
    def forward(ctx, f0, kn, lid_speed, spec):
        knv, uwv = kn.item(), lid_speed.item()
        f0 = f0.contiguous()
        if any(t.requires_grad for t in (f0, kn, lid_speed)):
            grad = torch.empty_like(f0)
            J, dkn, duw = lid_shear_and_gradient(spec, f0, knv, uwv, grad)
            ctx.save_for_backward(grad)
            ctx.dkn, ctx.duw = dkn, duw
            ctx.devices = (kn.device, lid_speed.device)
        else:
            J = lid_shear(spec, f0, knv, uwv)
        return torch.tensor(J, dtype=torch.float64, device=f0.device)

    @staticmethod
    def backward(ctx, gJ):
        (grad,) = ctx.saved_tensors
        g_f0 = gJ * grad if ctx.needs_input_grad[0] else None
        g_kn = (gJ * ctx.dkn).to(ctx.devices[0], torch.float64) if ctx.needs_input_grad[1] else None
        g_uw = (gJ * ctx.duw).to(ctx.devices[1], torch.float64) if ctx.needs_input_grad[2] else None
        return g_f0, g_kn, g_uw, None


def lid_shear_fn(f0: torch.Tensor, kn: torch.Tensor, lid_speed: torch.Tensor, spec: dict) -> torch.Tensor:
    """Differentiable J (see ``LidShear``)."""
    return LidShear.apply(f0, kn, lid_speed, spec)
