"""torch.autograd.Function around the library's adjoint (lb_adjoint_step).

LBLoss.apply(kappa, T, rho0, case, nsteps, u_from, s_final, ckpt_every, precision)
returns L = sum_{n >= u_from} sum_x |u^n|^2 + sum_x s_final rho^N for a run of
`case` (an lbfe.Case; its kappa and T are replaced by the tensors) started from
rho0, and back-propagates dL/dkappa, dL/dT and dL/drho0 from one forward and
one reverse sweep of the CUDA kernels (checkpointed; in FP64 by default, or
in FP32 with precision=lbfe.FP32). Gradients for other losses of the final
density enter through s_final (dL/drho^N). When no input needs a gradient
(inference, or torch.no_grad()), forward runs the steps alone and sums the
loss from the exported fields, with no checkpoints and no reverse sweep.
"""
from __future__ import annotations

import dataclasses

import torch

from . import lbfe


class LBLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, kappa, T, rho0, case, nsteps, u_from, s_final=None, ckpt_every=0, precision=lbfe.FP64):
        c = dataclasses.replace(case, kappa=float(kappa), T=float(T))
        lat = lbfe.Lattice([c], precision=precision, device=rho0.device if rho0.is_cuda else None)
        r0 = rho0.detach().to(torch.float64)
        sf = None if s_final is None else s_final.detach().to(torch.float64).to(r0.device)
        if not any(ctx.needs_input_grad[:3]):
            L = _forward_loss(lat, r0, nsteps, u_from, sf)
            lat.close()
            return torch.tensor(L, dtype=torch.float64, device=rho0.device)
        L, g, gk, gT = lat.adjoint(0, r0, nsteps, u_from, sf, ckpt_every)
        lat.close()
        g = torch.as_tensor(g, dtype=torch.float64, device=rho0.device)
        ctx.save_for_backward(g)
        ctx.gk, ctx.gT = gk, gT
        ctx.kdev, ctx.Tdev = kappa.device, T.device
        return torch.tensor(L, dtype=torch.float64, device=rho0.device)

    @staticmethod
    def backward(ctx, gout):
        (g,) = ctx.saved_tensors
        go = float(gout)
        gk = torch.tensor(go * ctx.gk, dtype=torch.float64, device=ctx.kdev)
        gT = torch.tensor(go * ctx.gT, dtype=torch.float64, device=ctx.Tdev)
        return gk, gT, go * g, None, None, None, None, None, None


def _forward_loss(lat, r0, nsteps: int, u_from: int, sf) -> float:
    """The loss of LBLoss from steps alone: sum over n = u_from .. nsteps of
    sum_x |u^n|^2 (u of Eq. 12 exported after n steps), plus sum_x s_final
    rho^N, the sums in FP64."""
    dev = lat.device
    lat.init_fields(0, r0)
    if u_from > 0:
        lat.step(min(u_from, nsteps))
    total = torch.zeros((), dtype=torch.float64, device=dev)
    m = None
    for n in range(min(u_from, nsteps), nsteps + 1):
        m = lat.moments(0, on_device=True)
        if n >= u_from:
            total += (m["ux"] ** 2 + m["uy"] ** 2).sum()
        if n < nsteps:
            lat.step(1)
    if sf is not None:
        total += (sf.to(dev) * m["rho"]).sum()
    return float(total)
