"""Differentiable rollout of the relative-velocity scheme for PyTorch.

``Rollout.apply(u0, s_nu, amp, sim, n, seg, rho0)`` sets the state of ``sim`` to the
equilibrium of (rho0, u0), advances n steps with checkpoints every ``seg`` steps, and
returns the final density and velocity fields. Its backward pass runs the hand-written
discrete adjoint of the library (moments adjoint, reverse sweep, equilibrium adjoint),
giving gradients with respect to the initial velocity field, the shear rate s_nu (the
shared rate of p_xx and p_xy) and the amplitude of a prescribed relative velocity.
All arithmetic runs in the CUDA library; this module only moves tensors.
"""
from __future__ import annotations

import math

import torch


class Rollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u0, s_nu, amp, sim, n, seg, rho0):
        s = list(sim.s)
        s[4] = s[5] = float(s_nu)
        sim.set_rates(s)
        sim.set_utilde(sim._ut0, float(amp), sim.period)
        u0c = u0.detach().to(device=sim.device, dtype=torch.float32).contiguous()
        rho0c = None if rho0 is None else rho0.detach().to(sim.device, torch.float32).contiguous()
        rho_in = rho0c if rho0c is not None else torch.ones((sim.ny, sim.nx), device=sim.device)
        sim.init_equilibrium(rho_in, u0c[0], u0c[1])
        seg = int(seg) if seg else max(1, int(math.ceil(math.sqrt(n))))
        ws = sim.adjoint_workspace(n, seg)
        sim.forward_checkpointed(n, seg, ws)
        rho, ux, uy = sim.moments()
        ctx.sim, ctx.n, ctx.seg, ctx.ws = sim, n, seg, ws
        ctx.meta = [(t.dtype, t.device) if torch.is_tensor(t) else (torch.float64, None)
                    for t in (s_nu, amp)]
        ctx.save_for_backward(u0c, rho_in)
        return rho, torch.stack([ux, uy])

    @staticmethod
    def backward(ctx, grad_rho, grad_u):
        sim = ctx.sim
        u0c, rho_in = ctx.saved_tensors
        dL_dS = sim.moments_vjp(grad_rho, grad_u)
        d0, ds, da, _ = sim.adjoint(ctx.n, ctx.seg, ctx.ws, dL_dS)
        _, du0 = sim.equilibrium_vjp(rho_in, u0c, d0)
        (sd, sdev), (ad, adev) = ctx.meta
        g_snu = torch.tensor(ds[4] + ds[5], dtype=sd, device=sdev)
        g_amp = torch.tensor(da, dtype=ad, device=adev)
        return du0.to(u0c.dtype), g_snu, g_amp, None, None, None, None
