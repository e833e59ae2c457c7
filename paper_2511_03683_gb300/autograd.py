"""Reverse-mode derivatives of rt-BTE trajectories through the C ABI.

``trajectory(dev, f0, g2, dt, nsteps, every)`` returns f after nsteps classic RK4 steps of
df/dt = I[f] (Eq. 2, Eq. 1 with no field) as a differentiable function of the initial
occupations f0 and of the couplings |g|^2 (one entry per stored channel, in the CSR order
of ``Channels.export``).  The forward pass keeps f every ``every`` steps; the backward pass
recomputes each segment from its checkpoint and applies ``pb_rtbte_rk4_vjp`` step by step
in reverse.  On a device made with adjoint=True the steps only accumulate the two stage sums
per state pair that dL/d|g|^2 needs, and one flush at the end spreads them over the channels.
Every arithmetic step runs in libpb.so; this module only orders the calls.
"""
from __future__ import annotations

import torch


class _Trajectory(torch.autograd.Function):
    @staticmethod
    def forward(ctx, f0, g2, dev, dt, nsteps, every):
        if g2.numel() > 0:
            # the trajectory (and so its gradient) is taken at the couplings given: push them to
            # the device when they differ from the ones it holds
            if g2.numel() != dev.nchannels:
                raise ValueError(f"g2 has {g2.numel()} values; the device stores {dev.nchannels} channels")
            g2d = g2.detach()
            if not torch.equal(dev.g2_values(), g2d):
                dev.set_g2(g2d.to(dtype=torch.float64).contiguous())
        f = f0.detach().clone().contiguous()
        ckpts = []
        n = 0
        while n < nsteps:
            m = min(every, nsteps - n)
            ckpts.append((n, m, f.clone()))
            dev.rk4(f, dt, m)
            n += m
        ctx.dev, ctx.dt = dev, float(dt)
        ctx.ckpts = ckpts
        ctx.want_g2 = g2 is not None and g2.requires_grad
        return f

    @staticmethod
    def backward(ctx, gout):
        dev, dt = ctx.dev, ctx.dt
        lam = gout.detach().clone().contiguous()
        gg2 = torch.zeros(dev.nchannels, dtype=torch.float64, device=lam.device) if ctx.want_g2 else None
        y = torch.empty_like(lam)
        for n0, m, fck in reversed(ctx.ckpts):
            states = [fck]
            y.copy_(fck)
            for _ in range(m - 1):
                dev.rk4(y, dt, 1)
                states.append(y.clone())
            for k in reversed(range(m)):
                if gg2 is not None and dev.deferred:
                    dev.rk4_vjp_defer(states[k], lam, dt)
                else:
                    dev.rk4_vjp(states[k], lam, dt, grad_g2=gg2)
        if gg2 is not None and dev.deferred:
            dev.g2grad_flush(gg2)
        return lam, gg2, None, None, None, None


def trajectory(dev, f0, g2=None, dt=1.0, nsteps=1, every=20):
    """Differentiable RK4 trajectory on ``dev`` (a Device of the FF, G32, G16 or H16 variant).
    ``g2`` is a CUDA float64 tensor of the stored couplings (CSR order, e.g. from ``g2_tensor``);
    the trajectory is computed at these values (they are pushed to the device with
    ``Device.set_g2`` when they differ from the ones it holds).  Pass it with requires_grad to
    get dL/dg2."""
    if g2 is None:
        g2 = torch.zeros(0, dtype=torch.float64, device=f0.device)
    return _Trajectory.apply(f0, g2, dev, dt, int(nsteps), int(every))


def g2_tensor(channels, device="cuda"):
    """The stored couplings in CSR order as a CUDA float64 tensor."""
    return torch.tensor(channels.export()["g2"], dtype=torch.float64, device=device)
