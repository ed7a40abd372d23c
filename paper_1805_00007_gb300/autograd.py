"""Differentiable evolution of the order parameter: torch.autograd over the CUDA step and its adjoint.

`evolve(phi0, scale, params, nsteps)` returns phi after `nsteps` steps of the library's step kernel, with
the prescribed velocity multiplied by `scale`.  Its backward pass runs the library's hand-written adjoint
(lb_ch_adjoint_*): the forward pass stores a checkpoint of the full state every `segment` steps (default
about sqrt(nsteps), so memory grows as sqrt(nsteps)); the backward pass reloads each checkpoint from the
last to the first, re-runs that segment while recording phi of each step (the adjoint needs only phi),
and sweeps the segment backwards.  All arithmetic runs in the CUDA library; torch supplies the device
buffers and the stream.
"""
from __future__ import annotations

import math

import torch

from . import abi

_VELOCITY_KEYS = ("U0", "ux0", "uy0", "shear")


def scaled_params(params: dict, s: float) -> dict:
    """The configuration with its prescribed velocity multiplied by s."""
    q = dict(params)
    for k in _VELOCITY_KEYS:
        q[k] = params[k] * s
    return q


class _Evolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, phi0, scale, params, nsteps, prec, segment):
        dev = torch.device("cuda", torch.cuda.current_device())
        s = float(scale)
        if s == 0.0 or not math.isfinite(s):
            # the adjoint differentiates in a multiplier of the configured velocity at 1; with the velocity
            # scaled to zero it cannot give d/dscale back (that derivative would be divided by zero)
            raise ValueError(f"evolve: scale must be finite and nonzero (got {s})")
        stream = torch.cuda.current_stream(dev).cuda_stream
        sim = abi.Simulation(scaled_params(params, s), phi0.detach().double().cpu().numpy(), prec=prec,
                             stream=stream)
        seg = int(segment) if segment else max(1, math.isqrt(int(nsteps)))
        nbytes = abi.lb_ch_state_bytes(sim.h)
        ckpts = []
        n = 0
        while n < nsteps:
            buf = torch.empty(nbytes, dtype=torch.uint8, device=dev)
            abi.lb_ch_state_save(sim.h, buf.data_ptr())
            k = min(seg, nsteps - n)
            ckpts.append((n, n + k, buf))
            sim.step(k)
            n += k
        phiT = torch.from_numpy(sim.phi()).to(device=phi0.device, dtype=phi0.dtype)
        ctx.sim, ctx.ckpts, ctx.scale, ctx.dev = sim, ckpts, s, dev
        ctx.tape_dtype = torch.float64 if prec in ("f64", abi.LBCH_F64) else torch.float32
        ctx.phi0_meta = (phi0.device, phi0.dtype)
        return phiT

    @staticmethod
    def backward(ctx, grad_phiT):
        sim, dev, tdt = ctx.sim, ctx.dev, ctx.tape_dtype
        ny, nx = grad_phiT.shape
        g = grad_phiT.detach().to(device=dev, dtype=torch.float64).contiguous()
        abi.lb_ch_adjoint_begin(sim.h, g.data_ptr())
        for n0, n1, buf in reversed(ctx.ckpts):
            abi.lb_ch_state_load(sim.h, buf.data_ptr())
            tape = torch.empty((n1 - n0, ny, nx), dtype=tdt, device=dev)
            for k in range(n1 - n0):
                abi.lb_ch_tape_phi(sim.h, tape[k].data_ptr())
                sim.step(1)
            for k in range(n1 - n0 - 1, -1, -1):
                abi.lb_ch_adjoint_step(sim.h, tape[k].data_ptr(), n0 + k)
        dphi0 = torch.empty((ny, nx), dtype=torch.float64, device=dev)
        dLds = abi.lb_ch_adjoint_end(sim.h, dphi0.data_ptr())
        sim.close()
        ctx.ckpts = None
        device, dtype = ctx.phi0_meta
        # the adjoint returns dL/ds' for u = s' (scale u_cfg) at s' = 1, which is scale * dL/dscale
        dscale = torch.tensor(dLds / ctx.scale, dtype=torch.float64)
        return dphi0.to(device=device, dtype=dtype), dscale, None, None, None, None


def evolve(phi0: torch.Tensor, scale: torch.Tensor, params: dict, nsteps: int, prec: str = "f32",
           segment: int | None = None) -> torch.Tensor:
    """phi after nsteps steps from phi0 (shape (ny, nx)) with the velocity scaled by `scale`;
    differentiable in phi0 and scale.  Single-instance, periodic configurations."""
    return _Evolve.apply(phi0, scale, params, int(nsteps), prec, segment)
