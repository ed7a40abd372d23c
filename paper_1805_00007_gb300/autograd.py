"""Differentiable evolution of the order parameter: torch.autograd over the CUDA step and its adjoint.

`evolve(phi0, scale, params, nsteps)` returns phi after `nsteps` steps of the library's step kernel, with
the prescribed velocity multiplied by `scale`.  Its backward pass runs the library's hand-written adjoint
(lb_ch_adjoint_*), which needs the forward phi of every step, in reverse order.  Those are recomputed from
checkpoints of the full state under a binomial (revolve) schedule: with `checkpoints` stored states the
reverse sweep runs each step forward at most r times, where r is the least repetition number whose binomial
capacity C(checkpoints + r, checkpoints + 1) covers the run, counted in leaves of `leaf` steps.  A leaf is replayed once
with its phi written to a tape (lb_ch_step_taped) and swept backwards in one call (lb_ch_adjoint_sweep).
All arithmetic runs in the CUDA library; torch supplies the device buffers and the stream.
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


def revolve_schedule(nsteps: int, checkpoints: int, leaf: int):
    """The actions that reverse `nsteps` steps, starting from the initial state (held in slot 0) on the device:
      ("advance", n)   n forward steps (no tape)
      ("save", k) / ("load", k) / ("free", k)   the full state into / out of / off checkpoint slot k
      ("tape", n0, n)  n forward steps from step n0, phi of each written to the tape
      ("sweep", n0, n) the adjoint of steps n0 + n - 1 .. n0 from that tape
    Binomial checkpointing (Griewank's revolve) over leaves of `leaf` steps: a range of u leaves with s free
    slots and repetition number r (the least with C(s + r, s + 1) >= u) is split where both parts stay within
    the binomial bounds and the forward steps are fewest; the right part is reversed first with one slot
    fewer, the left part after it.  Returns
    (actions, stats) with stats = {"forward_steps": steps run forward (tapes included), "slots": peak
    number of stored states (slot 0 included), "repetitions": r at the top level}."""
    if nsteps < 1 or checkpoints < 0 or leaf < 1:
        raise ValueError("need nsteps >= 1, checkpoints >= 0, leaf >= 1")
    acts = []
    st = {"forward_steps": 0, "slots": 1, "cur": 0, "live": {0}, "repetitions": 0}

    def new_slot():
        k = 1
        while k in st["live"]:
            k += 1
        st["live"].add(k)
        st["slots"] = max(st["slots"], len(st["live"]))
        return k

    def goto(l, slot_l, target):
        """Bring the device state to step `target` >= l from the state l held in slot_l."""
        if not l <= st["cur"] <= target:
            acts.append(("load", slot_l))
            st["cur"] = l
        if target > st["cur"]:
            acts.append(("advance", target - st["cur"]))
            st["forward_steps"] += target - st["cur"]
            st["cur"] = target

    def leaf_rev(a, n):
        acts.append(("tape", a, n))
        st["forward_steps"] += n
        st["cur"] = a + n
        acts.append(("sweep", a, n))

    def reverse(l, n, s, slot_l, top=False):
        # the state at l is in slot_l; the device state is at l or will be brought there
        if n <= leaf:
            goto(l, slot_l, l)
            leaf_rev(l, n)
            return
        u = -(-n // leaf)
        if s == 0:
            for j in range(u - 1, -1, -1):
                a = j * leaf
                goto(l, slot_l, l + a)
                leaf_rev(l + a, min(n, a + leaf) - a)
            if top:
                st["repetitions"] = u
            return
        # eta(s, r) = C(s + r, s + 1) leaves can be reversed with s free slots when every step runs forward at
        # most r times (taped run included): eta(0, r) = r, eta(s, 1) = 1, eta(s, r) = eta(s - 1, r) + eta(s, r - 1)
        eta = lambda s_, r_: math.comb(s_ + r_, s_ + 1) if r_ > 0 else 0
        r = 1
        while eta(s, r) < u:
            r += 1
        if top:
            st["repetitions"] = r
        # the split that also minimises the forward steps (Griewank): the right part fits s - 1 slots, the left
        # part one repetition fewer, and within those bounds the least total
        lo = max(eta(s, r - 2), u - eta(s - 1, r), 1)
        hi = min(eta(s, r - 1), u - eta(s - 1, r - 1))
        m = max(lo, min(hi, u - 1)) * leaf
        goto(l, slot_l, l + m)
        k = new_slot()
        acts.append(("save", k))
        reverse(l + m, n - m, s - 1, k)
        acts.append(("free", k))
        st["live"].discard(k)
        reverse(l, m, s, slot_l)

    reverse(0, int(nsteps), int(checkpoints), 0, top=True)
    return acts, {k: st[k] for k in ("forward_steps", "slots", "repetitions")}


class _Evolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, phi0, scale, params, nsteps, prec, checkpoints, leaf):
        dev = torch.device("cuda", torch.cuda.current_device())
        s = float(scale)
        if s == 0.0 or not math.isfinite(s):
            # the adjoint differentiates in a multiplier of the configured velocity at 1; with the velocity
            # scaled to zero it cannot give d/dscale back (that derivative would be divided by zero)
            raise ValueError(f"evolve: scale must be finite and nonzero (got {s})")
        stream = torch.cuda.current_stream(dev).cuda_stream
        sim = abi.Simulation(scaled_params(params, s), phi0.detach().double().cpu().numpy(), prec=prec,
                             stream=stream)
        nsteps = int(nsteps)
        leaf = max(1, min(int(leaf), nsteps))
        acts, stats = revolve_schedule(nsteps, int(checkpoints), leaf)
        ny, nx = phi0.shape
        tdt = torch.float64 if prec in ("f64", abi.LBCH_F64) else torch.float32
        nbytes = abi.lb_ch_state_bytes(sim.h)
        slots = {0: torch.empty(nbytes, dtype=torch.uint8, device=dev)}
        abi.lb_ch_state_save(sim.h, slots[0].data_ptr())
        tape = torch.empty((leaf, ny, nx), dtype=tdt, device=dev)
        # the forward pass runs the schedule up to the first sweep: it places the checkpoints along the way and
        # leaves the last leaf on the tape, with the state at nsteps
        first = next(i for i, a in enumerate(acts) if a[0] == "sweep")
        _run(sim, acts[:first], slots, tape, nbytes, dev)
        phiT = torch.from_numpy(sim.phi()).to(device=phi0.device, dtype=phi0.dtype)
        ctx.sim, ctx.slots, ctx.tape, ctx.rest, ctx.scale, ctx.dev = sim, slots, tape, acts[first:], s, dev
        ctx.nbytes = nbytes
        ctx.stats = stats
        ctx.phi0_meta = (phi0.device, phi0.dtype)
        return phiT

    @staticmethod
    def backward(ctx, grad_phiT):
        sim, dev = ctx.sim, ctx.dev
        ny, nx = grad_phiT.shape
        g = grad_phiT.detach().to(device=dev, dtype=torch.float64).contiguous()
        abi.lb_ch_adjoint_begin(sim.h, g.data_ptr())
        _run(sim, ctx.rest, ctx.slots, ctx.tape, ctx.nbytes, dev)
        dphi0 = torch.empty((ny, nx), dtype=torch.float64, device=dev)
        dLds = abi.lb_ch_adjoint_end(sim.h, dphi0.data_ptr())
        sim.close()
        ctx.slots = ctx.tape = ctx.rest = None
        device, dtype = ctx.phi0_meta
        # the adjoint returns dL/ds' for u = s' (scale u_cfg) at s' = 1, which is scale * dL/dscale
        dscale = torch.tensor(dLds / ctx.scale, dtype=torch.float64)
        return dphi0.to(device=device, dtype=dtype), dscale, None, None, None, None, None


def _run(sim, acts, slots, tape, nbytes, dev):
    h = sim.h
    for a in acts:
        kind = a[0]
        if kind == "advance":
            abi.lb_ch_step(h, a[1])
        elif kind == "save":
            if a[1] not in slots:
                slots[a[1]] = torch.empty(nbytes, dtype=torch.uint8, device=dev)
            abi.lb_ch_state_save(h, slots[a[1]].data_ptr())
        elif kind == "load":
            abi.lb_ch_state_load(h, slots[a[1]].data_ptr())
        elif kind == "free":
            pass  # the buffer is kept for the next save into that slot
        elif kind == "tape":
            abi.lb_ch_step_taped(h, a[2], tape.data_ptr())
        elif kind == "sweep":
            abi.lb_ch_adjoint_sweep(h, tape.data_ptr(), a[1], a[2])


def evolve(phi0: torch.Tensor, scale: torch.Tensor, params: dict, nsteps: int, prec: str = "f32",
           checkpoints: int = 16, leaf: int = 64) -> torch.Tensor:
    """phi after nsteps steps from phi0 (shape (ny, nx)) with the velocity scaled by `scale`;
    differentiable in phi0 and scale.  Single-instance, periodic configurations.  The reverse sweep keeps
    `checkpoints` full states besides the initial one and a tape of `leaf` steps of phi (see
    revolve_schedule for what it recomputes)."""
    return _Evolve.apply(phi0, scale, params, int(nsteps), prec, int(checkpoints), int(leaf))


def schedule_stats(nsteps: int, checkpoints: int = 16, leaf: int = 64) -> dict:
    """Forward steps, peak stored states and repetition number of the reverse sweep evolve() would run."""
    return revolve_schedule(nsteps, checkpoints, max(1, min(leaf, nsteps)))[1]
