"""The hand-written adjoint on the GPU, against the FP64 CPU adjoint of the oracle and against central
finite differences of the GPU forward map.

Tolerances: FP64 adjoint vs the oracle adjoint 1e-10 relative (the same linear algebra in another
order); FP32 adjoint vs the oracle adjoint and vs finite differences 1e-4 relative (the tolerance the
single-vortex workload states for its gradient).  The loss is L = 1/2 sum (phi(T) - phi_ref)^2 with phi_ref = phi0 detached.
"""
import numpy as np
import pytest

import oracle
from paper_1805_00007_gb300 import abi
from paper_1805_00007_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

from paper_1805_00007_gb300.autograd import evolve, scaled_params  # noqa: E402


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _grad(p, phi0, nsteps, prec, checkpoints=16, leaf=64, ref=None):
    x = torch.tensor(phi0, dtype=torch.float64, requires_grad=True)
    s = torch.tensor(1.0, dtype=torch.float64, requires_grad=True)
    phiT = evolve(x, s, p, nsteps, prec=prec, checkpoints=checkpoints, leaf=leaf)
    target = torch.tensor(phi0 if ref is None else ref, dtype=torch.float64)
    loss = 0.5 * torch.sum((phiT - target) ** 2)
    loss.backward()
    return x.grad.numpy(), float(s.grad.detach()), float(loss.detach()), phiT.detach().numpy()


CASES = [
    dict(vel=wl.VEL_VORTEX, model=2, tau=1.0),
    dict(vel=wl.VEL_ROTATION, model=2, tau=0.85),
    dict(vel=wl.VEL_UNIFORM, model=1, tau=1.3),
]


@pytest.mark.parametrize("case", CASES)
def test_gpu_adjoint_matches_oracle_adjoint(case):
    nx, ny, nsteps = 40, 36, 30
    p = wl.make_params(nx=nx, ny=ny, U0=0.05, ux0=0.04, uy0=-0.03, xc=20.0, yc=18.0, half=20.0, Tper=25.0,
                       M=0.02, sigma=0.03, W=3.0, rhoB=0.4, **case)
    phi0 = np.clip(wl.random_smooth_phi(nx, ny, seed=3) + 0.6 * wl.circle_phi(nx, ny, 19.0, 17.0, 8.0, 3.0) - 0.3,
                   0, 1)
    phiT_ref, _ = oracle.simulate(p, phi0, nsteps)
    d_ref, s_ref = oracle.adjoint(p, phi0, nsteps, phiT_ref - phi0)
    d64, s64, _, _ = _grad(p, phi0, nsteps, "f64", checkpoints=2, leaf=7)
    assert _rel(d64, d_ref) <= 1e-10
    assert abs(s64 - s_ref) <= 1e-10 * abs(s_ref)
    d32, s32, _, _ = _grad(p, phi0, nsteps, "f32", checkpoints=2, leaf=7)
    assert _rel(d32, d_ref) <= 1e-4
    assert abs(s32 - s_ref) <= 1e-4 * abs(s_ref)


def test_checkpoint_schedule_does_not_change_the_gradient():
    """The reverse sweep recomputes the forward states it needs; whichever schedule it follows (one tape of the
    whole run, binomial checkpointing over short tapes, one-step tapes with a few stored states, or none
    besides the initial one) the recomputed phi are the same bits, and so is the gradient."""
    p, phi0, _ = wl.single_vortex(n=64, T=60)
    a = _grad(p, phi0, 60, "f64", checkpoints=0, leaf=60)
    for ck, leaf in ((2, 7), (5, 1), (0, 9), (3, 64)):
        b = _grad(p, phi0, 60, "f64", checkpoints=ck, leaf=leaf)
        assert np.array_equal(a[0], b[0]) and a[1] == b[1], (ck, leaf)


def test_taped_replay_equals_single_steps():
    """lb_ch_step_taped (captured in a graph for long replays) writes the same phi as lb_ch_tape_phi between
    single steps, and leaves the same state; lb_ch_adjoint_sweep equals the adjoint steps one by one."""
    p, phi0, _ = wl.single_vortex(n=48, T=50)
    dev = torch.device("cuda")
    n = 20
    for prec, tdt in (("f64", torch.float64), ("f32", torch.float32)):
        with abi.Simulation(p, phi0, prec=prec) as a, abi.Simulation(p, phi0, prec=prec) as b:
            a.step(3)
            b.step(3)
            ta = torch.empty((n, 48, 48), dtype=tdt, device=dev)
            tb = torch.empty_like(ta)
            abi.lb_ch_step_taped(a.h, n, ta.data_ptr())
            for k in range(n):
                abi.lb_ch_tape_phi(b.h, tb[k].data_ptr())
                b.step(1)
            torch.cuda.synchronize()  # the handles' own streams do not synchronise with torch's
            assert torch.equal(ta, tb) and np.array_equal(a.phi(), b.phi())
            abi.lb_ch_step_taped(a.h, n, ta.data_ptr())  # the graph is replayed, not captured again
            for k in range(n):
                abi.lb_ch_tape_phi(b.h, tb[k].data_ptr())
                b.step(1)
            torch.cuda.synchronize()
            assert torch.equal(ta, tb) and np.array_equal(a.phi(), b.phi())
            seed = torch.ones((48, 48), dtype=torch.float64, device=dev)
            abi.lb_ch_adjoint_begin(a.h, seed.data_ptr())
            abi.lb_ch_adjoint_begin(b.h, seed.data_ptr())
            abi.lb_ch_adjoint_sweep(a.h, ta.data_ptr(), 23, n)
            for k in range(n - 1, -1, -1):
                abi.lb_ch_adjoint_step(b.h, tb[k].data_ptr(), 23 + k)
            ga, gb = torch.empty_like(seed), torch.empty_like(seed)
            sa = abi.lb_ch_adjoint_end(a.h, ga.data_ptr())
            sb = abi.lb_ch_adjoint_end(b.h, gb.data_ptr())
            assert torch.equal(ga, gb) and sa == sb


def test_evolve_rejects_zero_scale():
    p, phi0, _ = wl.single_vortex(n=32, T=10)
    x = torch.tensor(phi0, dtype=torch.float64, requires_grad=True)
    with pytest.raises(ValueError):
        evolve(x, torch.tensor(0.0, dtype=torch.float64, requires_grad=True), p, 10)


def test_state_save_load_round_trip():
    p, phi0, _ = wl.zalesak(n=64)
    dev = torch.device("cuda")
    for prec in ("f64", "f32", "f16s"):
        with abi.Simulation(p, phi0, prec=prec) as sim:
            sim.step(13)
            buf = torch.empty(abi.lb_ch_state_bytes(sim.h), dtype=torch.uint8, device=dev)
            abi.lb_ch_state_save(sim.h, buf.data_ptr())
            sim.step(70)
            a = sim.phi()
            abi.lb_ch_state_load(sim.h, buf.data_ptr())
            assert sim.observe(abi.LBCH_OBS_STEP) == 13
            sim.step(70)
            assert np.array_equal(a, sim.phi())


def test_state_load_rejects_a_buffer_of_another_layout():
    """A saved state carries the layout it was saved for; loading it into a handle of another size,
    precision or model, or loading a buffer that holds no saved state, is refused before anything is
    copied, and the handle's own state is left as it was."""
    dev = torch.device("cuda")
    p_small, f_small, _ = wl.zalesak(n=32)
    p_big, f_big, _ = wl.zalesak(n=64)
    with abi.Simulation(p_small, f_small, prec="f32") as small:
        small.step(3)
        buf = torch.empty(abi.lb_ch_state_bytes(small.h), dtype=torch.uint8, device=dev)
        abi.lb_ch_state_save(small.h, buf.data_ptr())
    for prec, params, field in (("f32", p_big, f_big), ("f64", p_small, f_small), ("f16s", p_small, f_small)):
        with abi.Simulation(params, field, prec=prec) as sim:
            sim.step(5)
            before = sim.phi()
            with pytest.raises(abi.LbchError) as ei:
                abi.lb_ch_state_load(sim.h, buf.data_ptr())
            assert ei.value.status == abi.LBCH_EINVAL and "does not fit" in str(ei.value)
            assert sim.observe(abi.LBCH_OBS_STEP) == 5 and np.array_equal(before, sim.phi())
    q = wl.make_params(nx=32, ny=32, model=1, vel=wl.VEL_UNIFORM, ux0=0.01, uy0=0.0, M=0.02)
    with abi.Simulation(q, f_small, prec="f32") as sim:  # the same layout but Model I: the hash tells
        with pytest.raises(abi.LbchError) as ei:
            abi.lb_ch_state_load(sim.h, buf.data_ptr())
        assert ei.value.status == abi.LBCH_EINVAL
    with abi.Simulation(p_small, f_small, prec="f32") as sim:
        zeros = torch.zeros_like(buf)
        torch.cuda.synchronize()  # the fill runs on torch's stream, the load on the handle's
        with pytest.raises(abi.LbchError) as ei:
            abi.lb_ch_state_load(sim.h, zeros.data_ptr())
        assert ei.value.status == abi.LBCH_EINVAL and "does not hold a saved state" in str(ei.value)
        abi.lb_ch_state_load(sim.h, buf.data_ptr())  # the matching handle still takes it
        assert sim.observe(abi.LBCH_OBS_STEP) == 3


def test_single_vortex_adjoint_vs_finite_differences():
    """The 512 x 512 single-vortex workload (R = 76.8 at (256, 384), U0 = 0.04, Pe = 1000) for its full
    reversal period T = 8000 steps: the FP32 adjoint (checkpointed) against central differences of the
    FP64 forward map, for dL/ds and for the derivative along a random direction of phi0."""
    p, phi0, T = wl.single_vortex()
    d32, s32, _, _ = _grad(p, phi0, T, "f32")
    ref = phi0

    def loss64(phi_init, s):
        with abi.Simulation(scaled_params(p, s), phi_init, prec="f64") as sim:
            sim.step(T)
            return 0.5 * float(np.sum((sim.phi() - ref) ** 2))

    h = 1e-4
    fds = (loss64(phi0, 1 + h) - loss64(phi0, 1 - h)) / (2 * h)
    assert abs(s32 - fds) <= 1e-4 * abs(fds)
    v = np.random.default_rng(7).normal(size=phi0.shape) * (np.abs(phi0 - 0.5) < 0.49)
    hv = 1e-4
    fdv = (loss64(phi0 + hv * v, 1.0) - loss64(phi0 - hv * v, 1.0)) / (2 * hv)
    assert abs(np.sum(d32 * v) - fdv) <= 1e-4 * abs(fdv)


def test_adjoint_rejects_walls_and_ensembles():
    p = wl.make_params(nx=16, ny=16, walls=1, vel=wl.VEL_SHEAR, shear=1e-3, M=0.02)
    dev = torch.device("cuda")
    g = torch.zeros(256, dtype=torch.float64, device=dev)
    with abi.Simulation(p, np.full((16, 16), 0.5), prec="f64") as sim:
        with pytest.raises(abi.LbchError) as ei:
            abi.lb_ch_adjoint_begin(sim.h, g.data_ptr())
        assert ei.value.status == abi.LBCH_EINVAL
