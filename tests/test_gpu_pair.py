"""The two-step kernel: two steps of Eq. LB per launch for periodic instances with tau_g = 1 (where the
state is phi alone), through the C ABI.

Its per-node arithmetic is that of the one-step kernels, and a halo node is computed as the periodic image
it stands for, so it must give the same bits as the one-step kernels -- which the parity tests pin to the
FP64 oracle -- for every tile shape, every split of the steps into calls (odd counts put a one-step launch
after the pairs; 64 and more run from CUDA graphs), time-dependent flows and ragged ensembles down to
domains smaller than its six-node halo.  It is compared with the oracle directly as well.
"""
import numpy as np
import pytest

import oracle
from paper_1805_00007_gb300 import abi
from paper_1805_00007_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5}
SCHEDULE = (37, 1, 70, 130, 2)  # step counts of successive calls: odd tails, graphs, a lone pair


def _ensemble():
    """Periodic instances with tau_g = 1: several tiles with ragged tails, time-dependent flows (the two
    steps of a launch take different time factors), Model I and II, and domains of 4 to 7 nodes."""
    specs = [
        (45, 37, wl.VEL_ROTATION, 2), (70, 52, wl.VEL_VORTEX, 1), (33, 64, wl.VEL_DEFORM, 2),
        (7, 5, wl.VEL_UNIFORM, 2), (4, 4, wl.VEL_REV_SHEAR, 2), (64, 17, wl.VEL_REV_SHEAR, 1),
    ]
    out = []
    for k, (nx, ny, vel, model) in enumerate(specs):
        p = wl.make_params(nx=nx, ny=ny, vel=vel, walls=0, model=model, U0=0.03, ux0=0.03, uy0=-0.02,
                           xc=nx / 2, yc=ny / 2, half=nx / 2, Tper=40.0, tau=1.0, M=0.02, sigma=0.02, W=3.0,
                           rhoB=0.4, nvort=2)
        phi0 = np.clip(wl.random_smooth_phi(nx, ny, 11 + k)
                       + 0.6 * wl.circle_phi(nx, ny, 0.45 * nx, 0.55 * ny, 0.25 * min(nx, ny), 2.0) - 0.3, -0.2, 1.2)
        out.append((p, phi0))
    return out


def _run(params, fields, prec, pair, shape=0, schedule=SCHEDULE):
    with abi.Simulation(list(params), list(fields), prec=prec) as sim:
        abi.lb_ch_test_hook(sim.h, abi.LBCH_HOOK_TILE_KERNEL, 0)  # the row sweep, one step per launch
        if pair:
            abi.lb_ch_test_hook(sim.h, abi.LBCH_HOOK_TWO_STEP, 1)
            abi.lb_ch_test_hook(sim.h, abi.LBCH_HOOK_TILE_SHAPE, shape)
            k = sim.kernel()
            assert k["form"] == "pair_tau1" and k["shape"] == shape
        out = []
        for n in schedule:
            sim.step(n)
            out.append([sim.phi(i) for i in range(len(params))])
        assert sim.observe(abi.LBCH_OBS_STEP) == sum(schedule)
        return out


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_two_step_kernel_gives_the_same_bits(prec):
    params, fields = zip(*_ensemble())
    ref = _run(params, fields, prec, pair=False)
    for shape in range(4):
        got = _run(params, fields, prec, pair=True, shape=shape)
        for a_call, b_call in zip(got, ref):
            for a, b in zip(a_call, b_call):
                assert np.array_equal(a, b), f"shape {shape}"


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_two_step_kernel_matches_oracle(prec):
    (p, phi0), (q, psi0) = _ensemble()[:2]
    for par, f in ((p, phi0), (q, psi0)):
        ref, _ = oracle.simulate(par, f, 51)
        got = _run([par], [f], prec, pair=True, schedule=(51,))[0][0]
        assert float(np.max(np.abs(got - ref))) <= TOL[prec]


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_two_step_state_save_load_round_trip(prec):
    """After an odd number of steps the two-step kernel has left the state in the other buffer of the pair;
    a checkpoint taken then reloads into the buffers of its step index and continues bit for bit."""
    torch = pytest.importorskip("torch")
    p, phi0 = _ensemble()[1]
    with abi.Simulation(p, phi0, prec=prec) as sim, abi.Simulation(p, phi0, prec=prec) as one:
        abi.lb_ch_test_hook(sim.h, abi.LBCH_HOOK_TWO_STEP, 1)
        sim.step(33)
        buf = torch.empty(abi.lb_ch_state_bytes(sim.h), dtype=torch.uint8, device="cuda")
        abi.lb_ch_state_save(sim.h, buf.data_ptr())
        sim.step(69)
        a = sim.phi()
        abi.lb_ch_state_load(sim.h, buf.data_ptr())
        assert sim.observe(abi.LBCH_OBS_STEP) == 33
        sim.step(69)
        assert np.array_equal(a, sim.phi())
        one.step(102)
        assert np.array_equal(a, one.phi())


def test_two_step_hook_needs_periodic_tau1():
    """Walls, tau_g != 1 and the half-storage path are refused; the handle keeps its one-step kernel."""
    cases = [(dict(walls=1, vel=wl.VEL_SHEAR, shear=1e-3, tau=1.0), "f32"), (dict(tau=0.8), "f64"),
             (dict(tau=1.0), "f16s")]
    for kw, prec in cases:
        p = wl.make_params(**dict(dict(nx=40, ny=32, vel=wl.VEL_UNIFORM, ux0=0.02, uy0=0.01, walls=0, M=0.02), **kw))
        phi0 = wl.circle_phi(40, 32, 20.0, 16.0, 8.0, 3.0)
        with abi.Simulation(p, phi0, prec=prec) as sim:
            form = sim.kernel()["form"]
            with pytest.raises(abi.LbchError):
                abi.lb_ch_test_hook(sim.h, abi.LBCH_HOOK_TWO_STEP, 1)
            assert sim.kernel()["form"] == form


def test_two_step_kernel_counts_half_the_bytes():
    """The two-step kernel reads and writes phi once per two lattice updates."""
    p, phi0 = _ensemble()[0]
    with abi.Simulation(p, phi0, prec="f32") as sim:
        abi.lb_ch_test_hook(sim.h, abi.LBCH_HOOK_TILE_KERNEL, 0)
        one = sim.info()["bytes_per_lu"]
        abi.lb_ch_test_hook(sim.h, abi.LBCH_HOOK_TWO_STEP, 1)
        assert sim.info()["bytes_per_lu"] == one / 2 == 8.0


def test_small_periodic_tau1_grids_default_to_two_steps():
    """Before tuning, a grid that fits the device in one wave of two-step tiles steps with the two-step
    kernel; a larger one, or one with walls, with the row sweep."""
    p, phi0 = _ensemble()[1]
    with abi.Simulation(p, phi0, prec="f32") as sim:
        assert sim.kernel()["form"] == "pair_tau1"
    big = wl.make_params(nx=512, ny=512, vel=wl.VEL_UNIFORM, ux0=0.02, uy0=0.01, M=0.02)
    with abi.Simulation(big, wl.circle_phi(512, 512, 256.0, 256.0, 64.0, 3.0), prec="f32") as sim:
        assert sim.kernel()["form"] == "sweep_tau1"
    walls = wl.make_params(nx=64, ny=64, vel=wl.VEL_SHEAR, walls=1, shear=1e-3, M=0.02)
    with abi.Simulation(walls, wl.circle_phi(64, 64, 32.0, 32.0, 12.0, 3.0), prec="f32") as sim:
        assert sim.kernel()["form"] == "sweep_tau1"
