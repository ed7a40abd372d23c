"""Reads of unwritten device memory, without a memory checker: before stepping, every buffer the next
step writes is filled with NaN (all bits set, LBCH_HOOK_POISON).  A kernel that reads a cell of them it
did not write first -- a halo, a ghost image, a padding cell that enters the arithmetic -- carries NaN into
phi.  Each kernel form, precision and boundary must give the same bits as the same run without the
poison, with the poison laid again in the middle of the run (after an odd step count, so the other buffer
of the pair is hit as well)."""
import numpy as np
import pytest

from paper_1805_00007_gb300 import abi
from paper_1805_00007_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

SCHEDULE = (37, 70)


def _periodic(tau):
    specs = [(45, 37, wl.VEL_ROTATION, 2), (7, 5, wl.VEL_UNIFORM, 2), (64, 17, wl.VEL_REV_SHEAR, 1)]
    out = []
    for k, (nx, ny, vel, model) in enumerate(specs):
        p = wl.make_params(nx=nx, ny=ny, vel=vel, walls=0, model=model, U0=0.03, ux0=0.03, uy0=-0.02,
                           xc=nx / 2, yc=ny / 2, half=nx / 2, Tper=40.0, tau=tau, M=0.02, sigma=0.02, W=3.0,
                           rhoB=0.4)
        out.append((p, wl.circle_phi(nx, ny, 0.45 * nx, 0.55 * ny, 0.3 * min(nx, ny), 2.0)))
    return out


def _walls(tau):
    p = wl.make_params(nx=40, ny=27, vel=wl.VEL_SHEAR, walls=1, shear=1e-3, tau=tau, M=0.02, model=2, rhoB=0.4)
    return [(p, wl.circle_phi(40, 27, 20.0, 13.0, 8.0, 3.0))]


def _run(cases, prec, form, poison):
    params, fields = zip(*cases)
    with abi.Simulation(list(params), list(fields), prec=prec) as sim:
        if form == "sweep":
            abi.lb_ch_test_hook(sim.h, abi.LBCH_HOOK_TILE_KERNEL, 0)
        elif form == "tile":
            abi.lb_ch_test_hook(sim.h, abi.LBCH_HOOK_TILE_KERNEL, 1)
        elif form == "pair":
            abi.lb_ch_test_hook(sim.h, abi.LBCH_HOOK_TILE_KERNEL, 0)
            abi.lb_ch_test_hook(sim.h, abi.LBCH_HOOK_TWO_STEP, 1)
        out = []
        for n in SCHEDULE:
            if poison:
                abi.lb_ch_test_hook(sim.h, abi.LBCH_HOOK_POISON, 1)
            sim.step(n)
            out.append([sim.phi(i) for i in range(len(params))])
        return out


@pytest.mark.parametrize("prec,form,setup,tau", [
    ("f32", "pair", "periodic", 1.0), ("f64", "pair", "periodic", 1.0),
    ("f32", "sweep", "periodic", 1.0), ("f16s", "sweep", "periodic", 1.0), ("f64", "tile", "periodic", 1.0),
    ("f32", "sweep", "walls", 1.0), ("f32", "tile", "walls", 1.0),
    ("f32", "sweep", "periodic", 0.8), ("f16s", "tile", "walls", 0.8), ("f64", "sweep", "walls", 0.8),
])
def test_no_kernel_reads_unwritten_cells(prec, form, setup, tau):
    cases = _periodic(tau) if setup == "periodic" else _walls(tau)
    ref = _run(cases, prec, form, poison=False)
    got = _run(cases, prec, form, poison=True)
    for a_call, b_call in zip(got, ref):
        for a, b in zip(a_call, b_call):
            assert np.all(np.isfinite(a)) and np.array_equal(a, b)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_coupled_step_reads_no_unwritten_cells(prec):
    p, phi0 = wl.rayleigh_taylor(nx=20, ny=37, Re=300.0)
    res = []
    for poison in (False, True):
        with abi.Simulation(p, phi0, prec=prec) as sim:
            for n in (5, 8):
                if poison:
                    abi.lb_ch_test_hook(sim.h, abi.LBCH_HOOK_POISON, 1)
                sim.step(n)
            res.append((sim.phi(), sim.velocity(), sim.pressure()))
    (a, ua, pa), (b, ub, pb) = res
    assert np.all(np.isfinite(b)) and np.array_equal(a, b)
    assert np.array_equal(ua[0], ub[0]) and np.array_equal(ua[1], ub[1]) and np.array_equal(pa, pb)
