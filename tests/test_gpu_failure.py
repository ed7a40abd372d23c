"""Failure paths of the CUDA library, exercised without faulting the GPU.

The step kernel waits on TMA completions with a bounded number of polls.  The test hook makes one
thread block skip its first copy, so that wait runs out: the kernel must record the error, finish
cleanly, and the host must see LBCH_ETIMEOUT; the CUDA context must stay usable afterwards.
"""
import numpy as np
import pytest

import oracle
from paper_1805_00007_gb300 import abi
from paper_1805_00007_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_bounded_wait_runs_out_and_reports_etimeout(prec):
    p, phi0, _ = wl.zalesak(n=64)
    with abi.Simulation(p, phi0, prec=prec) as sim:
        abi.lb_ch_test_hook(sim.h, abi.LBCH_HOOK_TILE_KERNEL, 0)  # the row sweep: its copies have bounded waits
        abi.lb_ch_test_hook(sim.h, abi.LBCH_HOOK_SKIP_FIRST_LOAD, 1)
        sim.step(1)
        with pytest.raises(abi.LbchError) as ei:
            sim.observe(abi.LBCH_OBS_MASS)
        assert ei.value.status == abi.LBCH_ETIMEOUT
    # the context is intact: a fresh simulation runs and matches the oracle
    ref, _ = oracle.simulate(p, phi0, 10)
    with abi.Simulation(p, phi0, prec="f64") as sim:
        sim.step(10)
        assert np.max(np.abs(sim.phi() - ref)) <= 1e-12


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_two_step_kernel_wait_runs_out_and_reports_etimeout(prec):
    """The two-step kernel's bounded wait on its table copy: with the copy withheld from one thread block,
    the wait runs out, the block drains and leaves, and the host sees LBCH_ETIMEOUT."""
    p, phi0, _ = wl.zalesak(n=64)
    with abi.Simulation(p, phi0, prec=prec) as sim:
        abi.lb_ch_test_hook(sim.h, abi.LBCH_HOOK_TWO_STEP, 1)
        assert sim.kernel()["form"] == "pair_tau1"
        abi.lb_ch_test_hook(sim.h, abi.LBCH_HOOK_SKIP_FIRST_LOAD, 1)
        sim.step(2)
        with pytest.raises(abi.LbchError) as ei:
            sim.observe(abi.LBCH_OBS_MASS)
        assert ei.value.status == abi.LBCH_ETIMEOUT
    ref, _ = oracle.simulate(p, phi0, 10)
    with abi.Simulation(p, phi0, prec="f64") as sim:
        sim.step(10)
        assert np.max(np.abs(sim.phi() - ref)) <= 1e-12


def test_unknown_hook_rejected():
    p, phi0, _ = wl.zalesak(n=32)
    with abi.Simulation(p, phi0, prec="f32") as sim:
        with pytest.raises(abi.LbchError) as ei:
            abi.lb_ch_test_hook(sim.h, 99, 1)
        assert ei.value.status == abi.LBCH_EINVAL
