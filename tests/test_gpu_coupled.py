"""Parity of the coupled Cahn-Hilliard / Navier-Stokes path (Rayleigh-Taylor) with the FP64 oracle.

Tolerances: FP64 1e-12 on phi, u and p; FP32 (plain float storage) 1e-5 on phi and 1e-7 on u and p
over at most a few hundred steps (the instability grows differences exponentially, so long runs are
compared through invariants: exact mass and the mirror symmetry of the setup)."""
import numpy as np
import pytest

import oracle
from paper_1805_00007_gb300 import abi
from paper_1805_00007_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _run(p, phi0, nsteps, prec):
    with abi.Simulation(p, phi0, prec=prec) as sim:
        sim.step(nsteps)
        return sim.phi(), sim.velocity(), sim.pressure()


@pytest.mark.parametrize("model", [1, 2])
def test_small_rayleigh_taylor_matches_oracle(model):
    p, phi0 = wl.rayleigh_taylor(nx=40, ny=72, Re=300.0, model=model)
    nsteps = 120
    phi_r, ux_r, uy_r, pr_r, _, _ = oracle.ns_simulate(p, phi0, nsteps)
    phi, u, pr = _run(p, phi0, nsteps, "f64")
    assert np.max(np.abs(phi - phi_r)) <= 1e-12
    assert np.max(np.abs(u[0] - ux_r)) <= 1e-12 and np.max(np.abs(u[1] - uy_r)) <= 1e-12
    assert np.max(np.abs(pr - pr_r)) <= 1e-12
    phi, u, pr = _run(p, phi0, nsteps, "f32")
    assert np.max(np.abs(phi - phi_r)) <= 1e-5
    assert np.max(np.abs(u[1] - uy_r)) <= 1e-7 and np.max(np.abs(pr - pr_r)) <= 1e-7


def test_full_size_rayleigh_taylor_first_steps():
    """The 256 x 1024 Rayleigh-Taylor workload (Atwood 0.5, Re 3000, Pe 1000, W 5, sqrt(g lambda) = 0.04)."""
    p, phi0 = wl.rayleigh_taylor()
    nsteps = 30
    phi_r, ux_r, uy_r, pr_r, _, _ = oracle.ns_simulate(p, phi0, nsteps)
    phi, u, pr = _run(p, phi0, nsteps, "f64")
    assert np.max(np.abs(phi - phi_r)) <= 1e-12
    assert np.max(np.abs(u[1] - uy_r)) <= 1e-12 and np.max(np.abs(pr - pr_r)) <= 1e-12
    phi, u, pr = _run(p, phi0, nsteps, "f32")
    assert np.max(np.abs(phi - phi_r)) <= 1e-5


def test_shear_wave_periodic_matches_oracle():
    nx, ny = 8, 64
    p = wl.make_params(nx=nx, ny=ny, vel=wl.VEL_COUPLED, phiA=1.0, phiB=-1.0, rhoA=1.0, rhoB=0.5, sigma=0.01,
                       W=4.0, M=0.01, tau=1.0, nu=0.05)
    phi0 = np.clip(0.9 + 0.1 * wl.random_smooth_phi(nx, ny, seed=2, amp=1.0, mean=0.0), -1, 1)
    phi_r, ux_r, uy_r, pr_r, _, _ = oracle.ns_simulate(p, phi0, 80)
    phi, u, pr = _run(p, phi0, 80, "f64")
    assert np.max(np.abs(phi - phi_r)) <= 1e-12 and np.max(np.abs(u[0] - ux_r)) <= 1e-12


@pytest.mark.parametrize("nx,ny,model,tau", [(20, 37, 2, 0.8), (20, 37, 1, 1.0), (5, 6, 2, 1.0), (33, 9, 2, 1.0)])
def test_ragged_tiles_with_walls_match_oracle(nx, ny, model, tau):
    """Domains that do not fill the coupled kernels' 32 x 8 tiles -- narrower than a tile, ragged in x and
    y, fewer rows than a tile -- between walls (the stencil operands at the ghost rows are the mirror
    nodes' values), with an asymmetric field, gravity along both axes and tau_g != 1 for the
    Cahn-Hilliard lattice."""
    p = wl.make_params(nx=nx, ny=ny, walls=1, vel=wl.VEL_COUPLED, phiA=1.0, phiB=-1.0, rhoA=1.0, rhoB=0.4,
                       sigma=0.01, W=3.0, M=0.02, tau=tau, model=model, nu=0.05, gx=1e-5, gy=-2e-5)
    phi0 = np.clip(wl.random_smooth_phi(nx, ny, seed=7 + nx, amp=1.6, mean=0.0), -1, 1)
    phi_r, ux_r, uy_r, pr_r, _, _ = oracle.ns_simulate(p, phi0, 60)
    phi, u, pr = _run(p, phi0, 60, "f64")
    assert np.max(np.abs(phi - phi_r)) <= 1e-12
    assert np.max(np.abs(u[0] - ux_r)) <= 1e-12 and np.max(np.abs(u[1] - uy_r)) <= 1e-12
    assert np.max(np.abs(pr - pr_r)) <= 1e-12


def test_long_run_invariants():
    p, phi0 = wl.rayleigh_taylor(nx=64, ny=256, Re=1000.0)
    with abi.Simulation(p, phi0, prec="f32") as sim:
        sim.step(3000)
        phi = sim.phi()
        mass = sim.observe(abi.LBCH_OBS_MASS)
    assert abs(mass - phi0.sum()) <= 1e-5 * np.abs(phi0).sum()
    mirror = lambda a: np.roll(a[:, ::-1], 1, axis=1)
    assert np.max(np.abs(mirror(phi) - phi)) <= 1e-3
    assert np.all(np.isfinite(phi))


def test_coupled_rejects_unsupported():
    p, phi0 = wl.rayleigh_taylor(nx=16, ny=32)
    with pytest.raises(abi.LbchError):
        abi.Simulation(p, phi0, prec="f16s")
    with pytest.raises(abi.LbchError):
        abi.Simulation([p, p], [phi0, phi0], prec="f32")
