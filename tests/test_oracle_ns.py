"""Pins of the oracle's coupled Navier-Stokes lattice (the paper calls it standard and does not write it
out; the reading taken is the incompressible pressure-based single-relaxation-time form with forcing).
Pinned by textbook cases that hold for any correct implementation of that form: the decay rate of a
shear wave (nu k^2), the steady Poiseuille profile between bounce-back walls, exact conservation of
sum(phi), the mirror symmetry of a symmetric Rayleigh-Taylor setup and small currents at a flat
interface at rest."""
import numpy as np
import pytest

import oracle
from paper_1805_00007_gb300 import workloads as wl


def _single_phase(nx, ny, **kw):
    return wl.make_params(nx=nx, ny=ny, vel=wl.VEL_COUPLED, phiA=1.0, phiB=-1.0, rhoA=1.0, rhoB=0.5,
                          sigma=0.01, W=4.0, M=0.01, tau=1.0, **kw)


@pytest.mark.parametrize("nu", [0.02, 0.1])
def test_shear_wave_decays_at_nu_k2(nu):
    nx, ny, n = 4, 64, 300
    p = _single_phase(nx, ny, nu=nu)
    y = np.arange(ny)[:, None] * np.ones((1, nx))
    k = 2 * np.pi / ny
    U = 1e-4
    phi0 = np.ones((ny, nx))
    _, ux, uy, _, _, _ = oracle.ns_simulate(p, phi0, n, ux0=U * np.sin(k * y))
    amp = 2.0 / ny * np.sum(ux[:, 0] * np.sin(k * np.arange(ny)))
    assert abs(amp / U - np.exp(-nu * k * k * n)) < 2e-3
    assert np.max(np.abs(uy)) < 1e-5 * U     # second order in U (weak compressibility of the model)


def test_poiseuille_profile_between_walls():
    nx, ny, nu = 4, 16, 0.1
    F = 1e-6
    # single phase rho = rhoA = 1, buoyancy -(rho - 0.75) gx = F
    p = _single_phase(nx, ny, nu=nu, walls=1, gx=-F / 0.25)
    phi, ux, uy, pr, f, g = oracle.ns_simulate(p, np.ones((ny, nx)), 6000)
    y = np.arange(ny)
    exact = F / (2 * nu) * (y + 0.5) * (ny - 0.5 - y)
    assert np.max(np.abs(ux[:, 1] - exact)) < 0.01 * np.max(exact)
    assert np.max(np.abs(uy)) < 1e-5 * np.max(exact)  # transient pressure waves, decaying


def test_rayleigh_taylor_conserves_mass_and_mirror_symmetry():
    p, phi0 = wl.rayleigh_taylor(nx=16, ny=48, Re=300.0)
    phi, ux, uy, pr, _, _ = oracle.ns_simulate(p, phi0, 60)
    assert abs(phi.sum() - phi0.sum()) < 1e-12 * np.abs(phi0).sum()
    # x -> -x (mod nx) maps the cosine perturbation to itself
    mirror = lambda a: np.roll(a[:, ::-1], 1, axis=1)
    np.testing.assert_allclose(mirror(phi), phi, atol=1e-13)
    np.testing.assert_allclose(mirror(ux), -ux, atol=1e-13)
    # the flow has started: heavy fluid sinks where the interface is lowest
    assert np.max(np.abs(uy)) > 1e-8


def test_flat_interface_at_rest_stays_quiet():
    nx, ny = 8, 48
    p = wl.make_params(nx=nx, ny=ny, walls=1, vel=wl.VEL_COUPLED, phiA=1.0, phiB=-1.0, rhoA=1.0, rhoB=1 / 3,
                       sigma=1e-3, W=4.0, M=0.05, tau=1.0, nu=0.05)
    y = np.arange(ny)[:, None] * np.ones((1, nx))
    phi0 = wl.tanh_profile(y - ny / 2 + 0.5, 4.0, 1.0, -1.0)
    phi, ux, uy, pr, _, _ = oracle.ns_simulate(p, phi0, 400)
    assert np.max(np.hypot(ux, uy)) < 1e-5
    assert np.max(np.abs(phi - phi0)) < 0.02


def _shear_flow(nx, ny):
    """A divergence-free initial flow: ux depends on y only, uy on x only."""
    x = np.arange(nx)[None, :] * np.ones((ny, 1))
    y = np.arange(ny)[:, None] * np.ones((1, nx))
    return 1e-3 * np.sin(2 * np.pi * y / ny + 0.3), 7e-4 * np.cos(2 * np.pi * x / nx + 1.1)


@pytest.mark.parametrize("gravity", [False, True])
def test_initial_equilibria_invert_to_the_given_flow(gravity):
    """f = f_eq(p = 0, rho, u0) has sum_q f_q = 0 and sum_q c_q f_q = rho u0 (the moments of f_eq), and the
    velocity carries half the force (rho u = sum_q c_q f_q + F/2): a single phase at rest in pressure
    gives back u = u0 + F/(2 rho), and p = 0 when there is no force."""
    nx, ny = 24, 20
    g = (2e-6, -3e-6) if gravity else (0.0, 0.0)
    p = _single_phase(nx, ny, nu=0.05, gx=g[0], gy=g[1])
    ux0, uy0 = _shear_flow(nx, ny)
    ux, uy, pr = oracle.ns_fields(p, *oracle.ns_init(p, np.ones((ny, nx)), ux0, uy0))
    rho, rbar = p["rhoA"], 0.5 * (p["rhoA"] + p["rhoB"])   # phi = phiA everywhere
    Fx, Fy = -(rho - rbar) * g[0], -(rho - rbar) * g[1]
    assert np.max(np.abs(ux - (ux0 + Fx / (2 * rho)))) < 1e-16
    assert np.max(np.abs(uy - (uy0 + Fy / (2 * rho)))) < 1e-16
    if not gravity:
        assert np.max(np.abs(pr)) < 1e-17


@pytest.mark.parametrize("gravity", [False, True])
def test_total_momentum_grows_by_the_force(gravity):
    """On a periodic single phase the collision keeps sum_q c_q f_q and the forcing adds F (its first
    moment), so the total momentum sum_x rho u after n steps is rho sum u0 + (n + 1/2) N F: conserved to
    rounding without a force; with gravity to within the weak coupling through phi, whose O(u^2) changes
    move rho (about 1e-8 of n N F here, against an error of order N F from a wrong forcing moment or a
    missing half force)."""
    nx, ny, n = 24, 20, 50
    g = (2e-6, -3e-6) if gravity else (0.0, 0.0)
    p = _single_phase(nx, ny, nu=0.05, gx=g[0], gy=g[1])
    ux0, uy0 = _shear_flow(nx, ny)
    _, ux, uy, _, _, _ = oracle.ns_simulate(p, np.ones((ny, nx)), n, ux0=ux0, uy0=uy0)
    rho, rbar = p["rhoA"], 0.5 * (p["rhoA"] + p["rhoB"])
    N = nx * ny
    Fx, Fy = -(rho - rbar) * g[0], -(rho - rbar) * g[1]
    ex = rho * ux.sum() - (rho * ux0.sum() + (n + 0.5) * N * Fx)
    ey = rho * uy.sum() - (rho * uy0.sum() + (n + 0.5) * N * Fy)
    if gravity:
        assert abs(ex) < 1e-6 * abs(n * N * Fx) and abs(ey) < 1e-6 * abs(n * N * Fy)
    else:
        assert abs(ex) < 1e-15 and abs(ey) < 1e-15
