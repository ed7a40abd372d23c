"""Pins of the oracle's reverse-mode adjoint against central finite differences of the oracle's forward
map (no GPU needed).  The loss is L = 1/2 sum_x (phi(T) - phi_ref)^2 with phi_ref fixed; the gradient is
taken with respect to the initial field phi0 and to the scale s of the velocity field (u = s u_ref)."""
import numpy as np
import pytest

import oracle
from paper_1805_00007_gb300 import workloads as wl


def _scaled(p, s):
    q = dict(p)
    for k in ("U0", "ux0", "uy0", "shear"):
        q[k] = p[k] * s
    return q


def _loss(p, phi0, nsteps, ref):
    phi, _ = oracle.simulate(p, phi0, nsteps)
    return 0.5 * float(np.sum((phi - ref) ** 2))


CASES = [
    dict(vel=wl.VEL_VORTEX, model=2, tau=1.0),
    dict(vel=wl.VEL_ROTATION, model=2, tau=0.85),
    dict(vel=wl.VEL_UNIFORM, model=1, tau=1.3),
    dict(vel=wl.VEL_DEFORM, model=2, tau=0.7),
]


@pytest.mark.parametrize("case", CASES)
def test_adjoint_matches_finite_differences(case):
    nx, ny, nsteps = 12, 10, 8
    p = wl.make_params(nx=nx, ny=ny, U0=0.06, ux0=0.05, uy0=-0.03, xc=6.0, yc=5.0, half=6.0, Tper=20.0,
                       M=0.03, sigma=0.05, W=3.0, rhoB=0.4, nvort=2, **case)
    phi0 = np.clip(wl.random_smooth_phi(nx, ny, seed=4) + 0.5 * wl.circle_phi(nx, ny, 5.2, 4.7, 3.0, 3.0) - 0.25, 0, 1)
    ref = wl.random_smooth_phi(nx, ny, seed=9)
    phiT, _ = oracle.simulate(p, phi0, nsteps)
    dphi0, dLds = oracle.adjoint(p, phi0, nsteps, phiT - ref)
    h = 1e-5
    rng = np.random.default_rng(1)
    # a few single nodes
    for (j, i) in [(0, 0), (4, 7), (9, 11), (5, 2)]:
        e = np.zeros_like(phi0); e[j, i] = h
        fd = (_loss(p, phi0 + e, nsteps, ref) - _loss(p, phi0 - e, nsteps, ref)) / (2 * h)
        assert abs(fd - dphi0[j, i]) <= 1e-6 * max(1e-3, abs(fd)), (j, i, fd, dphi0[j, i])
    # a random direction over every node
    v = rng.normal(size=phi0.shape)
    fd = (_loss(p, phi0 + h * v, nsteps, ref) - _loss(p, phi0 - h * v, nsteps, ref)) / (2 * h)
    assert abs(fd - np.sum(dphi0 * v)) <= 1e-6 * abs(fd)
    # the velocity scale
    fds = (_loss(_scaled(p, 1 + h), phi0, nsteps, ref) - _loss(_scaled(p, 1 - h), phi0, nsteps, ref)) / (2 * h)
    assert abs(fds - dLds) <= 1e-6 * max(1e-3, abs(fds))


def test_adjoint_rejects_walls():
    p = wl.make_params(nx=8, ny=8, walls=1, vel=wl.VEL_SHEAR, shear=1e-3, M=0.02)
    with pytest.raises(ValueError):
        oracle.adjoint(p, np.full((8, 8), 0.5), 2, np.zeros((8, 8)))
