"""Seeded synthetic inputs shaped like the paper's benchmarks (Sec. III).

This module holds only input generators: parameter tables (plain numbers) and initial order-parameter
fields.  It contains none of the lattice Boltzmann arithmetic -- no equilibria, stencils, sources or
derived constants -- so that both the CUDA library and the independent CPU oracle can be fed the very
same inputs.  Every field is float64, row-major (ny, nx); node (i, j) sits at x = i, y = j.

The initial fields use the planar equilibrium profile of the paper (Eq. analytical),
phi = (phiA + phiB)/2 + (phiA - phiB)/2 tanh(2 d / W), with d the signed distance to the interface
(positive inside phase A).
"""
from __future__ import annotations

import math

import numpy as np

SEED_BASE = 20180501

# Velocity-field codes, shared by the library's parameter struct and the oracle's.
VEL_UNIFORM, VEL_ROTATION, VEL_VORTEX, VEL_SHEAR, VEL_REV_SHEAR, VEL_DEFORM, VEL_COUPLED = range(7)

_DEFAULTS = dict(walls=0, model=2, vel=VEL_UNIFORM, nvort=4, phiA=1.0, phiB=0.0, sigma=0.01, W=4.0,
                 M=0.0, Pe=0.0, Ustar=0.0, tau=1.0, rhoA=1.0, rhoB=0.5, U0=0.0, ux0=0.0, uy0=0.0,
                 xc=0.0, yc=0.0, half=1.0, Tper=1.0, shear=0.0, nu=0.0, gx=0.0, gy=0.0)


def make_params(**kw) -> dict:
    """A full parameter dict: the paper's defaults (Sec. III: tau_g = 1, rhoA/rhoB = 2, sigma = 0.01)
    overridden by the keyword arguments."""
    unknown = set(kw) - set(_DEFAULTS) - {"nx", "ny"}
    if unknown:
        raise KeyError(f"unknown parameters: {sorted(unknown)}")
    p = dict(_DEFAULTS)
    p.update(kw)
    return p


def tanh_profile(d: np.ndarray, W: float, phiA: float, phiB: float) -> np.ndarray:
    """Eq. analytical evaluated at signed distance d."""
    return 0.5 * (phiA + phiB) + 0.5 * (phiA - phiB) * np.tanh(2.0 * d / W)


def _grid(nx: int, ny: int):
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    return x, y


def circle_phi(nx, ny, xc, yc, R, W, phiA=1.0, phiB=0.0) -> np.ndarray:
    x, y = _grid(nx, ny)
    return tanh_profile(R - np.hypot(x - xc, y - yc), W, phiA, phiB)


def planar_phi(nx, ny, y0, W, phiA=1.0, phiB=0.0, periodic_pair=True) -> np.ndarray:
    """A band of phase A between y0 and ny - y0 (two planar interfaces on a periodic domain) or a single
    interface at y0 (phase A below)."""
    _, y = _grid(nx, ny)
    if periodic_pair:
        d = np.minimum(y - y0, (ny - y0) - y)
    else:
        d = y0 - y
    return tanh_profile(d, W, phiA, phiB)


def _seg_dist(px, py, ax, ay, bx, by):
    dx, dy = bx - ax, by - ay
    t = np.clip(((px - ax) * dx + (py - ay) * dy) / (dx * dx + dy * dy), 0.0, 1.0)
    return np.hypot(px - ax - t * dx, py - ay - t * dy)


def zalesak_sdf(nx, ny, xc=128.0, yc=160.0, R=64.0, slot_w=16.0, slot_depth=80.0) -> np.ndarray:
    """Exact signed distance (positive inside) to a disk with a vertical slot cut upward from its bottom.

    The slot spans x in [xc - w/2, xc + w/2] and y from below the disk up to (yc - R) + depth.  The boundary
    is the disk arc outside the slot opening, the two slot walls and the slot's top edge; the distance is
    the minimum over these pieces and the sign comes from the inside test."""
    x, y = _grid(nx, ny)
    xl, xr = xc - slot_w / 2, xc + slot_w / 2
    ytop = yc - R + slot_depth
    # where the slot walls meet the circle (lower intersections)
    h = math.sqrt(R * R - (slot_w / 2) ** 2)
    yw = yc - h
    inside_disk = np.hypot(x - xc, y - yc) < R
    in_slot = (x > xl) & (x < xr) & (y < ytop)
    inside = inside_disk & ~in_slot
    # arc distance: points whose polar angle falls outside the slot opening project onto the arc
    ang = np.arctan2(y - yc, x - xc)
    a_l = math.atan2(yw - yc, xl - xc)   # about -97 deg
    a_r = math.atan2(yw - yc, xr - xc)   # about -83 deg
    in_gap = (ang > a_l) & (ang < a_r)
    d_arc = np.abs(np.hypot(x - xc, y - yc) - R)
    d_ends = np.minimum(np.hypot(x - xl, y - yw), np.hypot(x - xr, y - yw))
    d_arc = np.where(in_gap, d_ends, d_arc)
    d_wl = _seg_dist(x, y, xl, yw, xl, ytop)
    d_wr = _seg_dist(x, y, xr, yw, xr, ytop)
    d_top = _seg_dist(x, y, xl, ytop, xr, ytop)
    d = np.minimum(np.minimum(d_arc, d_wl), np.minimum(d_wr, d_top))
    return np.where(inside, d, -d)


# ----------------------------------------------------------------------------- the benchmark setups

def translation(nx=100, W=4.0, U=0.04, M=0.01, tau=0.8, model=2):
    """Diagonal translation of a circular interface (Sec. III.A shape): R = nx/4 centred, uniform
    u = (U, U); one period is nx/U steps."""
    p = make_params(nx=nx, ny=nx, vel=VEL_UNIFORM, ux0=U, uy0=U, W=W, M=M, tau=tau, model=model)
    phi0 = circle_phi(nx, nx, nx / 2, nx / 2, nx / 4, W)
    return p, phi0, int(round(nx / U))


def zalesak(n=256, W=4.0, U0=0.02, M=0.005, tau=1.0, model=2):
    """Zalesak's slotted disk in solid-body rotation (Sec. III.B shape): radius n/4 at (n/2, 5n/8), slot
    width n/16 and depth 5n/16, u = (-U0 pi (y - n/2)/(n/2), U0 pi (x - n/2)/(n/2)); one revolution is
    n/U0 steps."""
    p = make_params(nx=n, ny=n, vel=VEL_ROTATION, U0=U0, xc=n / 2, yc=n / 2, half=n / 2, W=W, M=M,
                    tau=tau, model=model)
    sdf = zalesak_sdf(n, n, xc=n / 2, yc=5 * n / 8, R=n / 4, slot_w=n / 16, slot_depth=5 * n / 16)
    phi0 = tanh_profile(sdf, W, 1.0, 0.0)
    return p, phi0, int(round(n / U0))


def single_vortex(n=512, W=4.0, U0=0.04, T=8000, Pe=1000.0, tau=1.0, model=2):
    """Circle of radius 0.15 n at (n/2, 3n/4) in the time-reversed single-vortex field
    u = U0 (-sin^2(pi x/n) sin(2 pi y/n), sin(2 pi x/n) sin^2(pi y/n)) cos(pi t/T); M from Pe with U* = U0."""
    p = make_params(nx=n, ny=n, vel=VEL_VORTEX, U0=U0, Tper=float(T), W=W, Pe=Pe, Ustar=U0, tau=tau,
                    model=model)
    phi0 = circle_phi(n, n, n / 2, 3 * n / 4, 0.15 * n, W)
    return p, phi0, int(T)


def shear_ensemble(n_inst=256, sides=(64, 128, 256, 512), seed=SEED_BASE + 3, W=4.0, tau=1.0, model=2):
    """Ragged ensemble of circular interfaces in wall-driven shear: square instances of side drawn from
    `sides`, periodic in x, moving walls in y, R ~ U[0.15, 0.3] side, shear rate ~ U[1e-5, 1e-4],
    Pe ~ U[10, 1000] with U* = shear * side / 2 (the wall speed)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n_inst):
        s = int(rng.choice(sides))
        R = float(rng.uniform(0.15, 0.3)) * s
        gam = float(rng.uniform(1e-5, 1e-4))
        Pe = float(rng.uniform(10.0, 1000.0))
        p = make_params(nx=s, ny=s, walls=1, vel=VEL_SHEAR, shear=gam, Pe=Pe, Ustar=gam * s / 2, W=W,
                        tau=tau, model=model)
        out.append((p, circle_phi(s, s, s / 2, s / 2, R, W)))
    return out


def paper_translation(L0=200, U0=0.02, Pe=200.0, W=2.0, sigma=0.01, tau=0.5 + math.sqrt(3) / 6,
                      rho_ratio=1.0, model=2):
    """The paper's own diagonal-translation setup (Sec. III.A): phiA = -phiB = 1, R = L0/5 centred,
    u = (U0, U0); one period T = L0/U0 steps."""
    p = make_params(nx=L0, ny=L0, vel=VEL_UNIFORM, ux0=U0, uy0=U0, W=W, sigma=sigma, Pe=Pe, Ustar=U0,
                    tau=tau, phiA=1.0, phiB=-1.0, rhoA=1.0, rhoB=1.0 / rho_ratio, model=model)
    phi0 = circle_phi(L0, L0, L0 / 2, L0 / 2, L0 / 5, W, 1.0, -1.0)
    return p, phi0, int(round(L0 / U0))


def paper_shear_reversal(L0=200, U0=0.025, W=2.0, Pe=1000.0, tau=1.0, model=2):
    """The paper's circular interface in a reversing shear flow (Sec. III.C, Eq. shear): R = L0/5 at
    (L0/2, 0.3 L0), phiA = -phiB = 1, rhoA = 1, rhoB = 0.5, sigma = 0.01; the flow reverses at t = T with
    T = L0/U0 (the convective period of the other tests; the text does not state it), so the interface
    returns at t = 2T, the returned step count."""
    T = int(round(L0 / U0))
    p = make_params(nx=L0, ny=L0, vel=VEL_REV_SHEAR, U0=U0, Tper=float(T), W=W, Pe=Pe, Ustar=U0, tau=tau,
                    phiA=1.0, phiB=-1.0, rhoA=1.0, rhoB=0.5, sigma=0.01, model=model)
    phi0 = circle_phi(L0, L0, 0.5 * L0, 0.3 * L0, L0 / 5, W, 1.0, -1.0)
    return p, phi0, 2 * T


def paper_deformation(L0=500, U0=0.025, W=2.0, Pe=1000.0, nvort=4, tau=1.0, model=2):
    """The paper's deformation field (Sec. III.D, Eq. deformation): a circle R = L0/5 at the centre in n = 4
    vortices whose velocity carries the factor cos(pi t/T0), T0 = 5T/4 with T = L0/U0; the flow runs
    backwards after T0/2, so the interface returns at t = T0, the returned step count."""
    T0 = int(round(1.25 * L0 / U0))
    p = make_params(nx=L0, ny=L0, vel=VEL_DEFORM, nvort=nvort, U0=U0, Tper=float(T0), W=W, Pe=Pe, Ustar=U0,
                    tau=tau, phiA=1.0, phiB=-1.0, rhoA=1.0, rhoB=0.5, sigma=0.01, model=model)
    phi0 = circle_phi(L0, L0, 0.5 * L0, 0.5 * L0, L0 / 5, W, 1.0, -1.0)
    return p, phi0, T0


def rayleigh_taylor(nx=256, ny=1024, atwood=0.5, Re=3000.0, Pe=1000.0, W=5.0, sqrt_g_lambda=0.04,
                    amp=0.1, sigma=5e-5, tau=1.0, model=2):
    """Rayleigh-Taylor instability (Sec. III.E shape): heavy phase A (phi = 1) above y = ny/2 + amp nx
    cos(2 pi x/nx), light phase B (phi = -1) below; periodic in x, no-slip walls in y; lambda = nx,
    sqrt(g lambda) given, rho_h = 1, rho_l from the Atwood number, nu from Re = lambda sqrt(A g lambda/(1+A))/nu,
    M from Pe with U* = sqrt(g lambda)."""
    lam = float(nx)
    g = sqrt_g_lambda ** 2 / lam
    rho_h, rho_l = 1.0, (1.0 - atwood) / (1.0 + atwood)
    nu = lam * math.sqrt(atwood * g * lam / (1.0 + atwood)) / Re
    p = make_params(nx=nx, ny=ny, walls=1, vel=VEL_COUPLED, phiA=1.0, phiB=-1.0, rhoA=rho_h, rhoB=rho_l,
                    sigma=sigma, W=W, Pe=Pe, Ustar=sqrt_g_lambda, tau=tau, model=model, nu=nu, gx=0.0, gy=g)
    x, y = _grid(nx, ny)
    h = ny / 2 + amp * nx * np.cos(2 * np.pi * x / nx)
    phi0 = tanh_profile(y - h, W, 1.0, -1.0)
    return p, phi0


def random_smooth_phi(nx, ny, seed, amp=0.3, mean=0.5, modes=4) -> np.ndarray:
    """A smooth random periodic field (a few Fourier modes) for parity tests at odd sizes."""
    rng = np.random.default_rng(seed)
    x, y = _grid(nx, ny)
    f = np.full((ny, nx), mean)
    for _ in range(modes):
        kx, ky = rng.integers(0, 3, size=2)
        ph = rng.uniform(0, 2 * np.pi)
        f += amp / modes * np.cos(2 * np.pi * (kx * x / nx + ky * y / ny) + ph)
    return f


def moving_wall_case(nx=45, ny=37, shear=2e-3, tau=0.8, model=2, seed=SEED_BASE + 11):
    """A wall-bounded shear flow at tau_g != 1 with a field that varies along the walls: the walls move at
    -/+ shear * ny / 2, and the bounced populations carry the moving-wall term into phi one step later.
    Returns (params, phi0)."""
    p = make_params(nx=nx, ny=ny, walls=1, vel=VEL_SHEAR, shear=shear, model=model, tau=tau, M=0.02,
                    sigma=0.02, W=3.0)
    return p, random_smooth_phi(nx, ny, seed=seed)
