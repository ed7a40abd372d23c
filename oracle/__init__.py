"""FP64 CPU oracle of the high-order lattice Boltzmann model for the Cahn-Hilliard equation.

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU-baseline leg use this
package to check and time the CUDA library; the product path never imports it.  The arithmetic lives
in ``lbch_oracle.c`` (plain C, double precision, no fast-math, no FMA contraction); this module only
compiles it with gcc and marshals numpy arrays through ctypes.

Parity status of each oracle function (what pins it is in ``tests/test_oracle_pins.py`` and
``tests/test_oracle_chapman_enskog.py``):
  geq, source, dfdphi, grad, lap, div, mu, force, init, step, observe -- pinned
  (moment identities, exact stencil symbols, polynomial exactness, a linear-stability amplification
  matrix built independently, conservation, stationarity, special values of K, the co-moving uniform
  state between moving walls for the bounce-back term, and the Chapman-Enskog expansion of the update:
  the dispersion of small waves matches the exact series whose terms are the Cahn-Hilliard equation and
  the paper's third-order error R1 + R2).
  The long-time benchmark behaviour (paper Sec. III) is pinned only softly (printed max/min of phi);
  the paper's error curves are figures that are not available, so those are "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, fields

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbch_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liblbch_oracle.so")

VEL_UNIFORM, VEL_ROTATION, VEL_VORTEX, VEL_SHEAR, VEL_REV_SHEAR, VEL_DEFORM, VEL_COUPLED = range(7)


class _Params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("walls", ctypes.c_int), ("model", ctypes.c_int),
        ("vel", ctypes.c_int), ("nvort", ctypes.c_int),
        ("phiA", ctypes.c_double), ("phiB", ctypes.c_double),
        ("sigma", ctypes.c_double), ("W", ctypes.c_double),
        ("M", ctypes.c_double), ("Pe", ctypes.c_double), ("Ustar", ctypes.c_double),
        ("tau", ctypes.c_double), ("rhoA", ctypes.c_double), ("rhoB", ctypes.c_double),
        ("U0", ctypes.c_double), ("ux0", ctypes.c_double), ("uy0", ctypes.c_double),
        ("xc", ctypes.c_double), ("yc", ctypes.c_double), ("half", ctypes.c_double),
        ("Tper", ctypes.c_double), ("shear", ctypes.c_double),
        ("nu", ctypes.c_double), ("gx", ctypes.c_double), ("gy", ctypes.c_double),
    ]


class _Consts(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in ("beta", "kappa", "M", "eta", "a", "b", "K")]


@dataclass
class Consts:
    beta: float
    kappa: float
    M: float
    eta: float
    a: float
    b: float
    K: float


def build(force: bool = False, openmp: bool = True) -> str:
    """Compile the oracle into a shared library (gcc, -O2, strict IEEE double)."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    cmd = ["gcc", "-O2", "-fno-fast-math", "-ffp-contract=off", "-fPIC", "-shared", "-std=c99"]
    if openmp:
        cmd.append("-fopenmp")
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd += [_SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        P = ctypes.POINTER
        dp = P(ctypes.c_double)
        _lib.ora_derive.argtypes = [P(_Params), P(_Consts)]
        _lib.ora_velocity.argtypes = [P(_Params), ctypes.c_double, ctypes.c_double, ctypes.c_long, dp, dp]
        _lib.ora_geq.argtypes = [ctypes.c_double] * 5 + [dp]
        _lib.ora_source.argtypes = [ctypes.c_double, ctypes.c_double, dp]
        _lib.ora_dfdphi.argtypes = [ctypes.c_double] * 4
        _lib.ora_dfdphi.restype = ctypes.c_double
        _lib.ora_grad.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp, dp]
        _lib.ora_lap.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp]
        _lib.ora_div.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp, dp]
        _lib.ora_phi.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp]
        _lib.ora_mu.argtypes = [P(_Params), P(_Consts), dp, dp]
        _lib.ora_velocity_field.argtypes = [P(_Params), ctypes.c_long, dp, dp]
        _lib.ora_force.argtypes = [P(_Params), P(_Consts), dp, dp, dp, dp, dp, dp]
        _lib.ora_init.argtypes = [P(_Params), dp, dp]
        _lib.ora_step.argtypes = [P(_Params), dp, dp, ctypes.c_long]
        _lib.ora_set_threads.argtypes = [ctypes.c_int]
        _lib.ora_set_threads.restype = ctypes.c_int
        _lib.ora_run.argtypes = [P(_Params), dp, ctypes.c_long, ctypes.c_long]
        _lib.ora_run.restype = ctypes.c_int
        _lib.ora_step_full.argtypes = [P(_Params), dp, dp, dp, ctypes.c_int, ctypes.c_long]
        _lib.ora_run_full.argtypes = [P(_Params), dp, dp, ctypes.c_long, ctypes.c_long]
        _lib.ora_run_full.restype = ctypes.c_int
        _lib.ora_observe.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, dp]
        _lib.ora_d2fdphi2.argtypes = [ctypes.c_double] * 4
        _lib.ora_d2fdphi2.restype = ctypes.c_double
        _lib.ora_adjoint_step.argtypes = [P(_Params), dp, dp, dp, ctypes.c_long, dp]
        _lib.ora_adjoint_step.restype = ctypes.c_int
        _lib.ora_adjoint_init.argtypes = [P(_Params), dp, dp, dp, dp]
        _lib.ora_adjoint_init.restype = ctypes.c_int
        _lib.ora_ns_fields.argtypes = [P(_Params), dp, dp, dp, dp, dp]
        _lib.ora_ns_init.argtypes = [P(_Params), dp, dp, dp, dp, dp]
        _lib.ora_ns_step.argtypes = [P(_Params), dp, dp, dp, dp, ctypes.c_long]
    return _lib


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def params(cfg) -> _Params:
    """Marshal a configuration (any object or dict with the parameter names) into the C struct."""
    p = _Params()
    get = cfg.get if isinstance(cfg, dict) else (lambda k, d=None: getattr(cfg, k, d))
    for name, ctype in _Params._fields_:
        v = get(name, None)
        if v is None:
            v = {"nvort": 4, "model": 2, "phiA": 1.0, "phiB": 0.0, "rhoA": 1.0, "rhoB": 0.5,
                 "tau": 1.0}.get(name, 0)
        setattr(p, name, int(v) if ctype is ctypes.c_int else float(v))
    return p


def derive(cfg) -> Consts:
    p, c = params(cfg), _Consts()
    lib().ora_derive(ctypes.byref(p), ctypes.byref(c))
    return Consts(*[getattr(c, f.name) for f in fields(Consts)])


def _consts(cfg):
    p, c = params(cfg), _Consts()
    lib().ora_derive(ctypes.byref(p), ctypes.byref(c))
    return p, c


def velocity(cfg, x: float, y: float, n: int):
    p = params(cfg)
    ux, uy = ctypes.c_double(), ctypes.c_double()
    lib().ora_velocity(ctypes.byref(p), x, y, n, ctypes.byref(ux), ctypes.byref(uy))
    return ux.value, uy.value


def velocity_field(cfg, n: int):
    p = params(cfg)
    ux = np.zeros((p.ny, p.nx)); uy = np.zeros((p.ny, p.nx))
    lib().ora_velocity_field(ctypes.byref(p), n, _ptr(ux), _ptr(uy))
    return ux, uy


def geq(phi, mu, ux, uy, eta) -> np.ndarray:
    out = np.zeros(9)
    lib().ora_geq(phi, mu, ux, uy, eta, _ptr(out))
    return out


def source(Fx, Fy) -> np.ndarray:
    out = np.zeros(9)
    lib().ora_source(Fx, Fy, _ptr(out))
    return out


def dfdphi(phi, beta, phiA, phiB) -> float:
    return lib().ora_dfdphi(phi, beta, phiA, phiB)


def grad(psi, walls: int = 0):
    psi = _f64(psi); ny, nx = psi.shape
    gx = np.zeros_like(psi); gy = np.zeros_like(psi)
    lib().ora_grad(nx, ny, walls, _ptr(psi), _ptr(gx), _ptr(gy))
    return gx, gy


def lap(psi, walls: int = 0):
    psi = _f64(psi); ny, nx = psi.shape
    out = np.zeros_like(psi)
    lib().ora_lap(nx, ny, walls, _ptr(psi), _ptr(out))
    return out


def div(vx, vy, walls: int = 0):
    vx, vy = _f64(vx), _f64(vy); ny, nx = vx.shape
    out = np.zeros_like(vx)
    lib().ora_div(nx, ny, walls, _ptr(vx), _ptr(vy), _ptr(out))
    return out


def phi_of(g) -> np.ndarray:
    g = _f64(g); _, ny, nx = g.shape
    out = np.zeros((ny, nx))
    lib().ora_phi(nx, ny, _ptr(g), _ptr(out))
    return out


def mu(cfg, phi):
    p, c = _consts(cfg)
    phi = _f64(phi); out = np.zeros_like(phi)
    lib().ora_mu(ctypes.byref(p), ctypes.byref(c), _ptr(phi), _ptr(out))
    return out


def force(cfg, phi, mu_, ux, uy):
    p, c = _consts(cfg)
    phi, mu_, ux, uy = map(_f64, (phi, mu_, ux, uy))
    Fx = np.zeros_like(phi); Fy = np.zeros_like(phi)
    lib().ora_force(ctypes.byref(p), ctypes.byref(c), _ptr(phi), _ptr(mu_), _ptr(ux), _ptr(uy),
                    _ptr(Fx), _ptr(Fy))
    return Fx, Fy


def init(cfg, phi0) -> np.ndarray:
    p = params(cfg)
    phi0 = _f64(phi0)
    assert phi0.shape == (p.ny, p.nx)
    g = np.zeros((9, p.ny, p.nx))
    lib().ora_init(ctypes.byref(p), _ptr(phi0), _ptr(g))
    return g


def step(cfg, g, n: int) -> np.ndarray:
    p = params(cfg)
    g = _f64(g); out = np.zeros_like(g)
    lib().ora_step(ctypes.byref(p), _ptr(g), _ptr(out), n)
    return out


def set_threads(n: int = 0) -> int:
    """Threads of the oracle's parallel loops from now on (n > 0; 1 = single-threaded); 0 only queries.
    Returns the count in effect.  Results do not depend on it."""
    return int(lib().ora_set_threads(int(n)))


def run(cfg, g, nsteps: int, n0: int = 0) -> np.ndarray:
    """Advance a copy of g by nsteps steps starting at step index n0."""
    p = params(cfg)
    g = _f64(g).copy()
    rc = lib().ora_run(ctypes.byref(p), _ptr(g), n0, nsteps)
    if rc != 0:
        raise MemoryError("oracle run failed to allocate")
    return g


def run_full(cfg, g, H, nsteps: int, n0: int = 0):
    """Model III (model = 3): advance copies of g and of H (the stored part of the time-derivative terms of
    Eq. F2-1, 2 N values) by nsteps steps from step index n0; H is ignored when n0 = 0."""
    p = params(cfg)
    g = _f64(g).copy()
    H = np.zeros(2 * p.nx * p.ny) if H is None else _f64(H).copy()
    rc = lib().ora_run_full(ctypes.byref(p), _ptr(g), _ptr(H), n0, nsteps)
    if rc != 0:
        raise MemoryError("oracle run failed to allocate")
    return g, H


def step_full(cfg, g, H, n: int):
    """One Model III step n -> n+1; returns (g', H') (H is ignored at n = 0)."""
    p = params(cfg)
    out = np.empty_like(_f64(g))
    H = np.zeros(2 * p.nx * p.ny) if H is None else _f64(H).copy()
    lib().ora_step_full(ctypes.byref(p), _ptr(_f64(g)), _ptr(out), _ptr(H), int(n == 0), n)
    return out, H


def observe(phi, phi0) -> dict:
    phi, phi0 = _f64(phi), _f64(phi0)
    ny, nx = phi.shape
    out = np.zeros(6)
    lib().ora_observe(nx, ny, _ptr(phi), _ptr(phi0), _ptr(out))
    return {"mass": out[0], "err_l2": out[1], "max": out[2], "min": out[3],
            "err_num": out[4], "err_den": out[5]}


def simulate(cfg, phi0, nsteps: int, n0: int = 0):
    """phi after nsteps steps from the initial field phi0 (initial g from the equilibria)."""
    if int(cfg.get("model", 2)) == 3:
        if n0 != 0:
            raise ValueError("a Model III run from phi0 starts at step 0")
        g, _ = run_full(cfg, init(cfg, phi0), None, nsteps)
        return phi_of(g), g
    g = run(cfg, init(cfg, phi0), nsteps, n0)
    return phi_of(g), g


def d2fdphi2(phi, beta, phiA, phiB) -> float:
    return lib().ora_d2fdphi2(phi, beta, phiA, phiB)


def adjoint(cfg, phi0, nsteps: int, dL_dphiT):
    """Reverse-mode gradient of a loss of phi(nsteps): given dL/dphi(T), returns (dL/dphi0, dL/ds) where the
    velocity field is s * u (derivative at s = 1).  Stores every forward state (small grids only)."""
    p = params(cfg)
    phi0 = _f64(phi0)
    N = p.nx * p.ny
    states = [init(cfg, phi0)]
    for n in range(nsteps):
        states.append(step(cfg, states[-1], n))
    lam = np.repeat(_f64(dL_dphiT)[None], 9, axis=0).copy()   # phi = sum_q g_q
    dLds = ctypes.c_double(0.0)
    for n in range(nsteps - 1, -1, -1):
        out = np.zeros_like(lam)
        rc = lib().ora_adjoint_step(ctypes.byref(p), _ptr(states[n]), _ptr(lam), _ptr(out), n, ctypes.byref(dLds))
        if rc != 0:
            raise ValueError("the oracle adjoint supports periodic domains only")
        lam = out
    dphi0 = np.zeros((p.ny, p.nx))
    lib().ora_adjoint_init(ctypes.byref(p), _ptr(phi0), _ptr(np.ascontiguousarray(lam)), _ptr(dphi0), ctypes.byref(dLds))
    return dphi0, dLds.value


def ns_init(cfg, phi0, ux0=None, uy0=None):
    """Initial coupled state (f, g): g = g_eq(phi0, mu0, u0), f = f_eq(p = 0, rho(phi0), u0)."""
    p = params(cfg)
    phi0 = _f64(phi0)
    ux0 = np.zeros_like(phi0) if ux0 is None else _f64(ux0)
    uy0 = np.zeros_like(phi0) if uy0 is None else _f64(uy0)
    f = np.zeros((9, p.ny, p.nx)); g = np.zeros((9, p.ny, p.nx))
    lib().ora_ns_init(ctypes.byref(p), _ptr(phi0), _ptr(ux0), _ptr(uy0), _ptr(f), _ptr(g))
    return f, g


def ns_fields(cfg, f, g):
    p = params(cfg)
    f, g = _f64(f), _f64(g)
    ux = np.zeros((p.ny, p.nx)); uy = np.zeros_like(ux); pr = np.zeros_like(ux)
    lib().ora_ns_fields(ctypes.byref(p), _ptr(f), _ptr(g), _ptr(ux), _ptr(uy), _ptr(pr))
    return ux, uy, pr


def ns_simulate(cfg, phi0, nsteps: int, ux0=None, uy0=None):
    """Coupled Cahn-Hilliard / Navier-Stokes run: returns (phi, ux, uy, p, f, g) after nsteps."""
    p = params(cfg)
    f, g = ns_init(cfg, phi0, ux0, uy0)
    for n in range(nsteps):
        fo = np.zeros_like(f); go = np.zeros_like(g)
        lib().ora_ns_step(ctypes.byref(p), _ptr(f), _ptr(g), _ptr(fo), _ptr(go), n)
        f, g = fo, go
    ux, uy, pr = ns_fields(cfg, f, g)
    return phi_of(g), ux, uy, pr, f, g


def _simulate_one(args):
    cfg, phi0, nsteps = args
    set_threads(1)
    return simulate(cfg, phi0, nsteps)[0]


def simulate_many(cases, nsteps: int, processes: int | None = None) -> list:
    """phi after nsteps steps for each (cfg, phi0) of `cases` -- the same runs as simulate(), one
    single-threaded oracle per worker process, the workers started with `spawn` (never forked from a
    process that may hold a CUDA context).  Largest cases first, results in the order of `cases`."""
    import multiprocessing as mp
    order = sorted(range(len(cases)), key=lambda i: -int(cases[i][0]["nx"]) * int(cases[i][0]["ny"]))
    n = processes or os.cpu_count() or 1
    with mp.get_context("spawn").Pool(processes=min(n, len(cases))) as pool:
        res = pool.map(_simulate_one, [(cases[i][0], cases[i][1], nsteps) for i in order], chunksize=1)
    out = [None] * len(cases)
    for i, r in zip(order, res):
        out[i] = r
    return out
