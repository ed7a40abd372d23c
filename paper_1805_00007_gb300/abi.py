"""Thin ctypes binding of the C ABI in include/lbch.h: the same entry points, argument marshalling only.

Every step of the method runs in the CUDA library; this module never computes any part of it.  If the
library cannot be loaded the import of the entry points raises -- there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _build

LBCH_OK, LBCH_EINVAL, LBCH_ENOMEM, LBCH_ECUDA, LBCH_ETIMEOUT, LBCH_ENONFINITE = range(6)
LBCH_F64, LBCH_F32, LBCH_F16S = range(3)
LBCH_OBS_MASS, LBCH_OBS_ERR_L2, LBCH_OBS_MAX, LBCH_OBS_MIN, LBCH_OBS_PHI, LBCH_OBS_STEP, LBCH_OBS_U, LBCH_OBS_P = range(8)
PRECISIONS = {"f64": LBCH_F64, "f32": LBCH_F32, "f16s": LBCH_F16S}

# Exported symbols, as declared in include/lbch.h.
SYMBOLS = ("lb_ch_init", "lb_ch_step", "lb_ch_observe", "lb_ch_observe_all", "lb_ch_free",
           "lb_ch_strerror", "lb_ch_last_error", "lb_ch_info", "lb_ch_kernel_info", "lb_ch_stream", "lb_ch_test_hook",
           "lb_ch_field_stats_noalloc", "lb_ch_state_bytes", "lb_ch_state_save", "lb_ch_state_load",
           "lb_ch_tape_phi", "lb_ch_adjoint_begin", "lb_ch_adjoint_step", "lb_ch_adjoint_end", "lb_ch_tune",
           "lb_ch_alu_peak", "lb_ch_init_slab", "lb_ch_halo_bytes", "lb_ch_halo_export", "lb_ch_halo_import",
           "lb_ch_step_taped", "lb_ch_adjoint_sweep")
(LBCH_HOOK_SKIP_FIRST_LOAD, LBCH_HOOK_TILE_SHAPE, LBCH_HOOK_GENERAL_PATH, LBCH_HOOK_NO_PDL, LBCH_HOOK_TILE_KERNEL,
 LBCH_HOOK_TWO_STEP, LBCH_HOOK_POISON) = 1, 2, 3, 4, 5, 6, 7


class lbch_params(ctypes.Structure):
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


class LbchError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {msg} (status {status})")
        self.status = status


_lib = None


def load(path: str | None = None) -> ctypes.CDLL:
    """Load liblbch.so (building it in-tree first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _build.build()
    if not os.path.exists(path):
        raise OSError(f"CUDA library not found at {path}")
    lib = ctypes.CDLL(path)
    P = ctypes.POINTER
    dp = P(ctypes.c_double)
    vp = ctypes.c_void_p
    lib.lb_ch_init.argtypes = [P(lbch_params), ctypes.c_int, dp, ctypes.c_int, vp, P(vp)]
    lib.lb_ch_step.argtypes = [vp, ctypes.c_long]
    lib.lb_ch_observe.argtypes = [vp, ctypes.c_int, ctypes.c_int, dp]
    lib.lb_ch_observe_all.argtypes = [vp, ctypes.c_int, dp]
    lib.lb_ch_free.argtypes = [vp]
    lib.lb_ch_strerror.argtypes = [ctypes.c_int]
    lib.lb_ch_strerror.restype = ctypes.c_char_p
    lib.lb_ch_last_error.argtypes = []
    lib.lb_ch_last_error.restype = ctypes.c_char_p
    lib.lb_ch_info.argtypes = [vp, dp]
    lib.lb_ch_kernel_info.argtypes = [vp, P(ctypes.c_int)]
    lib.lb_ch_stream.argtypes = [vp]
    lib.lb_ch_stream.restype = vp
    lib.lb_ch_test_hook.argtypes = [vp, ctypes.c_int, ctypes.c_long]
    lib.lb_ch_field_stats_noalloc.argtypes = [vp, vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, vp]
    lib.lb_ch_state_bytes.argtypes = [vp, P(ctypes.c_longlong)]
    lib.lb_ch_state_save.argtypes = [vp, vp]
    lib.lb_ch_state_load.argtypes = [vp, vp]
    lib.lb_ch_tape_phi.argtypes = [vp, vp]
    lib.lb_ch_adjoint_begin.argtypes = [vp, vp]
    lib.lb_ch_adjoint_step.argtypes = [vp, vp, ctypes.c_long]
    lib.lb_ch_adjoint_end.argtypes = [vp, vp, dp]
    lib.lb_ch_tune.argtypes = [vp, ctypes.c_int, P(ctypes.c_int), P(ctypes.c_int)]
    lib.lb_ch_alu_peak.argtypes = [ctypes.c_int, vp, dp]
    lib.lb_ch_init_slab.argtypes = [P(lbch_params), ctypes.c_int, ctypes.c_int, dp, ctypes.c_int, vp, P(vp)]
    lib.lb_ch_halo_bytes.argtypes = [vp, P(ctypes.c_longlong)]
    lib.lb_ch_halo_export.argtypes = [vp, ctypes.c_int, vp]
    lib.lb_ch_halo_import.argtypes = [vp, ctypes.c_int, vp]
    lib.lb_ch_step_taped.argtypes = [vp, ctypes.c_long, vp]
    lib.lb_ch_adjoint_sweep.argtypes = [vp, vp, ctypes.c_long, ctypes.c_long]
    for name in ("lb_ch_init", "lb_ch_step", "lb_ch_observe", "lb_ch_observe_all", "lb_ch_free", "lb_ch_info",
                 "lb_ch_kernel_info",
                 "lb_ch_test_hook", "lb_ch_field_stats_noalloc", "lb_ch_state_bytes", "lb_ch_state_save",
                 "lb_ch_state_load", "lb_ch_tape_phi", "lb_ch_adjoint_begin", "lb_ch_adjoint_step",
                 "lb_ch_adjoint_end", "lb_ch_tune", "lb_ch_alu_peak", "lb_ch_init_slab", "lb_ch_halo_bytes",
                 "lb_ch_halo_export", "lb_ch_halo_import", "lb_ch_step_taped", "lb_ch_adjoint_sweep"):
        getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def _check(status: int, where: str):
    if status != LBCH_OK:
        lib = load()
        raise LbchError(status, where, lib.lb_ch_last_error().decode() or lib.lb_ch_strerror(status).decode())


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def make_params(cfg) -> lbch_params:
    p = lbch_params()
    for name, ctype in lbch_params._fields_:
        v = cfg[name]
        setattr(p, name, int(v) if ctype is ctypes.c_int else float(v))
    return p


# ----------------------------------------------------------------------------- entry points

def lb_ch_init(params, phi0, prec=LBCH_F64, stream=None):
    """params: one config dict or a list of them; phi0: one (ny, nx) array or a list.  Returns a handle."""
    lib = load()
    if isinstance(params, dict):
        params, phi0 = [params], [phi0]
    n = len(params)
    arr = (lbch_params * n)(*[make_params(p) for p in params])
    flat = np.ascontiguousarray(np.concatenate([np.ascontiguousarray(f, dtype=np.float64).ravel() for f in phi0]))
    for p, f in zip(params, phi0):
        if np.shape(f) != (p["ny"], p["nx"]):
            raise ValueError(f"phi0 of shape {np.shape(f)} does not match ny x nx = {p['ny']} x {p['nx']}")
    h = ctypes.c_void_p()
    _check(lib.lb_ch_init(arr, n, _dptr(flat), int(prec), ctypes.c_void_p(stream or 0), ctypes.byref(h)),
           "lb_ch_init")
    return h


def lb_ch_init_slab(params: dict, y0: int, ny_local: int, phi0_halo, prec=LBCH_F64, stream=None):
    """A handle for global rows y0 .. y0 + ny_local - 1 of the periodic problem `params`; phi0_halo holds
    ny_local + 6 rows (global rows y0 - 3 .. y0 + ny_local + 2, wrapped) of nx values."""
    lib = load()
    f = np.ascontiguousarray(phi0_halo, dtype=np.float64)
    if f.shape != (int(ny_local) + 6, params["nx"]):
        raise ValueError(f"phi0_halo of shape {f.shape} is not (ny_local + 6, nx) = ({ny_local + 6}, {params['nx']})")
    h = ctypes.c_void_p()
    p = make_params(params)
    _check(lib.lb_ch_init_slab(ctypes.byref(p), int(y0), int(ny_local), _dptr(f), int(prec),
                               ctypes.c_void_p(stream or 0), ctypes.byref(h)), "lb_ch_init_slab")
    return h


def lb_ch_halo_bytes(h) -> int:
    out = ctypes.c_longlong(0)
    _check(load().lb_ch_halo_bytes(h, ctypes.byref(out)), "lb_ch_halo_bytes")
    return out.value


def lb_ch_halo_export(h, side: int, dst_ptr: int):
    _check(load().lb_ch_halo_export(h, int(side), ctypes.c_void_p(dst_ptr)), "lb_ch_halo_export")


def lb_ch_halo_import(h, side: int, src_ptr: int):
    _check(load().lb_ch_halo_import(h, int(side), ctypes.c_void_p(src_ptr)), "lb_ch_halo_import")


def lb_ch_step(h, nsteps: int):
    _check(load().lb_ch_step(h, int(nsteps)), "lb_ch_step")


def lb_ch_observe(h, inst: int, what: int, shape=None):
    if what in (LBCH_OBS_PHI, LBCH_OBS_P):
        out = np.empty(shape, dtype=np.float64)
    elif what == LBCH_OBS_U:
        out = np.empty((2,) + tuple(shape), dtype=np.float64)
    else:
        out = np.empty(1, dtype=np.float64)
    _check(load().lb_ch_observe(h, int(inst), int(what), _dptr(out)), "lb_ch_observe")
    return out if what in (LBCH_OBS_PHI, LBCH_OBS_P, LBCH_OBS_U) else float(out[0])


def lb_ch_observe_all(h, what: int, n_inst: int) -> np.ndarray:
    out = np.empty(n_inst, dtype=np.float64)
    _check(load().lb_ch_observe_all(h, int(what), _dptr(out)), "lb_ch_observe_all")
    return out


def lb_ch_free(h):
    if h:
        _check(load().lb_ch_free(h), "lb_ch_free")


KERNEL_FORMS = {0: "tile", 1: "sweep_tau1", 2: "sweep", 3: "coupled", 4: "tile_tau1", 5: "pair_tau1"}


def lb_ch_kernel_info(h) -> dict:
    """The step kernel in use: its form, shape index, tile, rows per warp and threads per block."""
    out = (ctypes.c_int * 6)()
    _check(load().lb_ch_kernel_info(h, out), "lb_ch_kernel_info")
    return {"form": KERNEL_FORMS[out[0]], "shape": out[1], "tile": (out[2], out[3]), "rows_per_warp": out[4],
            "threads": out[5]}


def lb_ch_info(h) -> dict:
    out = np.zeros(4)
    _check(load().lb_ch_info(h, _dptr(out)), "lb_ch_info")
    return {"nodes": int(out[0]), "bytes_per_lu": out[1], "grid": int(out[2]), "step": int(out[3])}


def lb_ch_test_hook(h, hook: int, value: int):
    _check(load().lb_ch_test_hook(h, int(hook), int(value)), "lb_ch_test_hook")


def lb_ch_alu_peak(prec: int, stream: int | None = None) -> float:
    """Fused multiply-add throughput of the current device in prec (LBCH_F32 or LBCH_F64), flop/s."""
    out = ctypes.c_double(0.0)
    _check(load().lb_ch_alu_peak(int(prec), ctypes.c_void_p(stream or 0), ctypes.byref(out)), "lb_ch_alu_peak")
    return out.value


def lb_ch_field_stats_noalloc(phi_ptr: int, phi0_ptr: int, nx: int, ny: int, pitch: int, out_ptr: int,
                              stream: int = 0):
    """Statistics of a caller-owned device field (device pointers as integers) into a caller-owned
    device array of 6 doubles, without any device allocation."""
    _check(load().lb_ch_field_stats_noalloc(ctypes.c_void_p(phi_ptr), ctypes.c_void_p(phi0_ptr), int(nx), int(ny),
                                            int(pitch), ctypes.c_void_p(out_ptr), ctypes.c_void_p(stream or 0)),
           "lb_ch_field_stats_noalloc")


def lb_ch_state_bytes(h) -> int:
    out = ctypes.c_longlong(0)
    _check(load().lb_ch_state_bytes(h, ctypes.byref(out)), "lb_ch_state_bytes")
    return out.value


def lb_ch_state_save(h, dst_ptr: int):
    _check(load().lb_ch_state_save(h, ctypes.c_void_p(dst_ptr)), "lb_ch_state_save")


def lb_ch_state_load(h, src_ptr: int):
    _check(load().lb_ch_state_load(h, ctypes.c_void_p(src_ptr)), "lb_ch_state_load")


def lb_ch_tape_phi(h, dst_ptr: int):
    _check(load().lb_ch_tape_phi(h, ctypes.c_void_p(dst_ptr)), "lb_ch_tape_phi")


def lb_ch_adjoint_begin(h, dphiT_ptr: int):
    _check(load().lb_ch_adjoint_begin(h, ctypes.c_void_p(dphiT_ptr)), "lb_ch_adjoint_begin")


def lb_ch_adjoint_step(h, phi_n_ptr: int, n: int):
    _check(load().lb_ch_adjoint_step(h, ctypes.c_void_p(phi_n_ptr), int(n)), "lb_ch_adjoint_step")


def lb_ch_step_taped(h, nsteps: int, tape_ptr: int):
    _check(load().lb_ch_step_taped(h, int(nsteps), ctypes.c_void_p(tape_ptr)), "lb_ch_step_taped")


def lb_ch_adjoint_sweep(h, tape_ptr: int, n0: int, nsteps: int):
    _check(load().lb_ch_adjoint_sweep(h, ctypes.c_void_p(tape_ptr), int(n0), int(nsteps)), "lb_ch_adjoint_sweep")


def lb_ch_adjoint_end(h, dphi0_ptr: int) -> float:
    out = ctypes.c_double(0.0)
    _check(load().lb_ch_adjoint_end(h, ctypes.c_void_p(dphi0_ptr), ctypes.byref(out)), "lb_ch_adjoint_end")
    return out.value


def lb_ch_tune(h, steps: int = 20):
    """Time every built tile shape on this handle's problem and keep the fastest; returns (tx, ty)."""
    tx, ty = ctypes.c_int(0), ctypes.c_int(0)
    _check(load().lb_ch_tune(h, int(steps), ctypes.byref(tx), ctypes.byref(ty)), "lb_ch_tune")
    return tx.value, ty.value


def lb_ch_stream(h) -> int:
    return load().lb_ch_stream(h) or 0


# ----------------------------------------------------------------------------- convenience wrapper

class Simulation:
    """One handle: an instance or a ragged ensemble of instances advanced together."""

    def __init__(self, params, phi0, prec="f64", stream=None, tune: bool = False):
        self.params = [params] if isinstance(params, dict) else list(params)
        self.prec = PRECISIONS[prec] if isinstance(prec, str) else int(prec)
        self.h = lb_ch_init(self.params, [phi0] if isinstance(params, dict) else list(phi0), self.prec, stream)
        # enough timed steps per candidate that small grids (a few microseconds per step) are not decided
        # by timer noise: about 2e7 lattice updates, between 20 and 400 steps
        nodes = sum(int(p["nx"]) * int(p["ny"]) for p in self.params)
        self.tile = lb_ch_tune(self.h, max(20, min(400, 20_000_000 // max(nodes, 1)))) if tune else None

    def step(self, nsteps: int):
        lb_ch_step(self.h, nsteps)
        return self

    def phi(self, inst: int = 0) -> np.ndarray:
        p = self.params[inst]
        return lb_ch_observe(self.h, inst, LBCH_OBS_PHI, (p["ny"], p["nx"]))

    def observe(self, what: int, inst: int = 0) -> float:
        return lb_ch_observe(self.h, inst, what)

    def velocity(self, inst: int = 0) -> np.ndarray:
        """(2, ny, nx): the flow's velocity of a coupled handle."""
        p = self.params[inst]
        return lb_ch_observe(self.h, inst, LBCH_OBS_U, (p["ny"], p["nx"]))

    def pressure(self, inst: int = 0) -> np.ndarray:
        p = self.params[inst]
        return lb_ch_observe(self.h, inst, LBCH_OBS_P, (p["ny"], p["nx"]))

    def observe_all(self, what: int) -> np.ndarray:
        return lb_ch_observe_all(self.h, what, len(self.params))

    def info(self) -> dict:
        return lb_ch_info(self.h)

    def kernel(self) -> dict:
        return lb_ch_kernel_info(self.h)

    def close(self):
        if self.h:
            lb_ch_free(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
