"""Host-side checks of the C ABI that need no GPU: the library builds, loads and exports every entry
point include/*.h declares; argument validation fails cleanly without touching a device."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

from paper_1805_00007_gb300 import abi
from paper_1805_00007_gb300 import workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(hdr).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(lb_ch_\w+)\s*\(", text))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ("lb_ch_init", "lb_ch_step", "lb_ch_observe", "lb_ch_free"):
        assert required in names


def test_library_exports_every_declared_symbol():
    lib = abi.load()
    for name in declared_symbols():
        assert hasattr(lib, name), f"{name} declared in include/ but not exported"
    assert set(abi.SYMBOLS) <= set(declared_symbols())


def test_param_struct_layout_matches_header():
    """The ctypes mirror of lbch_params lists the header's fields in the header's order."""
    text = open(os.path.join(ROOT, "include", "lbch.h")).read()
    body = re.search(r"typedef struct \{(.*?)\} lbch_params;", text, flags=re.S).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl:
            continue
        parts = decl.split(None, 1)
        fields += [f.strip() for f in parts[1].split(",")]
    assert fields == [f for f, _ in abi.lbch_params._fields_]


def test_invalid_arguments_rejected_without_gpu():
    lib = abi.load()
    h = ctypes.c_void_p()
    p, phi0, _ = wl.translation(nx=8)
    bad = dict(p, nx=2, ny=2)
    arr = (abi.lbch_params * 1)(abi.make_params(bad))
    flat = np.zeros(4)
    st = lib.lb_ch_init(arr, 1, flat.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 0, None, ctypes.byref(h))
    assert st == abi.LBCH_EINVAL and not h.value
    assert b"nx" in lib.lb_ch_last_error()
    for kw in (dict(tau=0.5), dict(model=4), dict(model=0), dict(vel=9), dict(M=0.0, Pe=0.0),
               dict(model=3, vel=wl.VEL_COUPLED, nu=0.01)):
        arr = (abi.lbch_params * 1)(abi.make_params(dict(p, **kw)))
        flat = np.ascontiguousarray(phi0.ravel())
        st = lib.lb_ch_init(arr, 1, flat.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 0, None, ctypes.byref(h))
        assert st == abi.LBCH_EINVAL, kw
    assert lib.lb_ch_step(None, 1) == abi.LBCH_EINVAL
    assert lib.lb_ch_free(None) == abi.LBCH_OK
    assert lib.lb_ch_strerror(abi.LBCH_ENONFINITE) == b"non-finite order parameter"


def test_binding_rejects_shape_mismatch():
    p, phi0, _ = wl.translation(nx=8)
    with pytest.raises(ValueError):
        abi.lb_ch_init(p, phi0[:, :4])


def test_every_entry_point_rejects_null_arguments_without_gpu():
    """Each entry point checks its handle and pointers before touching a device: NULL gives LBCH_EINVAL
    (lb_ch_free(NULL) is a no-op, lb_ch_stream(NULL) is NULL) and sets the last-error message."""
    lib = abi.load()
    d = ctypes.c_double()
    i = ctypes.c_int()
    ll = ctypes.c_longlong()
    buf = ctypes.c_void_p(8)  # never dereferenced: the NULL handle is rejected first
    h = ctypes.c_void_p()
    calls = {
        "lb_ch_observe": lambda: lib.lb_ch_observe(None, 0, abi.LBCH_OBS_MASS, ctypes.byref(d)),
        "lb_ch_observe_all": lambda: lib.lb_ch_observe_all(None, abi.LBCH_OBS_MASS, ctypes.byref(d)),
        "lb_ch_info": lambda: lib.lb_ch_info(None, ctypes.byref(d)),
        "lb_ch_kernel_info": lambda: lib.lb_ch_kernel_info(None, ctypes.byref(i)),
        "lb_ch_tune": lambda: lib.lb_ch_tune(None, 8, ctypes.byref(i), ctypes.byref(i)),
        "lb_ch_state_bytes": lambda: lib.lb_ch_state_bytes(None, ctypes.byref(ll)),
        "lb_ch_state_save": lambda: lib.lb_ch_state_save(None, buf),
        "lb_ch_state_load": lambda: lib.lb_ch_state_load(None, buf),
        "lb_ch_tape_phi": lambda: lib.lb_ch_tape_phi(None, buf),
        "lb_ch_adjoint_begin": lambda: lib.lb_ch_adjoint_begin(None, buf),
        "lb_ch_adjoint_step": lambda: lib.lb_ch_adjoint_step(None, buf, 0),
        "lb_ch_adjoint_end": lambda: lib.lb_ch_adjoint_end(None, buf, ctypes.byref(d)),
        "lb_ch_test_hook": lambda: lib.lb_ch_test_hook(None, abi.LBCH_HOOK_POISON, 1),
        "lb_ch_field_stats_noalloc": lambda: lib.lb_ch_field_stats_noalloc(None, None, 4, 4, 4, None, None),
        "lb_ch_alu_peak (bad precision)": lambda: lib.lb_ch_alu_peak(abi.LBCH_F16S, None, ctypes.byref(d)),
        "lb_ch_init_slab": lambda: lib.lb_ch_init_slab(None, 0, 8, None, 0, None, ctypes.byref(h)),
        "lb_ch_halo_bytes": lambda: lib.lb_ch_halo_bytes(None, ctypes.byref(ll)),
        "lb_ch_halo_export": lambda: lib.lb_ch_halo_export(None, 0, buf),
        "lb_ch_halo_import": lambda: lib.lb_ch_halo_import(None, 1, buf),
        "lb_ch_step_taped": lambda: lib.lb_ch_step_taped(None, 4, buf),
        "lb_ch_adjoint_sweep": lambda: lib.lb_ch_adjoint_sweep(None, buf, 0, 4),
    }
    for name, call in calls.items():
        assert call() == abi.LBCH_EINVAL, name
        assert lib.lb_ch_last_error(), name
    assert lib.lb_ch_free(None) == abi.LBCH_OK
    assert lib.lb_ch_stream(None) is None


def test_missing_library_fails_loudly():
    """There is no fallback: a binding whose library is absent raises instead of computing anything."""
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = ("from paper_1805_00007_gb300 import abi\n"
            "abi.load('/nonexistent/liblbch.so')\n")
    r = subprocess.run([sys.executable, "-c", code], cwd=root, capture_output=True, text=True, timeout=120)
    assert r.returncode != 0 and "CUDA library not found" in r.stderr
