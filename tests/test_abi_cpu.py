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
