"""The C-ABI library loads and exports every symbol include/cpm.h declares (no GPU)."""
import ctypes
import os
import re

import pytest

from paper_2111_06704_gb300 import build, cpm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    text = open(os.path.join(ROOT, "include", "cpm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(cpm_\w+)\s*\(", text)))


def test_library_builds_and_loads():
    path = build.build()
    assert os.path.exists(path)
    lib = cpm.load()
    assert isinstance(lib, ctypes.CDLL)


def test_every_declared_symbol_is_exported():
    lib = cpm.load()
    names = _declared_functions()
    assert "cpm_build_E" in names and "cpm_solve" in names
    for name in names:
        assert hasattr(lib, name), name
    assert set(cpm.EXPORTS) <= set(names)


def test_default_parameters_follow_the_paper():
    p = cpm.default_params((19.68, 34.08, 90.0))
    assert p.g_ewald == 0.3 and p.rcut_real == 12.0 and p.kspace_eps == 1e-8
    # Sec. IV A: PCG-DC with g = 0.083 1/A at r_cut = 8 A
    assert p.precond == cpm.CPM_PRECOND_DC and p.g_dc == 0.083 and p.rcut_dc == 8.0
    assert p.slab == 1 and p.p_gap == 1


@pytest.mark.parametrize("field,value", [("g_ewald", 0.0), ("rcut_real", -1.0),
                                         ("kspace_eps", 2.0), ("precision", 9),
                                         ("precond", 7)])
def test_create_rejects_bad_parameters(field, value):
    lib = cpm.load()
    p = cpm.default_params((10.0, 10.0, 30.0))
    setattr(p, field, value)
    h = ctypes.c_void_p()
    assert lib.cpm_create(ctypes.byref(h), ctypes.byref(p)) == cpm.CPM_EINVAL
    assert not h.value


def test_create_rejects_missing_box():
    lib = cpm.load()
    p = cpm.default_params((0.0, 10.0, 30.0))
    h = ctypes.c_void_p()
    assert lib.cpm_create(ctypes.byref(h), ctypes.byref(p)) == cpm.CPM_EINVAL


def _null_args(fn):
    """NULL for every pointer argument, zero for every number (per the binding's argtypes)."""
    out = []
    for t in fn.argtypes:
        if t in (ctypes.c_int, ctypes.c_int64, ctypes.c_uint64):
            out.append(0)
        elif t in (ctypes.c_double, ctypes.c_float):
            out.append(0.0)
        else:
            out.append(None)
    return out


def test_every_call_rejects_a_null_handle():
    # a NULL context, batch or output handle is a bad argument (CPM_EINVAL): each call
    # checks it before any CUDA work, so this runs without a GPU
    lib = cpm.load()
    skip = {"cpm_default_params", "cpm_last_error", "cpm_batch_last_error"}
    for name in cpm.EXPORTS:
        if name in skip:
            continue
        fn = getattr(lib, name)
        assert fn(*_null_args(fn)) == cpm.CPM_EINVAL, name
    assert lib.cpm_last_error(None) == b"null context"
    assert lib.cpm_batch_last_error(None) == b"null batch"
