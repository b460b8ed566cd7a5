"""CPU checks of the C ABI: the library loads, exports every function that
include/*.h declares, and reports errors without a device (no compute call
is made here)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(px_\w+)\s*\(", text, re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2307_07931_b300 import build as b
    path = b.build()
    return ctypes.CDLL(path)


def test_header_declares_core_calls():
    names = declared_functions()
    for core in ("px_create", "px_destroy", "px_relax_n", "px_apply_stencil",
                 "px_residual_norm"):
        assert core in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings(lib):
    lib.px_status_string.restype = ctypes.c_char_p
    lib.px_status_string.argtypes = [ctypes.c_int]
    assert lib.px_status_string(0) == b"PX_OK"
    assert lib.px_status_string(1) == b"PX_EINVAL"
    assert lib.px_status_string(7) == b"PX_ENAN"
    assert lib.px_status_string(99) == b"PX_UNKNOWN"


def test_null_context_is_rejected(lib):
    lib.px_relax_n.restype = ctypes.c_int
    assert lib.px_relax_n(None, None, None, None, None, ctypes.c_double(0.5), 1, 0, None, 0,
                          None) == 1
    lib.px_destroy.restype = ctypes.c_int
    assert lib.px_destroy(None) == 0


def test_create_without_device_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    h = ctypes.c_void_p()
    lib.px_create.restype = ctypes.c_int
    s = lib.px_create(ctypes.byref(h), 0)
    assert s in (1, 2)  # PX_EINVAL (no device 0) or PX_ECUDA
    assert not h.value
    lib.px_last_error.restype = ctypes.c_char_p
    assert len(lib.px_last_error(None)) > 0


def test_binding_marshals_layout():
    import torch
    import paper_2307_07931_b300 as px
    t = torch.zeros(7, 12, dtype=torch.float32)
    g = px.grid_of(t, 0.25)
    assert (g.nx, g.ny, g.ld, g.ghost, g.dtype, g.h) == (12, 7, 12, 0, px.PX_F32, 0.25)
    t2 = torch.zeros(10, 20, dtype=torch.float64)[1:8, 2:14]
    g2 = px.grid_of(t2, 0.5)
    assert (g2.nx, g2.ny, g2.ld, g2.dtype) == (12, 7, 20, px.PX_F64)
    g3 = px.grid_of(torch.zeros(66, 66, dtype=torch.float64), 1 / 64, ghost=1)
    assert (g3.nx, g3.ny, g3.ld, g3.ghost) == (64, 64, 66, 1)
    with pytest.raises(TypeError):
        px.grid_of(torch.zeros(4, 4, dtype=torch.int32), 1.0)
    with pytest.raises(ValueError):
        px.grid_of(torch.zeros(4, 4, dtype=torch.float32).t(), 1.0)


def header_enum_values():
    """name -> value of every PX_* enumerator with an explicit value in include/*.h."""
    vals = {}
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        for body in re.findall(r"\benum\b[^{]*\{([^}]*)\}", text):
            for m in re.finditer(r"\b(PX_\w+)\s*=\s*(-?\d+)", body):
                vals[m.group(1)] = int(m.group(2))
    return vals


def test_binding_constants_match_header():
    """The binding's PX_* integers (statuses, dtypes, options, solve modes) are
    the header's enumerators, value for value."""
    import paper_2307_07931_b300 as px
    vals = header_enum_values()
    for must in ("PX_OK", "PX_F64", "PX_F32", "PX_OPT_FP32_FAMILY", "PX_OPT_RB_FP64_PASSES",
                 "PX_SOLVE_REFINE"):
        assert must in vals, must
    bound = {n: v for n, v in vals.items() if hasattr(px, n)}
    assert {n: getattr(px, n) for n in bound} == bound
    opts = [n for n in vals if n.startswith("PX_OPT_")]
    assert all(hasattr(px, n) for n in opts), [n for n in opts if not hasattr(px, n)]
