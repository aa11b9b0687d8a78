"""The C-ABI library builds for sm_103a, loads without a GPU and exports every declared symbol."""
import ctypes
import os
import re

import pytest

from paper_2411_14974_gb300 import _binding
from paper_2411_14974_gb300 import build as b

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"\b(cs_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def library():
    path = b.build()
    return ctypes.CDLL(path)


def test_library_exports_every_declared_symbol(library):
    names = declared_functions()
    assert len(names) >= 9
    missing = [n for n in names if not hasattr(library, n)]
    assert not missing, missing
    # the Python binding declares prototypes for exactly these entry points
    assert sorted(_binding.exported_symbols()) == names


def test_no_gpu_calls_on_cpu(library):
    """Host-only entry points work without a device; device calls fail with a status, no crash."""
    s = _binding.CsSettings()
    library.cs_default_settings(ctypes.byref(s))
    assert abs(s.tau - 1 / 255) < 1e-9 and abs(s.alpha_max - 0.99) < 1e-7 and s.dist_power == 1.0
    lib = _binding.lib()
    assert lib.cs_last_error() is not None
    import torch
    if not torch.cuda.is_available():
        h = ctypes.c_void_p()
        code = lib.cs_context_create(0, ctypes.byref(h))
        assert code != 0 and not h.value
        assert len(lib.cs_last_error()) > 0


def test_static_forward_reports_a_failed_runtime_call_on_cpu(library):
    """cs_forward_static with valid arguments but no usable device: the first runtime call fails
    on the host and the entry point returns that failure with a message (no crash, no CS_OK)."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("needs a machine without a usable GPU")
    lib = _binding.lib()
    buf = (ctypes.c_float * 64)()
    p = ctypes.cast(buf, ctypes.c_void_p)
    sc = _binding.CsScene(points=p, delta=p, sigma=p, opacity=p, sh=p, n=1, k=3, sh_degree=0, activation=0,
                          storage=0)
    cam = _binding.CsCamera(width=16, height=16, fx=10.0, fy=10.0, cx=8.0, cy=8.0, z_near=0.2)
    cam.R[0] = cam.R[4] = cam.R[8] = 1.0
    s = _binding.CsSettings()
    lib.cs_default_settings(ctypes.byref(s))
    code = lib.cs_forward_static(ctypes.byref(sc), ctypes.byref(cam), ctypes.byref(s), p, p, None)
    assert code == 2  # CS_ERR_CUDA
    assert len(lib.cs_last_error()) > 0


def test_checked_library_builds_and_exports_every_declared_symbol():
    """The bounds-checked variant (CS_CHECKED=1) links completely and loads without a GPU."""
    path = b.build(checked=True)
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
