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
