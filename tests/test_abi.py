"""The C ABI library builds for sm_103a, loads, and exports every entry point
declared in include/*.h; the binding covers the same names.  No GPU calls."""
import ctypes
import glob
import os
import re
import shutil

import pytest
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(ash_[a-z0-9_]+)\s*\(", text))
    return names


@pytest.fixture(scope="module")
def libpath():
    from paper_2110_00511_gb300 import build
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    return build.build()


def test_header_declares_entry_points():
    names = declared_symbols()
    for must in ("ash_create", "ash_destroy", "ash_insert", "ash_activate", "ash_find", "ash_erase",
                 "ash_get_active_indices", "ash_rehash", "ash_reserve", "ash_size", "ash_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in sorted(declared_symbols()) if not hasattr(lib, n)]
    assert not missing, f"not exported: {missing}"


def test_binding_covers_header(libpath):
    from paper_2110_00511_gb300 import ash
    assert set(ash.exported_symbols()) == declared_symbols()
    ash.lib()  # loads and sets every signature


def test_last_error_without_gpu(libpath):
    lib = ctypes.CDLL(libpath)
    lib.ash_last_error.restype = ctypes.c_char_p
    assert isinstance(lib.ash_last_error(), bytes)


@pytest.mark.skipif(torch.cuda.is_available(), reason="checks the no-GPU failure path")
def test_no_cpu_fallback():
    from paper_2110_00511_gb300 import ash
    with pytest.raises(RuntimeError):
        ash.HashMap(3, 16)
