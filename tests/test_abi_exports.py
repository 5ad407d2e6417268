"""The C-ABI library builds for sm_103a, loads, and exports every entry point
declared in include/mpwos.h (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

from paper_2606_21883_b300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for hdr in os.listdir(os.path.join(ROOT, "include")):
        if hdr.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", hdr)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(mpwos_[a-z0-9_]+)\s*\(", txt))
    return names


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(B.build())
    names = _declared()
    assert len(names) >= 10
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing


def test_library_targets_sm103a():
    assert any("compute_103a,code=sm_103a" in a for a in B.ARCH)


def test_autotune_calls_reject_null_context():
    """Host-side argument checks of the autotuner's entry points (no GPU needed)."""
    lib = ctypes.CDLL(B.build())
    lib.mpwos_set_autotune.argtypes = [ctypes.c_void_p, ctypes.c_int]
    lib.mpwos_autotune_entries.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                           ctypes.POINTER(ctypes.c_int)]
    einval = 1
    assert lib.mpwos_set_autotune(None, 1) == einval
    n = ctypes.c_int(-1)
    assert lib.mpwos_autotune_entries(None, None, 0, ctypes.byref(n)) == einval
