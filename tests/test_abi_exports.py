"""The C-ABI library loads and exports every entry point declared in include/*.h
(no compute call: this runs without a GPU)."""
import ctypes
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(precode_[a-z0-9_]+)\s*\(",
                             src, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    from paper_2304_12745_gb300 import build
    lib_path = build.build()
    lib = ctypes.CDLL(lib_path)
    names = declared_functions()
    assert "precode_solve" in names and "precode_plan" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings_without_gpu():
    from paper_2304_12745_gb300 import capi
    capi.LIB.precode_status_str.restype = ctypes.c_char_p
    assert capi.LIB.precode_status_str(0) == b"ok"
    assert capi.LIB.precode_status_str(1) == b"invalid argument"


def test_instance_descriptor_packing_matches_abi_layout():
    import numpy as np
    from paper_2304_12745_gb300.precoder import inst_table
    t = inst_table([0, 4096], [2, 4098], [0, 8], [64, 256], [8, 32]).numpy()
    assert t.shape == (2, 4) and t.dtype == np.int64
    raw = t.view(np.int32).reshape(2, 8)
    assert list(t[1, :3]) == [4096, 4098, 8]
    assert list(raw[0, 6:]) == [64, 8] and list(raw[1, 6:]) == [256, 32]
