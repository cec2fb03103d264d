"""The C-ABI library builds, loads and exports every symbol of include/rips.h
(no GPU needed: no compute call is made)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    src = open(os.path.join(ROOT, "include", "rips.h")).read()
    return sorted(set(re.findall(r"RIPS_API\s+[\w\s\*]+?\b(rips_\w+)\s*\(", src)))


def test_header_declarations_match_binding():
    from paper_1908_02518_gb300 import _lib
    assert _declared_symbols() == sorted(_lib.EXPORTS)


def test_library_exports_every_symbol():
    from paper_1908_02518_gb300 import _lib, build
    path = build.build()
    lib = ctypes.CDLL(path)
    for name in _declared_symbols():
        assert hasattr(lib, name), name
    _lib.load()


def test_status_strings_without_gpu():
    from paper_1908_02518_gb300 import _lib
    lib = _lib.load()
    for code in range(0, -8, -1):
        s = lib.rips_status_string(code)
        assert s and s != b"unknown status"


def test_argument_checks_without_gpu():
    """Invalid arguments are rejected on the host before any device work."""
    import numpy as np
    from paper_1908_02518_gb300 import _lib
    lib = _lib.load()
    out = ctypes.c_void_p()
    d = np.zeros((4, 4), dtype=np.float32)
    fp = d.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
    assert lib.rips_barcodes(fp, 4, 1, ctypes.c_float(1.0), 4, ctypes.byref(out)) == -2   # p = 4
    assert lib.rips_barcodes(fp, 4, 1, ctypes.c_float(1.0), 65537, ctypes.byref(out)) == -2
    assert lib.rips_barcodes(fp, 0, 1, ctypes.c_float(1.0), 2, ctypes.byref(out)) == -1   # n = 0
    assert lib.rips_barcodes(fp, 4, -1, ctypes.c_float(1.0), 2, ctypes.byref(out)) == -1  # dim_max < 0
    assert lib.rips_barcodes(fp, 4, 1, ctypes.c_float(-1.0), 2, ctypes.byref(out)) == -1  # t < 0
    assert lib.rips_barcodes(None, 4, 1, ctypes.c_float(1.0), 2, ctypes.byref(out)) == -1
    # C(n, dim_max + 2) >= 2^63
    assert lib.rips_barcodes(fp, 40000, 7, ctypes.c_float(1.0), 2, ctypes.byref(out)) == -3


def test_no_oracle_import_in_product():
    """The product package never imports the oracle."""
    pkg = os.path.join(ROOT, "paper_1908_02518_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "rips_oracle" not in txt, f


def test_options_reject_unknown_bits():
    from paper_1908_02518_gb300 import _lib
    lib = _lib.load()
    assert lib.rips_set_options(1 << 7) == -1
    assert lib.rips_set_options(3) == 0 and lib.rips_get_options() == 3
    assert lib.rips_set_options(0) == 0 and lib.rips_get_options() == 0
