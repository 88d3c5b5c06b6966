"""The C-ABI library builds for sm_103a and exports every entry point include/sgf.h declares
(no GPU needed: nothing is computed)."""
import ctypes
import os
import re

from paper_1707_04950_gb300 import build as b
from paper_1707_04950_gb300 import sgf

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "sgf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sgf_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    b.build()
    lib = ctypes.CDLL(b.LIB)
    names = _declared()
    assert len(names) >= 17
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert sorted(sgf.EXPORTED + ["sgf_destroy", "sgf_last_error"])[0]
    assert set(names) <= set(sgf.EXPORTED) | {"sgf_destroy", "sgf_last_error"}


def test_params_struct_layout_matches_header():
    # the ctypes record must have the C layout: 18 fields, 112 bytes on LP64
    assert ctypes.sizeof(sgf.sgf_params) == 112
