"""CPU checks of the C ABI: the library loads, exports every symbol the header
declares, and the binding's structs match the header's layout."""
import ctypes
import os
import re

import pytest

from paper_2410_14088_gb300 import qsim

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    txt = open(os.path.join(ROOT, "include", "qsim.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(qsim_[a-z0-9_]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol():
    L = qsim.lib()
    names = header_functions()
    assert len(names) >= 20
    for name in names:
        assert hasattr(L, name), name
    assert set(names) == set(qsim.SIGNATURES), set(names) ^ set(qsim.SIGNATURES)


def test_struct_sizes_match_header():
    # sizes from the C layout (x86-64 / aarch64 LP64 agree)
    assert ctypes.sizeof(qsim.Gate) == 48
    assert ctypes.sizeof(qsim.Config) == 4 * 12 + 8 * 4 + 8 * 6
    assert ctypes.sizeof(qsim.Stats) == 8 * 16
    assert ctypes.sizeof(qsim.OpInfo) == 4 * 14 + 8 + 8 + 8
    assert ctypes.sizeof(qsim.TrainConfig) == 24


def test_defaults_and_worst_case():
    c = qsim.default_config()
    assert (c.m, c.inner, c.k, c.streams, c.eps) == (20, 2, 4, 2, 1e-3)
    # 32 + pad16(4 * 2) + 1 * (pad16(2 * 32) + 8 * 1024) for m = 10
    assert qsim.worst_case_bytes(10) == 32 + 16 + 64 + 8192
    assert qsim.worst_case_bytes(4) == 0 and qsim.worst_case_bytes(27) == 0
