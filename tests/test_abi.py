"""The C-ABI library builds, loads and exports every entry point its header declares.

CPU only: these calls either touch no CUDA state or fail argument validation first.
"""
import ctypes
import os
import re

import pytest

import paper_1710_08591_gb300 as fb

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(fftbf_[a-z0-9_]+)\s*\(", txt))
    return sorted(names)


@pytest.fixture(scope="module")
def L():
    fb.build()
    return fb.lib()


def test_every_declared_symbol_is_exported(L):
    names = _declared()
    assert "fftbf_execute" in names and "fftbf_tied_beams" in names
    for n in names:
        assert hasattr(L, n), n


def test_header_names_match_binding():
    for n in _declared():
        short = n[len("fftbf_"):]
        assert hasattr(fb, short), f"binding lacks {short}"


def test_plan_create_rejects_bad_sizes(L):
    assert not L.fftbf_plan_create(0, 16, 2, 32, 1, 8, 16, None)
    assert "must all be >= 1" in fb.last_error()
    assert not L.fftbf_plan_create(4, 256, 65, 512, 2, 8, 16, None)
    assert "limits" in fb.last_error()


def test_null_plan_and_bad_T(L):
    assert L.fftbf_execute(None, None, 0, None, None) == -1
    assert L.fftbf_tied_beams(None, None, 0, 1, None, None, None, None) == -1
    assert L.fftbf_plan_sync(None) == -1
    L.fftbf_destroy(None)
    assert L.fftbf_debug_unpack(None, -1, None, None) == -1


def test_python_errors_carry_status():
    with pytest.raises(fb.FftbfError) as e:
        fb.plan_create(4, 256, 4, 512, 0, 8, 16)
    assert e.value.code == -1
