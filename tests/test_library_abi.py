"""CPU checks of the C ABI: the library builds and loads, exports every entry
point include/sr.h declares, and its host-only calls behave (no GPU needed).

The phase generator is checked bit for bit against the independent Python
Philox4x32-10 of ``synthetic`` (two implementations of the published
generator; neither is derived from the other).
"""
import ctypes as C
import os
import re

import numpy as np
import pytest
import torch

import synthetic as S
from paper_2409_05734_gb300 import _lib
from paper_2409_05734_gb300.buildlib import build as build_library

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build_library()
    return _lib.load()


def _declared_functions():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(sr_[a-z0-9_]+)\s*\(", text))
    return names


def test_every_declared_symbol_is_exported(lib):
    names = _declared_functions()
    assert {"sr_plan_create", "sr_forward", "sr_adjoint", "sr_loss_grad", "sr_spectral_init",
            "sr_gd_solve"} <= names
    for name in names:
        assert hasattr(lib, name), name
    declared_in_binding = {s[0] for s in _lib.SIGNATURES}
    assert names <= declared_in_binding


@pytest.mark.parametrize("seed,L,m", [(0, 1, 16), (20240905, 2, 256), (2**40 + 7, 3, 1000), (123, 2, 65536)])
def test_host_phases_match_independent_generator(lib, seed, L, m):
    out = np.empty(L * m, dtype=np.float64)
    _lib.check(lib.sr_phases(seed, L, m, out.ctypes.data_as(C.POINTER(C.c_double))), "sr_phases")
    ref = S.phases(seed, L, m).reshape(-1)
    assert np.array_equal(out, ref)


def test_host_argument_errors(lib):
    assert lib.sr_phases(1, 0, 16, None) == 1
    out = np.empty(4)
    assert lib.sr_phases(1, 0, 4, out.ctypes.data_as(C.POINTER(C.c_double))) == 1
    assert "L >= 1" in lib.sr_last_error().decode()
    h = C.c_void_p()
    # sizes are validated before any CUDA call
    assert lib.sr_plan_create(10, 20, 2, 0, C.byref(h)) == 2   # m neither 2^a nor 3 * 2^a
    assert lib.sr_plan_create(5, 6, 2, 0, C.byref(h)) == 2     # m = 3 * 2 (radix-3 needs 3 * 2^a, 2^a >= 4)
    assert lib.sr_plan_create(3, 9, 2, 0, C.byref(h)) == 2     # 3^2 is not supported
    assert lib.sr_plan_create(20, 16, 2, 0, C.byref(h)) == 2   # n > m
    assert lib.sr_plan_create(4, 16, 0, 0, C.byref(h)) == 2    # L < 1
    assert lib.sr_plan_create(4, 16, 9, 0, C.byref(h)) == 2    # L > 8
    assert lib.sr_plan_create(1, 2, 1, 0, C.byref(h)) == 2     # m < 4
    assert lib.sr_plan_create(4, 16, 2, 0, None) == 1
    assert lib.sr_forward(None, None, None, 1, None) == 1
    assert lib.sr_plan_destroy(None) == 0
    assert lib.sr_status_string(0).decode() == "ok"
    assert lib.sr_status_string(2).decode() == "unsupported size"


@pytest.mark.skipif(torch.cuda.is_available(), reason="checks the no-GPU error path")
def test_plan_create_without_gpu_reports_cuda_error(lib):
    h = C.c_void_p()
    assert lib.sr_plan_create(64, 256, 2, 0, C.byref(h)) == 4
    assert not h.value
