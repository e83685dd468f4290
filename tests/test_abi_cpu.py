"""C ABI checks that need no GPU: the library builds for sm_103a, loads, and
exports every function include/rsv.h declares; the binding's record layouts
match the header."""
import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

from paper_1401_1757_gb300 import _build, rsv

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rsv.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rsv_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib_path():
    return _build.build_library()


def test_library_exports_every_declared_function(lib_path):
    names = declared_functions()
    assert len(names) >= 12
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\b(rsv_[a-z0-9_]+)\b", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    assert set(names) == set(rsv.EXPORTS)


def test_library_loads_without_gpu(lib_path):
    lib = rsv.load_library(lib_path)
    for n in declared_functions():
        assert hasattr(lib, n)
    # pure host queries need no device
    assert lib.rsv_variant_count(2) >= 2
    assert b"comp" in lib.rsv_variant_name(2, 0)
    assert lib.rsv_variant_count(3) >= 4
    assert b"deflated" in lib.rsv_variant_name(3, 0)
    assert lib.rsv_variant_name(3, 99) == b""
    assert lib.rsv_variant_count(7) == 0
    assert lib.rsv_last_error(None) == b"NULL context"


def test_record_layouts_match_header():
    src = open(HEADER).read()
    assert "(48 bytes)" in src
    assert C.sizeof(rsv.rsv_policy) == 48
    assert C.sizeof(rsv.rsv_opts) == 32
    assert C.sizeof(rsv.rsv_out) == 5 * 8
    assert rsv.POLICY_DTYPE.itemsize == 48


def test_null_arguments_are_rejected_without_gpu(lib_path):
    lib = rsv.load_library(lib_path)
    assert lib.rsv_create(None, 0, None) == rsv.RSV_E_ARG
    assert lib.rsv_destroy(None) == rsv.RSV_OK
    assert lib.rsv_load_portfolio(None, None, 0) == rsv.RSV_E_ARG
    assert lib.rsv_compute_reserves(None, None, None) == rsv.RSV_E_ARG


def test_generator_math_selftest_arguments_without_gpu(lib_path):
    """The generator-math test entry point checks its arguments before any CUDA
    call: a negative count or missing buffers are RSV_E_ARG, an empty call is a
    no-op (the device functions themselves are checked in the GPU tests)."""
    lib = rsv.load_library(lib_path)
    buf = np.zeros(8)
    w = np.zeros(2, np.uint32)
    assert lib.rsv_selftest_generator_math(0, None, None, None, -1, None) == rsv.RSV_E_ARG
    assert lib.rsv_selftest_generator_math(0, None, None, buf.ctypes.data, 2, buf.ctypes.data) == rsv.RSV_E_ARG
    assert lib.rsv_selftest_generator_math(0, None, w.ctypes.data, None, 2, buf.ctypes.data) == rsv.RSV_E_ARG
    assert lib.rsv_selftest_generator_math(0, None, w.ctypes.data, buf.ctypes.data, 2, None) == rsv.RSV_E_ARG
    assert lib.rsv_selftest_generator_math(0, None, None, None, 0, None) == rsv.RSV_OK
    with pytest.raises(ValueError):
        rsv.rsv_selftest_generator_math(np.zeros(3, np.uint32), np.zeros(2))


def test_noalloc_refuses_oversized_calls_without_gpu(lib_path):
    """rsv_reserves_noalloc checks its sizes in 64-bit arithmetic before any CUDA
    call: a scenario or step count near 2^31, or a portfolio beyond the scratch,
    is RSV_E_LIMIT (the pointers are never read, so placeholders serve)."""
    lib = rsv.load_library(lib_path)
    fake = C.c_void_p(4096)
    big = 2 ** 31 - 100
    for n_pol, n_scen, n_steps in [(1, big, 1), (1, 1, big), (1, big, big), (10 ** 9, 1000, 1200), (100_000, 1000, 20_000)]:
        st = lib.rsv_reserves_noalloc(0, None, fake, n_pol, fake, 1440, fake, n_scen, n_steps, fake, None)
        assert st == rsv.RSV_E_LIMIT, (n_pol, n_scen, n_steps)
    assert lib.rsv_reserves_noalloc(0, None, fake, 1, fake, 1440, fake, 0, 1, fake, None) == rsv.RSV_E_ARG
