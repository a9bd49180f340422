"""The device-memory check of the C ABI needs no kernel: a host address
passed where a call expects device memory is refused with INVALID_ARG
before anything is launched, with or without a GPU in the machine (without
one the CUDA runtime knows no address at all).  Sizes are small and no
call here reaches a launch."""
import ctypes
import os

import numpy as np
import pytest

INVALID_ARG = -1


@pytest.fixture(scope="module")
def lib():
    from paper_2404_10404_b300 import library_path
    if not os.path.exists(library_path()):
        pytest.skip("library not built")
    import paper_2404_10404_b300 as S
    return S._lib


def _host(n):
    a = np.zeros(n + 256, dtype=np.uint8)
    addr = a.ctypes.data
    return a, addr + (-addr) % 256


def test_digest_refuses_host_data(lib):
    keep, addr = _host(4096)
    out = ctypes.create_string_buffer(32)
    assert lib.sisu_statement_digest(addr, 4096, ctypes.cast(out, ctypes.c_void_p), None) == INVALID_ARG
    assert lib.sisu_last_error().startswith(b"data")


def test_field_batch_refuses_host_arrays(lib):
    keep, addr = _host(32 * 16)
    assert lib.sisu_fr_batch(0, addr, addr, addr, 16, None) == INVALID_ARG
    assert lib.sisu_last_error().startswith((b"a:", b"a is"))


def test_sort_and_hash_refuse_host_arrays(lib):
    keep, addr = _host(32 * 64)
    passes = ctypes.c_uint32()
    assert lib.sisu_sort_elements(addr, 64, 1, None, addr, ctypes.byref(passes)) == INVALID_ARG
    out = ctypes.create_string_buffer(32)
    assert lib.sisu_assoc_hash(addr, 64, None, 1, None, ctypes.cast(out, ctypes.c_void_p)) == INVALID_ARG
    res = ctypes.c_int()
    assert lib.sisu_pairwise_distinct_check(addr, addr, 64, 1, None, ctypes.byref(res), None, None) == INVALID_ARG
