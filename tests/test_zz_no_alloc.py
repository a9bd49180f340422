"""The allocation-free statement digest (sisu_statement_digest_noalloc).

Some callers cannot let a library allocate device memory: a serving loop
or framework that owns every byte through its own pool, or code running
while that pool is locked.  The entry point keeps its scratch in a fixed
array inside the library.  This file runs last (pytest collects it last),
so a failure here comes after every other test has run; it also passes
alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

from gpu_util import from_device, to_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    import paper_2404_10404_b300 as S
    return S


@pytest.mark.parametrize("n", [0, 1, 31, 1024, 1025, 3 * 1024 + 5, 1 << 20, 64 << 20])
def test_matches_allocating_digest_twice(S, n):
    import torch
    data = torch.randint(0, 256, (max(16, n),), dtype=torch.uint8, device="cuda", generator=None)
    want = S.statement_digest(data, n)
    out = to_device(bytes(32))
    stream = torch.cuda.current_stream()
    for _ in range(2):  # the shared scratch keeps the previous call's contents
        out.zero_()
        S.statement_digest_noalloc(data, n, out, stream)
        torch.cuda.synchronize()
        assert from_device(out, 32) == want


@pytest.mark.parametrize("n", [0, 5, 1024, 4 * 1024 + 17, 40000])
def test_matches_oracle_digest(S, n, oracle):
    import torch
    rng = np.random.default_rng(n + 11)
    raw = rng.integers(0, 256, size=n, dtype=np.uint8).tobytes()
    data = to_device(raw)
    out = to_device(bytes(32))
    S.statement_digest_noalloc(data, n, out, torch.cuda.current_stream())
    torch.cuda.synchronize()
    assert from_device(out, 32) == oracle.statement_digest(raw)


def test_free_device_memory_unchanged(S):
    import torch
    data = torch.randint(0, 256, (1 << 22,), dtype=torch.uint8, device="cuda")
    out = to_device(bytes(32))
    stream = torch.cuda.current_stream()
    S.statement_digest_noalloc(data, 1 << 22, out, stream)  # kernels loaded, scratch address looked up
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        S.statement_digest_noalloc(data, 1 << 22, out, stream)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_rejects_inputs_beyond_the_limit(S):
    import torch
    data = torch.zeros(16, dtype=torch.uint8, device="cuda")
    out = to_device(bytes(32))
    with pytest.raises(S.SisuError) as e:
        S.statement_digest_noalloc(data, (64 << 20) + 1, out)
    assert e.value.code == -9
    assert "64 MiB" in str(e.value)


def test_refuses_host_buffers_without_launching(S):
    import torch
    dev_data = to_device(bytes(range(64)))
    dev_out = to_device(bytes(32))
    host = np.zeros(64, dtype=np.uint8)
    before = S.kernel_launches()
    # the binding refuses host arrays before calling the library
    with pytest.raises(S.SisuError):
        S.statement_digest_noalloc(host, 64, dev_out)
    with pytest.raises(S.SisuError):
        S.statement_digest_noalloc(dev_data, 64, host)
    # raw host addresses reach the C entry point, which refuses them
    pinned = torch.zeros(64, dtype=torch.uint8).pin_memory()
    lib = S._lib
    for data, out in ((host.ctypes.data, dev_out.data_ptr()), (dev_data.data_ptr(), host.ctypes.data),
                      (pinned.data_ptr(), dev_out.data_ptr()), (dev_data.data_ptr(), pinned.data_ptr())):
        rc = lib.sisu_statement_digest_noalloc(ctypes.c_void_p(data), 64, ctypes.c_void_p(out), None)
        assert rc == -1
        assert b"device memory" in lib.sisu_last_error()
    assert S.kernel_launches() == before
