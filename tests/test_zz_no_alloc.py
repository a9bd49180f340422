"""The allocation-free statement digest (sisu_statement_digest_noalloc).

Some callers cannot let a library allocate device memory: a serving loop
or framework that owns every byte through its own pool, or code running
while that pool is locked.  The entry point keeps its scratch in a fixed
array inside the library.  This file runs last (pytest collects it last),
so a failure here comes after every other test has run; it also passes
alone in a fresh process.
"""
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


def test_rejects_inputs_beyond_the_limit(S):
    import torch
    data = torch.zeros(16, dtype=torch.uint8, device="cuda")
    out = to_device(bytes(32))
    with pytest.raises(S.SisuError) as e:
        S.statement_digest_noalloc(data, (64 << 20) + 1, out)
    assert e.value.code == -9
    assert "64 MiB" in str(e.value)
