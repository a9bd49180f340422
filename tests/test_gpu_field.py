"""GPU field core (Sec. 4.1, BN254 scalar field) and device digests, through
the C ABI, against Python integers and the CPU oracle."""
import random

import pytest

from gpu_util import bytes_of, from_device, ints_of, to_device

pytestmark = pytest.mark.gpu

P = 0x30644E72E131A029B85045B68181585D2833E84879B9709143E1F593F0000001
EDGE = [0, 1, 2, 3, P - 1, P - 2, (P - 1) // 2, (P + 1) // 2, 1 << 253, (1 << 254) - P + 7,
        (1 << 128) - 1, 1 << 64, (1 << 32) - 1, 0xF0000001]


@pytest.fixture(scope="module")
def S():
    import paper_2404_10404_b300 as S
    return S


def _run(S, op, a, b):
    n = len(a)
    da, db, do = to_device(bytes_of(a)), to_device(bytes_of(b)), to_device(bytes(32 * n))
    S.fr_batch(op, da, db, do, n)
    return ints_of(from_device(do, 32 * n))


@pytest.mark.parametrize("op,fn", [
    (0, lambda a, b: (a + b) % P), (1, lambda a, b: (a - b) % P), (2, lambda a, b: a * b % P),
    (4, lambda a, b: (a * b + (1 - a) * (1 - b)) % P)])
def test_ops_vs_python_ints(S, op, fn):
    rng = random.Random(op)
    a = [rng.randrange(P) for _ in range(20000)] + [x for x in EDGE for _ in EDGE]
    b = [rng.randrange(P) for _ in range(20000)] + [y for _ in EDGE for y in EDGE]
    assert _run(S, op, a, b) == [fn(x, y) for x, y in zip(a, b)]


@pytest.mark.parametrize("op", [7, 8])
def test_square_vs_python_ints(S, op):
    """The squaring routine (op 7) and the same on the other representative
    of each Montgomery form in [r, 2r) (op 8) against a^2 mod r."""
    rng = random.Random(70 + op)
    a = [rng.randrange(P) for _ in range(50000)] + EDGE + [P - k for k in range(1, 200)] + list(range(200))
    a += [(1 << k) % P for k in range(256)] + [((1 << k) - 1) % P for k in range(1, 256)]
    assert _run(S, op, a, a) == [x * x % P for x in a]


def test_million_products_vs_oracle(S, oracle):
    import numpy as np
    rng = np.random.default_rng(12)
    n = 1 << 20
    raw = rng.integers(0, 1 << 63, size=(2, n, 4), dtype=np.uint64)
    raw[..., 3] &= np.uint64((1 << 61) - 1)  # below 2^253 < r
    a, b = raw[0].tobytes(), raw[1].tobytes()
    da, db, do = to_device(a), to_device(b), to_device(bytes(32 * n))
    S.fr_batch(2, da, db, do, n)
    got = from_device(do, 32 * n)
    assert got == oracle.fr_op(2, a, b)


def test_batched_inverse(S):
    rng = random.Random(5)
    a = [rng.randrange(1, P) for _ in range(1001)] + [1, P - 1, 2]
    got = _run(S, 3, a, a)
    assert got == [pow(x, -1, P) for x in a]


def test_inverse_of_zero_reported(S):
    a = [5, 0, 7, 11, 0, 13, 17, 19, 23]
    da, do = to_device(bytes_of(a)), to_device(bytes(32 * len(a)))
    with pytest.raises(S.SisuError) as e:
        S.fr_batch(3, da, da, do, len(a))
    assert e.value.code == -8
    got = ints_of(from_device(do, 32 * len(a)))
    assert got == [pow(x, -1, P) if x else 0 for x in a]


def test_non_canonical_rejected(S):
    for bad in (P, P + 5, (1 << 256) - 1):
        da, do = to_device(bytes_of([bad, 1])), to_device(bytes(64))
        with pytest.raises(S.SisuError) as e:
            S.fr_batch(2, da, da, do, 2)
        assert e.value.code == -3


@pytest.mark.parametrize("n", [0, 1, 31, 1023, 1024, 1025, 4096, 3 * 1024 + 5, 100000])
def test_device_digest_vs_oracle(S, oracle, n):
    rng = random.Random(n)
    data = bytes(rng.getrandbits(8) for _ in range(n))
    assert S.statement_digest(to_device(data), n) == oracle.statement_digest(data)


def test_microbench_runs(S):
    for kind in (0, 1, 2, 3, 4, 5, 7, 8, 9, 11):
        ms, ops = S.microbench(kind, 148, 256, 64)
        assert ms > 0 and ops > 0


def test_product_formulations_agree(S):
    """The carry-chain and the 64-bit-partial-product Montgomery products
    give identical limbs on chained inputs (every thread of every block)."""
    ms, bad = S.microbench(6, 148 * 4, 256, 256)
    assert bad == 0


def test_karatsuba_forms_agree(S):
    """The lazy 512-bit product by Karatsuba (the kernels' form) equals the
    schoolbook product on arbitrary 256-bit operands, all-ones words
    included; the Karatsuba-based Montgomery product equals the CIOS one."""
    ms, bad = S.microbench(10, 148 * 4, 256, 256)
    assert bad == 0
    ms, bad = S.microbench(12, 148 * 4, 256, 256)
    assert bad == 0


def test_lazy_dot_products_vs_python_ints(S):
    """op 5: prefix sums of products within aligned runs of 64, through the
    544-bit accumulator and one reduction per sum."""
    rng = random.Random(55)
    n = 64 * 40 + 17  # ragged last run
    a = [rng.randrange(P) for _ in range(n)]
    b = [rng.randrange(P) for _ in range(n)]
    a[:len(EDGE)] = EDGE
    b[64:64 + len(EDGE)] = EDGE
    a[128:192] = [P - 1] * 64  # the largest canonical operands in a full run
    b[128:192] = [P - 1] * 64
    want, run = [], 0
    for i in range(n):
        run = (0 if i % 64 == 0 else run) + a[i] * b[i]
        want.append(run % P)
    assert _run(S, 5, a, b) == want


@pytest.mark.parametrize("fixed", [1, 2, P - 1, (1 << 253) + 12345, 0xF0000001, None])
def test_fixed_multiplier_products_vs_python_ints(S, fixed):
    """op 6: a[i] * b[0] through the fixed-multiplier product (the fold's)."""
    rng = random.Random(66 if fixed is None else fixed % 1000)
    b0 = rng.randrange(P) if fixed is None else fixed
    a = [rng.randrange(P) for _ in range(3000)] + EDGE
    b = [b0] + [0] * (len(a) - 1)
    assert _run(S, 6, a, b) == [x * b0 % P for x in a]
