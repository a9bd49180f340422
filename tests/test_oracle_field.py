"""Pins of the oracle's BN254 scalar-field arithmetic (Sec. 4.1 picks BN254).

The oracle reduces with Barrett's method on 64-bit words; these tests check
it against Python's arbitrary-precision integers (an independent library
routine), against identities that hold in any prime field, and at the edge
values of the canonical range.
"""
import random

import pytest

from oracle.binding import ERR_CANON, ints_to_bytes, bytes_to_ints

P = 0x30644E72E131A029B85045B68181585D2833E84879B9709143E1F593F0000001
EDGE = [0, 1, 2, P - 1, P - 2, (P - 1) // 2, (P + 1) // 2, 1 << 253, (1 << 128) - 1, 1 << 64]


def _rand(rng, n):
    return [rng.randrange(P) for _ in range(n)]


@pytest.mark.parametrize("op,fn", [
    (0, lambda a, b: (a + b) % P),
    (1, lambda a, b: (a - b) % P),
    (2, lambda a, b: (a * b) % P),
    (4, lambda a, b: (a * b + (1 - a) * (1 - b)) % P),
])
def test_binary_ops_match_python_ints(oracle, op, fn):
    rng = random.Random(1000 + op)
    a = _rand(rng, 3000) + [x for x in EDGE for _ in EDGE]
    b = _rand(rng, 3000) + [y for _ in EDGE for y in EDGE]
    got = bytes_to_ints(oracle.fr_op(op, ints_to_bytes(a), ints_to_bytes(b)))
    assert got == [fn(x, y) for x, y in zip(a, b)]


def test_inverse(oracle):
    rng = random.Random(7)
    a = _rand(rng, 200) + [1, 2, P - 1, (P + 1) // 2]
    inv = bytes_to_ints(oracle.fr_op(3, ints_to_bytes(a)))
    assert inv == [pow(x, -1, P) for x in a]
    assert all(x * y % P == 1 for x, y in zip(a, inv))
    assert bytes_to_ints(oracle.fr_op(3, ints_to_bytes([0]))) == [0]


def test_identities(oracle):
    # (p-1)^2 = 1, 2 * (p+1)/2 = 1, and Fermat a^(p-1) = 1 via repeated squaring
    sq = bytes_to_ints(oracle.fr_op(2, ints_to_bytes([P - 1]), ints_to_bytes([P - 1])))
    assert sq == [1]
    half = bytes_to_ints(oracle.fr_op(2, ints_to_bytes([2]), ints_to_bytes([(P + 1) // 2])))
    assert half == [1]
    # p - 1 = 2^28 * odd: squaring a 2^28-th root of unity 28 times gives 1
    odd = (P - 1) >> 28
    assert odd % 2 == 1
    w = pow(5, odd, P)
    x = [w]
    for _ in range(28):
        x = bytes_to_ints(oracle.fr_op(2, ints_to_bytes(x), ints_to_bytes(x)))
    assert x == [1]


def test_barrett_reduction_full_range(oracle):
    rng = random.Random(11)
    vals = [rng.getrandbits(512) for _ in range(3000)]
    vals += [0, 1, P, P * P - 1, P * P, (1 << 512) - 1, (1 << 511), P * (1 << 258), (P - 1) * (P - 1)]
    vals += [k * P + e for k in (1, 2, 3, (1 << 258) - 1) for e in (0, 1, P - 1)]
    for v in vals:
        assert oracle.reduce512(v) == v % P, hex(v)


def test_non_canonical_rejected(oracle):
    for bad in (P, P + 1, (1 << 256) - 1, 1 << 254):
        with pytest.raises(ValueError) as e:
            oracle.fr_op(0, ints_to_bytes([bad]), ints_to_bytes([1]))
        assert str(ERR_CANON) in str(e.value)
