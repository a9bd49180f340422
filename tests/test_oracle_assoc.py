"""Pins of the oracle's associative hash (Sec. 3.4.1, Algorithm 1) and
pairwise-distinct check (Sec. 3.4.2, Algorithm 2).

F(e) starts from r = 0 and three times replaces r by (r + e + 2^32 - 1)^3;
the hash of a list is the sum of F over it.  The pins do not re-type that
formula: they use values the composition takes in closed form, the degree
and leading coefficient of F as a polynomial in e (finite differences), the
algebra of a sum (order independence, concatenation), the paper's own
bit-change experiment (Fig. 5), and the plain meaning of "pairwise
distinct" on small lists.
"""
import math
import os
import random
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import brute
from oracle.binding import bytes_to_ints, ints_to_bytes

P = brute.P
BIG = 2**32 - 1


def F_c(oracle, vals):
    return bytes_to_ints(oracle.assoc_F(ints_to_bytes(vals)))


@pytest.mark.parametrize("a,expected", [(0, 0), (1, 729), (P - 1, P - 729), (2, 1006012008)])
def test_closed_forms(oracle, a, expected):
    # e = a - (2^32 - 1): the first base is a, then a^3 + a, then (a^3 + a)^3 + a:
    # a = 1 gives 1, 8, 9^3; a = -1 gives -1, -8, -9^3; a = 2 gives 8, 10^3, 1002^3
    e = (a - BIG) % P
    assert F_c(oracle, [e]) == [expected]
    assert brute.assoc_F(e) == expected


@pytest.mark.parametrize("e0", [0, 1, 12345, P - 20])
def test_degree_27_monic(oracle, e0):
    # F is a monic polynomial of degree 3^3 = 27 in e: its 27th forward
    # difference with step 1 is 27!, the 28th is 0
    vals = F_c(oracle, [(e0 + k) % P for k in range(29)])
    def diff(v, order):
        return sum((-1) ** (order - k) * math.comb(order, k) * v[k] for k in range(order + 1)) % P
    assert diff(vals, 27) == math.factorial(27) % P
    assert diff(vals, 28) == 0


def test_c_and_python_agree(oracle):
    rng = random.Random(11)
    vals = [rng.randrange(P) for _ in range(200)] + [0, 1, P - 1, P - BIG, BIG]
    assert F_c(oracle, vals) == [brute.assoc_F(v) for v in vals]


def test_hash_is_a_sum(oracle):
    rng = random.Random(12)
    A = [rng.randrange(P) for _ in range(97)]
    h = int.from_bytes(oracle.assoc_hash(ints_to_bytes(A)), "little")
    assert h == sum(F_c(oracle, A)) % P
    assert h == brute.assoc_hash(A)
    # order independence (the defining property of Sec. 3.4.1)
    B = A[:]
    rng.shuffle(B)
    assert oracle.assoc_hash(ints_to_bytes(B)) == oracle.assoc_hash(ints_to_bytes(A))
    # continuation: H_cur = AH(later list) continued from H_pre = AH(earlier list)
    pre = oracle.assoc_hash(ints_to_bytes(A[:40]))
    assert oracle.assoc_hash(ints_to_bytes(A[40:]), pre) == oracle.assoc_hash(ints_to_bytes(A))
    # empty list: the continuation value itself, 0 without one
    assert oracle.assoc_hash(b"", pre) == pre
    assert oracle.assoc_hash(b"") == bytes(32)


def test_noncanonical_rejected(oracle):
    with pytest.raises(ValueError):
        oracle.assoc_hash(ints_to_bytes([5, P]))
    with pytest.raises(ValueError):
        oracle.assoc_F(ints_to_bytes([P + 3]))
    with pytest.raises(ValueError):
        oracle.pairwise_distinct_check(ints_to_bytes([1, 2]), ints_to_bytes([1, P]))


def test_bit_change_rate(oracle):
    """Sec. 3.4.1, Fig. 5: over x = 1 .. 10^6, each little-endian output bit
    of F changes between F(x) and F(x+1) with probability within 0.5 +- 0.1;
    the figure drops at the top, where values below p are not uniform in
    their highest bits.  Reading: "bit change" is the XOR of the two outputs.
    p lies in [1.5 * 2^253, 1.53 * 2^253), so bits 252 and 253 of a uniform
    value below p are each set with probability q = 1 - 2^253/p (about 0.34)
    and change with probability 2q(1-q) (about 0.45); bits 254 and 255 never
    change.  The bits of the difference F(x+1) - F(x) mod p follow the same
    band below bit 252; bits 252 and 253 are set at the rate q itself: the
    drop."""
    n = 10**6
    xs = list(range(1, n + 2))
    f = np.frombuffer(oracle.assoc_F(ints_to_bytes(xs)), dtype=np.uint8).reshape(n + 1, 32)
    bits = np.unpackbits(f, axis=1, bitorder="little")  # bit k of the LE integer in column k
    change = (bits[1:] ^ bits[:-1]).mean(axis=0)
    assert np.all((change[:254] > 0.4) & (change[:254] < 0.6)), change[:254].min()
    assert change[254] == 0 and change[255] == 0
    q = 1 - 2**253 / P
    assert np.all(np.abs(change[252:254] - 2 * q * (1 - q)) < 0.01)
    d = np.frombuffer(oracle.fr_op(1, f[1:].tobytes(), f[:-1].tobytes()), dtype=np.uint8).reshape(n, 32)
    dbits = np.unpackbits(d, axis=1, bitorder="little").mean(axis=0)
    assert np.all((dbits[:252] > 0.4) & (dbits[:252] < 0.6))
    assert np.all(np.abs(dbits[252:254] - q) < 0.01) and np.all(dbits[252:254] < 0.4)
    assert dbits[254] == 0 and dbits[255] == 0


def _check(oracle, A, S):
    return oracle.pairwise_distinct_check(ints_to_bytes(A), ints_to_bytes(S))


def test_pairwise_distinct_definition(oracle):
    """With A* the sorted list, Algorithm 2 answers whether A's elements are
    pairwise distinct: compared with the plain set-size definition."""
    rng = random.Random(13)
    for trial in range(60):
        n = rng.randrange(0, 12)
        pool = rng.randrange(1, 30)
        A = [rng.randrange(pool) if trial % 2 else rng.randrange(P) for _ in range(n)]
        S = sorted(A)
        want = int(len(set(A)) == len(A))
        assert _check(oracle, A, S) == want
        assert brute.pairwise_distinct_check(A, S) == want


def test_pairwise_distinct_rejects(oracle):
    rng = random.Random(14)
    A = rng.sample(range(10**6), 50)
    S = sorted(A)
    assert _check(oracle, A, S) == 1
    # the claimed sort is not ascending (a permutation, same hash)
    T = S[:]
    T[3], T[4] = T[4], T[3]
    assert _check(oracle, A, T) == 0
    # the claimed sort is ascending but not a permutation of A
    U = S[:]
    U[10] += 1 if U[10] + 1 < U[11] else 0
    U[-1] += 1
    assert _check(oracle, A, U) == 0
    # a duplicate: its sorted list is not strictly ascending
    D = A[:-1] + [A[0]]
    assert _check(oracle, D, sorted(D)) == 0
    # empty and single lists are pairwise distinct
    assert _check(oracle, [], []) == 1
    assert _check(oracle, [P - 1], [P - 1]) == 1
    assert _check(oracle, [5], [6]) == 0
