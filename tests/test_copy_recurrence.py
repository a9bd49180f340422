"""The identity behind the copy phase's recurrence form, checked on Python
integers in the BN254 scalar field (no GPU, no library).

For a table T of n = 2h rows over the positions of layer i + 1, gates g
with weights w(g), op_g(x, y) = x + y or x y of the entries at in1 g and
in2 g of a row, write U(j) = sum_g w(g) op_g(T(j, in1 g), T(j, in2 g)) and
c_j = sum over mul gates of w (T(j + h, in1) - T(j, in1))(T(j + h, in2) -
T(j, in2)).  Then

  * the copy round's per-pair sum at t is S_j(t) = U(j) + t (U(j + h) -
    U(j)) + (t^2 - t) c_j (degree 2 in t, from the rows T_t = T(j) + t
    (T(j + h) - T(j))), and
  * after the fold T'(j) = T(j) + r (T(j + h) - T(j)) the next round's row
    sums are U'(j) = (1 - r) U(j) + r U(j + h) + (r^2 - r) c_j.

The GPU prover's copy rounds form only c_j per pair and carry U by the
second identity (its proofs are compared byte for byte with the oracle's
elsewhere); these tests check both identities directly, over whole folding
chains and for gates with several entries (accumulation layers).
"""
import random

import pytest

P = 0x30644E72E131A029B85045B68181585D2833E84879B9709143E1F593F0000001


def rand_fe(rng):
    return rng.randrange(P)


def make_gates(rng, w_in, n_entries, mul_share):
    # (type, in1, in2, weight); several entries may share a weight (one gate)
    gates = []
    for _ in range(n_entries):
        gates.append((1 if rng.random() < mul_share else 0, rng.randrange(w_in), rng.randrange(w_in),
                      rand_fe(rng)))
    return gates


def op(t, x, y):
    return x * y % P if t else (x + y) % P


def row_sum(gates, row):
    return sum(w * op(t, row[a], row[b]) for t, a, b, w in gates) % P


def t2_coeff(gates, lo, hi):
    return sum(w * (hi[a] - lo[a]) * (hi[b] - lo[b]) for t, a, b, w in gates if t) % P


def fold(T, r):
    h = len(T) // 2
    return [[(T[j][x] + r * (T[j + h][x] - T[j][x])) % P for x in range(len(T[0]))] for j in range(h)]


@pytest.mark.parametrize("n,w_in,n_entries,mul_share,seed", [
    (2, 4, 3, 0.5, 1), (8, 16, 12, 0.7, 2), (16, 8, 20, 1.0, 3), (32, 16, 16, 0.0, 4), (64, 32, 40, 0.4, 5),
])
def test_round_sums_and_fold_recurrence(n, w_in, n_entries, mul_share, seed):
    rng = random.Random(seed)
    gates = make_gates(rng, w_in, n_entries, mul_share)
    T = [[rand_fe(rng) for _ in range(w_in)] for _ in range(n)]
    U = [row_sum(gates, row) for row in T]
    while len(T) > 1:
        h = len(T) // 2
        c = [t2_coeff(gates, T[j], T[j + h]) for j in range(h)]
        # the round's per-pair sums at t = 0..3 from the rows T_t
        for j in range(h):
            for t in range(4):
                Tt = [(T[j][x] + t * (T[j + h][x] - T[j][x])) % P for x in range(w_in)]
                want = row_sum(gates, Tt)
                got = (U[j] + t * (U[j + h] - U[j]) + (t * t - t) * c[j]) % P
                assert got == want, (len(T), j, t)
        r = rand_fe(rng)
        T = fold(T, r)
        U_next = [((1 - r) * U[j] + r * U[j + h] + (r * r - r) * c[j]) % P for j in range(h)]
        assert U_next == [row_sum(gates, row) for row in T], len(T)
        U = U_next


def test_special_challenges():
    # r = 0 and r = 1 select a half; r = 2 extrapolates (t^2 - t = 2)
    rng = random.Random(7)
    gates = make_gates(rng, 8, 10, 0.6)
    T = [[rand_fe(rng) for _ in range(8)] for _ in range(4)]
    U = [row_sum(gates, row) for row in T]
    c = [t2_coeff(gates, T[j], T[j + 2]) for j in range(2)]
    for r in (0, 1, 2, P - 1):
        Tn = fold(T, r)
        for j in range(2):
            assert ((1 - r) * U[j] + r * U[j + 2] + (r * r - r) * c[j]) % P == row_sum(gates, Tn[j])


def test_a_dropped_correction_is_caught():
    # without the (r^2 - r) c_j term the recurrence fails whenever a mul
    # gate's inputs differ between the two rows
    rng = random.Random(11)
    gates = [(1, 0, 1, 5), (0, 1, 2, 7)]
    T = [[rand_fe(rng) for _ in range(3)] for _ in range(2)]
    U = [row_sum(gates, row) for row in T]
    r = rand_fe(rng)
    wrong = ((1 - r) * U[0] + r * U[1]) % P
    assert wrong != row_sum(gates, fold(T, r)[0])
