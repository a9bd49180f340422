"""Pins of the oracle's evaluator, multilinear extensions, prover and verifier.

- Multilinear extensions (Sec. 2.2): folding equals the explicit eq-sum and
  reproduces the table at boolean points.
- Evaluator (the layer relation of Sec. 2.2): closed forms on doubling and
  squaring circuits.
- Prover: byte-identical to the brute-force generic sumcheck of
  ``oracle/brute.py`` (which asserts g(0)+g(1) = claim every round, the check
  of Sec. 3.2.1, before leaving g(1) out of the message, and the final
  identity of every layer) on micro circuits,
  including padded widths and copy counts (Sec. 2.2 padding), all-add,
  all-mul and in1 = in2 wiring.
- Verifier: accepts honest proofs, rejects tampered proofs, outputs, inputs,
  wiring and domains.
"""
import random

import numpy as np
import pytest

import synth
from oracle import brute
from oracle.binding import ERR_REJECT, ints_to_bytes, bytes_to_ints

P = brute.P


def _mk(C, widths, pct=50, seed=9):
    circ = synth.micro(seed, C, widths, pct)
    x = synth.inputs_for(circ)
    return circ, synth.fr_bytes(x), synth.fr_ints(x)


# -- multilinear extensions --------------------------------------------------

@pytest.mark.parametrize("m", [0, 1, 2, 3, 5])
def test_mle_folding_equals_eq_sum(oracle, m):
    rng = random.Random(m)
    table = [rng.randrange(P) for _ in range(1 << m)]
    for _ in range(4):
        pt = [rng.randrange(P) for _ in range(m)]
        got = bytes_to_ints(oracle.mle(ints_to_bytes(table), m, ints_to_bytes(pt)))[0]
        assert got == brute.mle(table, pt)


def test_mle_boolean_points_and_linearity(oracle):
    rng = random.Random(3)
    m = 4
    table = [rng.randrange(P) for _ in range(1 << m)]
    tb = ints_to_bytes(table)
    for j in range(1 << m):
        pt = brute.bits_msb(j, m)
        assert bytes_to_ints(oracle.mle(tb, m, ints_to_bytes(pt)))[0] == table[j]
    # affine in each coordinate: f(t) = (1 - t) f(0) + t f(1)
    base = [rng.randrange(P) for _ in range(m)]
    for k in range(m):
        f = lambda t: bytes_to_ints(oracle.mle(tb, m, ints_to_bytes(base[:k] + [t] + base[k + 1:])))[0]
        t = rng.randrange(P)
        assert f(t) == ((1 - t) * f(0) + t * f(1)) % P


# -- evaluator closed forms ----------------------------------------------------

def _structured(kind, C, W, d):
    g = np.arange(W, dtype=np.uint32)
    t = np.full(W, 0 if kind == "double" else 1, dtype=np.uint8)
    return synth.Circuit([W] * (d + 1), [t] * d, [g] * d, [g] * d, C, name=kind)


@pytest.mark.parametrize("kind", ["double", "square"])
def test_eval_closed_forms(oracle, kind):
    C, W, d = 3, 5, 4
    circ = _structured(kind, C, W, d)
    x = synth.draw_fr_rows(17, b"cf", C, W)
    outs = bytes_to_ints(oracle.outputs(circ, synth.fr_bytes(x)))
    ins = synth.fr_ints(x)
    want = [(v << d) % P for v in ins] if kind == "double" else [pow(v, 1 << d, P) for v in ins]
    assert outs == want


def test_eval_matches_bruteforce_layers(oracle):
    circ, xb, xi = _mk(3, [6, 3, 7], 50, seed=4)
    pc = brute.Padded(circ)
    V = brute.evaluate(pc, xi)
    for layer in range(circ.depth + 1):
        assert bytes_to_ints(oracle.eval_layer(circ, xb, layer)) == V[layer]


# -- prover vs brute force -----------------------------------------------------

MICRO = [
    (1, [1, 1], 50), (1, [2, 2], 50), (1, [4, 4, 4], 50), (2, [2, 2, 2], 50),
    (4, [4, 4, 4], 50), (4, [4, 2, 8], 100), (4, [4, 4, 4], 0), (8, [8, 8], 50),
    (3, [3, 5, 2], 50), (5, [2, 3, 3], 60), (2, [1, 2, 1], 50), (8, [2, 4, 2, 4], 50),
    (2, [8, 8], 100), (16, [2, 2], 50),
]


@pytest.mark.parametrize("C,widths,pct", MICRO)
def test_prover_matches_bruteforce(oracle, C, widths, pct):
    circ, xb, xi = _mk(C, widths, pct)
    p1 = oracle.prove(circ, xb)
    p2 = brute.prove(circ, xi)
    assert len(p1) == oracle.proof_len(circ)
    assert p1 == p2
    assert oracle.verify(circ, xb, oracle.outputs(circ, xb), p1) == 0


def _random_shapes(n, seed=2024):
    """Seeded random micro shapes: copy counts 1-9 and widths 1-9 (powers of
    two or not: padding on both), depths 1-4, every mul share."""
    rng = random.Random(seed)
    out = []
    for _ in range(n):
        C = rng.randint(1, 9)
        widths = [rng.randint(1, 9) for _ in range(rng.randint(2, 5))]
        out.append((rng.randrange(1 << 30), C, widths, rng.choice([0, 25, 50, 75, 100])))
    return out


@pytest.mark.parametrize("seed,C,widths,pct", _random_shapes(24))
def test_prover_matches_bruteforce_random_shapes(oracle, seed, C, widths, pct):
    circ, xb, xi = _mk(C, widths, pct, seed=seed)
    p1 = oracle.prove(circ, xb)
    assert p1 == brute.prove(circ, xi)
    assert oracle.verify(circ, xb, oracle.outputs(circ, xb), p1) == 0


def test_in1_equals_in2_and_domain(oracle):
    circ, xb, xi = _mk(4, [4, 4, 4], 50, seed=21)
    for i in range(circ.depth):
        circ.in2[i] = circ.in1[i].copy()
    dom = b"another-domain"
    p1 = oracle.prove(circ, xb, dom)
    assert p1 == brute.prove(circ, xi, dom)
    outs = oracle.outputs(circ, xb)
    assert oracle.verify(circ, xb, outs, p1, dom) == 0
    assert oracle.verify(circ, xb, outs, p1) == ERR_REJECT


def test_proof_length_formula(oracle):
    for C, widths in [(16, [1024] * 9), (1024, [4096] * 21), (32768, [1024] * 25), (3, [3, 5, 2])]:
        circ = synth.Circuit(widths, [np.zeros(w, np.uint8) for w in widths[:-1]],
                             [np.zeros(w, np.uint32) for w in widths[:-1]],
                             [np.zeros(w, np.uint32) for w in widths[:-1]], C)
        d = len(widths) - 1
        c = brute.log2_ceil(C)
        s = [brute.log2_ceil(w) for w in widths]
        # per layer: 3 values per copy round, 2 per x and y round (g(1) left
        # out), then v_x and v_y
        assert oracle.proof_len(circ) == 8 + 4 * (d + 3) + 32 * sum(3 * c + 4 * s[i + 1] + 2 for i in range(d))
    assert oracle.proof_len(synth.tiny()) == 13876


# -- verifier: tampering -------------------------------------------------------

@pytest.fixture(scope="module")
def tiny_case(oracle):
    circ = synth.uniform_circuit(1, 4, [64] * 5, 50)
    xb = synth.fr_bytes(synth.inputs_for(circ))
    return circ, xb, oracle.outputs(circ, xb), oracle.prove(circ, xb)


def test_verifier_accepts(oracle, tiny_case):
    circ, xb, outs, proof = tiny_case
    assert oracle.verify(circ, xb, outs, proof) == 0


def test_tampered_elements_rejected(oracle, tiny_case):
    circ, xb, outs, proof = tiny_case
    hdr = 8 + 4 * (circ.depth + 3)
    n = (len(proof) - hdr) // 32
    rng = random.Random(2)
    positions = sorted(set([0, 1, 2, 3, n - 1, n - 2] + [rng.randrange(n) for _ in range(40)]))
    for k in positions:
        bad = bytearray(proof)
        bad[hdr + 32 * k + rng.randrange(31)] ^= 1 << rng.randrange(8)
        assert oracle.verify(circ, xb, outs, bytes(bad)) != 0, k
    for k in range(hdr):
        bad = bytearray(proof)
        bad[k] ^= 0x10
        assert oracle.verify(circ, xb, outs, bytes(bad)) != 0
    assert oracle.verify(circ, xb, outs, proof[:-32]) != 0
    assert oracle.verify(circ, xb, outs, proof + bytes(32)) != 0


def test_tampered_statement_rejected(oracle, tiny_case):
    circ, xb, outs, proof = tiny_case
    bad_out = bytearray(outs); bad_out[5] ^= 1
    assert oracle.verify(circ, xb, bytes(bad_out), proof) != 0
    bad_in = bytearray(xb); bad_in[32 * 7] ^= 1
    assert oracle.verify(circ, bytes(bad_in), outs, proof) != 0
    # swapping two wiring entries changes the statement
    c2 = synth.Circuit(list(circ.widths), [t.copy() for t in circ.types], [a.copy() for a in circ.in1],
                       [b.copy() for b in circ.in2], circ.n_copies)
    c2.in1[1][[3, 4]] = c2.in1[1][[4, 3]]
    assert oracle.verify(c2, xb, outs, proof) != 0


def test_non_canonical_inputs_rejected(oracle):
    circ, xb, xi = _mk(2, [2, 2], 50)
    bad = bytearray(xb)
    bad[0:32] = P.to_bytes(32, "little")
    with pytest.raises(ValueError):
        oracle.prove(circ, bytes(bad))


def test_invalid_circuits_rejected(oracle):
    good = synth.micro(1, 2, [2, 2])
    bad_idx = synth.Circuit([2, 2], [np.array([0, 1], np.uint8)], [np.array([0, 2], np.uint32)],
                            [np.array([0, 1], np.uint32)], 2)
    bad_type = synth.Circuit([2, 2], [np.array([0, 3], np.uint8)], [np.array([0, 1], np.uint32)],
                             [np.array([0, 1], np.uint32)], 2)
    oracle.proof_len(good)
    for c in (bad_idx, bad_type):
        with pytest.raises(ValueError):
            oracle.proof_len(c)


# --- accumulation gates (Sec. 3.4.3) ---------------------------------------

def _acc(widths, C, layers):
    """Circuit from per-layer entry lists [(out, type, in1, in2), ...]."""
    outs = [np.array([e[0] for e in L], np.uint32) for L in layers]
    types = [np.array([e[1] for e in L], np.uint8) for L in layers]
    in1 = [np.array([e[2] for e in L], np.uint32) for L in layers]
    in2 = [np.array([e[3] for e in L], np.uint32) for L in layers]
    return synth.Circuit(list(widths), types, in1, in2, C, outs=outs)


def test_accumulation_gate_closed_forms(oracle):
    """The paper's example: one gate of two add entries sums four inputs in
    one layer; a mul and an add entry give x0 x1 + x2 + x3; a gate with no
    entry is 0."""
    rng = random.Random(3)
    circ = _acc([3, 4], 2, [[(0, 0, 0, 1), (0, 0, 2, 3), (1, 1, 0, 1), (1, 0, 2, 3)]])
    x = [rng.randrange(P) for _ in range(8)]
    out = bytes_to_ints(oracle.outputs(circ, ints_to_bytes(x)))
    for b in range(2):
        v = x[4 * b:4 * b + 4]
        assert out[3 * b:3 * b + 3] == [sum(v) % P, (v[0] * v[1] + v[2] + v[3]) % P, 0]


def test_accumulation_with_one_entry_a_gate_is_the_plain_circuit(oracle):
    """Writing every gate as a single entry changes nothing: same wiring
    digest, same proof bytes."""
    plain = synth.micro(17, 4, [6, 5, 7], 50)
    layers = [[(g, int(plain.types[i][g]), int(plain.in1[i][g]), int(plain.in2[i][g]))
               for g in range(plain.widths[i])] for i in range(plain.depth)]
    acc = _acc(plain.widths, 4, layers)
    assert acc.accumulates
    xb = synth.fr_bytes(synth.inputs_for(plain))
    assert oracle.wiring_digest(acc) == oracle.wiring_digest(plain)
    assert oracle.prove(acc, xb) == oracle.prove(plain, xb)


@pytest.mark.parametrize("seed,C,widths,k", [(1, 2, [3, 4, 5], 3), (2, 4, [4, 4, 4], 4), (3, 3, [5, 2, 3, 4], 2),
                                             (4, 1, [2, 2], 5), (5, 8, [6, 3, 8], 3)])
def test_accumulation_prover_matches_bruteforce(oracle, seed, C, widths, k):
    circ = synth.accumulation_circuit(seed, C, widths, k)
    x = synth.inputs_for(circ)
    xb = synth.fr_bytes(x)
    proof = oracle.prove(circ, xb)
    assert proof == brute.prove(circ, synth.fr_ints(x))
    assert oracle.wiring_digest(circ) == brute.digest(brute.Padded(circ).wiring_bytes())
    V = brute.evaluate(brute.Padded(circ), synth.fr_ints(x))
    pc = brute.Padded(circ)
    for layer in range(circ.depth + 1):
        want = b"".join(brute.fe(V[layer][b * pc.W[layer] + g]) for b in range(pc.C) for g in range(pc.W[layer]))
        assert oracle.eval_layer(circ, xb, layer) == want
    outs = oracle.outputs(circ, xb)
    assert oracle.verify(circ, xb, outs, proof) == 0
    bad = bytearray(outs)
    bad[0] ^= 1
    assert oracle.verify(circ, xb, bytes(bad), proof) == ERR_REJECT
    hdr = 8 + 4 * (circ.depth + 3)
    for kk in range(0, (len(proof) - hdr) // 32, 5):
        t = bytearray(proof)
        t[hdr + 32 * kk + 1] ^= 2
        assert oracle.verify(circ, xb, outs, bytes(t)) == ERR_REJECT


def _random_accumulation(n, seed=3032):
    rng = random.Random(seed)
    return [(rng.randrange(1 << 30), rng.randint(1, 8), [rng.randint(1, 8) for _ in range(rng.randint(2, 4))],
             rng.randint(1, 5)) for _ in range(n)]


@pytest.mark.parametrize("seed,C,widths,k", _random_accumulation(12))
def test_accumulation_prover_matches_bruteforce_random_shapes(oracle, seed, C, widths, k):
    """Seeded random accumulation shapes: 1-8 copies, widths 1-8, up to 1-5
    entries a gate (gates with none are 0)."""
    circ = synth.accumulation_circuit(seed, C, widths, k)
    x = synth.inputs_for(circ)
    xb = synth.fr_bytes(x)
    proof = oracle.prove(circ, xb)
    assert proof == brute.prove(circ, synth.fr_ints(x))
    assert oracle.verify(circ, xb, oracle.outputs(circ, xb), proof) == 0


def test_accumulation_wiring_is_bound(oracle):
    """Moving one entry to another gate, or swapping two entries' order
    inside a gate with different types, changes the wiring digest."""
    base = _acc([2, 4], 1, [[(0, 0, 0, 1), (0, 1, 2, 3), (1, 0, 1, 2)]])
    moved = _acc([2, 4], 1, [[(0, 0, 0, 1), (1, 1, 2, 3), (1, 0, 1, 2)]])
    swapped = _acc([2, 4], 1, [[(0, 1, 2, 3), (0, 0, 0, 1), (1, 0, 1, 2)]])
    d = {oracle.wiring_digest(c) for c in (base, moved, swapped)}
    assert len(d) == 3


def test_thread_count_leaves_proofs_unchanged(oracle):
    """The oracle's OpenMP loops (copy pairs, fold rows, evaluation copies)
    only regroup exact field sums, so any thread count gives the same bytes;
    brute force fixes the one-thread proof on a micro circuit."""
    micro, mx, mi = _mk(8, [16, 8, 16], 50)
    circ = synth.uniform_circuit(2, 64, [128, 256, 64], 60, name="threads")
    x = synth.fr_bytes(synth.inputs_for(circ))
    try:
        one = oracle.prove(circ, x)
        micro_one = oracle.prove(micro, mx)
        for n in (2, 3, 8):
            assert oracle.set_threads(n) >= 1
            assert oracle.prove(circ, x) == one
            assert oracle.prove(micro, mx) == micro_one
    finally:
        oracle.set_threads(1)
    assert micro_one == brute.prove(micro, mi)
