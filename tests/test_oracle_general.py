"""General circuits (Sec. 2.7) in the oracle, pinned against what fixes
them: the brute-force prover (Python integers, every round by enumeration
over the hypercube, asserting g(0) + g(1) = claim and each layer's final
identity), the layered protocol (a general circuit whose second inputs all
come from the next layer is a layered circuit, and its proof must be the
layered proof byte for byte), closed forms of the evaluation, and the
verifier's accept and reject behaviour."""
import numpy as np
import pytest

import synth
from oracle import brute

P = brute.P


def _case(seed, C, widths, pct_mul=50, far=40):
    g = synth.general_circuit(seed, C, widths, pct_mul, far)
    x = synth.inputs_for(g)
    return g, synth.fr_bytes(x), synth.fr_ints(x)


LAYERED = [(2, [4, 4, 4], 50), (4, [4, 8, 4, 8], 60), (1, [8, 4], 50), (8, [16, 8, 16], 100), (3, [5, 3, 6], 0)]


@pytest.mark.parametrize("C,widths,pct", LAYERED)
def test_layered_circuit_gives_the_layered_proof(oracle, C, widths, pct):
    circ = synth.micro(9, C, widths, pct)
    x = synth.inputs_for(circ)
    xb = synth.fr_bytes(x)
    want = oracle.prove(circ, xb)
    assert oracle.prove_general(circ, xb) == want
    assert brute.prove_general(circ, synth.fr_ints(x)) == want


GENERAL = [(5, 4, [8, 8, 6, 8], 50, 40), (6, 2, [4, 4, 4, 4, 4], 60, 60), (7, 8, [8, 4, 8, 2, 8], 70, 70),
           (8, 1, [4, 4, 4], 50, 100), (9, 4, [5, 3, 6], 50, 50), (10, 3, [6, 7, 5, 9], 0, 50),
           (11, 4, [8, 8, 8, 8], 100, 30)]


@pytest.mark.parametrize("seed,C,widths,pct,far", GENERAL)
def test_general_proof_equals_brute_force(oracle, seed, C, widths, pct, far):
    g, xb, xi = _case(seed, C, widths, pct, far)
    assert g.general or g.depth < 2
    proof = oracle.prove_general(g, xb)
    assert proof == brute.prove_general(g, xi)
    assert len(proof) == oracle.general_proof_len(g)
    assert oracle.verify_general(g, xb, oracle.outputs_general(g, xb), proof) == 0


def _random_general(n, seed=4048):
    """Seeded random general shapes: 1-8 copies, 3-5 layers of widths 1-9,
    every mul share and share of far second inputs."""
    import random
    rng = random.Random(seed)
    out = []
    for _ in range(n):
        widths = [rng.randint(1, 9) for _ in range(rng.randint(3, 5))]
        out.append((rng.randrange(1 << 30), rng.randint(1, 8), widths, rng.choice([0, 50, 100]),
                    rng.choice([20, 50, 100])))
    return out


@pytest.mark.parametrize("seed,C,widths,pct,far", _random_general(12))
def test_general_proof_equals_brute_force_random_shapes(oracle, seed, C, widths, pct, far):
    g, xb, xi = _case(seed, C, widths, pct, far)
    proof = oracle.prove_general(g, xb)
    assert proof == brute.prove_general(g, xi)
    assert oracle.verify_general(g, xb, oracle.outputs_general(g, xb), proof) == 0


def test_used_gates_indexing():
    """The virtual layer: layer i + 1 in full, then the used gates of each
    deeper layer in ascending order; indexes differ from positions."""
    g, _, _ = _case(5, 4, [8, 8, 6, 8], 50, 40)
    pc = brute.GeneralPadded(g)
    for i in range(g.depth):
        src = g.layer_src(i)
        assert pc.blocks[i][0] == (i + 1, 0, list(range(pc.W[i + 1])))
        base = pc.W[i + 1]
        for j, b0, ys in pc.blocks[i][1:]:
            assert j > i + 1 and b0 == base and ys == sorted(set(int(y) for y, s in zip(g.in2[i], src) if s == j))
            base += len(ys)
        assert 1 << pc.sx[i] >= base > (1 << pc.sx[i]) // 2 or base == 1
        for gate, u in enumerate(pc.u2[i]):
            j, y = int(src[gate]), int(g.in2[i][gate])
            if j == i + 1:
                assert u == y
            else:
                blk = next(b for b in pc.blocks[i] if b[0] == j)
                assert u == blk[1] + blk[2].index(y)


def test_skip_connection_closed_form(oracle):
    """layer 1 = 2 x (add gates x + x), layer 0 = layer 1 times the input
    (second input from the input layer): outputs 2 x^2."""
    W, C = 4, 2
    g = synth.Circuit([W, W, W], [np.ones(W, np.uint8), np.zeros(W, np.uint8)],
                      [np.arange(W, dtype=np.uint32)] * 2, [np.arange(W, dtype=np.uint32)] * 2, C,
                      name="skip", src=[np.full(W, 2, np.uint32), np.full(W, 2, np.uint32)])
    x = synth.inputs_for(g)
    xi = synth.fr_ints(x)
    outs = oracle.outputs_general(g, synth.fr_bytes(x))
    assert [int.from_bytes(outs[32 * k:32 * k + 32], "little") for k in range(C * W)] == [2 * v * v % P for v in xi]
    assert oracle.prove_general(g, synth.fr_bytes(x)) == brute.prove_general(g, xi)


def test_verifier_rejects(oracle):
    g, xb, xi = _case(5, 4, [8, 8, 6, 8], 50, 40)
    proof = oracle.prove_general(g, xb)
    outs = oracle.outputs_general(g, xb)
    assert oracle.verify_general(g, xb, outs, proof) == 0
    hdr = 8 + 4 * (g.depth + 3)
    for k in range((len(proof) - hdr) // 32):  # every element of the proof
        bad = bytearray(proof)
        bad[hdr + 32 * k + 5] ^= 0x10
        assert oracle.verify_general(g, xb, outs, bytes(bad)) != 0, k
    assert oracle.verify_general(g, xb, outs, proof[:-32]) != 0
    bad_out = bytearray(outs)
    bad_out[0] ^= 1
    assert oracle.verify_general(g, xb, bytes(bad_out), proof) != 0
    bad_in = bytearray(xb)
    bad_in[32 * 3] ^= 1
    assert oracle.verify_general(g, bytes(bad_in), outs, proof) != 0
    # the wiring digest binds the second input's layer
    moved = synth.general_circuit(5, 4, [8, 8, 6, 8], 50, 40)
    i = next(i for i in range(moved.depth) if (moved.layer_src(i) != i + 1).any())
    gate = int(np.nonzero(moved.layer_src(i) != i + 1)[0][0])
    moved.src[i] = moved.layer_src(i).copy()
    moved.src[i][gate] = i + 1
    moved.in2[i] = np.array(moved.in2[i]).copy()
    moved.in2[i][gate] = 0
    assert oracle.verify_general(moved, xb, oracle.outputs_general(moved, xb), proof) != 0
    # another domain
    assert oracle.verify_general(g, xb, outs, proof, b"other") != 0
    assert oracle.verify_general(g, xb, outs, oracle.prove_general(g, xb, b"other"), b"other") == 0


@pytest.mark.parametrize("seed,C,widths", [(31, 4, [8] * 7), (32, 2, [4, 8, 4, 8, 4, 8, 4, 8]), (33, 3, [5] * 10)])
def test_layers_reading_many_layers(oracle, seed, C, widths):
    """Every second input far: a layer reads up to d - i layers, so its end
    absorbs two values for each of five to nine blocks in one message."""
    g, xb, xi = _case(seed, C, widths, 50, 100)
    pc = brute.GeneralPadded(g)
    assert max(len(b) for b in pc.blocks) >= 5
    proof = oracle.prove_general(g, xb)
    assert proof == brute.prove_general(g, xi)
    assert oracle.verify_general(g, xb, oracle.outputs_general(g, xb), proof) == 0
