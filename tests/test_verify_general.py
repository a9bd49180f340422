"""The library's host verifier on general circuits (Sec. 2.7), on CPU
(circuits created for host verification only): it accepts the oracle's
proofs and rejects any tampered element, other outputs or inputs, and a
circuit whose second inputs come from other layers."""
import numpy as np
import pytest

import synth


@pytest.fixture(scope="module")
def S():
    import paper_2404_10404_b300 as S
    return S


@pytest.mark.parametrize("seed,C,widths,far", [(5, 4, [8, 8, 6, 8], 40), (7, 8, [8, 4, 8, 2, 8], 70),
                                               (9, 4, [5, 3, 6], 50), (8, 1, [4, 4, 4], 100),
                                               # layers reading five to nine layers: long 'V' absorbs
                                               (31, 4, [8] * 7, 100), (33, 3, [5] * 10, 100)])
def test_host_verifier_on_general_proofs(S, oracle, seed, C, widths, far):
    g = synth.general_circuit(seed, C, widths, 50, far)
    xb = synth.fr_bytes(synth.inputs_for(g))
    gc = S.Circuit.from_spec(g, host_only=True)
    proof = oracle.prove_general(g, xb)
    outs = oracle.outputs_general(g, xb)
    assert gc.proof_len == len(proof)
    assert S.verify(gc, xb, outs, proof) == 0
    hdr = 8 + 4 * (g.depth + 3)
    for k in range(0, (len(proof) - hdr) // 32, 2):
        bad = bytearray(proof)
        bad[hdr + 32 * k + 3] ^= 0x40
        assert S.verify(gc, xb, outs, bytes(bad)) != 0
    bad_out = bytearray(outs)
    bad_out[33] ^= 1
    assert S.verify(gc, xb, bytes(bad_out), proof) != 0
    bad_in = bytearray(xb)
    bad_in[-40] ^= 1
    assert S.verify(gc, bytes(bad_in), outs, proof) != 0


def test_layer_of_second_input_is_bound(S, oracle):
    g = synth.general_circuit(5, 4, [8, 8, 6, 8], 50, 40)
    xb = synth.fr_bytes(synth.inputs_for(g))
    proof = oracle.prove_general(g, xb)
    i = next(i for i in range(g.depth) if (g.layer_src(i) != i + 1).any())
    gate = int(np.nonzero(g.layer_src(i) != i + 1)[0][0])
    moved = synth.Circuit(g.widths, g.types, g.in1, [b.copy() for b in g.in2], g.n_copies,
                          src=[s.copy() for s in g.src])
    moved.src[i][gate] = i + 1
    moved.in2[i][gate] = 0
    gm = S.Circuit.from_spec(moved, host_only=True)
    assert S.verify(gm, xb, oracle.outputs_general(moved, xb), proof) != 0
