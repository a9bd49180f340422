"""General circuits (Sec. 2.7) on the GPU: gates whose second input comes
from any deeper layer, proven over virtual layers of the used gates.  Every
proof must equal the oracle's general prover byte for byte (itself pinned
against brute force), a layered circuit given as a general one must give
the layered proof, and the host verifier must accept."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    import paper_2404_10404_b300 as S
    return S


MICRO = [(5, 4, [8, 8, 6, 8], 50, 40), (6, 2, [4, 4, 4, 4, 4], 60, 60), (7, 8, [8, 4, 8, 2, 8], 70, 70),
         (8, 1, [4, 4, 4], 50, 100), (9, 4, [5, 3, 6], 50, 50), (10, 3, [6, 7, 5, 9], 0, 50),
         (11, 16, [32, 64, 16, 32], 100, 30)]


@pytest.mark.parametrize("seed,C,widths,pct,far", MICRO)
def test_general_micro_equals_oracle(S, oracle, seed, C, widths, pct, far):
    g = synth.general_circuit(seed, C, widths, pct, far)
    xb = synth.fr_bytes(synth.inputs_for(g))
    gc = S.Circuit.from_spec(g)
    assert gc.proof_len == oracle.general_proof_len(g)
    ev = S.Eval(gc, xb)
    assert ev.outputs() == oracle.outputs_general(g, xb)
    want = oracle.prove_general(g, xb)
    for _ in range(3):  # the second proof and later replay the captured graph
        assert S.prove(gc, ev) == want
    assert S.verify(gc, xb, ev.outputs(), want) == 0


def test_layered_given_as_general_is_the_layered_proof(S, oracle):
    spec = synth.uniform_circuit(12, 64, [64, 32, 128, 64], 60, name="as-general")
    gen = synth.Circuit(spec.widths, spec.types, spec.in1, spec.in2, spec.n_copies, name="as-general-g",
                        src=[np.full(w, i + 1, np.uint32) for i, w in enumerate(spec.widths[:-1])])
    xb = synth.fr_bytes(synth.inputs_for(spec))
    want = oracle.prove(spec, xb)
    gl, gg = S.Circuit.from_spec(spec), S.Circuit.from_spec(gen)
    assert S.prove(gl, S.Eval(gl, xb)) == want
    assert S.prove(gg, S.Eval(gg, xb)) == want


def test_general_several_tiles_and_domain(S, oracle):
    """Rounds spanning many CTAs (256 copies, 1024-wide layers, several
    readers of one layer), with another transcript domain."""
    g = synth.general_circuit(13, 256, [1024, 1024, 512, 1024, 1024], 50, 30)
    xb = synth.fr_bytes(synth.inputs_for(g))
    gc = S.Circuit.from_spec(g)
    ev = S.Eval(gc, xb)
    tr = S.Transcript(b"general-domain")
    want = oracle.prove_general(g, xb, b"general-domain")
    assert S.prove(gc, ev, tr) == want
    assert S.verify(gc, xb, ev.outputs(), want, b"general-domain") == 0
    assert S.verify(gc, xb, ev.outputs(), want) != 0


def test_general_in_a_batch(S, oracle):
    specs = [synth.general_circuit(20 + k, 2 ** (k + 1), [16 * (k + 1), 32, 16, 32], 60, 40) for k in range(4)]
    specs.append(synth.uniform_circuit(30, 8, [32, 32, 32], 50, name="layered-in-batch"))
    xs = [synth.fr_bytes(synth.inputs_for(c)) for c in specs]
    gcs = [S.Circuit.from_spec(c) for c in specs]
    evs = [S.Eval(g, x) for g, x in zip(gcs, xs)]
    want = [oracle.prove_general(c, x) if c.src is not None else oracle.prove(c, x) for c, x in zip(specs, xs)]
    for k in (1, 3):
        assert S.prove_batch(gcs, evs, concurrency=k) == want


def test_general_errors(S):
    g = synth.general_circuit(5, 4, [8, 8, 6, 8], 50, 40)
    bad = synth.Circuit(g.widths, g.types, g.in1, g.in2, g.n_copies, src=[s.copy() for s in g.src])
    bad.src[1][0] = 1  # not below the gate's layer
    with pytest.raises(S.SisuError) as e:
        S.Circuit.from_spec(bad)
    assert e.value.code == -2
    bad.src[1][0] = 4  # beyond the inputs
    with pytest.raises(S.SisuError):
        S.Circuit.from_spec(bad)
    bad.src[1][0] = 3
    bad.in2 = [b.copy() for b in g.in2]
    bad.in2[1][0] = 8  # layer 3 has 8 gates
    with pytest.raises(S.SisuError):
        S.Circuit.from_spec(bad)
    gc = S.Circuit.from_spec(g)
    srv = S.Server(1 << 30, 2)
    with pytest.raises(S.SisuError):
        srv.submit(gc, synth.fr_bytes(synth.inputs_for(g)))
    srv.close()


@pytest.mark.parametrize("seed,C,widths", [(31, 4, [8] * 7), (33, 3, [5] * 10), (34, 64, [256] * 9)])
def test_layers_reading_many_layers(S, oracle, seed, C, widths):
    """Every second input far: a layer's end absorbs two values for each of
    up to d - i blocks (five to nine here) in one message."""
    g = synth.general_circuit(seed, C, widths, 50, 100)
    xb = synth.fr_bytes(synth.inputs_for(g))
    gc = S.Circuit.from_spec(g)
    ev = S.Eval(gc, xb)
    want = oracle.prove_general(g, xb)
    assert S.prove(gc, ev) == want
    assert S.verify(gc, xb, ev.outputs(), want) == 0


def test_general_and_accumulation_handles_take_new_inputs(S, oracle):
    """A handle's later proofs replay its captured graph: after new inputs
    (host, then device) the virtual layers are gathered again and every
    proof is the oracle's for the current inputs."""
    from gpu_util import to_device
    specs = [(synth.general_circuit(41, 32, [64, 32, 64, 16, 64], 50, 60), oracle.prove_general),
             (synth.accumulation_circuit(42, 32, [64, 32, 64, 16], 4), oracle.prove)]
    for circ, prove in specs:
        x1 = synth.fr_bytes(synth.inputs_for(circ))
        x2 = synth.fr_bytes(synth.inputs_for(circ, seed=99))
        gc = S.Circuit.from_spec(circ)
        ev = S.Eval(gc, x1)
        p1 = S.prove(gc, ev)
        assert p1 == prove(circ, x1) == S.prove(gc, ev)
        ev.update(x2)
        assert S.prove(gc, ev) == prove(circ, x2)
        ev.update(to_device(x1))
        assert S.prove(gc, ev) == p1
