"""GPU evaluation and proving through the C ABI, byte for byte against the
CPU oracle (GKR layer sumcheck, Sec. 2.2-2.3; data-parallel copies).

Proofs are deterministic and every element is exact, so parity is byte
equality of the whole proof.  Small cases call the oracle live; the
full-size workloads compare with hashes written by
tests/golden/make_golden.py, which calls only the oracle.
"""
import numpy as np
import pytest

import synth
from gpu_util import golden, sha, to_device

pytestmark = pytest.mark.gpu

P = synth.FR_MODULUS


@pytest.fixture(scope="module")
def S():
    import paper_2404_10404_b300 as S
    return S


def _case(S, oracle, circ, domain=None, device_inputs=False):
    xb = synth.fr_bytes(synth.inputs_for(circ))
    gc = S.Circuit.from_spec(circ)
    ev = S.Eval(gc, to_device(xb) if device_inputs else xb)
    tr = S.Transcript(domain) if domain else None
    proof = S.prove(gc, ev, tr)
    want = oracle.prove(circ, xb, domain)
    assert len(proof) == len(want) == gc.proof_len
    assert proof == want, _first_diff(proof, want, circ)
    outs = ev.outputs()
    assert outs == oracle.outputs(circ, xb)
    assert S.verify(gc, xb, outs, proof, domain) == 0
    return gc, ev, xb, proof


def _first_diff(a, b, circ):
    for i, (x, y) in enumerate(zip(a, b)):
        if x != y:
            hdr = 8 + 4 * (circ.depth + 3)
            return f"first differing byte {i} (element {(i - hdr) // 32} after the header)"
    return "lengths differ"


MICRO = [
    (1, [1, 1], 50), (1, [2, 2], 50), (1, [4, 4, 4], 50), (2, [2, 2, 2], 50), (4, [4, 4, 4], 50),
    (4, [4, 2, 8], 100), (4, [4, 4, 4], 0), (8, [8, 8], 50), (3, [3, 5, 2], 50), (5, [2, 3, 3], 60),
    (2, [1, 2, 1], 50), (8, [2, 4, 2, 4], 50), (2, [8, 8], 100), (16, [2, 2], 50), (64, [32, 16, 64], 50),
]


@pytest.mark.parametrize("C,widths,pct", MICRO)
def test_micro_parity(S, oracle, C, widths, pct):
    _case(S, oracle, synth.micro(9, C, widths, pct))


@pytest.mark.parametrize("C,widths,pct", [
    (1000, [1000, 1000, 1000], 50),     # padded copies and widths: absent gates, ragged tails
    (37, [300, 257, 513, 129], 70),
    (1, [4096, 4096, 4096], 50),        # one copy: the copy phase is empty
    (4096, [1, 1, 1], 50),              # one gate: x and y phases are empty
    (2, [2048, 8], 50),                 # fan-in from a narrow layer
    (256, [16, 2048, 16], 50),
    (512, [1024] * 4, 100), (512, [1024] * 4, 0),
    (2048, [3, 5, 2], 50),              # many pairs a warp: segments of a few gates each
    (600, [70, 33, 9], 40),             # padded copies, more pairs than CTAs, ragged segments
])
def test_shapes_parity(S, oracle, C, widths, pct):
    _case(S, oracle, synth.micro(11, C, widths, pct))


def test_wide_next_layer_parity(S, oracle):
    """A layer reading from more than 2^16 gates takes the one-launch-per-
    round path of Libra's phases instead of the cluster kernel."""
    _case(S, oracle, synth.micro(13, 2, [1024, 1 << 17], 50))
    _case(S, oracle, synth.micro(14, 4, [3000, 70000, 5000], 60))


def test_mixing_parity(S, oracle):
    _case(S, oracle, synth.mixing_circuit(3, 64, 256, 6))


def test_in1_equals_in2(S, oracle):
    circ = synth.micro(21, 16, [64, 64, 64], 50)
    for i in range(circ.depth):
        circ.in2[i] = circ.in1[i].copy()
    _case(S, oracle, circ)


def test_domain_and_device_inputs(S, oracle):
    circ = synth.micro(23, 32, [128, 64, 128], 50)
    _case(S, oracle, circ, domain=b"custom-domain", device_inputs=True)


def test_tiny_parity_and_golden(S, oracle):
    circ = synth.tiny()
    gc, ev, xb, proof = _case(S, oracle, circ)
    g = golden("tiny")
    if g:
        assert sha(proof) == g["proof_sha256"]


def test_layers_match_oracle(S, oracle):
    circ = synth.micro(31, 48, [100, 200, 300, 50], 50)
    xb = synth.fr_bytes(synth.inputs_for(circ))
    ev = S.Eval(S.Circuit.from_spec(circ), xb)
    for layer in range(circ.depth + 1):
        assert ev.layer(layer) == oracle.eval_layer(circ, xb, layer), layer


def test_repeat_and_update(S, oracle):
    """Workspace reuse: several proofs on one handle, then new inputs."""
    circ = synth.micro(41, 128, [256, 256, 256], 50)
    x1 = synth.fr_bytes(synth.inputs_for(circ))
    x2 = synth.fr_bytes(synth.inputs_for(circ, seed=99))
    gc = S.Circuit.from_spec(circ)
    ev = S.Eval(gc, x1)
    p1 = S.prove(gc, ev)
    assert S.prove(gc, ev) == p1 == S.prove_alloc(gc, ev)
    ev.update(to_device(x2))
    assert S.prove(gc, ev) == oracle.prove(circ, x2)
    ev.update(x1)
    assert S.prove(gc, ev) == p1


def test_errors(S):
    circ = synth.micro(1, 4, [4, 4])
    gc = S.Circuit.from_spec(circ)
    bad = bytearray(synth.fr_bytes(synth.inputs_for(circ)))
    bad[32:64] = P.to_bytes(32, "little")
    with pytest.raises(S.SisuError) as e:
        S.Eval(gc, bytes(bad))
    assert e.value.code == -3
    with pytest.raises(S.SisuError) as e:
        S.Circuit([4, 4], [np.zeros(4, np.uint8)], [np.array([0, 1, 2, 4], np.uint32)],
                  [np.zeros(4, np.uint32)], 4)
    assert e.value.code == -2
    with pytest.raises(S.SisuError) as e:
        S.Circuit([2, 2], [np.array([0, 5], np.uint8)], [np.zeros(2, np.uint32)], [np.zeros(2, np.uint32)], 4)
    assert e.value.code == -1
    with pytest.raises(S.SisuError) as e:
        S.Circuit([2, 2], [np.zeros(2, np.uint8)], [np.zeros(2, np.uint32)], [np.zeros(2, np.uint32)], 0)
    assert e.value.code == -1
    host_only = S.Circuit.from_spec(circ, host_only=True)
    with pytest.raises(S.SisuError):
        S.Eval(host_only, synth.fr_bytes(synth.inputs_for(circ)))


def test_tampered_gpu_proof_rejected(S):
    circ = synth.micro(51, 32, [64, 64, 64], 50)
    xb = synth.fr_bytes(synth.inputs_for(circ))
    gc = S.Circuit.from_spec(circ)
    ev = S.Eval(gc, xb)
    proof = S.prove(gc, ev)
    outs = ev.outputs()
    assert S.verify(gc, xb, outs, proof) == 0
    hdr = 8 + 4 * (circ.depth + 3)
    for k in range(0, (len(proof) - hdr) // 32, 7):
        bad = bytearray(proof)
        bad[hdr + 32 * k + 3] ^= 0x40
        assert S.verify(gc, xb, outs, bytes(bad)) == -7


@pytest.mark.parametrize("name", ["medium", "slot"])
def test_full_size_golden(S, name):
    """Full-size workloads, in the launch configuration the benchmark times:
    proof and outputs equal to the oracle's (stored hashes)."""
    g = golden(name)
    if g is None:
        pytest.skip(f"no oracle record for {name}")
    circ = {"medium": synth.medium, "slot": synth.slot}[name]()
    xb = synth.fr_bytes(synth.inputs_for(circ))
    assert sha(xb) == g["inputs_sha256"]
    gc = S.Circuit.from_spec(circ)
    ev = S.Eval(gc, to_device(xb))
    del xb
    proof = S.prove(gc, ev)
    assert len(proof) == g["proof_len"]
    assert sha(proof) == g["proof_sha256"]
    assert sha(ev.outputs()) == g["outputs_sha256"]


def test_chunked_host_inputs(S, oracle):
    """Host inputs of 32 MiB and more arrive in chunks of copies that are
    evaluated while the next chunk is in transfer: the proof equals the
    oracle's, and re-evaluating the handle from host and device inputs in
    turn on one stream keeps every proof identical."""
    circ = synth.uniform_circuit(8, 256, [4096, 4096, 4096], 50)
    xb = synth.fr_bytes(synth.inputs_for(circ))
    assert len(xb) >= 32 << 20
    gc = S.Circuit.from_spec(circ)
    ev = S.Eval(gc, xb)
    want = oracle.prove(circ, xb)
    assert S.prove(gc, ev) == want
    dev = to_device(xb)
    for src in (dev, xb, xb, dev, xb):
        ev.update(src)
        assert S.prove(gc, ev) == want


def test_full_size_golden_host_inputs(S):
    """The medium workload evaluated from host bytes (the chunked transfer)
    gives the oracle's proof and outputs (stored hashes)."""
    g = golden("medium")
    if g is None:
        pytest.skip("no oracle record for medium")
    circ = synth.medium()
    xb = synth.fr_bytes(synth.inputs_for(circ))
    gc = S.Circuit.from_spec(circ)
    ev = S.Eval(gc, xb)
    proof = S.prove(gc, ev)
    assert sha(proof) == g["proof_sha256"]
    assert sha(ev.outputs()) == g["outputs_sha256"]


@pytest.mark.parametrize("seed,C,widths,k", [
    (1, 2, [3, 4, 5], 3), (2, 4, [4, 4, 4], 4), (3, 37, [300, 257, 513], 3),  # padded copies and widths
    (4, 1, [64, 64, 64], 6),                                                  # one copy: no copy phase
    (5, 512, [1024, 1024, 1024], 2), (6, 64, [16, 2048, 16], 5),
    (7, 16, [1, 8, 1], 4),                                                    # one gate: no x, y phases
])
def test_accumulation_parity(S, oracle, seed, C, widths, k):
    """Accumulation gates (Sec. 3.4.3): a gate sums several fan-in-2
    entries; proofs and every layer's values equal the oracle's."""
    circ = synth.accumulation_circuit(seed, C, widths, k)
    _, ev, xb, _ = _case(S, oracle, circ)
    for layer in range(circ.depth + 1):
        assert ev.layer(layer) == oracle.eval_layer(circ, xb, layer), layer


def test_accumulation_wide_next_layer(S, oracle):
    """Entries over a layer wider than 2^16 take the one-launch-per-round
    path of Libra's phases."""
    _case(S, oracle, synth.accumulation_circuit(8, 2, [512, 1 << 17], 3))


def test_one_entry_a_gate_equals_plain(S, oracle):
    """The plain circuit written as one entry a gate proves the same bytes."""
    plain = synth.micro(19, 64, [128, 96, 128], 50)
    outs = [np.arange(w, dtype=np.uint32) for w in plain.widths[:-1]]
    acc = synth.Circuit(plain.widths, plain.types, plain.in1, plain.in2, plain.n_copies, outs=outs)
    xb = synth.fr_bytes(synth.inputs_for(plain))
    gp = S.Circuit.from_spec(plain)
    p_plain = S.prove(gp, S.Eval(gp, xb))
    ga = S.Circuit.from_spec(acc)
    assert S.prove(ga, S.Eval(ga, xb)) == p_plain == oracle.prove(plain, xb)
