"""The C-ABI library loads and exports every entry point include/sisu.h
declares; its host-only verifier (no CUDA call) accepts the oracle's proofs
and rejects tampered ones.  Runs without a GPU."""
import ctypes
import os
import re

import pytest

import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "sisu.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sisu_[a-z0-9_]+)\s*\(", src)))


def test_header_symbols_exported():
    from paper_2404_10404_b300 import ENTRY_POINTS, library_path
    if not os.path.exists(library_path()):
        pytest.skip("library not built")
    lib = ctypes.CDLL(library_path())
    names = _declared()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(ENTRY_POINTS) == names


def test_host_verifier_against_oracle(oracle):
    import paper_2404_10404_b300 as S
    if not os.path.exists(S.library_path()):
        pytest.skip("library not built")
    for circ in (synth.micro(3, 4, [4, 4, 4]), synth.micro(4, 3, [3, 5, 2]), synth.micro(5, 64, [64, 32, 64])):
        xb = synth.fr_bytes(synth.inputs_for(circ))
        proof, outs = oracle.prove(circ, xb), oracle.outputs(circ, xb)
        hc = S.Circuit.from_spec(circ, host_only=True)
        assert hc.proof_len == len(proof)
        assert S.verify(hc, xb, outs, proof) == 0
        hdr = 8 + 4 * (circ.depth + 3)
        for k in range(0, (len(proof) - hdr) // 32, 3):
            bad = bytearray(proof)
            bad[hdr + 32 * k] ^= 1
            assert S.verify(hc, xb, outs, bytes(bad)) == -7
        assert S.verify(hc, xb, outs, proof, b"other-domain") == -7
        bad_out = bytearray(outs)
        bad_out[0] ^= 1
        assert S.verify(hc, xb, bytes(bad_out), proof) == -7


def test_host_verifier_rejects_forgeries():
    """Round-consistent forgeries (the oracle's pins) fail the library's
    final-identity and input checks too."""
    import paper_2404_10404_b300 as S
    from oracle import brute
    if not os.path.exists(S.library_path()):
        pytest.skip("library not built")
    circ = synth.micro(6, 4, [4, 4], 50)
    x = synth.fr_ints(synth.inputs_for(circ))
    hc = S.Circuit.from_spec(circ, host_only=True)
    xb = brute.fe(0)[:0] + b"".join(brute.fe(v) for v in x)
    outs = brute.evaluate(brute.Padded(circ), x)[0]
    fake = list(outs)
    fake[0] = (fake[0] + 1) % brute.P
    forged = brute.forge_one_layer(circ, x, fake)
    assert S.verify(hc, xb, b"".join(brute.fe(v) for v in fake), forged) == -7
    forged = brute.forge_vy_one_layer(circ, x)
    assert S.verify(hc, xb, b"".join(brute.fe(v) for v in outs), forged) == -7
    honest = brute.prove(circ, x)
    assert S.verify(hc, xb, b"".join(brute.fe(v) for v in outs), honest) == 0


def test_host_verifier_accumulation_gates(oracle):
    """Accumulation gates (Sec. 3.4.3) through sisu_circuit_create_acc_host:
    the host verifier accepts the oracle's proofs and rejects tampering;
    invalid entries are refused."""
    import numpy as np

    import paper_2404_10404_b300 as S
    if not os.path.exists(S.library_path()):
        pytest.skip("library not built")
    for circ in (synth.accumulation_circuit(1, 2, [3, 4, 5], 3), synth.accumulation_circuit(5, 8, [6, 3, 8], 3),
                 synth.accumulation_circuit(6, 1, [4, 4], 5)):
        xb = synth.fr_bytes(synth.inputs_for(circ))
        proof, outs = oracle.prove(circ, xb), oracle.outputs(circ, xb)
        hc = S.Circuit.from_spec(circ, host_only=True)
        assert hc.proof_len == len(proof)
        assert S.verify(hc, xb, outs, proof) == 0
        hdr = 8 + 4 * (circ.depth + 3)
        for k in range(0, (len(proof) - hdr) // 32, 4):
            bad = bytearray(proof)
            bad[hdr + 32 * k] ^= 1
            assert S.verify(hc, xb, outs, bytes(bad)) == -7
    u32 = lambda v: np.array(v, np.uint32)
    with pytest.raises(S.SisuError) as e:  # entry's gate beyond the layer's width
        S.Circuit([2, 2], [np.zeros(1, np.uint8)], [u32([0])], [u32([1])], 1, host_only=True, outs=[u32([2])])
    assert e.value.code == -2
    with pytest.raises(S.SisuError) as e:  # input index beyond the next layer
        S.Circuit([2, 2], [np.zeros(1, np.uint8)], [u32([0])], [u32([2])], 1, host_only=True, outs=[u32([0])])
    assert e.value.code == -2
    with pytest.raises(S.SisuError) as e:  # type 2
        S.Circuit([2, 2], [np.full(1, 2, np.uint8)], [u32([0])], [u32([1])], 1, host_only=True, outs=[u32([0])])
    assert e.value.code == -1
