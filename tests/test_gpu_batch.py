"""Batched proving of independent instances of uneven size (the batched
workload's distribution, scaled to sizes the oracle finishes quickly): every proof
equals the oracle's and the single-instance GPU proof, at every concurrency,
on repeated calls (CUDA-graph replay) and in any order."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    import paper_2404_10404_b300 as S
    return S


def _instances():
    rng = np.random.default_rng(7)
    out = []
    for j in range(7):
        C = int(2 ** rng.integers(2, 8))
        W = int(2 ** rng.integers(3, 9))
        d = int(rng.integers(1, 5))
        out.append(synth.uniform_circuit(4 * (1 << 32) + j, C, [W] * (d + 1), 60, name=f"b{j}"))
    out.append(synth.micro(99, 37, [300, 257, 513], 70))  # padded shape in the mix
    return out


@pytest.fixture(scope="module")
def batch(S, oracle):
    circs = _instances()
    xs = [synth.fr_bytes(synth.inputs_for(c)) for c in circs]
    gcs = [S.Circuit.from_spec(c) for c in circs]
    evs = [S.Eval(g, x) for g, x in zip(gcs, xs)]
    want = [oracle.prove(c, x) for c, x in zip(circs, xs)]
    return circs, xs, gcs, evs, want


@pytest.mark.parametrize("k", [1, 3, 8])
def test_batch_equals_oracle(S, batch, k):
    circs, xs, gcs, evs, want = batch
    for _ in range(2):  # second call replays the captured graphs
        assert S.prove_batch(gcs, evs, concurrency=k) == want


def test_batch_equals_single_and_order_free(S, batch):
    circs, xs, gcs, evs, want = batch
    singles = [S.prove(g, e) for g, e in zip(gcs, evs)]
    assert singles == want
    order = [5, 0, 7, 2, 6, 1, 3, 4]
    got = S.prove_batch([gcs[i] for i in order], [evs[i] for i in order], concurrency=4)
    assert got == [want[i] for i in order]
    for g, x, e, p in zip(gcs, xs, evs, want):
        assert S.verify(g, x, e.outputs(), p) == 0


def test_batch_domain_and_repeat_rejected(S, batch, oracle):
    circs, xs, gcs, evs, want = batch
    tr = S.Transcript(b"batch-domain")
    got = S.prove_batch(gcs[:3], evs[:3], tr, concurrency=2)
    assert got == [oracle.prove(c, x, b"batch-domain") for c, x in zip(circs[:3], xs[:3])]
    with pytest.raises(S.SisuError) as e:
        S.prove_batch([gcs[0], gcs[0]], [evs[0], evs[0]])
    assert e.value.code == -1


# instances of the batched workload itself (C = 2^U{6..14}, W = 2^U{8..12},
# d = U{8..24}, 60% mul, seeds 4*2^32+j): the nine smallest of its first 64,
# up to 2.9 M gates each, among them the widest width (4096)
BATCHED_SMALL = [21, 29, 56, 57, 33, 30, 22, 34, 10]


def test_batched_workload_instances_equal_oracle(S):
    import os

    from oracle import Oracle
    o = Oracle()
    o.set_threads(os.cpu_count() or 1)  # the proof bytes do not depend on it
    circs = [synth.batched_instance(j) for j in BATCHED_SMALL]
    xs = [synth.fr_bytes(synth.inputs_for(c)) for c in circs]
    gcs = [S.Circuit.from_spec(c) for c in circs]
    evs = [S.Eval(g, x) for g, x in zip(gcs, xs)]
    want = [o.prove(c, x) for c, x in zip(circs, xs)]
    for k in (1, 4, 9):
        assert S.prove_batch(gcs, evs, concurrency=k) == want


# larger instances of the same workload (8 to 55 M gates, up to its largest
# copy count, 2^14, and its widest width, 4096), compared with the oracle's
# proof hashes written by tests/golden/make_golden.py
BATCHED_MID = [36, 40, 35, 62, 38, 27, 31, 12]


def test_batched_workload_mid_size_instances_equal_oracle_hashes(S):
    from gpu_util import golden, sha
    gold = [golden(f"batched_{j}") for j in BATCHED_MID]
    if any(g is None for g in gold):
        pytest.skip("no oracle record for the batched instances")
    circs = [synth.batched_instance(j) for j in BATCHED_MID]
    xs = [synth.fr_bytes(synth.inputs_for(c)) for c in circs]
    for x, g in zip(xs, gold):
        assert sha(x) == g["inputs_sha256"]
    gcs = [S.Circuit.from_spec(c) for c in circs]
    evs = [S.Eval(g, x) for g, x in zip(gcs, xs)]
    del xs
    proofs = S.prove_batch(gcs, evs, concurrency=4)
    for j, p, ev, g in zip(BATCHED_MID, proofs, evs, gold):
        assert len(p) == g["proof_len"], j
        assert sha(p) == g["proof_sha256"], j
        assert sha(ev.outputs()) == g["outputs_sha256"], j
