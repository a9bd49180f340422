"""Seeded random shapes on the GPU, byte for byte against the CPU oracle:
layered circuits with padded copy counts and widths (every mul share,
depths 1-4, up to a few hundred copies and gates, so that rounds span
several CTAs with ragged tails), accumulation layers and general circuits.
The same seeds give the same shapes on every run."""
import random

import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    import paper_2404_10404_b300 as S
    return S


def _layered(n, seed=77):
    rng = random.Random(seed)
    out = []
    for _ in range(n):
        big = rng.random() < 0.4
        C = rng.randint(1, 300 if big else 9)
        widths = [rng.randint(1, 300 if big else 9) for _ in range(rng.randint(2, 5))]
        out.append((rng.randrange(1 << 30), C, widths, rng.choice([0, 30, 50, 70, 100])))
    return out


def _check(S, oracle, circ, prove_oracle):
    xb = synth.fr_bytes(synth.inputs_for(circ))
    gc = S.Circuit.from_spec(circ)
    ev = S.Eval(gc, xb)
    proof = S.prove(gc, ev)
    assert proof == prove_oracle(circ, xb)
    assert S.verify(gc, xb, ev.outputs(), proof) == 0


@pytest.mark.parametrize("seed,C,widths,pct", _layered(20))
def test_layered_random_shapes(S, oracle, seed, C, widths, pct):
    _check(S, oracle, synth.micro(seed, C, widths, pct), oracle.prove)


@pytest.mark.parametrize("seed,C,widths,k", [
    (s, c, w, k) for s, c, w, k in
    ((lambda r: [(r.randrange(1 << 30), r.randint(1, 64), [r.randint(1, 64) for _ in range(r.randint(2, 4))],
                  r.randint(1, 5)) for _ in range(6)])(random.Random(78)))])
def test_accumulation_random_shapes(S, oracle, seed, C, widths, k):
    _check(S, oracle, synth.accumulation_circuit(seed, C, widths, k), oracle.prove)


@pytest.mark.parametrize("seed,C,widths,pct,far", [
    (s, c, w, p, f) for s, c, w, p, f in
    ((lambda r: [(r.randrange(1 << 30), r.randint(1, 64), [r.randint(1, 64) for _ in range(r.randint(3, 5))],
                  r.choice([0, 50, 100]), r.choice([20, 50, 100])) for _ in range(6)])(random.Random(79)))])
def test_general_random_shapes(S, oracle, seed, C, widths, pct, far):
    _check(S, oracle, synth.general_circuit(seed, C, widths, pct, far), oracle.prove_general)
