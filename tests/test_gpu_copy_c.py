"""The layered circuits' copy round (the recurrence form) on shapes chosen
for its work splits, byte for byte against the CPU oracle:

  * many pairs a CTA, so that a CTA's pairs go in several chunks of at most
    128 (2^17 copies of narrow layers);
  * pairs split between warps at every kind of boundary (mul-entry counts
    that do not divide the warps' ranges);
  * few pairs, so that a pair's mul entries go to several shares whose t^2
    terms are combined by the last block;
  * layers with no mul entry (every round's c_j = 0) and with mul entries
    only;
  * every launch shape the autotuner can pick (CTA width, whole pairs or
    shares, share size), set through the tuning table.
"""
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    import paper_2404_10404_b300 as S
    return S


def _check(S, oracle, circ):
    xb = synth.fr_bytes(synth.inputs_for(circ))
    gc = S.Circuit.from_spec(circ)
    proof = S.prove(gc, S.Eval(gc, xb))
    want = oracle.prove(circ, xb)
    assert proof == want, circ.name
    return gc, xb, proof


@pytest.mark.parametrize("C,widths,pct", [
    (1 << 17, [8, 16, 8], 60),     # 2^16 pairs in the first round: 222 a CTA, two chunks
    (1 << 12, [48, 37, 64], 70),   # padded widths, mul counts that split pairs between warps
    (8, [4096, 4096], 50),         # four pairs of 2048 mul entries: shares of a pair
    (2, [2048, 1024], 100),        # one pair, mul entries only
    (64, [512, 512, 256], 0),      # no mul entry: c_j = 0 in every round
])
def test_split_shapes(S, oracle, C, widths, pct):
    oracle.set_threads(16)
    try:
        _check(S, oracle, synth.uniform_circuit(11 * (1 << 32) + C + len(widths), C, widths, pct,
                                                name=f"copy_c_C{C}_W{widths[0]}"))
    finally:
        oracle.set_threads(1)


def test_every_launch_shape(S, oracle):
    from paper_2404_10404_b300 import tune
    spec = synth.uniform_circuit(11 * (1 << 32) + 99, 512, [256, 128, 256], 60, name="copy_c_shapes")
    classes = sorted(tune.classes_of([spec]))
    xb = synth.fr_bytes(synth.inputs_for(spec))
    want = oracle.prove(spec, xb)
    try:
        for bd in tune.CTA_THREADS:
            for form in tune.FORMS:
                for mi in tune.MIN_ITEMS:
                    for sn, lh in classes:
                        S.tune_copy_round(sn, lh, bd, form, mi * bd)
                    gc = S.Circuit.from_spec(spec)
                    assert S.prove(gc, S.Eval(gc, xb)) == want, (bd, form, mi)
    finally:
        tune.reset(classes)
