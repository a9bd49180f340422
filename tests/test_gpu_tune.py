"""The copy round's autotuner: every candidate launch shape gives the same
proof (the tuner checks it), the chosen table is cached on disk per GPU and
reloads, and proofs under the tuned table equal the oracle's."""
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    import paper_2404_10404_b300 as S
    return S


def test_tune_cache_and_parity(S, oracle, tmp_path):
    from paper_2404_10404_b300 import tune
    spec = synth.uniform_circuit(31, 64, [128, 64, 128], 60, name="tuned")
    classes = sorted(tune.classes_of([spec]))
    assert (6, 5) in classes and (7, 0) in classes
    path = str(tmp_path / "copy_round.json")
    try:
        table = tune.tune(classes[:4], path, min_items=0)
        assert set(table) == set(classes[:4])
        for bd, form, mi in table.values():
            assert bd in tune.CTA_THREADS and form in tune.FORMS
        assert tune.load(path) == table
        # a second call finds every class cached and tunes nothing
        assert tune.tune(classes[:4], path, min_items=0) == table
        # classes below the item floor keep the default without being timed
        small = tune.tune(classes[4:], str(tmp_path / "small.json"))
        assert all(v == tune.DEFAULT_SHAPE for v in small.values())
        # every launch shape on every round of a fresh handle
        for bd in tune.CTA_THREADS:
            for form in tune.FORMS:
                for sn, lh in classes:
                    S.tune_copy_round(sn, lh, bd, form, 2 * bd)
                xb = synth.fr_bytes(synth.inputs_for(spec))
                gc = S.Circuit.from_spec(spec)
                assert S.prove(gc, S.Eval(gc, xb)) == oracle.prove(spec, xb), (bd, form)
    finally:
        tune.reset(classes)
    with pytest.raises(S.SisuError):
        S.tune_copy_round(6, 5, 300)
