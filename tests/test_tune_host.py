"""Host logic of the copy round's autotuner (no GPU): the classes a set of
circuits needs, and the on-disk cache read back per GPU name."""
import json

import pytest

import synth
from paper_2404_10404_b300 import tune


def test_classes_of_counts_every_copy_round():
    # 8 copies (rounds of 4, 2 and 1 pairs) over next layers of 16 and 8 gates
    c = synth.uniform_circuit(1, 8, [8, 16, 8], 50)
    assert tune.classes_of([c]) == {(4, 2), (4, 1), (4, 0), (3, 2), (3, 1), (3, 0)}
    # padded shapes: 5 copies pad to 8, a width of 9 to 16
    p = synth.uniform_circuit(2, 5, [4, 9], 50)
    assert tune.classes_of([p]) == {(4, 2), (4, 1), (4, 0)}
    # one copy: no copy round
    assert tune.classes_of([synth.uniform_circuit(3, 1, [4, 4], 50)]) == set()


def test_cache_is_read_per_gpu_name(tmp_path, monkeypatch):
    path = tmp_path / "copy_round.json"
    data = {"GPU A": {"table": {"10,14": [384, 1, 768], "12,9": [128, 1, 256]},
                      "timings_us": {"10,14": {"default": 534.7, "384,1,768": 506.0},
                                     "12,9": {"default": 190.5, "128,1,256": 163.7}}},
            "GPU B": {"table": {"10,14": [256, 0, 0]}, "timings_us": {}}}
    path.write_text(json.dumps(data))
    monkeypatch.setattr(tune, "_gpu_name", lambda: "GPU A")
    assert tune.load(str(path)) == {(10, 14): (384, 1, 768), (12, 9): (128, 1, 256)}
    assert tune.gains([(10, 14), (12, 9)], str(path)) == [pytest.approx(725.2), pytest.approx(669.7)]
    monkeypatch.setattr(tune, "_gpu_name", lambda: "GPU C")
    assert tune.load(str(path)) is None
    assert tune.gains([(10, 14)], str(path)) is None
    assert tune.load(str(tmp_path / "missing.json")) is None


def test_candidates_cover_the_table_of_shapes():
    cands = list(tune.candidates())
    assert len(cands) == 27 and len(set(cands)) == 27
    assert {c[0] for c in cands} == set(tune.CTA_THREADS)
    assert all(mi % bd == 0 for bd, _, mi in cands)
