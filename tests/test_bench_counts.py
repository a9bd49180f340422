"""Host-side counts of bench.py's roofline lines, checked by hand on small
circuits (no GPU): the copy phase's item-by-item product count is 2 + 4 f
products a (pair, gate) item plus one a folded row element, summed over
the copy rounds of every layer (C/2 + C/4 + ... + 1 pairs a layer)."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402
import synth  # noqa: E402


def _circuit(C, widths, types):
    d = len(widths) - 1
    z = [np.zeros(widths[i], np.uint32) for i in range(d)]
    return synth.Circuit(list(widths), [np.asarray(t, np.uint8) for t in types], z, z, C, name="counts")


BD = {"row_sums": {"ms": 0.25}, "copy_round": {"ms": 0.5}, "copy_fold": {"ms": 0.25}}


def test_one_layer_by_hand():
    # 4 copies: rounds of 2 and 1 pairs; 2 mul and 2 add gates over 4 inputs
    c = _circuit(4, [4, 4], [[1, 1, 0, 0]])
    r = bench.copy_phase_equivalent(c, BD, 10.0)
    assert r["item_by_item_products"] == 3 * (2 * 4 + 4 * 2) + 3 * 4
    assert r["ms_per_step"] == pytest.approx(1.0)
    assert r["achieved"] == pytest.approx(60 * 264 / 1e-3 / 1e12)
    assert r["frac_equivalent"] == pytest.approx(r["achieved"] / 10.0)


def test_layers_of_other_widths_and_mixes():
    # 8 copies (7 pairs over 3 rounds); layer 0: 2 gates, both mul, over 8
    # inputs; layer 1: 8 gates, 1 mul, over 4 inputs
    c = _circuit(8, [2, 8, 4], [[1, 1], [1, 0, 0, 0, 0, 0, 0, 0]])
    r = bench.copy_phase_equivalent(c, BD, 10.0)
    want = 7 * (2 * 2 + 4 * 2) + 7 * 8 + 7 * (2 * 8 + 4 * 1) + 7 * 4
    assert r["item_by_item_products"] == want


def test_one_copy_has_no_copy_phase():
    c = _circuit(1, [4, 4], [[1, 0, 1, 0]])
    assert bench.copy_phase_equivalent(c, BD, 10.0)["item_by_item_products"] == 0
    assert bench.copy_phase_equivalent(c, {k: {"ms": 0.0} for k in BD}, 10.0) is None


def test_step_count_by_hand():
    # 4 copies; layer 0: 2 mul + 2 add gates, layer 1: 4 add gates
    c = _circuit(4, [4, 4, 4], [[1, 1, 0, 0], [0, 0, 0, 0]])
    r = bench.step_equivalent(c, 2.0, 10.0)
    assert r["per_step_products"] == 4 * (3 * 4 + 5 * 2) + 4 * (3 * 4)
    assert r["achieved"] == pytest.approx(r["per_step_products"] * 264 / 2e-3 / 1e12)
    assert r["frac_equivalent"] == pytest.approx(r["achieved"] / 10.0)
    assert bench.step_equivalent(c, 0.0, 10.0) is None


def test_slot_counts_match_the_per_gate_formula():
    # the slot-shaped mixing layers alternate 100% and 40% mul: 3 + 5 f a gate
    c = synth.mixing_circuit(3, 8, 1024, 4)
    mul = sum(int(np.count_nonzero(np.asarray(t) == 1)) for t in c.types)
    gates = 8 * 1024 * 4
    r = bench.step_equivalent(c, 1.0, 1.0)
    assert r["per_step_products"] == 3 * gates + 5 * 8 * mul
    assert abs(mul / (1024 * 4) - 0.7) < 0.02
