"""The C ABI's wiring validation on host-only circuits (no GPU): valid
circuits are accepted; every kind of invalid wiring returns its error code
(an input index beyond the next layer, an entry's gate beyond its layer, a
second input from a layer that is not below, a gate type other than add or
mul, zero copies, a zero width, no gate layer) instead of reading outside
the arrays.  Seeded random circuits and corruptions."""
import random

import numpy as np
import pytest

import synth

OK, INVALID_ARG, INDEX_OOB = 0, -1, -2


@pytest.fixture(scope="module")
def S():
    import paper_2404_10404_b300 as S
    if not __import__("os").path.exists(S.library_path()):
        pytest.skip("library not built")
    return S


def _code(S, spec, n_copies=None):
    try:
        S.Circuit.from_spec(spec, host_only=True, n_copies=n_copies)
    except S.SisuError as e:
        return e.code
    return OK


def _copy(c, **kw):
    f = dict(widths=list(c.widths), types=[np.array(t) for t in c.types], in1=[np.array(a) for a in c.in1],
             in2=[np.array(b) for b in c.in2], n_copies=c.n_copies, name=c.name,
             outs=None if c.outs is None else [None if o is None else np.array(o) for o in c.outs],
             src=None if c.src is None else [None if s is None else np.array(s) for s in c.src])
    f.update(kw)
    return synth.Circuit(**f)


def _shapes(n, seed):
    rng = random.Random(seed)
    return [(rng.randrange(1 << 30), rng.randint(1, 9), [rng.randint(1, 12) for _ in range(rng.randint(2, 5))])
            for _ in range(n)]


@pytest.mark.parametrize("seed,C,widths", _shapes(12, 5150))
def test_layered_wiring(S, seed, C, widths):
    c = synth.micro(seed, C, widths, 50)
    assert _code(S, c) == OK
    rng = random.Random(seed)
    i = rng.randrange(c.depth)
    g = rng.randrange(c.widths[i])
    for arr in ("in1", "in2"):
        bad = _copy(c)
        getattr(bad, arr)[i][g] = c.widths[i + 1] + rng.randrange(3)
        assert _code(S, bad) == INDEX_OOB
    bad = _copy(c)
    bad.types[i][g] = rng.randint(2, 255)
    assert _code(S, bad) == INVALID_ARG
    assert _code(S, c, n_copies=0) == INVALID_ARG
    w = rng.randrange(c.depth + 1)
    zero = _copy(c, widths=[0 if k == w else c.widths[k] for k in range(c.depth + 1)])
    if w < c.depth:
        zero.types[w] = zero.types[w][:0]
        zero.in1[w] = zero.in1[w][:0]
        zero.in2[w] = zero.in2[w][:0]
    assert _code(S, zero) in (INVALID_ARG, INDEX_OOB)
    assert _code(S, _copy(c, widths=[c.widths[0]], types=[], in1=[], in2=[])) == INVALID_ARG


@pytest.mark.parametrize("seed,C,widths", _shapes(8, 5151))
def test_accumulation_wiring(S, seed, C, widths):
    c = synth.accumulation_circuit(seed, C, widths, 3)
    assert _code(S, c) == OK
    rng = random.Random(seed)
    layers = [i for i in range(c.depth) if len(c.outs[i])]
    if not layers:
        pytest.skip("no entries drawn")
    i = rng.choice(layers)
    e = rng.randrange(len(c.outs[i]))
    bad = _copy(c)
    bad.outs[i][e] = c.widths[i] + rng.randrange(3)
    assert _code(S, bad) == INDEX_OOB
    bad = _copy(c)
    bad.in1[i][e] = c.widths[i + 1]
    assert _code(S, bad) == INDEX_OOB
    bad = _copy(c)
    bad.types[i][e] = 7
    assert _code(S, bad) == INVALID_ARG


@pytest.mark.parametrize("seed,C,widths", _shapes(8, 5152))
def test_general_wiring(S, seed, C, widths):
    if len(widths) < 3:
        widths = widths + [5]
    c = synth.general_circuit(seed, C, widths, 50, 50)
    assert _code(S, c) == OK
    rng = random.Random(seed)
    i = rng.randrange(c.depth)
    g = rng.randrange(c.widths[i])
    for j in (i, c.depth + 1 + rng.randrange(3)):  # not below layer i, or beyond the inputs
        bad = _copy(c)
        bad.src[i][g] = j
        assert _code(S, bad) == INDEX_OOB
    bad = _copy(c)
    j = int(bad.src[i][g])
    bad.in2[i][g] = c.widths[j]
    assert _code(S, bad) == INDEX_OOB
    bad = _copy(c)
    bad.types[i][g] = 2
    assert _code(S, bad) == INVALID_ARG
