"""GPU associative hash (Sec. 3.4.1, Algorithm 1) and pairwise-distinct
check (Sec. 3.4.2, Algorithm 2) through the C ABI against the CPU oracle.

Hash values are field elements: compared byte for byte.  The check's answer
is an integer: compared exactly, with the oracle's answer and with the plain
meaning of the inputs (distinct or not)."""
import random

import numpy as np
import pytest

import synth
from gpu_util import to_device

pytestmark = pytest.mark.gpu

P = synth.FR_MODULUS


@pytest.fixture(scope="module")
def S():
    import paper_2404_10404_b300 as S
    return S


def _elems(seed, n):
    return synth.fr_bytes(synth.draw_fr_rows(seed, b"assoc", 1, n)[0]) if n else b""


@pytest.mark.parametrize("n", [0, 1, 31, 256, 257, 4095, 4097, 70001])
def test_hash_parity(S, oracle, n):
    x = _elems(n + 1, n)
    assert S.assoc_hash(x) == oracle.assoc_hash(x)
    if n:
        # the same values from device memory
        assert S.assoc_hash(to_device(x), n) == oracle.assoc_hash(x)


def test_hash_continuation(S, oracle):
    x = _elems(3, 5000)
    pre = oracle.assoc_hash(x[:32 * 1234])
    assert S.assoc_hash(x[32 * 1234:], h_pre=pre) == oracle.assoc_hash(x)
    assert S.assoc_hash(b"", 0, h_pre=pre) == pre
    edge = synth.fr_bytes(np.array([[0, 0, 0, 0], [(P - 1) & (2**64 - 1), (P - 1) >> 64 & (2**64 - 1),
                                                   (P - 1) >> 128 & (2**64 - 1), (P - 1) >> 192]], dtype=np.uint64))
    assert S.assoc_hash(edge) == oracle.assoc_hash(edge)


def test_segments(S, oracle):
    rng = random.Random(5)
    lens = [rng.choice([0, 0, 1, 7, 255, 256, 300, 4096, 5000]) for _ in range(120)]
    offs = np.concatenate([[0], np.cumsum(lens)]).astype(np.uint64)
    x = _elems(6, int(offs[-1]))
    pre = b"".join(oracle.assoc_hash(_elems(100 + g, 3)) for g in range(len(lens)))
    got = S.assoc_hash_segments(x, offs, h_pre=pre)
    got_dev = S.assoc_hash_segments(to_device(x), offs)
    for g in range(len(lens)):
        seg = x[32 * int(offs[g]):32 * int(offs[g + 1])]
        assert got[g] == oracle.assoc_hash(seg, pre[32 * g:32 * g + 32]), g
        assert got_dev[g] == oracle.assoc_hash(seg), g


def test_validator_indexes(S, oracle):
    idx = synth.validator_indexes(7, 100000, 20)
    x = synth.fr_bytes(idx)
    assert S.assoc_hash(x) == oracle.assoc_hash(x)
    # order independence: the sorted list hashes the same
    xs = synth.fr_bytes(idx[np.argsort(idx[:, 0], kind="stable")])
    assert S.assoc_hash(xs) == S.assoc_hash(x)


def _sorted(idx):
    return idx[np.argsort(idx[:, 0], kind="stable")]


def test_pairwise_distinct(S, oracle):
    idx = synth.validator_indexes(8, 50000, 22)
    a, s = synth.fr_bytes(idx), synth.fr_bytes(_sorted(idx))
    res, ha, hs = S.pairwise_distinct_check(a, s)
    assert res == 1 == oracle.pairwise_distinct_check(a, s)
    assert ha == hs == oracle.assoc_hash(a)
    res_dev, _, _ = S.pairwise_distinct_check(to_device(a), to_device(s), len(a) // 32)
    assert res_dev == 1
    # a repeated index: the sorted list has two equal neighbours
    dup = idx.copy()
    dup[-1] = dup[0]
    a2, s2 = synth.fr_bytes(dup), synth.fr_bytes(_sorted(dup))
    assert S.pairwise_distinct_check(a2, s2)[0] == 0 == oracle.pairwise_distinct_check(a2, s2)
    # a claimed sort that is not ascending (same multiset, same hash)
    bad = _sorted(idx).copy()
    bad[[100, 101]] = bad[[101, 100]]
    s3 = synth.fr_bytes(bad)
    r3, h3a, h3s = S.pairwise_distinct_check(a, s3)
    assert r3 == 0 == oracle.pairwise_distinct_check(a, s3) and h3a == h3s
    # an ascending list that is not a permutation of a (the last index moved up)
    other = _sorted(idx).copy()
    other[-1, 0] += 1
    s4 = synth.fr_bytes(other)
    r4, h4a, h4s = S.pairwise_distinct_check(a, s4)
    assert r4 == 0 == oracle.pairwise_distinct_check(a, s4) and h4a != h4s
    # chunk boundaries: an unordered pair straddling two chunks is seen
    n = 20000
    big = synth.validator_indexes(9, n, 24)
    srt = _sorted(big).copy()
    for k in (4095, 4096, 8191, n - 2):
        t = srt.copy()
        t[[k, k + 1]] = t[[k + 1, k]]
        assert S.pairwise_distinct_check(synth.fr_bytes(big), synth.fr_bytes(t))[0] == 0, k


def test_pairwise_segments(S, oracle):
    """Independent checks side by side (one per epoch or sub-circuit): each
    segment's answer and hashes equal the oracle's for that segment alone;
    a segment that starts below the previous one's last element is not
    unordered."""
    rng = random.Random(15)
    A, Srt, offs = [], [], [0]
    for g in range(40):
        n = rng.choice([0, 1, 2, 50, 4096, 5000])
        idx = synth.validator_indexes(200 + g, n, 16)
        srt = _sorted(idx).copy()
        kind = rng.randrange(4)
        if kind == 1 and n >= 2:      # a repeat
            idx[-1] = idx[0]
            srt = _sorted(idx).copy()
        elif kind == 2 and n >= 2:    # not ascending
            k = rng.randrange(n - 1)
            srt[[k, k + 1]] = srt[[k + 1, k]]
        elif kind == 3 and n >= 1:    # not a permutation
            srt[-1, 0] += 1 << 20
        A.append(idx)
        Srt.append(srt)
        offs.append(offs[-1] + n)
    a = synth.fr_bytes(np.concatenate(A)) if offs[-1] else b""
    s = synth.fr_bytes(np.concatenate(Srt)) if offs[-1] else b""
    res, ha, hs = S.pairwise_distinct_check_segments(a, s, offs)
    for g in range(40):
        ag, sg = a[32 * offs[g]:32 * offs[g + 1]], s[32 * offs[g]:32 * offs[g + 1]]
        assert res[g] == oracle.pairwise_distinct_check(ag, sg), g
        assert ha[g] == oracle.assoc_hash(ag) and hs[g] == oracle.assoc_hash(sg), g
    assert 0 < sum(res) < 40
    res_dev, _, _ = S.pairwise_distinct_check_segments(to_device(a), to_device(s), offs)
    assert res_dev == res


def test_pairwise_small_cases(S, oracle):
    assert S.pairwise_distinct_check(b"", b"")[0] == 1
    one = _elems(10, 1)
    assert S.pairwise_distinct_check(one, one)[0] == 1
    rng = random.Random(11)
    for trial in range(40):
        n = rng.randrange(1, 40)
        vals = [rng.randrange(20) for _ in range(n)]
        a = b"".join(v.to_bytes(32, "little") for v in vals)
        s = b"".join(v.to_bytes(32, "little") for v in sorted(vals))
        want = int(len(set(vals)) == n)
        assert S.pairwise_distinct_check(a, s)[0] == want == oracle.pairwise_distinct_check(a, s)


def test_errors(S):
    bad = (P).to_bytes(32, "little")
    good = _elems(12, 3)
    with pytest.raises(S.SisuError):
        S.assoc_hash(good + bad)
    with pytest.raises(S.SisuError):
        S.assoc_hash(good, h_pre=bad)
    with pytest.raises(S.SisuError):
        S.pairwise_distinct_check(good + bad, good + bad)
    t = to_device(good + bytes(16))
    with pytest.raises(S.SisuError):  # device arrays must be 16-byte aligned
        S.assoc_hash(t.data_ptr() + 8, 3)
    with pytest.raises(S.SisuError):  # offsets must not decrease
        S.assoc_hash_segments(good, [0, 2, 1, 3])


def test_full_size_sampled(S, oracle):
    """The benchmark workload (64 epochs x 2^20 indexes, one segment per slot
    of 32768): every segment hashed on the GPU; eight segments against the
    oracle, and all segments of the first epoch summed against the epoch's
    own hash (the sum form continues across segments)."""
    n, seg = 1 << 26, 1 << 15
    idx = synth.validator_indexes(13, n, 27)
    x = idx.tobytes()
    offs = np.arange(0, n + 1, seg, dtype=np.uint64)
    got = S.assoc_hash_segments(x, offs)
    rng = random.Random(14)
    for g in rng.sample(range(len(offs) - 1), 8):
        assert got[g] == oracle.assoc_hash(x[32 * g * seg:32 * (g + 1) * seg]), g
    epoch = sum(int.from_bytes(h, "little") for h in got[:32]) % P
    assert int.from_bytes(S.assoc_hash(x[:32 * (1 << 20)]), "little") == epoch


# ---------------------------------------------------------------------------
# the prover's sort (A* of Algorithm 2), against the plain definition

def _ints(b):
    return [int.from_bytes(b[i:i + 32], "little") for i in range(0, len(b), 32)]


@pytest.mark.parametrize("n", [1, 2, 255, 256, 257, 4096 + 13, 100000])
def test_sort_uniform_elements(S, n):
    x = _elems(300 + n, n)
    got, passes = S.sort_elements(x)
    assert _ints(got) == sorted(_ints(x))
    assert passes == (0 if n == 1 else 32)


def test_sort_validator_indexes_and_repeats(S):
    idx = synth.validator_indexes(17, 300000, 21)
    x = synth.fr_bytes(idx)
    got, passes = S.sort_elements(x)
    assert _ints(got) == sorted(_ints(x)) and passes == 3
    # repeats, an already sorted list, a reversed one, all equal
    vals = [v % 1000 for v in _ints(x)[:50000]]
    for case in (vals, sorted(vals), sorted(vals, reverse=True), [7] * 5000):
        b = b"".join(v.to_bytes(32, "little") for v in case)
        got, _ = S.sort_elements(b)
        assert _ints(got) == sorted(case)
    # device memory, in place
    t = to_device(x)
    S.sort_elements(t, t, len(idx))
    assert _ints(t[:len(x)].cpu().numpy().tobytes()) == sorted(_ints(x))


def test_sort_feeds_the_check(S):
    """The sorted list the prover produces is accepted by Algorithm 2, and a
    list with a repeat is rejected."""
    idx = synth.validator_indexes(18, 1 << 20, 21)
    a = synth.fr_bytes(idx)
    s, _ = S.sort_elements(a)
    assert S.pairwise_distinct_check(a, s)[0] == 1
    dup = idx.copy()
    dup[5] = dup[6]
    a2 = synth.fr_bytes(dup)
    s2, _ = S.sort_elements(a2)
    assert S.pairwise_distinct_check(a2, s2)[0] == 0


def test_sort_errors(S):
    with pytest.raises(S.SisuError):
        S.sort_elements(_elems(19, 3) + (P).to_bytes(32, "little"))
    assert S.sort_elements(b"")[0] == b""


def test_assoc_epochs(S, oracle):
    """Slot hashes and Algorithm 2 per epoch in one call: the slot hashes,
    every epoch's answer and both epoch hashes equal the oracle's on the
    same lists, for accepted epochs, repeats, unordered claims and claims
    that are not permutations; host and device inputs agree."""
    rng = random.Random(21)
    spe, nslots = 4, 24
    lens = [rng.choice([0, 1, 5, 300, 4096, 5000]) for _ in range(nslots)]
    offs = np.concatenate([[0], np.cumsum(lens)]).astype(np.uint64)
    A, Srt = [], []
    for e in range(nslots // spe):
        n = int(offs[(e + 1) * spe] - offs[e * spe])
        idx = synth.validator_indexes(300 + e, n, 20)
        srt = _sorted(idx).copy()
        kind = e % 4
        if kind == 1 and n >= 2:      # a repeat
            idx[-1] = idx[0]
            srt = _sorted(idx).copy()
        elif kind == 2 and n >= 2:    # not ascending
            k = rng.randrange(n - 1)
            srt[[k, k + 1]] = srt[[k + 1, k]]
        elif kind == 3 and n >= 1:    # not a permutation
            srt[-1, 0] += 1 << 21
        A.append(idx)
        Srt.append(srt)
    a, s = synth.fr_bytes(np.concatenate(A)), synth.fr_bytes(np.concatenate(Srt))
    sh, res, ha, hs = S.assoc_epochs(a, s, offs, spe)
    for g in range(nslots):
        assert sh[g] == oracle.assoc_hash(a[32 * int(offs[g]):32 * int(offs[g + 1])]), g
    for e in range(nslots // spe):
        lo, hi = int(offs[e * spe]), int(offs[(e + 1) * spe])
        ae, se = a[32 * lo:32 * hi], s[32 * lo:32 * hi]
        assert res[e] == oracle.pairwise_distinct_check(ae, se), e
        assert ha[e] == oracle.assoc_hash(ae) and hs[e] == oracle.assoc_hash(se), e
    assert 0 < sum(res) < nslots // spe
    assert S.assoc_epochs(to_device(a), to_device(s), offs, spe) == (sh, res, ha, hs)
    with pytest.raises(S.SisuError):  # the slots must make whole epochs
        S.assoc_epochs(a, s, offs, 5)


def test_assoc_epochs_errors(S):
    """Non-canonical elements in either list, and offsets that decrease,
    are refused; an empty epoch is accepted with the empty hash."""
    bad = (P).to_bytes(32, "little")
    good = _elems(22, 4)
    with pytest.raises(S.SisuError):
        S.assoc_epochs(good[:96] + bad, good, [0, 2, 4], 2)
    with pytest.raises(S.SisuError):
        S.assoc_epochs(good, good[:96] + bad, [0, 2, 4], 2)
    with pytest.raises(S.SisuError):
        S.assoc_epochs(good, good, [0, 3, 2, 4], 3)
    sh, res, ha, hs = S.assoc_epochs(b"", b"", [0, 0, 0], 2)
    assert res == [1] and ha == hs and sh[0] == sh[1] == ha[0]
