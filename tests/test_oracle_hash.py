"""Pins of the oracle's SHA-256 and statement digests.

SHA-256 is checked against the FIPS 180 example vectors (golden files with
their citations) and against ``hashlib``; the oracle derives its round
constants from the primes, and those are checked against the printed table.
The Merkle statement digest is a project convention (the paper fixes no
transcript), checked against the independent pure-Python implementation.
"""
import hashlib
import os
import random

import pytest

from oracle import brute

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _fips_vectors():
    out = []
    for line in open(os.path.join(GOLDEN, "sha256_fips180.txt")):
        if not line.strip() or line.startswith("#"):
            continue
        msg, dig = line.split()
        if msg == "empty":
            m = b""
        elif msg.startswith("repeat:"):
            _, byte, count = msg.split(":")
            m = bytes([int(byte, 16)]) * int(count)
        else:
            m = bytes.fromhex(msg)
        out.append((m, bytes.fromhex(dig)))
    return out


def test_fips_vectors(oracle):
    vecs = _fips_vectors()
    assert len(vecs) == 4
    for m, d in vecs:
        assert oracle.sha256(m) == d


def test_derived_constants_match_fips_table(oracle):
    k, h = oracle.sha256_constants()
    rows = [l.split() for l in open(os.path.join(GOLDEN, "sha256_constants.txt")) if l[:1] in "KH"]
    K = [int(x, 16) for r in rows if r[0] == "K" for x in r[1:]]
    H = [int(x, 16) for r in rows if r[0] == "H" for x in r[1:]]
    assert (k, h) == (K, H)


def test_random_lengths_match_hashlib(oracle):
    rng = random.Random(5)
    for n in list(range(0, 140)) + [rng.randrange(200, 5000) for _ in range(40)]:
        m = bytes(rng.getrandbits(8) for _ in range(n))
        assert oracle.sha256(m) == hashlib.sha256(m).digest(), n


@pytest.mark.parametrize("n", [0, 1, 31, 32, 1023, 1024, 1025, 2048, 3 * 1024 + 5, 5 * 1024, 9 * 1024 + 1])
def test_statement_digest_matches_independent(oracle, n):
    rng = random.Random(n)
    data = bytes(rng.getrandbits(8) for _ in range(n))
    assert oracle.statement_digest(data) == brute.digest(data)


def test_statement_digest_structure(oracle):
    # closed forms of the convention: empty input, one chunk, two chunks
    H = lambda *p: hashlib.sha256(b"".join(p)).digest()
    assert oracle.statement_digest(b"") == H(H(b"\x02"), (0).to_bytes(8, "little"), b"\x03")
    one = b"\x07" * 100
    assert oracle.statement_digest(one) == H(H(one, b"\x00"), (100).to_bytes(8, "little"), b"\x03")
    two = bytes(range(256)) * 5
    l0, l1 = H(two[:1024], b"\x00"), H(two[1024:], b"\x00")
    assert oracle.statement_digest(two) == H(H(l0, l1, b"\x01"), (1280).to_bytes(8, "little"), b"\x03")
    three = b"\x01" * 2500
    ls = [H(three[i:i + 1024], b"\x00") for i in (0, 1024, 2048)]
    root = H(H(ls[0], ls[1], b"\x01"), ls[2], b"\x01")
    assert oracle.statement_digest(three) == H(root, (2500).to_bytes(8, "little"), b"\x03")


def _sha256_by_compress(m: bytes) -> bytes:
    # FIPS 180-4 Sec. 5.1.1 padding, then the compression function block by block
    padded = m + b"\x80" + bytes(-(len(m) + 9) % 64) + (8 * len(m)).to_bytes(8, "big")
    h = b"".join(v.to_bytes(4, "big") for v in brute.SHA_IV)
    for i in range(0, len(padded), 64):
        h = brute.compress(h, padded[i:i + 64])
    return h


def test_python_compression_function_matches_hashlib():
    """The transcript's compression function (the pure-Python one; the C
    oracle's is pinned through its full SHA-256 above) chained over the
    FIPS padding is SHA-256."""
    rng = random.Random(9)
    for m, d in _fips_vectors():
        assert _sha256_by_compress(m) == d
    for n in list(range(0, 130)) + [rng.randrange(200, 3000) for _ in range(20)]:
        m = bytes(rng.getrandbits(8) for _ in range(n))
        assert _sha256_by_compress(m) == hashlib.sha256(m).digest(), n


def test_python_constants_match_fips_table():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "sha256_constants.txt")) if l[:1] in "KH"]
    assert brute.SHA_K == [int(x, 16) for r in rows if r[0] == "K" for x in r[1:]]
    assert brute.SHA_IV == [int(x, 16) for r in rows if r[0] == "H" for x in r[1:]]


def test_transcript_challenges_are_uniform_field_elements():
    """Every challenge is below r, consecutive challenges differ, and a
    different tag or element count changes the state."""
    t = brute.Transcript(None, 1, 2, [3, 3], b"\x01" * 32, b"\x02" * 32, b"\x03" * 32)
    seen = set()
    for i in range(200):
        if i % 3 == 0:
            t.absorb(b"R", [i, 2 * i])
        x = t.challenge()
        assert 0 <= x < brute.P and x not in seen
        seen.add(x)
    a = brute.Transcript(None, 1, 2, [3, 3], b"\x01" * 32, b"\x02" * 32, b"\x03" * 32)
    b = brute.Transcript(None, 1, 2, [3, 3], b"\x01" * 32, b"\x02" * 32, b"\x03" * 32)
    c = brute.Transcript(None, 1, 2, [3, 3], b"\x01" * 32, b"\x02" * 32, b"\x03" * 32)
    a.absorb(b"R", [5, 6])
    b.absorb(b"V", [5, 6])
    c.absorb(b"R", [5, 6, 0])
    assert len({a.st, b.st, c.st}) == 3
