"""Seeded synthetic workloads for the data-parallel GKR prover.

This module only draws random circuits and inputs; it holds none of the
prover's arithmetic.  Both the CPU oracle (under ``oracle/``) and the CUDA
library are fed from it, so the two see identical bytes.

Randomness
----------
Every stream is SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014).  SplitMix64 is counter based:
the k-th output (k = 0, 1, ...) of the stream with seed ``s`` is
``mix(s + (k + 1) * GAMMA)``, so whole streams are produced with vectorised
numpy code.  A stream is keyed by ``(seed, tag, i)``: its 64-bit seed is the
first 8 bytes (little endian) of ``SHA256(u64le(seed) || tag || u32le(i))``.

Field elements
--------------
An element of the BN254 scalar field (Sec. 4.1 of the paper picks BN254) is
drawn as four stream words forming a 256-bit little-endian integer; the top
two bits are cleared (value below 2^254) and the draw is rejected and
repeated when the value is not below the modulus r.  Elements are returned
as ``uint64[..., 4]`` limb arrays (little-endian); ``.tobytes()`` of such an
array is the canonical 32-byte little-endian encoding.

Circuits
--------
A circuit is a layered fan-in-2 arithmetic circuit (Sec. 2.2): layer 0 holds
the outputs, layer d the inputs, and gate g of layer i < d reads gates
``in1[g]`` and ``in2[g]`` of layer i + 1.  Gate type 0 is add, 1 is mul.  All
copies share the wiring (the data-parallel setting of Sec. 2.2).
"""
from __future__ import annotations

import hashlib
import struct
from dataclasses import dataclass, field

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
# BN254 scalar-field modulus, as little-endian 64-bit words (used only to
# reject out-of-range draws).
FR_MODULUS = 0x30644E72E131A029B85045B68181585D2833E84879B9709143E1F593F0000001
_MOD_WORDS = [(FR_MODULUS >> (64 * k)) & 0xFFFFFFFFFFFFFFFF for k in range(4)]


def stream_seed(seed: int, tag: bytes, i: int) -> int:
    """64-bit seed of the stream keyed by (seed, tag, i)."""
    h = hashlib.sha256(struct.pack("<Q", seed & 0xFFFFFFFFFFFFFFFF) + tag +
                       struct.pack("<I", i & 0xFFFFFFFF)).digest()
    return int.from_bytes(h[:8], "little")


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def splitmix_words(seeds, start: int, count: int) -> np.ndarray:
    """Words start .. start+count-1 of the streams with the given seeds.

    ``seeds`` is an int or a uint64 array of shape (n,); the result has shape
    (count,) or (n, count).
    """
    scalar = np.isscalar(seeds) or isinstance(seeds, int)
    s = np.atleast_1d(np.asarray(seeds, dtype=np.uint64))
    k = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = s[:, None] + k[None, :] * GAMMA
        out = _mix(z)
    return out[0] if scalar else out


def _below_modulus(w: np.ndarray) -> np.ndarray:
    """Lexicographic test (w3, w2, w1, w0) < r over the last axis."""
    less = np.zeros(w.shape[:-1], dtype=bool)
    equal = np.ones(w.shape[:-1], dtype=bool)
    for k in (3, 2, 1, 0):
        mk = np.uint64(_MOD_WORDS[k])
        less |= equal & (w[..., k] < mk)
        equal &= w[..., k] == mk
    return less


def draw_fr_rows(seed: int, tag: bytes, rows: int, width: int,
                 row_offset: int = 0) -> np.ndarray:
    """Uniform field elements, one stream per row: uint64[rows, width, 4]."""
    out = np.empty((rows, width, 4), dtype=np.uint64)
    chunk = max(1, (1 << 24) // max(1, width))  # bound the scratch per pass
    top_mask = np.uint64((1 << 62) - 1)
    for r0 in range(0, rows, chunk):
        r1 = min(rows, r0 + chunk)
        seeds = np.array([stream_seed(seed, tag, row_offset + r)
                          for r in range(r0, r1)], dtype=np.uint64)
        groups = int(width / 0.757 + 6.0 * np.sqrt(width) + 16)
        while True:
            w = splitmix_words(seeds, 0, 4 * groups).reshape(r1 - r0, groups, 4)
            w[..., 3] &= top_mask
            ok = _below_modulus(w)
            if (ok.sum(axis=1) >= width).all():
                break
            groups *= 2
        order = np.argsort(~ok, axis=1, kind="stable")[:, :width]
        out[r0:r1] = np.take_along_axis(w, order[:, :, None], axis=1)
    return out


@dataclass
class Circuit:
    """Layered circuit shared by ``n_copies`` copies.

    ``widths[i]`` is the number of gates of layer i (0 = outputs,
    d = inputs); ``types[i]``, ``in1[i]``, ``in2[i]`` describe layer i < d.
    Widths need not be powers of two: the prover pads (Sec. 2.2).

    Accumulation gates (Sec. 3.4.3): when ``outs`` is given and
    ``outs[i]`` is not None, layer i is a list of fan-in-2 entries:
    ``types[i]``, ``in1[i]``, ``in2[i]`` and ``outs[i]`` have one element
    per entry, and gate g's value is the sum over the entries with
    ``outs[i] == g`` (a gate with no entry is 0).

    General circuits (Sec. 2.7): when ``src`` is given and ``src[i]`` is
    not None, the second input of gate g of layer i is gate ``in2[i][g]``
    of layer ``src[i][g]`` (any layer below i: i + 1 .. d); the first input
    always comes from layer i + 1.
    """
    widths: list
    types: list
    in1: list
    in2: list
    n_copies: int
    name: str = ""
    seed: int = 0
    meta: dict = field(default_factory=dict)
    outs: list | None = None
    src: list | None = None

    def layer_src(self, i: int):
        """Layer of every entry's second input (i + 1 unless general)."""
        if self.src is not None and self.src[i] is not None:
            return np.asarray(self.src[i], dtype=np.uint32)
        return np.full(len(self.in1[i]), i + 1, dtype=np.uint32)

    @property
    def general(self) -> bool:
        return self.src is not None and any(
            s is not None and (np.asarray(s) != i + 1).any() for i, s in enumerate(self.src))

    def layer_outs(self, i: int):
        """Output gate of every entry of layer i (one entry per gate when plain)."""
        if self.outs is not None and self.outs[i] is not None:
            return np.asarray(self.outs[i], dtype=np.uint32)
        return np.arange(self.widths[i], dtype=np.uint32)

    @property
    def accumulates(self) -> bool:
        return self.outs is not None and any(o is not None for o in self.outs)

    @property
    def depth(self) -> int:
        return len(self.widths) - 1

    def gates_per_copy(self) -> int:
        return int(sum(self.widths[:-1]))

    def flat(self):
        """Concatenated (widths, types, in1, in2) arrays for C callers."""
        return (np.ascontiguousarray(self.widths, dtype=np.uint32),
                np.ascontiguousarray(np.concatenate(self.types), dtype=np.uint8),
                np.ascontiguousarray(np.concatenate(self.in1), dtype=np.uint32),
                np.ascontiguousarray(np.concatenate(self.in2), dtype=np.uint32))

    def flat_entries(self):
        """(widths, entries per layer, outs, types, in1, in2), concatenated."""
        outs = [self.layer_outs(i) for i in range(self.depth)]
        return (np.ascontiguousarray(self.widths, dtype=np.uint32),
                np.ascontiguousarray([len(o) for o in outs], dtype=np.uint32),
                np.ascontiguousarray(np.concatenate(outs), dtype=np.uint32),
                np.ascontiguousarray(np.concatenate(self.types), dtype=np.uint8),
                np.ascontiguousarray(np.concatenate(self.in1), dtype=np.uint32),
                np.ascontiguousarray(np.concatenate(self.in2), dtype=np.uint32))


def uniform_layer(seed: int, i: int, width: int, next_width: int, pct_mul: int):
    """Gate types (mul with probability pct_mul %) and uniform wiring."""
    u = splitmix_words(stream_seed(seed, b"wiring", i), 0, 3 * width).reshape(width, 3)
    hi = u >> np.uint64(32)
    types = (((hi[:, 0] * np.uint64(100)) >> np.uint64(32)) < np.uint64(pct_mul)).astype(np.uint8)
    in1 = ((hi[:, 1] * np.uint64(next_width)) >> np.uint64(32)).astype(np.uint32)
    in2 = ((hi[:, 2] * np.uint64(next_width)) >> np.uint64(32)).astype(np.uint32)
    return types, in1, in2


def mixing_layer(seed: int, i: int, width: int, pct_mul: int):
    """Hash-like mixing layer: in1 = pi(g), in2 = pi((g + rho) mod W).

    ``pi`` is a seeded Fisher-Yates permutation and ``rho`` a seeded odd
    offset, so every value of the next layer feeds exactly two gates.
    """
    u = splitmix_words(stream_seed(seed, b"perm", i), 0, width)
    perm = np.arange(width, dtype=np.int64)
    for k in range(width - 1, 0, -1):
        j = int((int(u[width - 1 - k]) >> 32) * (k + 1) >> 32)
        perm[k], perm[j] = perm[j], perm[k]
    w0 = int(splitmix_words(stream_seed(seed, b"rho", i), 0, 1)[0])
    half = max(1, width // 2)
    rho = (2 * (((w0 >> 32) * half) >> 32) + 1) % max(1, width)
    t = splitmix_words(stream_seed(seed, b"type", i), 0, width) >> np.uint64(32)
    types = (((t * np.uint64(100)) >> np.uint64(32)) < np.uint64(pct_mul)).astype(np.uint8)
    g = np.arange(width)
    in1 = perm[g].astype(np.uint32)
    in2 = perm[(g + rho) % width].astype(np.uint32)
    return types, in1, in2


def uniform_circuit(seed: int, n_copies: int, widths, pct_mul: int, name: str = "") -> Circuit:
    widths = [int(w) for w in widths]
    d = len(widths) - 1
    T, A, B = [], [], []
    for i in range(d):
        t, a, b = uniform_layer(seed, i, widths[i], widths[i + 1], pct_mul)
        T.append(t); A.append(a); B.append(b)
    return Circuit(widths, T, A, B, int(n_copies), name=name, seed=seed,
                   meta={"wiring": "uniform", "pct_mul": pct_mul})


def mixing_circuit(seed: int, n_copies: int, width: int, depth: int, name: str = "") -> Circuit:
    """Alternating 100 % mul (even layers) and 40 % mul (odd layers)."""
    T, A, B = [], [], []
    for i in range(depth):
        t, a, b = mixing_layer(seed, i, width, 100 if i % 2 == 0 else 40)
        T.append(t); A.append(a); B.append(b)
    return Circuit([width] * (depth + 1), T, A, B, int(n_copies), name=name, seed=seed,
                   meta={"wiring": "mixing", "pct_mul": 70})


def general_circuit(seed: int, n_copies: int, widths, pct_mul: int, pct_far: int, name: str = "") -> Circuit:
    """A general circuit (Sec. 2.7): uniform wiring and gate types as in
    uniform_circuit, and with probability pct_far % a gate's second input
    comes from a deeper layer than i + 1, drawn uniformly among layers
    i + 2 .. d (the gate in it uniform); the first input stays in i + 1."""
    widths = [int(w) for w in widths]
    d = len(widths) - 1
    T, A, B, R = [], [], [], []
    for i in range(d):
        t, a, b = uniform_layer(seed, i, widths[i], widths[i + 1], pct_mul)
        src = np.full(widths[i], i + 1, dtype=np.uint32)
        if i + 2 <= d:
            u = splitmix_words(stream_seed(seed, b"far", i), 0, 3 * widths[i]).reshape(widths[i], 3) >> np.uint64(32)
            far = ((u[:, 0] * np.uint64(100)) >> np.uint64(32)) < np.uint64(pct_far)
            layer = (i + 2 + ((u[:, 1] * np.uint64(d - i - 1)) >> np.uint64(32))).astype(np.uint32)
            src = np.where(far, layer, src).astype(np.uint32)
            wsrc = np.asarray(widths, dtype=np.uint64)[src]
            b = np.where(far, ((u[:, 2] * wsrc) >> np.uint64(32)).astype(np.uint32), b).astype(np.uint32)
        T.append(t); A.append(a); B.append(b); R.append(src)
    return Circuit(widths, T, A, B, int(n_copies), name=name, seed=seed,
                   meta={"wiring": "general", "pct_mul": pct_mul, "pct_far": pct_far}, src=R)


def inputs_for(circ: Circuit, seed: int | None = None) -> np.ndarray:
    """Uniform inputs, uint64[n_copies, widths[d], 4] (one stream per copy)."""
    s = circ.seed if seed is None else seed
    return draw_fr_rows(s, b"inputs", circ.n_copies, circ.widths[-1])


# ---------------------------------------------------------------------------
# Named workloads (the shapes of the paper's setting: many identical copies,
# about 32,000 per slot, Sec. 1 and Sec. 4.1).

def tiny() -> Circuit:
    """16 copies x 1024 wide x 8 layers, 50 % mul, uniform wiring (seed 1)."""
    return uniform_circuit(1, 16, [1024] * 9, 50, name="tiny_C16_W1024_d8")


def medium() -> Circuit:
    """1024 copies x 4096 wide x 20 layers, 50 % mul, uniform wiring (seed 2)."""
    return uniform_circuit(2, 1024, [4096] * 21, 50, name="medium_C1024_W4096_d20")


def slot() -> Circuit:
    """32768 copies x 1024 wide x 24 mixing layers, 70 % mul (seed 3)."""
    return mixing_circuit(3, 32768, 1024, 24, name="slot_C32768_W1024_d24")


def batched_instance(j: int) -> Circuit:
    """Instance j of the batched workload: C = 2^U{6..14}, W = 2^U{8..12},
    d = U{8..24}, 60 % mul, uniform wiring, seed 4 * 2^32 + j."""
    seed = 4 * (1 << 32) + j
    u = splitmix_words(stream_seed(seed, b"shape", 0), 0, 3) >> np.uint64(32)
    c = 6 + int((int(u[0]) * 9) >> 32)
    s = 8 + int((int(u[1]) * 5) >> 32)
    d = 8 + int((int(u[2]) * 17) >> 32)
    return uniform_circuit(seed, 1 << c, [1 << s] * (d + 1), 60,
                           name=f"batched_{j}_C{1 << c}_W{1 << s}_d{d}")


def micro(seed: int, n_copies: int, widths, pct_mul: int = 50) -> Circuit:
    return uniform_circuit(seed, n_copies, widths, pct_mul,
                           name=f"micro_s{seed}_C{n_copies}_W{'-'.join(map(str, widths))}")


def accumulation_circuit(seed: int, n_copies: int, widths, max_entries: int = 4, pct_mul: int = 50,
                         name: str = "") -> Circuit:
    """Layers of accumulation gates (Sec. 3.4.3) with uniform wiring: gate g
    of layer i gets U{0..max_entries} fan-in-2 entries (so some gates are
    plain, some are 0), each entry mul with probability pct_mul % and its two
    inputs uniform over layer i+1.  Entries are listed by gate."""
    d = len(widths) - 1
    types, in1, in2, outs = [], [], [], []
    for i in range(d):
        cnt = splitmix_words(stream_seed(seed, b"acc-count", i), 0, widths[i]) >> np.uint64(32)
        cnt = ((cnt * np.uint64(max_entries + 1)) >> np.uint64(32)).astype(np.int64)
        ne = int(cnt.sum())
        u = splitmix_words(stream_seed(seed, b"acc-wiring", i), 0, 3 * max(ne, 1)).reshape(-1, 3)[:ne]
        hi = u >> np.uint64(32)
        types.append((((hi[:, 0] * np.uint64(100)) >> np.uint64(32)) < np.uint64(pct_mul)).astype(np.uint8))
        in1.append(((hi[:, 1] * np.uint64(widths[i + 1])) >> np.uint64(32)).astype(np.uint32))
        in2.append(((hi[:, 2] * np.uint64(widths[i + 1])) >> np.uint64(32)).astype(np.uint32))
        outs.append(np.repeat(np.arange(widths[i], dtype=np.uint32), cnt))
    return Circuit(list(widths), types, in1, in2, n_copies,
                   name=name or f"acc_s{seed}_C{n_copies}_W{'-'.join(map(str, widths))}", seed=seed,
                   meta={"pct_mul": pct_mul, "wiring": f"accumulation, U{{0..{max_entries}}} entries a gate"},
                   outs=outs)


def validator_indexes(seed: int, n: int, log_universe: int) -> np.ndarray:
    """n distinct validator indexes below 2^log_universe (n <= 2^log_universe)
    in a seeded order, as field elements uint64[n, 4].

    The inputs of the associative hash and of the pairwise-distinct check
    (Sec. 3.4.1 and 3.4.2) are validator indexes, each below the number of
    active validators, distinct within an epoch.  Index j is
    (a j + b) mod 2^log_universe with a odd and b drawn from the stream
    (seed, b"idx", 0): a bijection, so the n indexes are distinct."""
    assert 0 <= n <= (1 << log_universe) and log_universe <= 62
    w = splitmix_words(np.array([stream_seed(seed, b"idx", 0)], dtype=np.uint64), 0, 2)[0]
    mask = np.uint64((1 << log_universe) - 1)
    a, b = (w[0] | np.uint64(1)) & mask | np.uint64(1), w[1] & mask
    j = np.arange(n, dtype=np.uint64)
    out = np.zeros((n, 4), dtype=np.uint64)
    with np.errstate(over="ignore"):
        out[:, 0] = (a * j + b) & mask
    return out


def fr_bytes(elems: np.ndarray) -> bytes:
    """Canonical little-endian bytes of a uint64[..., 4] element array."""
    return np.ascontiguousarray(elems, dtype="<u8").tobytes()


def fr_ints(elems: np.ndarray) -> list:
    """Python ints of a uint64[..., 4] element array (flattened)."""
    e = np.asarray(elems, dtype=np.uint64).reshape(-1, 4)
    return [int(a) | (int(b) << 64) | (int(c) << 128) | (int(d) << 192) for a, b, c, d in e]
