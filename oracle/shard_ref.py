"""One rank of a copy-sharded proof, restated on Python integers (TEST
INFRASTRUCTURE ONLY: the tests drive it with the library's sharding driver
over gloo ranks and compare rank 0's proof with the one-rank proofs of
``sisu_oracle.c`` and ``brute.py``).

The distributed GKR of Sec. 3.2.1 splits the variables into machine bits
and local bits: each machine sums the round polynomial over its own part of
the hypercube, a master adds the parts, and once the local variables are
bound the master continues on a table with one entry per machine.  Here the
machine index is the low part of the copy index (rank q holds copies
b = j * world + q), so a rank's first c - log2(world) copy rounds bind its
own copy bits.  Per copy round k the rank's part is

    g_q(t) = sum_{j < h} E_t(j) sum_e w(out e) op_e(T_t(j, in1 e), T_t(j, in2 e)),

with T its copy rows folded by the challenges so far, E its copy weights
eq(z, j * world + q) folded alike, and X_t(j) = X(j) + t (X(j + h) - X(j));
the round polynomial is the sum of the parts.  After the local rounds rank
q's table is one row V~(r, q, .) with weight E(q); rank 0 takes the rows as
a table of ``world`` copies and finishes the layer: the remaining copy
rounds as above, then the x and y phases, each round polynomial summed over
the gates from its definition (no bookkeeping tables).

Exchange buffers are torch uint8 host tensors; the state buffer carries
rank 0's transcript and challenges to every rank after each layer.
"""
from __future__ import annotations

import pickle
import struct

from . import brute
from .brute import P, H, fe, eq, bits_msb

STATE_BYTES = 1 << 16


def _ints(t, n=None):
    b = t.numpy().tobytes()
    m = len(b) // 32 if n is None else n
    return [int.from_bytes(b[32 * i:32 * i + 32], "little") for i in range(m)]


def _put(t, vals):
    import torch
    b = b"".join(fe(v) for v in vals)
    t[:len(b)].copy_(torch.frombuffer(bytearray(b), dtype=torch.uint8))


def _merkle(leaves):
    """Root of a perfect binary tree over the leaf hashes."""
    while len(leaves) > 1:
        leaves = [H(leaves[i], leaves[i + 1], b"\x01") for i in range(0, len(leaves), 2)]
    return leaves[0]


def _copy_roots(table, C, W):
    """Per copy: the Merkle root over its row's 1 KiB chunks."""
    out = []
    for b in range(C):
        row = b"".join(fe(v) for v in table[b * W:(b + 1) * W])
        out.append(_merkle([H(row[i:i + brute.CHUNK], b"\x00") for i in range(0, len(row), brute.CHUNK)]))
    return out


def _fold(T, n, width, r):
    h = n // 2
    for j in range(h):
        for x in range(width):
            lo, hi = T[j * width + x], T[(j + h) * width + x]
            T[j * width + x] = (lo + r * (hi - lo)) % P


class OracleRank:
    """Rank ``rank`` of ``world`` for circuit ``spec`` (its inputs: the rows
    of copies j * world + rank, as ints)."""

    def __init__(self, spec, local_inputs, rank: int, world: int, domain: bytes | None = None):
        import torch

        self.rank, self.world, self.domain = rank, world, domain
        self.cq = world.bit_length() - 1
        assert 1 << self.cq == world and spec.n_copies % world == 0
        local = type("LocalSpec", (), {})()
        for a in ("widths", "types", "in1", "in2"):
            setattr(local, a, getattr(spec, a))
        local.n_copies = spec.n_copies // world
        local.depth = spec.depth
        local.layer_outs = spec.layer_outs
        self.pc = brute.Padded(local)
        pc = self.pc
        assert pc.C == pc.Creal, "no padded copies"
        self.V = brute.evaluate(pc, local_inputs)
        self.depth, self.local_rounds = pc.d, pc.c
        self.c = pc.c + self.cq
        self.wmax = max(pc.W[1:])
        n_local = pc.C
        sizes = {"roots_send": 64 * n_local, "roots_recv": 64 * n_local * world, "sums_send": 128,
                 "sums_recv": 128 * world, "row_send": 32 * (self.wmax + 1),
                 "row_recv": 32 * (self.wmax + 1) * world, "state": STATE_BYTES}
        self.bufs = {k: torch.zeros(v, dtype=torch.uint8) for k, v in sizes.items()}
        self.out = bytearray()

    def buf(self, name):
        return self.bufs[name]

    # statement and transcript ---------------------------------------------
    def roots(self, stream=None):
        pc = self.pc
        r_in = _copy_roots(self.V[pc.d], pc.C, pc.W[pc.d])
        r_out = _copy_roots(self.V[0], pc.C, pc.W[0])
        b = b"".join(r_in) + b"".join(r_out)
        import torch
        self.bufs["roots_send"][:len(b)].copy_(torch.frombuffer(bytearray(b), dtype=torch.uint8))

    def begin(self, stream=None):
        pc, N = self.pc, self.world
        raw = self.bufs["roots_recv"].numpy().tobytes()
        n = pc.C
        C = n * N
        r_in, r_out = [None] * C, [None] * C
        for q in range(N):
            part = raw[q * 64 * n:(q + 1) * 64 * n]
            for j in range(n):
                r_in[j * N + q] = part[32 * j:32 * j + 32]
                r_out[j * N + q] = part[32 * (n + j):32 * (n + j) + 32]
        dig_in = H(_merkle(r_in), struct.pack("<Q", C * pc.W[pc.d] * 32), b"\x03")
        dig_out = H(_merkle(r_out), struct.pack("<Q", C * pc.W[0] * 32), b"\x03")
        self.tr = brute.Transcript(self.domain, pc.d, self.c, pc.s, brute.digest(pc.wiring_bytes()), dig_in, dig_out)
        self.out = bytearray(b"SISUGKR2" + struct.pack("<II", pc.d, self.c) +
                             b"".join(struct.pack("<I", v) for v in pc.s))
        self.zb = [self.tr.challenge() for _ in range(self.c)]
        self.zg = [self.tr.challenge() for _ in range(pc.s[0])]
        self.rb, self.rx, self.ry, self.alpha, self.beta = [], [], [], None, None

    def _save_state(self):
        blob = pickle.dumps((self.tr.st, self.tr.fresh, self.rb, self.rx, self.ry, self.alpha, self.beta,
                             bytes(self.out)))
        import torch
        assert len(blob) + 4 <= STATE_BYTES
        self.bufs["state"][:4 + len(blob)].copy_(
            torch.frombuffer(bytearray(struct.pack("<I", len(blob)) + blob), dtype=torch.uint8))

    def _load_state(self):
        raw = self.bufs["state"].numpy().tobytes()
        n = struct.unpack("<I", raw[:4])[0]
        st, fresh, self.rb, self.rx, self.ry, self.alpha, self.beta, out = pickle.loads(raw[4:4 + n])
        self.tr.st, self.tr.fresh = st, fresh
        if self.rank != 0:  # rank 0's proof so far (the others' lack the finished parts)
            self.out = bytearray(out)

    # one layer ------------------------------------------------------------
    def layer_begin(self, i, stream=None):
        pc = self.pc
        if i > 0:
            self._load_state()
        self.layer = i
        W = pc.W[i]
        if i == 0:
            self.omega = [eq(self.zg, bits_msb(g, pc.s[0])) for g in range(W)]
            z = self.zb
        else:
            self.omega = [(self.alpha * eq(self.rx, bits_msb(g, pc.s[i])) +
                           self.beta * eq(self.ry, bits_msb(g, pc.s[i]))) % P for g in range(W)]
            z = self.rb
        self.E = [eq(z, bits_msb(j * self.world + self.rank, self.c)) for j in range(pc.C)]
        self.T = list(self.V[i + 1])
        self.n = pc.C
        self.rb = []

    def _round_sums(self, T, E, n):
        pc, i = self.pc, self.layer
        Wn, h = pc.W[i + 1], n // 2
        g = [0, 0, 0, 0]
        for j in range(h):
            for t in range(4):
                e = (E[j] + t * (E[j + h] - E[j])) % P
                lo, hi = T[j * Wn:(j + 1) * Wn], T[(j + h) * Wn:(j + h + 1) * Wn]
                S = 0
                for o, ty, a, b in pc.entries[i]:
                    u = lo[a] + t * (hi[a] - lo[a])
                    v = lo[b] + t * (hi[b] - lo[b])
                    S += self.omega[o] * ((u + v) if ty == 0 else u * v)
                g[t] = (g[t] + e * S) % P
        return g

    def _send(self, g, n):
        sent = [g[0]] + g[2:n]
        self.out += b"".join(fe(v) for v in sent)
        self.tr.absorb(b"R", sent)
        return self.tr.challenge()

    def copy_round(self, i, k, stream=None):
        _put(self.bufs["sums_send"], self._round_sums(self.T, self.E, self.n))

    def absorb(self, i, k, stream=None):
        parts = _ints(self.bufs["sums_recv"], 4 * self.world)
        g = [sum(parts[4 * q + t] for q in range(self.world)) % P for t in range(4)]
        r = self._send(g, 4)
        self.rb.append(r)
        _fold(self.T, self.n, self.pc.W[self.layer + 1], r)
        _fold(self.E, self.n, 1, r)
        self.n //= 2

    def row(self, i, stream=None):
        Wn = self.pc.W[i + 1]
        _put(self.bufs["row_send"], self.T[:Wn] + [self.E[0]])

    def finish(self, i, stream=None):
        pc, N = self.pc, self.world
        Wn, s = pc.W[i + 1], pc.s[i + 1]
        rows = _ints(self.bufs["row_recv"], N * (self.wmax + 1))
        T, E = [], []
        for q in range(N):
            part = rows[q * (self.wmax + 1):(q + 1) * (self.wmax + 1)]
            T += part[:Wn]
            E.append(part[Wn])
        n = N
        while n > 1:  # the remaining copy rounds, over one row a rank
            r = self._send(self._round_sums(T, E, n), 4)
            self.rb.append(r)
            _fold(T, n, Wn, r)
            _fold(E, n, 1, r)
            n //= 2
        A0, e = T[:Wn], E[0]
        ents = pc.entries[i]
        # phase over x: sum over the gates of w eq(r_x so far, in1 top bits)
        # eq1(t, bit k of in1) op(A_t(rest of in1), A0(in2)), times e
        A = list(A0)
        self.rx = []
        for k in range(s):
            m = 1 << (s - k)
            h = m // 2
            g = []
            for t in range(3):
                acc = 0
                for o, ty, a, b in ents:
                    pre = eq(self.rx, bits_msb(a >> (s - k), k)) if k else 1
                    bit = (a >> (s - 1 - k)) & 1
                    lo = a & (h - 1)
                    at = A[lo] + t * (A[lo + h] - A[lo])
                    op = (at + A0[b]) if ty == 0 else at * A0[b]
                    acc += self.omega[o] * pre * (t if bit else 1 - t) * op
                g.append(e * acc % P)
            r = self._send(g, 3)
            self.rx.append(r)
            _fold(A, m, 1, r)
        vx = A[0]
        # phase over y, with x bound to r_x
        A = list(A0)
        self.ry = []
        for k in range(s):
            m = 1 << (s - k)
            h = m // 2
            g = []
            for t in range(3):
                acc = 0
                for o, ty, a, b in ents:
                    pre = eq(self.rx, bits_msb(a, s)) * (eq(self.ry, bits_msb(b >> (s - k), k)) if k else 1)
                    bit = (b >> (s - 1 - k)) & 1
                    lo = b & (h - 1)
                    at = A[lo] + t * (A[lo + h] - A[lo])
                    op = (vx + at) if ty == 0 else vx * at
                    acc += self.omega[o] * pre * (t if bit else 1 - t) * op
                g.append(e * acc % P)
            r = self._send(g, 3)
            self.ry.append(r)
            _fold(A, m, 1, r)
        vy = A[0]
        self.out += fe(vx) + fe(vy)
        self.tr.absorb(b"V", [vx, vy])
        if i + 1 < pc.d:
            self.alpha, self.beta = self.tr.challenge(), self.tr.challenge()
        self._save_state()

    def proof(self, stream=None):
        return bytes(self.out)
