"""Brute-force GKR prover and verifier in pure Python (TEST INFRASTRUCTURE ONLY).

This is the pin of the C oracle: an independent, exponential-time
implementation on Python integers and ``hashlib`` that shares no code with
``sisu_oracle.c``.  It runs the layer sumcheck of GKR (Sec. 2.2) as a
*generic* sumcheck over all variables (copy bits b, then x, then y) of

    f(b, x, y) = eq(z_b, b) * sum_g w(g) eq(x, in1 g) eq(y, in2 g) op_g(V~(b,x), V~(b,y)),

each round polynomial evaluated by enumerating every boolean value of the
still-free variables, and every multilinear extension evaluated as the
explicit sum  V~(p) = sum_j eq(p, bits(j)) V[j]  over the whole table.
Only micro circuits (a few hundred hypercube points) are feasible.

The transcript and proof conventions are the project's own (the paper fixes
none): Fiat-Shamir on the SHA-256 compression function, with statement
digests (full SHA-256) over 1024-byte chunks.  The compression function is
written out here from FIPS 180-4 and checked against ``hashlib``.
"""
from __future__ import annotations

import hashlib
import struct

P = 0x30644E72E131A029B85045B68181585D2833E84879B9709143E1F593F0000001
DOMAIN = b"SISU-GKR-v1"
CHUNK = 1024


def H(*parts: bytes) -> bytes:
    return hashlib.sha256(b"".join(parts)).digest()


def _iroot(n: int, k: int) -> int:
    """floor(n^(1/k)) for a non-negative integer n."""
    lo, hi = 0, 1 << (n.bit_length() // k + 1)
    while hi - lo > 1:
        mid = (lo + hi) // 2
        if mid ** k <= n:
            lo = mid
        else:
            hi = mid
    return lo


def _primes(n: int):
    out, v = [], 2
    while len(out) < n:
        if all(v % q for q in out if q * q <= v):
            out.append(v)
        v += 1
    return out


# FIPS 180-4 Sec. 4.2.2 and 5.3.3: the first 32 fraction bits of the cube
# roots of the first 64 primes and of the square roots of the first 8
_PR = _primes(64)
SHA_K = [_iroot(p << 96, 3) & 0xFFFFFFFF for p in _PR]
SHA_IV = [_iroot(p << 64, 2) & 0xFFFFFFFF for p in _PR[:8]]


def _rotr(x: int, n: int) -> int:
    return ((x >> n) | (x << (32 - n))) & 0xFFFFFFFF


def compress(h: bytes, block: bytes) -> bytes:
    """SHA-256 compression function (FIPS 180-4 Sec. 6.2.2, steps 1-4) of a
    32-byte chaining value (big-endian words) and one 64-byte block."""
    assert len(h) == 32 and len(block) == 64
    w = list(struct.unpack(">16I", block))
    for t in range(16, 64):
        s0 = _rotr(w[t - 15], 7) ^ _rotr(w[t - 15], 18) ^ (w[t - 15] >> 3)
        s1 = _rotr(w[t - 2], 17) ^ _rotr(w[t - 2], 19) ^ (w[t - 2] >> 10)
        w.append((w[t - 16] + s0 + w[t - 7] + s1) & 0xFFFFFFFF)
    hv = list(struct.unpack(">8I", h))
    a, b, c, d, e, f, g, hh = hv
    for t in range(64):
        S1 = _rotr(e, 6) ^ _rotr(e, 11) ^ _rotr(e, 25)
        ch = (e & f) ^ (~e & g)
        t1 = (hh + S1 + ch + SHA_K[t] + w[t]) & 0xFFFFFFFF
        S0 = _rotr(a, 2) ^ _rotr(a, 13) ^ _rotr(a, 22)
        maj = (a & b) ^ (a & c) ^ (b & c)
        hh, g, f, e, d, c, b, a = g, f, e, (d + t1) & 0xFFFFFFFF, c, b, a, (t1 + S0 + maj) & 0xFFFFFFFF
    return struct.pack(">8I", *[(x + y) & 0xFFFFFFFF for x, y in zip(hv, (a, b, c, d, e, f, g, hh))])


def digest(data: bytes) -> bytes:
    """Binary Merkle tree over 1024-byte chunks, then a length-binding hash."""
    if not data:
        root = H(b"\x02")
    else:
        level = [H(data[i:i + CHUNK], b"\x00") for i in range(0, len(data), CHUNK)]
        while len(level) > 1:
            nxt = [H(level[i], level[i + 1], b"\x01") for i in range(0, len(level) - 1, 2)]
            if len(level) % 2:
                nxt.append(level[-1])
            level = nxt
        root = level[0]
    return H(root, struct.pack("<Q", len(data)), b"\x03")


def fe(x: int) -> bytes:
    return (x % P).to_bytes(32, "little")


class Transcript:
    """State: a SHA-256 chaining value.  absorb tweaks it with the tag and
    the element count and compresses the elements 64 bytes at a time;
    the first challenge after an absorb reads the state itself, later ones
    compress a squeeze block first.  A challenge is x 2^-256 mod r for the
    state's low 254 bits x (rejected and squeezed again when x >= r)."""

    def __init__(self, domain, d, c, s, dig_w, dig_in, dig_out):
        dom = DOMAIN if domain is None else domain
        self.st = H(dom, b"\x00", struct.pack("<II", d, c),
                    b"".join(struct.pack("<I", v) for v in s), dig_w, dig_in, dig_out)
        self.fresh = True

    def absorb(self, tag: bytes, elems):
        msg = b"".join(fe(e) for e in elems)
        msg += bytes(-len(msg) % 64)
        tweak = 256 * tag[0] + len(elems)
        h = self.st[:28] + (int.from_bytes(self.st[28:], "big") ^ tweak).to_bytes(4, "big")
        for i in range(0, len(msg), 64):
            h = compress(h, msg[i:i + 64])
        self.st, self.fresh = h, True

    def _squeeze(self, ctr: int):
        self.st = compress(self.st, b"C" + struct.pack("<I", ctr) + bytes(59))

    def challenge(self) -> int:
        ctr = 0
        if not self.fresh:
            self._squeeze(ctr)
            ctr += 1
        self.fresh = False
        while True:
            x = int.from_bytes(self.st, "little") % (1 << 254)
            if x < P:
                return x * pow(2, -256, P) % P
            self._squeeze(ctr)
            ctr += 1


def log2_ceil(v: int) -> int:
    s = 0
    while (1 << s) < v:
        s += 1
    return s


class Padded:
    """Circuit padded to power-of-two widths and copy count.

    Layer i is a list of fan-in-2 entries (out, type, in1, in2): gate g's
    value is the sum of op(V(in1), V(in2)) over the entries with out = g
    (Sec. 3.4.3, accumulation gates); a plain gate is one entry and a
    padding gate has none."""

    def __init__(self, circ):
        self.d = circ.depth
        self.Creal = circ.n_copies
        self.c = log2_ceil(circ.n_copies)
        self.C = 1 << self.c
        self.wreal = list(circ.widths)
        self.s = [log2_ceil(w) for w in circ.widths]
        self.W = [1 << s for s in self.s]
        self.entries = []
        for i in range(self.d):
            outs = [int(o) for o in circ.layer_outs(i)]
            ent = [(o, int(t), int(a), int(b)) for o, t, a, b in zip(outs, circ.types[i], circ.in1[i], circ.in2[i])]
            self.entries.append(sorted(ent, key=lambda e: e[0]))  # stable: order within a gate kept

    def wiring_bytes(self) -> bytes:
        """Per padded gate: its one entry as u8 type || u32 in1 || u32 in2;
        no entry as (2, 0, 0); k >= 2 entries as u8 3 || u32 k || k records."""
        out = bytearray()
        for i in range(self.d):
            by_gate = [[] for _ in range(self.W[i])]
            for o, t, a, b in self.entries[i]:
                by_gate[o].append((t, a, b))
            for recs in by_gate:
                if not recs:
                    out += struct.pack("<BII", 2, 0, 0)
                elif len(recs) == 1:
                    out += struct.pack("<BII", *recs[0])
                else:
                    out += struct.pack("<BI", 3, len(recs))
                    for r in recs:
                        out += struct.pack("<BII", *r)
        return bytes(out)


def evaluate(pc: Padded, inputs):
    """inputs: ints, n_copies x widths[d] row-major. Returns padded layers."""
    d = pc.d
    V = [None] * (d + 1)
    V[d] = [0] * (pc.C * pc.W[d])
    for b in range(pc.Creal):
        for x in range(pc.wreal[d]):
            V[d][b * pc.W[d] + x] = inputs[b * pc.wreal[d] + x] % P
    for i in range(d - 1, -1, -1):
        V[i] = [0] * (pc.C * pc.W[i])
        for b in range(pc.C):
            row = V[i + 1][b * pc.W[i + 1]:(b + 1) * pc.W[i + 1]]
            for g, t, a1, a2 in pc.entries[i]:
                u, v = row[a1], row[a2]
                k = b * pc.W[i] + g
                V[i][k] = (V[i][k] + ((u + v) if t == 0 else u * v)) % P
    return V


def bits_msb(v: int, m: int):
    return [(v >> (m - 1 - k)) & 1 for k in range(m)]


def eq(p, q) -> int:
    acc = 1
    for a, b in zip(p, q):
        acc = acc * (a * b + (1 - a) * (1 - b)) % P
    return acc


def mle(table, point) -> int:
    """sum_j eq(point, bits(j)) table[j] (the first coordinate is the top bit)."""
    m = len(point)
    return sum(eq(point, bits_msb(j, m)) * table[j] for j in range(1 << m)) % P


def interpolate(g, x: int) -> int:
    n = len(g)
    acc = 0
    for i in range(n):
        num, den = 1, 1
        for j in range(n):
            if j != i:
                num = num * (x - j) % P
                den = den * (i - j) % P
        acc = (acc + g[i] * num * pow(den, P - 2, P)) % P
    return acc


def _layer_function(pc: Padded, i: int, V_next, zb, omega):
    """f(b, x, y) for layer i, as a function of a full point."""
    c, s = pc.c, pc.s[i + 1]
    gates = [(t, bits_msb(a1, s), bits_msb(a2, s), omega[g]) for g, t, a1, a2 in pc.entries[i]]
    memo = {}

    def Vt(point):
        key = tuple(point)
        if key not in memo:
            memo[key] = mle(V_next, point)
        return memo[key]

    def f(point):
        b, x, y = point[:c], point[c:c + s], point[c + s:]
        vx, vy = Vt(b + x), Vt(b + y)
        acc = 0
        for t, a1, a2, w in gates:
            op = (vx + vy) if t == 0 else vx * vy
            acc += w * eq(x, a1) * eq(y, a2) * op
        return eq(zb, b) * acc % P

    return f, Vt


def prove(circ, inputs, domain: bytes | None = None, check: bool = True,
          statement_inputs=None) -> bytes:
    """Proof bytes, every round polynomial by brute-force enumeration.

    ``statement_inputs`` (tests only) puts other inputs into the transcript's
    statement than the ones evaluated, which yields a proof that is
    consistent in every round but false at the input check.
    """
    pc = Padded(circ)
    d, c = pc.d, pc.c
    V = evaluate(pc, inputs)
    Vs = V[d] if statement_inputs is None else evaluate(pc, statement_inputs)[d]
    tr = Transcript(domain, d, c, pc.s, digest(pc.wiring_bytes()),
                    digest(b"".join(fe(v) for v in Vs)),
                    digest(b"".join(fe(v) for v in V[0])))
    out = bytearray(b"SISUGKR2" + struct.pack("<II", d, c) + b"".join(struct.pack("<I", v) for v in pc.s))
    zb = [tr.challenge() for _ in range(c)]
    zg = [tr.challenge() for _ in range(pc.s[0])]
    claim = mle(V[0], zb + zg)
    alpha = beta = None
    prx = pry = None
    for i in range(d):
        s = pc.s[i + 1]
        if i == 0:
            omega = [eq(zg, bits_msb(g, pc.s[0])) for g in range(pc.W[0])]
        else:
            omega = [(alpha * eq(prx, bits_msb(g, pc.s[i])) + beta * eq(pry, bits_msb(g, pc.s[i]))) % P
                     for g in range(pc.W[i])]
        f, Vt = _layer_function(pc, i, V[i + 1], zb, omega)
        nvars = c + 2 * s
        bound = []
        for k in range(nvars):
            nodes = 4 if k < c else 3
            rest = nvars - k - 1
            g = []
            for t in range(nodes):
                g.append(sum(f(bound + [t] + bits_msb(u, rest)) for u in range(1 << rest)) % P)
            if check:
                assert (g[0] + g[1]) % P == claim, f"layer {i} round {k}: g(0)+g(1) != claim"
            sent = [g[0]] + g[2:]  # g(1) = claim - g(0) is left to the verifier
            out += b"".join(fe(v) for v in sent)
            tr.absorb(b"R", sent)
            r = tr.challenge()
            claim = interpolate(g, r)
            bound.append(r)
        rb, rx, ry = bound[:c], bound[c:c + s], bound[c + s:]
        vx, vy = Vt(rb + rx), Vt(rb + ry)
        if check:
            assert claim == f(bound), f"layer {i}: final identity fails"
        out += fe(vx) + fe(vy)
        tr.absorb(b"V", [vx, vy])
        if i + 1 < d:
            alpha, beta = tr.challenge(), tr.challenge()
            claim = (alpha * vx + beta * vy) % P
            zb, prx, pry = rb, rx, ry
    return bytes(out)


def forge_one_layer(circ, inputs, fake_outputs, domain: bytes | None = None) -> bytes:
    """A proof for a one-layer circuit that claims ``fake_outputs``.

    Every round message is chosen so that g(0) + g(1) equals the running
    claim (g = [claim, 0, 0, ...]) and v_x, v_y are the true values of the
    input layer at the final point, so only the verifier's final per-layer
    identity can expose it.  Tests only.
    """
    pc = Padded(circ)
    assert pc.d == 1
    c, s = pc.c, pc.s[1]
    V = evaluate(pc, inputs)
    V0 = [0] * (pc.C * pc.W[0])
    for b in range(pc.Creal):
        for g in range(pc.wreal[0]):
            V0[b * pc.W[0] + g] = fake_outputs[b * pc.wreal[0] + g]
    tr = Transcript(domain, 1, c, pc.s, digest(pc.wiring_bytes()),
                    digest(b"".join(fe(v) for v in V[1])), digest(b"".join(fe(v) for v in V0)))
    out = bytearray(b"SISUGKR2" + struct.pack("<II", 1, c) + b"".join(struct.pack("<I", v) for v in pc.s))
    zb = [tr.challenge() for _ in range(c)]
    zg = [tr.challenge() for _ in range(pc.s[0])]
    claim = mle(V0, zb + zg)
    bound = []
    for k in range(c + 2 * s):
        g = [claim] + [0] * (3 if k < c else 2)  # g(1) = claim - g(0) = 0
        sent = [g[0]] + g[2:]
        out += b"".join(fe(v) for v in sent)
        tr.absorb(b"R", sent)
        r = tr.challenge()
        claim = interpolate(g, r)
        bound.append(r)
    rb, rx, ry = bound[:c], bound[c:c + s], bound[c + s:]
    vx, vy = mle(V[1], rb + rx), mle(V[1], rb + ry)
    out += fe(vx) + fe(vy)
    return bytes(out)


def forge_vy_one_layer(circ, inputs, domain: bytes | None = None) -> bytes:
    """A proof for a one-layer circuit whose v_y is false.

    The copy and x phases are honest; the y-phase messages are g = [claim,
    0, 0] and v_y is solved from the final per-layer identity (affine in
    v_y), so every check passes except the input check on v_y.  Tests only.
    """
    pc = Padded(circ)
    assert pc.d == 1
    c, s = pc.c, pc.s[1]
    V = evaluate(pc, inputs)
    tr = Transcript(domain, 1, c, pc.s, digest(pc.wiring_bytes()),
                    digest(b"".join(fe(v) for v in V[1])), digest(b"".join(fe(v) for v in V[0])))
    out = bytearray(b"SISUGKR2" + struct.pack("<II", 1, c) + b"".join(struct.pack("<I", v) for v in pc.s))
    zb = [tr.challenge() for _ in range(c)]
    zg = [tr.challenge() for _ in range(pc.s[0])]
    claim = mle(V[0], zb + zg)
    omega = [eq(zg, bits_msb(g, pc.s[0])) for g in range(pc.W[0])]
    f, Vt = _layer_function(pc, 0, V[1], zb, omega)
    nvars = c + 2 * s
    bound = []
    for k in range(nvars):
        if k < c + s:
            nodes, rest = (4 if k < c else 3), nvars - k - 1
            g = [sum(f(bound + [t] + bits_msb(u, rest)) for u in range(1 << rest)) % P for t in range(nodes)]
        else:
            g = [claim, 0, 0]
        sent = [g[0]] + g[2:]
        out += b"".join(fe(v) for v in sent)
        tr.absorb(b"R", sent)
        r = tr.challenge()
        claim = interpolate(g, r)
        bound.append(r)
    rb, rx, ry = bound[:c], bound[c:c + s], bound[c + s:]
    vx = Vt(rb + rx)
    e = eq(zb, rb)
    A = B = 0
    for g, t, a1, a2 in pc.entries[0]:
        w = omega[g] * eq(rx, bits_msb(a1, s)) * eq(ry, bits_msb(a2, s)) % P
        if t == 0:
            A, B = (A + w * vx) % P, (B + w) % P
        else:
            B = (B + w * vx) % P
    vy = (claim - e * A) * pow(e * B % P, P - 2, P) % P
    out += fe(vx) + fe(vy)
    return bytes(out)


# ---------------------------------------------------------------------------
# Associative hash (Sec. 3.4.1, Algorithm 1) and the pairwise-distinct check
# (Sec. 3.4.2, Algorithm 2) on Python integers.

ASSOC_ADD = 4294967295  # 2^32 - 1, the constant Algorithm 1 adds every round


def assoc_F(e: int) -> int:
    """Algorithm 1: from r = 0, three times r <- (r + e + 2^32 - 1)^3 mod p."""
    r = 0
    for _ in range(3):
        r = pow(r + e + ASSOC_ADD, 3, P)
    return r


def assoc_hash(elems, h_pre: int = 0) -> int:
    """h_pre + F(e_1) + ... + F(e_n) mod p (the sum form of Sec. 3.4.1)."""
    h = h_pre % P
    for e in elems:
        h = (h + assoc_F(e)) % P
    return h


def pairwise_distinct_check(A, A_sorted) -> int:
    """Algorithm 2: equal hashes, then a strictly ascending claimed sort."""
    if assoc_hash(A) != assoc_hash(A_sorted):
        return 0
    for i in range(1, len(A_sorted)):
        if A_sorted[i] <= A_sorted[i - 1]:
            return 0
    return 1

# ---------------------------------------------------------------------------
# General circuits (Sec. 2.7): the second input of a gate of layer i may come
# from any deeper layer j (i + 1 <= j <= d); the first input stays in layer
# i + 1.  Layer i's sumcheck runs over a virtual layer X_i: layer i + 1 in
# full (block 0), then, for each deeper layer j that layer i reads, only the
# gates of j it uses, in ascending order (the "used gates" indexing of Sec.
# 2.7: their indexes differ from their positions in layer j), padded to a
# power of two.  After the sumcheck the prover sends, for both final points
# r_x and r_y, the part of X~_i(r_b, r) carried by each block:
#     v_beta(r) = sum_{u in block beta} eq(r, u) X~_i(r_b, u),
# which are claims on the block's layer (a weighted sum of its values at copy
# point r_b).  A layer receives such claims from every layer that reads it;
# they are combined by random coefficients into one claim, each term keeping
# its own copy point:
#     sum_T sum_b eq(z_T, b) sum_g M_T(g) V_j(b, g),
#     M_T(g) = alpha_x eq(r_x, u(g)) + alpha_y eq(r_y, u(g))   (g used by T's block),
# which is the next layer sumcheck's starting claim.  The input layer's claims
# are checked against the clear inputs.  With every second input in layer
# i + 1 this is exactly the layered protocol above (one block, one term).

class GeneralPadded:
    """A general circuit padded to power-of-two widths and copy count, with
    the virtual layers X_i of its gate layers."""

    def __init__(self, circ):
        self.d = circ.depth
        self.Creal = circ.n_copies
        self.c = log2_ceil(circ.n_copies)
        self.C = 1 << self.c
        self.wreal = list(circ.widths)
        self.s = [log2_ceil(w) for w in circ.widths]
        self.W = [1 << s for s in self.s]
        self.gates, self.blocks, self.sx, self.u2 = [], [], [], []
        for i in range(self.d):
            srcs = [int(v) for v in circ.layer_src(i)]
            gates = [(g, int(t), int(a), int(j), int(b)) for g, (t, a, j, b) in
                     enumerate(zip(circ.types[i], circ.in1[i], srcs, circ.in2[i]))]
            blocks = [(i + 1, 0, list(range(self.W[i + 1])))]
            base = self.W[i + 1]
            for j in range(i + 2, self.d + 1):
                used = sorted({b for (_, _, _, jj, b) in gates if jj == j})
                if used:
                    blocks.append((j, base, used))
                    base += len(used)
            sx = log2_ceil(base)
            index = {}
            for j, b0, ys in blocks:
                for k, y in enumerate(ys):
                    index[(j, y)] = b0 + k
            self.gates.append(gates)
            self.blocks.append(blocks)
            self.sx.append(sx)
            self.u2.append([index[(j, b)] for (_, _, _, j, b) in gates])

    def wiring_bytes(self) -> bytes:
        """Per padded gate: u8 type || u32 in1 || u32 in2 when the second
        input is in layer i + 1, u8 (4 + type) || u32 in1 || u32 in2 ||
        u32 layer when it is deeper, (2, 0, 0) for a padding gate."""
        out = bytearray()
        for i in range(self.d):
            by_gate = {g: (t, a, j, b) for g, t, a, j, b in self.gates[i]}
            for g in range(self.W[i]):
                if g not in by_gate:
                    out += struct.pack("<BII", 2, 0, 0)
                    continue
                t, a, j, b = by_gate[g]
                out += struct.pack("<BII", t, a, b) if j == i + 1 else struct.pack("<BIII", 4 + t, a, b, j)
        return bytes(out)


def evaluate_general(pc: GeneralPadded, inputs):
    d = pc.d
    V = [None] * (d + 1)
    V[d] = [0] * (pc.C * pc.W[d])
    for b in range(pc.Creal):
        for x in range(pc.wreal[d]):
            V[d][b * pc.W[d] + x] = inputs[b * pc.wreal[d] + x] % P
    for i in range(d - 1, -1, -1):
        V[i] = [0] * (pc.C * pc.W[i])
        for b in range(pc.C):
            for g, t, a, j, y in pc.gates[i]:
                u, v = V[i + 1][b * pc.W[i + 1] + a], V[j][b * pc.W[j] + y]
                V[i][b * pc.W[i] + g] = ((u + v) if t == 0 else u * v) % P
    return V


def prove_general(circ, inputs, domain: bytes | None = None, check: bool = True) -> bytes:
    """Proof bytes of a general circuit, every round polynomial by
    brute-force enumeration over the hypercube."""
    pc = GeneralPadded(circ)
    d, c = pc.d, pc.c
    V = evaluate_general(pc, inputs)
    tr = Transcript(domain, d, c, pc.s, digest(pc.wiring_bytes()),
                    digest(b"".join(fe(v) for v in V[d])), digest(b"".join(fe(v) for v in V[0])))
    out = bytearray(b"SISUGKR2" + struct.pack("<II", d, c) + b"".join(struct.pack("<I", v) for v in pc.s))
    zb = [tr.challenge() for _ in range(c)]
    zg = [tr.challenge() for _ in range(pc.s[0])]
    # terms[j]: the combined claim on layer j as (copy point, gate weights)
    terms = {0: [(zb, [eq(zg, bits_msb(g, pc.s[0])) for g in range(pc.W[0])])]}
    claim = mle(V[0], zb + zg)
    claims = {j: 0 for j in range(d + 1)}
    for i in range(d):
        sx, WX = pc.sx[i], 1 << pc.sx[i]
        X = [0] * (pc.C * WX)
        for j, b0, ys in pc.blocks[i]:
            for k, y in enumerate(ys):
                for b in range(pc.C):
                    X[b * WX + b0 + k] = V[j][b * pc.W[j] + y]
        gates = [(g, t, bits_msb(a, sx), bits_msb(u, sx)) for (g, t, a, _, _), u in zip(pc.gates[i], pc.u2[i])]
        memo = {}

        def Xt(point):
            key = tuple(point)
            if key not in memo:
                memo[key] = mle(X, point)
            return memo[key]

        def f(point, gates=gates, layer_terms=terms[i], sx=sx):
            b, x, y = point[:c], point[c:c + sx], point[c + sx:]
            vx, vy = Xt(b + x), Xt(b + y)
            acc = 0
            for zt, M in layer_terms:
                part = 0
                for g, t, a1, a2 in gates:
                    op = (vx + vy) if t == 0 else vx * vy
                    part += M[g] * eq(x, a1) * eq(y, a2) * op
                acc += eq(zt, b) * part
            return acc % P

        if i > 0:
            claim = claims[i]
        nvars = c + 2 * sx
        bound = []
        for k in range(nvars):
            nodes = 4 if k < c else 3
            rest = nvars - k - 1
            g = [sum(f(bound + [t] + bits_msb(u, rest)) for u in range(1 << rest)) % P for t in range(nodes)]
            if check:
                assert (g[0] + g[1]) % P == claim, f"layer {i} round {k}: g(0)+g(1) != claim"
            sent = [g[0]] + g[2:]
            out += b"".join(fe(v) for v in sent)
            tr.absorb(b"R", sent)
            r = tr.challenge()
            claim = interpolate(g, r)
            bound.append(r)
        rb, rx, ry = bound[:c], bound[c:c + sx], bound[c + sx:]
        if check:
            assert claim == f(bound), f"layer {i}: final identity fails"
        col = [sum(eq(rb, bits_msb(b, c)) * X[b * WX + u] for b in range(pc.C)) % P for u in range(WX)]
        vb = {}
        for name, r in (("x", rx), ("y", ry)):
            vb[name] = [sum(eq(r, bits_msb(b0 + k, sx)) * col[b0 + k] for k in range(len(ys))) % P
                        for _, b0, ys in pc.blocks[i]]
            if check:
                assert sum(vb[name]) % P == Xt(rb + r)
        out += b"".join(fe(v) for v in vb["x"] + vb["y"])
        tr.absorb(b"V", vb["x"] + vb["y"])
        for beta, (j, b0, ys) in enumerate(pc.blocks[i]):
            if j == d:
                continue
            ax, ay = tr.challenge(), tr.challenge()
            M = [0] * pc.W[j]
            for k, y in enumerate(ys):
                M[y] = (ax * eq(rx, bits_msb(b0 + k, sx)) + ay * eq(ry, bits_msb(b0 + k, sx))) % P
            terms.setdefault(j, []).append((rb, M))
            claims[j] = (claims[j] + ax * vb["x"][beta] + ay * vb["y"][beta]) % P
    return bytes(out)
