/*
 * Plain CPU oracle for the data-parallel GKR prover of Sisu (arXiv 2404.10404).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code with
 * the CUDA library: its field arithmetic, SHA-256, circuit evaluator, prover
 * and verifier are written here from the definitions, deliberately plain and
 * slow.
 *
 * What it computes (paper sections):
 *   - Field: the BN254 scalar field r (Sec. 4.1 picks BN254).  Elements are
 *     4 x 64-bit little-endian words in [0, r); products are reduced with
 *     Barrett's method (Handbook of Applied Cryptography, Alg. 14.42), unlike
 *     the Montgomery form the GPU uses.
 *   - Circuit: layer 0 = outputs ... layer d = inputs; gate g of layer i adds
 *     or multiplies gates in1(g), in2(g) of layer i+1 (Sec. 2.2, the layer
 *     relation V_i(g) = sum add_i(g,x,y)(V(x)+V(y)) + mult_i(g,x,y)V(x)V(y)).
 *     Widths are padded to powers of two with absent gates of value 0
 *     (Sec. 2.2 allows padding gates).  All copies share the wiring
 *     (data-parallel GKR, Sec. 2.2).
 *   - Prover: the GKR layer sumcheck (Sec. 2.2) over the variables
 *     (copy bits b, left input x, right input y), bound in that order, x and y
 *     forming Libra's two phases (Sec. 2.3).  Every round message is computed
 *     straight from its definition as a sum over gates of the layer
 *     polynomial
 *        P(b,x,y) = eq(z_b,b) * sum_g w(g) eq(x,in1 g) eq(y,in2 g)
 *                   * op_g(V~(b,x), V~(b,y)),
 *     summed over the boolean values of the variables not yet bound.  Partial
 *     evaluations of the multilinear extension V~ are obtained by folding the
 *     value table one variable at a time (the multilinear identity
 *     f(r, rest) = (1-r) f(0, rest) + r f(1, rest)).  No bookkeeping tables.
 *   - Verifier: checks g(0)+g(1) = claim every round (the round check of
 *     Sec. 3.2.1), the final per-layer identity by summing the wiring
 *     predicates over gates, the output claim from the clear outputs and the
 *     input claims from the clear inputs.
 *   - Associative hash (Sec. 3.4.1, Algorithm 1) and the pairwise-distinct
 *     check (Sec. 3.4.2, Algorithm 2), on the same field: F(e) starts from
 *     0 and three times replaces r by (r + e + 4294967295)^3; the hash of a
 *     list is the sum of F over it (the form Sec. 3.4.1 settles on), and
 *     the check compares the hashes of a list and of its claimed sorted
 *     permutation, then requires the latter strictly ascending.
 *   - Transcript: SHA-256 Fiat-Shamir; statement digests are binary Merkle
 *     trees over 1024-byte chunks.  The paper fixes neither: these are the
 *     project's conventions, pinned by the FIPS 180 vectors and by the
 *     independent hashlib-based implementation in brute.py.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Threads of the copy-phase sums, folds and evaluation (OpenMP over copy
 * pairs, rows and copies; 1 unless so_set_threads is called).  Field sums
 * are exact, so the result does not depend on the thread count. */
static int g_threads = 1;

typedef unsigned __int128 u128;

#define SO_OK 0
#define SO_ERR_ARG (-1)
#define SO_ERR_CANON (-2)
#define SO_ERR_REJECT (-3)
#define SO_ERR_OOM (-4)
#define SO_MAX_DEPTH 64

/* ------------------------------------------------------------------ */
/* Multi-word unsigned integers, little-endian 64-bit words.           */

static int mw_cmp(const uint64_t *a, const uint64_t *b, int n) {
    for (int i = n - 1; i >= 0; --i)
        if (a[i] != b[i]) return a[i] < b[i] ? -1 : 1;
    return 0;
}

static uint64_t mw_add(uint64_t *out, const uint64_t *a, const uint64_t *b, int n) {
    uint64_t carry = 0;
    for (int i = 0; i < n; ++i) {
        u128 s = (u128)a[i] + b[i] + carry;
        out[i] = (uint64_t)s;
        carry = (uint64_t)(s >> 64);
    }
    return carry;
}

static uint64_t mw_sub(uint64_t *out, const uint64_t *a, const uint64_t *b, int n) {
    uint64_t borrow = 0;
    for (int i = 0; i < n; ++i) {
        uint64_t ai = a[i], bi = b[i];
        uint64_t d = ai - bi - borrow;
        borrow = (ai < bi) || (ai == bi && borrow) ? 1 : 0;
        out[i] = d;
    }
    return borrow;
}

/* out[0 .. na+nb-1] = a * b (schoolbook). */
static void mw_mul(uint64_t *out, const uint64_t *a, int na, const uint64_t *b, int nb) {
    for (int i = 0; i < na + nb; ++i) out[i] = 0;
    for (int i = 0; i < na; ++i) {
        uint64_t carry = 0;
        for (int j = 0; j < nb; ++j) {
            u128 t = (u128)a[i] * b[j] + out[i + j] + carry;
            out[i + j] = (uint64_t)t;
            carry = (uint64_t)(t >> 64);
        }
        out[i + nb] = carry;
    }
}

/* ------------------------------------------------------------------ */
/* The field F_r, r the BN254 scalar-field modulus.                    */

typedef struct { uint64_t w[4]; } fr;

static const uint64_t MODW[4] = {0x43e1f593f0000001ULL, 0x2833e84879b97091ULL,
                                 0xb85045b68181585dULL, 0x30644e72e131a029ULL};
static uint64_t MU[5]; /* floor(2^512 / r), Barrett's constant */
static int mu_ready = 0;

/* floor(2^512 / r) by restoring long division, one bit at a time. */
static void init_mu(void) {
    uint64_t rem[5] = {0, 0, 0, 0, 0}, q[9] = {0};
    uint64_t mod5[5] = {MODW[0], MODW[1], MODW[2], MODW[3], 0};
    for (int pos = 512; pos >= 0; --pos) {
        /* rem = 2 * rem + (bit pos of 2^512) */
        for (int k = 4; k > 0; --k) rem[k] = (rem[k] << 1) | (rem[k - 1] >> 63);
        rem[0] = (rem[0] << 1) | (pos == 512 ? 1u : 0u);
        if (mw_cmp(rem, mod5, 5) >= 0) {
            mw_sub(rem, rem, mod5, 5);
            q[pos / 64] |= 1ULL << (pos % 64);
        }
    }
    for (int k = 0; k < 5; ++k) MU[k] = q[k];
    mu_ready = 1;
}

/* x mod r for x < 2^512 (8 words), HAC Alg. 14.42 with b = 2^64, k = 4. */
static fr fr_reduce512(const uint64_t x[8]) {
    uint64_t q2[10], q3[5], r2full[9], r1[5], r2[5], r[5];
    uint64_t mod5[5] = {MODW[0], MODW[1], MODW[2], MODW[3], 0};
    /* q1 = floor(x / b^(k-1)) = words 3..7 */
    mw_mul(q2, x + 3, 5, MU, 5);
    /* q3 = floor(q2 / b^(k+1)) = words 5..9 */
    for (int i = 0; i < 5; ++i) q3[i] = q2[5 + i];
    /* r1 = x mod b^(k+1), r2 = q3 * r mod b^(k+1) */
    for (int i = 0; i < 5; ++i) r1[i] = x[i];
    mw_mul(r2full, q3, 5, MODW, 4);
    for (int i = 0; i < 5; ++i) r2[i] = r2full[i];
    mw_sub(r, r1, r2, 5); /* wraps modulo b^(k+1) as the algorithm allows */
    while (mw_cmp(r, mod5, 5) >= 0) mw_sub(r, r, mod5, 5);
    fr out;
    for (int i = 0; i < 4; ++i) out.w[i] = r[i];
    return out;
}

static fr fr_zero(void) { fr z = {{0, 0, 0, 0}}; return z; }
static fr fr_u64(uint64_t v) { fr z = {{v, 0, 0, 0}}; return z; }
static int fr_eq(fr a, fr b) { return mw_cmp(a.w, b.w, 4) == 0; }

static fr fr_add(fr a, fr b) {
    fr s;
    mw_add(s.w, a.w, b.w, 4); /* a, b < r < 2^254: no carry out */
    if (mw_cmp(s.w, MODW, 4) >= 0) mw_sub(s.w, s.w, MODW, 4);
    return s;
}

static fr fr_sub(fr a, fr b) {
    fr d;
    if (mw_sub(d.w, a.w, b.w, 4)) mw_add(d.w, d.w, MODW, 4);
    return d;
}

static fr fr_mul(fr a, fr b) {
    uint64_t t[8];
    mw_mul(t, a.w, 4, b.w, 4);
    return fr_reduce512(t);
}

static fr fr_pow(fr a, const uint64_t e[4]) {
    fr acc = fr_u64(1);
    for (int i = 255; i >= 0; --i) {
        acc = fr_mul(acc, acc);
        if ((e[i / 64] >> (i % 64)) & 1) acc = fr_mul(acc, a);
    }
    return acc;
}

/* Fermat: a^(r-2) = a^-1 for a != 0 (returns 0 for 0). */
static fr fr_inv(fr a) {
    uint64_t e[4], two[4] = {2, 0, 0, 0};
    mw_sub(e, MODW, two, 4);
    return fr_pow(a, e);
}

/* eq1(a, b) = a b + (1 - a)(1 - b): the one-variable identity polynomial. */
static fr eq1(fr a, fr b) {
    fr one = fr_u64(1);
    return fr_add(fr_mul(a, b), fr_mul(fr_sub(one, a), fr_sub(one, b)));
}

static int fr_from_bytes(fr *out, const uint8_t *b) {
    for (int i = 0; i < 4; ++i) {
        uint64_t v = 0;
        for (int k = 7; k >= 0; --k) v = (v << 8) | b[8 * i + k];
        out->w[i] = v;
    }
    return mw_cmp(out->w, MODW, 4) < 0 ? SO_OK : SO_ERR_CANON;
}

static void fr_to_bytes(uint8_t *b, fr a) {
    for (int i = 0; i < 4; ++i)
        for (int k = 0; k < 8; ++k) b[8 * i + k] = (uint8_t)(a.w[i] >> (8 * k));
}

/* ------------------------------------------------------------------ */
/* SHA-256 (FIPS 180-4).  The round constants and initial hash value    */
/* are derived here from their definition: the first 32 bits of the    */
/* fractional parts of the cube roots of the first 64 primes, and of    */
/* the square roots of the first 8 primes.                              */

static uint32_t SHA_K[64], SHA_H0[8];
static int sha_ready = 0;

static uint64_t icbrt128(u128 n) { /* largest x with x^3 <= n, n < 2^105 */
    uint64_t lo = 0, hi = 1ULL << 36;
    while (hi - lo > 1) {
        uint64_t mid = lo + (hi - lo) / 2;
        if ((u128)mid * mid * mid <= n) lo = mid; else hi = mid;
    }
    return lo;
}

static uint64_t isqrt128(u128 n) { /* largest x with x^2 <= n, n < 2^70 */
    uint64_t lo = 0, hi = 1ULL << 36;
    while (hi - lo > 1) {
        uint64_t mid = lo + (hi - lo) / 2;
        if ((u128)mid * mid <= n) lo = mid; else hi = mid;
    }
    return lo;
}

static void sha_init_constants(void) {
    int found = 0;
    for (uint32_t p = 2; found < 64; ++p) {
        int prime = 1;
        for (uint32_t q = 2; q * q <= p; ++q)
            if (p % q == 0) { prime = 0; break; }
        if (!prime) continue;
        SHA_K[found] = (uint32_t)icbrt128((u128)p << 96);
        if (found < 8) SHA_H0[found] = (uint32_t)isqrt128((u128)p << 64);
        ++found;
    }
    sha_ready = 1;
}

typedef struct {
    uint32_t h[8];
    uint8_t buf[64];
    size_t buflen;
    uint64_t total;
} sha_ctx;

static uint32_t rotr(uint32_t x, int n) { return (x >> n) | (x << (32 - n)); }

static void sha_block(uint32_t h[8], const uint8_t blk[64]) {
    uint32_t w[64];
    for (int t = 0; t < 16; ++t)
        w[t] = ((uint32_t)blk[4 * t] << 24) | ((uint32_t)blk[4 * t + 1] << 16) |
               ((uint32_t)blk[4 * t + 2] << 8) | blk[4 * t + 3];
    for (int t = 16; t < 64; ++t) {
        uint32_t s0 = rotr(w[t - 15], 7) ^ rotr(w[t - 15], 18) ^ (w[t - 15] >> 3);
        uint32_t s1 = rotr(w[t - 2], 17) ^ rotr(w[t - 2], 19) ^ (w[t - 2] >> 10);
        w[t] = w[t - 16] + s0 + w[t - 7] + s1;
    }
    uint32_t a = h[0], b = h[1], c = h[2], d = h[3], e = h[4], f = h[5], g = h[6], hh = h[7];
    for (int t = 0; t < 64; ++t) {
        uint32_t S1 = rotr(e, 6) ^ rotr(e, 11) ^ rotr(e, 25);
        uint32_t ch = (e & f) ^ (~e & g);
        uint32_t t1 = hh + S1 + ch + SHA_K[t] + w[t];
        uint32_t S0 = rotr(a, 2) ^ rotr(a, 13) ^ rotr(a, 22);
        uint32_t maj = (a & b) ^ (a & c) ^ (b & c);
        uint32_t t2 = S0 + maj;
        hh = g; g = f; f = e; e = d + t1; d = c; c = b; b = a; a = t1 + t2;
    }
    h[0] += a; h[1] += b; h[2] += c; h[3] += d; h[4] += e; h[5] += f; h[6] += g; h[7] += hh;
}

static void sha_begin(sha_ctx *c) {
    if (!sha_ready) sha_init_constants();
    memcpy(c->h, SHA_H0, sizeof SHA_H0);
    c->buflen = 0;
    c->total = 0;
}

static void sha_update(sha_ctx *c, const uint8_t *p, size_t n) {
    c->total += n;
    while (n > 0) {
        size_t take = 64 - c->buflen;
        if (take > n) take = n;
        memcpy(c->buf + c->buflen, p, take);
        c->buflen += take; p += take; n -= take;
        if (c->buflen == 64) { sha_block(c->h, c->buf); c->buflen = 0; }
    }
}

static void sha_end(sha_ctx *c, uint8_t out[32]) {
    uint64_t bits = c->total * 8;
    uint8_t pad = 0x80, zero = 0, len[8];
    sha_update(c, &pad, 1);
    while (c->buflen != 56) sha_update(c, &zero, 1);
    for (int i = 0; i < 8; ++i) len[i] = (uint8_t)(bits >> (56 - 8 * i));
    sha_update(c, len, 8);
    for (int i = 0; i < 8; ++i) {
        out[4 * i] = (uint8_t)(c->h[i] >> 24); out[4 * i + 1] = (uint8_t)(c->h[i] >> 16);
        out[4 * i + 2] = (uint8_t)(c->h[i] >> 8); out[4 * i + 3] = (uint8_t)c->h[i];
    }
}

static void sha256(const uint8_t *p, size_t n, uint8_t out[32]) {
    sha_ctx c;
    sha_begin(&c);
    sha_update(&c, p, n);
    sha_end(&c, out);
}

/* ------------------------------------------------------------------ */
/* Statement digest: a binary Merkle tree over 1024-byte chunks.        */
/*   leaf = SHA256(chunk || 0x00)   (the last chunk may be short)       */
/*   node = SHA256(left || right || 0x01); an odd last node moves up    */
/*   empty input: root = SHA256(0x02)                                   */
/*   digest = SHA256(root || u64le(length) || 0x03)                     */

#define DIGEST_CHUNK 1024

static int statement_digest(const uint8_t *data, size_t len, uint8_t out[32]) {
    uint8_t root[32];
    if (len == 0) {
        uint8_t t = 0x02;
        sha256(&t, 1, root);
    } else {
        size_t n = (len + DIGEST_CHUNK - 1) / DIGEST_CHUNK;
        uint8_t *lvl = (uint8_t *)malloc(n * 32);
        if (!lvl) return SO_ERR_OOM;
        for (size_t i = 0; i < n; ++i) {
            size_t off = i * DIGEST_CHUNK, m = len - off < DIGEST_CHUNK ? len - off : DIGEST_CHUNK;
            sha_ctx c;
            uint8_t tag = 0x00;
            sha_begin(&c); sha_update(&c, data + off, m); sha_update(&c, &tag, 1);
            sha_end(&c, lvl + 32 * i);
        }
        while (n > 1) {
            size_t m = 0;
            for (size_t i = 0; i + 1 < n; i += 2) {
                uint8_t msg[65];
                memcpy(msg, lvl + 32 * i, 32);
                memcpy(msg + 32, lvl + 32 * (i + 1), 32);
                msg[64] = 0x01;
                uint8_t h[32];
                sha256(msg, 65, h);
                memcpy(lvl + 32 * m, h, 32);
                ++m;
            }
            if (n % 2) { memmove(lvl + 32 * m, lvl + 32 * (n - 1), 32); ++m; }
            n = m;
        }
        memcpy(root, lvl, 32);
        free(lvl);
    }
    uint8_t msg[41];
    memcpy(msg, root, 32);
    for (int i = 0; i < 8; ++i) msg[32 + i] = (uint8_t)((uint64_t)len >> (8 * i));
    msg[40] = 0x03;
    sha256(msg, 41, out);
    return SO_OK;
}

/* ------------------------------------------------------------------ */
/* Fiat-Shamir transcript (the paper fixes no hash; this is our reading).*/
/* The state st is a SHA-256 chaining value (32 bytes, big-endian        */
/* words) and F(h, B) is the SHA-256 compression function (FIPS 180-4    */
/* Sec. 6.2.2) of chaining value h and a 64-byte block B.                */
/*   init:      st = SHA256(domain || 0x00 || u32le d || u32le c ||     */
/*                          u32le s_0..s_d || Dig(wiring) ||            */
/*                          Dig(inputs) || Dig(outputs)); fresh         */
/*   absorb:    h = st with word 7 xor (256 tag + n); for every 64-byte */
/*              block B of the n canonical LE elements, zero-padded to  */
/*              a multiple of 64 bytes: h = F(h, B).  st = h; fresh     */
/*   challenge: ctr = 0; unless fresh: st = F(st, Q(ctr++)); then while */
/*              x = LE(st) mod 2^254 is not below r: st = F(st,         */
/*              Q(ctr++)).  Not fresh any more.  The challenge is       */
/*              x 2^-256 mod r (x read as a Montgomery form).           */
/*              Q(c) = 'C' || u32le c || 59 zero bytes.                 */

typedef struct { uint8_t st[32]; int fresh; } transcript;

static const char DEFAULT_DOMAIN[] = "SISU-GKR-v1";

static void put_u32(uint8_t *p, uint32_t v) {
    for (int i = 0; i < 4; ++i) p[i] = (uint8_t)(v >> (8 * i));
}

static void tr_init(transcript *t, const uint8_t *domain, size_t dlen, uint32_t d, uint32_t c,
                    const uint32_t *s, const uint8_t dw[32], const uint8_t di[32],
                    const uint8_t dout[32]) {
    sha_ctx h;
    uint8_t u[4], zero = 0;
    if (!domain) { domain = (const uint8_t *)DEFAULT_DOMAIN; dlen = strlen(DEFAULT_DOMAIN); }
    sha_begin(&h);
    sha_update(&h, domain, dlen);
    sha_update(&h, &zero, 1);
    put_u32(u, d); sha_update(&h, u, 4);
    put_u32(u, c); sha_update(&h, u, 4);
    for (uint32_t i = 0; i <= d; ++i) { put_u32(u, s[i]); sha_update(&h, u, 4); }
    sha_update(&h, dw, 32);
    sha_update(&h, di, 32);
    sha_update(&h, dout, 32);
    sha_end(&h, t->st);
    t->fresh = 1;
}

/* st = F(st, blk), with st as 32 big-endian bytes */
static void tr_compress(uint8_t st[32], const uint8_t blk[64]) {
    uint32_t h[8];
    for (int i = 0; i < 8; ++i)
        h[i] = ((uint32_t)st[4 * i] << 24) | ((uint32_t)st[4 * i + 1] << 16) |
               ((uint32_t)st[4 * i + 2] << 8) | st[4 * i + 3];
    sha_block(h, blk);
    for (int i = 0; i < 8; ++i) {
        st[4 * i] = (uint8_t)(h[i] >> 24); st[4 * i + 1] = (uint8_t)(h[i] >> 16);
        st[4 * i + 2] = (uint8_t)(h[i] >> 8); st[4 * i + 3] = (uint8_t)h[i];
    }
}

/* The most elements one absorb takes: a general circuit's layer end sends
 * two values for each of its blocks, at most one block per layer below it
 * (SO_MAX_DEPTH + 1); every other absorb takes at most three. */
#define SO_MAX_ABSORB (2 * (SO_MAX_DEPTH + 1))

static void tr_absorb(transcript *t, uint8_t tag, const fr *e, int n) {
    uint8_t msg[32 * SO_MAX_ABSORB + 32]; /* n elements, zero-padded to whole 64-byte blocks */
    size_t len = 32 * (size_t)n, nb = (len + 63) / 64;
    memset(msg, 0, 64 * nb);
    for (int i = 0; i < n; ++i) fr_to_bytes(msg + 32 * i, e[i]);
    t->st[30] ^= tag;           /* word 7 xor (256 tag + n) */
    t->st[31] ^= (uint8_t)n;
    for (size_t b = 0; b < nb; ++b) tr_compress(t->st, msg + 64 * b);
    t->fresh = 1;
}

/* 2^-256 mod r */
static fr r_inverse(void) {
    fr x = fr_u64(2);
    for (int i = 0; i < 8; ++i) x = fr_mul(x, x); /* 2^(2^8) */
    return fr_inv(x);
}

static void tr_squeeze(transcript *t, uint32_t ctr) {
    uint8_t q[64] = {0};
    q[0] = 'C';
    put_u32(q + 1, ctr);
    tr_compress(t->st, q);
}

static fr tr_challenge(transcript *t) {
    uint32_t ctr = 0;
    if (!t->fresh) tr_squeeze(t, ctr++);
    t->fresh = 0;
    for (;;) {
        uint8_t hm[32];
        for (int i = 0; i < 32; ++i) hm[i] = t->st[i];
        hm[31] &= 0x3f; /* mod 2^254 */
        fr x;
        if (fr_from_bytes(&x, hm) == SO_OK) return fr_mul(x, r_inverse());
        tr_squeeze(t, ctr++);
    }
}

/* ------------------------------------------------------------------ */
/* Circuits.  Gate layer i is a list of ne[i] fan-in-2 entries (out, type,*/
/* in1, in2), type 0 add or 1 mul, sorted by output gate: gate g's value  */
/* is the sum of op(V_{i+1}(in1), V_{i+1}(in2)) over its entries (Sec.    */
/* 3.4.3, accumulation gates).  A plain gate has one entry; a gate with   */
/* none, such as a padding gate, is 0.                                     */

typedef struct so_circuit {
    uint32_t d, c, C, Creal;
    uint32_t s[SO_MAX_DEPTH + 1], W[SO_MAX_DEPTH + 1], wreal[SO_MAX_DEPTH + 1];
    uint32_t ne[SO_MAX_DEPTH];
    uint32_t *out[SO_MAX_DEPTH];
    uint8_t *type[SO_MAX_DEPTH];
    uint32_t *in1[SO_MAX_DEPTH], *in2[SO_MAX_DEPTH];
    uint8_t wiring_digest[32];
} so_circuit;

static fr op_gate(uint8_t t, fr a, fr b) { return t == 0 ? fr_add(a, b) : fr_mul(a, b); }

static uint32_t ceil_log2(uint64_t v) {
    uint32_t s = 0;
    while ((1ULL << s) < v) ++s;
    return s;
}

void so_circuit_free(so_circuit *cc) {
    if (!cc) return;
    for (uint32_t i = 0; i < cc->d; ++i) {
        free(cc->out[i]); free(cc->type[i]); free(cc->in1[i]); free(cc->in2[i]);
    }
    free(cc);
}

/* Wiring bytes: for i = 0..d-1 and each padded gate g = 0..W_i-1 in turn,
 *   one entry:   u8 type || u32le in1 || u32le in2
 *   no entry:    u8 2 || u32le 0 || u32le 0         (a padding gate)
 *   k >= 2:      u8 3 || u32le k, then k times u8 type || u32le in1 || u32le in2
 * The first byte of a record tells which form follows. */
static int wiring_digest(so_circuit *cc) {
    size_t n = 0;
    for (uint32_t i = 0; i < cc->d; ++i) n += (size_t)cc->W[i] * 9 + (size_t)cc->ne[i] * 9;
    uint8_t *buf = (uint8_t *)malloc(n ? n : 1), *p = buf;
    if (!buf) return SO_ERR_OOM;
    for (uint32_t i = 0; i < cc->d; ++i) {
        uint32_t e = 0;
        for (uint32_t g = 0; g < cc->W[i]; ++g) {
            uint32_t e1 = e;
            while (e1 < cc->ne[i] && cc->out[i][e1] == g) ++e1;
            uint32_t k = e1 - e;
            if (k == 0) {
                *p++ = 2; put_u32(p, 0); p += 4; put_u32(p, 0); p += 4;
            } else if (k == 1) {
                *p++ = cc->type[i][e]; put_u32(p, cc->in1[i][e]); p += 4; put_u32(p, cc->in2[i][e]); p += 4;
            } else {
                *p++ = 3; put_u32(p, k); p += 4;
                for (uint32_t q = e; q < e1; ++q) {
                    *p++ = cc->type[i][q]; put_u32(p, cc->in1[i][q]); p += 4; put_u32(p, cc->in2[i][q]); p += 4;
                }
            }
            e = e1;
        }
    }
    int rc = statement_digest(buf, (size_t)(p - buf), cc->wiring_digest);
    free(buf);
    return rc;
}

/* Shared constructor: layer i gets cnt[i] entries (outs, types, in1, in2
 * concatenated over the layers), kept in order of output gate (stable). */
static so_circuit *circuit_from_entries(uint32_t d, const uint32_t *widths, const uint32_t *cnt,
                                        const uint32_t *outs, const uint8_t *types, const uint32_t *in1,
                                        const uint32_t *in2, uint32_t n_copies, int *err) {
    if (!mu_ready) init_mu();
    if (!sha_ready) sha_init_constants();
    *err = SO_ERR_ARG;
    if (d < 1 || d > SO_MAX_DEPTH || n_copies < 1 || !widths) return NULL;
    for (uint32_t i = 0; i <= d; ++i)
        if (widths[i] < 1 || widths[i] > (1u << 24)) return NULL;
    so_circuit *cc = (so_circuit *)calloc(1, sizeof *cc);
    if (!cc) { *err = SO_ERR_OOM; return NULL; }
    cc->d = d;
    cc->Creal = n_copies;
    cc->c = ceil_log2(n_copies);
    cc->C = 1u << cc->c;
    for (uint32_t i = 0; i <= d; ++i) {
        cc->wreal[i] = widths[i];
        cc->s[i] = ceil_log2(widths[i]);
        cc->W[i] = 1u << cc->s[i];
    }
    size_t off = 0;
    for (uint32_t i = 0; i < d; ++i) {
        uint32_t n = cnt[i];
        cc->d = i + 1; /* so that so_circuit_free releases what exists */
        cc->ne[i] = n;
        cc->out[i] = (uint32_t *)calloc(n ? n : 1, 4);
        cc->type[i] = (uint8_t *)calloc(n ? n : 1, 1);
        cc->in1[i] = (uint32_t *)calloc(n ? n : 1, 4);
        cc->in2[i] = (uint32_t *)calloc(n ? n : 1, 4);
        if (!cc->out[i] || !cc->type[i] || !cc->in1[i] || !cc->in2[i]) {
            so_circuit_free(cc); *err = SO_ERR_OOM; return NULL;
        }
        uint32_t k = 0;
        for (uint32_t g = 0; g < widths[i]; ++g) /* stable by output gate */
            for (uint32_t e = 0; e < n; ++e) {
                if (outs[off + e] >= widths[i]) { so_circuit_free(cc); return NULL; }
                if (outs[off + e] != g) continue;
                uint8_t t = types[off + e];
                uint32_t a = in1[off + e], b = in2[off + e];
                if (t > 1 || a >= widths[i + 1] || b >= widths[i + 1]) { so_circuit_free(cc); return NULL; }
                cc->out[i][k] = g; cc->type[i][k] = t; cc->in1[i][k] = a; cc->in2[i][k] = b;
                ++k;
            }
        off += n;
    }
    cc->d = d;
    if (wiring_digest(cc) != SO_OK) { so_circuit_free(cc); *err = SO_ERR_OOM; return NULL; }
    *err = SO_OK;
    return cc;
}

so_circuit *so_circuit_new_entries(uint32_t d, const uint32_t *widths, const uint32_t *cnt, const uint32_t *outs,
                                   const uint8_t *types, const uint32_t *in1, const uint32_t *in2,
                                   uint32_t n_copies, int *err) {
    *err = SO_ERR_ARG;
    if (!cnt || !outs || !types || !in1 || !in2) return NULL;
    return circuit_from_entries(d, widths, cnt, outs, types, in1, in2, n_copies, err);
}

so_circuit *so_circuit_new(uint32_t d, const uint32_t *widths, const uint8_t *types,
                           const uint32_t *in1, const uint32_t *in2, uint32_t n_copies, int *err) {
    /* one entry per gate: entry e of layer i belongs to gate e */
    *err = SO_ERR_ARG;
    if (d < 1 || d > SO_MAX_DEPTH || !widths) return NULL;
    size_t total = 0;
    uint32_t cnt[SO_MAX_DEPTH];
    for (uint32_t i = 0; i < d; ++i) { cnt[i] = widths[i]; total += widths[i]; }
    uint32_t *outs = (uint32_t *)malloc(total ? total * 4 : 4);
    if (!outs) { *err = SO_ERR_OOM; return NULL; }
    size_t off = 0;
    for (uint32_t i = 0; i < d; ++i)
        for (uint32_t g = 0; g < widths[i]; ++g) outs[off++] = g;
    so_circuit *cc = circuit_from_entries(d, widths, cnt, outs, types, in1, in2, n_copies, err);
    free(outs);
    return cc;
}

uint32_t so_circuit_log_copies(const so_circuit *cc) { return cc->c; }
uint32_t so_circuit_log_width(const so_circuit *cc, uint32_t i) { return cc->s[i]; }

size_t so_proof_len(const so_circuit *cc) {
    size_t n = 8 + 4 * ((size_t)cc->d + 3);
    for (uint32_t i = 0; i < cc->d; ++i) n += 32 * (3 * (size_t)cc->c + 4 * (size_t)cc->s[i + 1] + 2);
    return n;
}

/* Evaluate every layer: V[i] holds C * W_i elements, copy-major. */
static int eval_all(const so_circuit *cc, const uint8_t *inputs, fr **V) {
    uint32_t d = cc->d;
    for (uint32_t i = 0; i <= d; ++i) V[i] = NULL;
    for (uint32_t i = 0; i <= d; ++i) {
        V[i] = (fr *)calloc((size_t)cc->C * cc->W[i], sizeof(fr));
        if (!V[i]) return SO_ERR_OOM;
    }
    for (uint32_t b = 0; b < cc->Creal; ++b)
        for (uint32_t x = 0; x < cc->wreal[d]; ++x) {
            size_t src = (size_t)b * cc->wreal[d] + x;
            if (fr_from_bytes(&V[d][(size_t)b * cc->W[d] + x], inputs + 32 * src) != SO_OK)
                return SO_ERR_CANON;
        }
    for (int i = (int)d - 1; i >= 0; --i) {
        uint32_t W = cc->W[i], Wn = cc->W[i + 1];
#pragma omp parallel for num_threads(g_threads) schedule(static)
        for (uint32_t b = 0; b < cc->C; ++b) {
            const fr *in = V[i + 1] + (size_t)b * Wn;
            fr *out = V[i] + (size_t)b * W;
            for (uint32_t g = 0; g < W; ++g) out[g] = fr_zero();
            for (uint32_t e = 0; e < cc->ne[i]; ++e) /* each entry adds to its gate */
                out[cc->out[i][e]] = fr_add(out[cc->out[i][e]],
                                            op_gate(cc->type[i][e], in[cc->in1[i][e]], in[cc->in2[i][e]]));
        }
    }
    return SO_OK;
}

static void free_layers(fr **V, uint32_t n) {
    for (uint32_t i = 0; i < n; ++i) free(V[i]);
}

static int table_digest(const fr *T, size_t n, uint8_t out[32]) {
    uint8_t *buf = (uint8_t *)malloc(n ? n * 32 : 1);
    if (!buf) return SO_ERR_OOM;
    for (size_t i = 0; i < n; ++i) fr_to_bytes(buf + 32 * i, T[i]);
    int rc = statement_digest(buf, n * 32, out);
    free(buf);
    return rc;
}

/* bit m (1-based, most significant first) of an s-bit index */
static int bit_msb(uint32_t v, uint32_t s, uint32_t m) { return (int)((v >> (s - m)) & 1u); }

/* eq(r_1..r_s, v) = prod_m eq1(r_m, bit_m(v)) for an s-bit index v. */
static fr eq_point_index(const fr *r, uint32_t s, uint32_t v) {
    fr acc = fr_u64(1), one = fr_u64(1);
    for (uint32_t m = 1; m <= s; ++m)
        acc = fr_mul(acc, bit_msb(v, s, m) ? r[m - 1] : fr_sub(one, r[m - 1]));
    return acc;
}


/* MLE of a table of 2^m entries at point r (r_1 binds the top index bit). */
static fr mle_by_folding(const fr *T, uint32_t m, const fr *r) {
    size_t n = (size_t)1 << m;
    fr *w = (fr *)malloc(n * sizeof(fr));
    if (!w) return fr_zero();
    memcpy(w, T, n * sizeof(fr));
    for (uint32_t k = 0; k < m; ++k) {
        n /= 2;
        for (size_t j = 0; j < n; ++j) w[j] = fr_add(w[j], fr_mul(r[k], fr_sub(w[j + n], w[j])));
    }
    fr v = w[0];
    free(w);
    return v;
}

/* Lagrange interpolation through (0, g0), ..., (n-1, g_{n-1}) at x. */
static fr interpolate(const fr *g, int n, fr x) {
    fr acc = fr_zero();
    for (int i = 0; i < n; ++i) {
        fr num = fr_u64(1), den = fr_u64(1);
        for (int j = 0; j < n; ++j) {
            if (j == i) continue;
            num = fr_mul(num, fr_sub(x, fr_u64((uint64_t)j)));
            den = fr_mul(den, fr_sub(fr_u64((uint64_t)i), fr_u64((uint64_t)j)));
        }
        acc = fr_add(acc, fr_mul(g[i], fr_mul(num, fr_inv(den))));
    }
    return acc;
}

/* ------------------------------------------------------------------ */
/* Prover.                                                              */

typedef struct {
    uint8_t *buf;
    size_t len, cap;
} writer;

static void put_fr(writer *w, fr x) {
    if (w->len + 32 <= w->cap) fr_to_bytes(w->buf + w->len, x);
    w->len += 32;
}

static void put_hdr(writer *w, const so_circuit *cc) {
    static const char magic[8] = {'S', 'I', 'S', 'U', 'G', 'K', 'R', '2'};
    uint8_t u[4];
    if (w->cap >= 8) memcpy(w->buf, magic, 8);
    w->len = 8;
    put_u32(u, cc->d); if (w->len + 4 <= w->cap) memcpy(w->buf + w->len, u, 4); w->len += 4;
    put_u32(u, cc->c); if (w->len + 4 <= w->cap) memcpy(w->buf + w->len, u, 4); w->len += 4;
    for (uint32_t i = 0; i <= cc->d; ++i) {
        put_u32(u, cc->s[i]);
        if (w->len + 4 <= w->cap) memcpy(w->buf + w->len, u, 4);
        w->len += 4;
    }
}

/* Round k (1-based) of the copy phase for one layer.
 * T: the layer-(i+1) table folded by r_1..r_{k-1}: n rows of Wn values.
 * g(t) = sum_{j < n/2} eq(z_b, (r_1..r_{k-1}, t, bits(j)))
 *        * sum_g w(g) op_g(T_t(j, in1 g), T_t(j, in2 g)),
 * with T_t(j, x) = T(j, x) + t (T(j + n/2, x) - T(j, x)). */
static void copy_round(const so_circuit *cc, uint32_t i, const fr *T, size_t n, const fr *omega,
                       const fr *zb, const fr *rb, uint32_t k, fr out[4]) {
    uint32_t c = cc->c, Wn = cc->W[i + 1];
    size_t h = n / 2;
    fr prefix = fr_u64(1);
    for (uint32_t m = 1; m < k; ++m) prefix = fr_mul(prefix, eq1(zb[m - 1], rb[m - 1]));
    for (int t = 0; t < 4; ++t) out[t] = fr_zero();
#pragma omp parallel num_threads(g_threads)
    {
        fr part[4] = {fr_zero(), fr_zero(), fr_zero(), fr_zero()}; /* this thread's pairs */
        fr *row = (fr *)malloc(Wn * sizeof(fr));
#pragma omp for schedule(static)
        for (size_t j = 0; j < h; ++j) {
            fr suffix = fr_u64(1);
            for (uint32_t m = k + 1; m <= c; ++m)
                suffix = fr_mul(suffix, eq1(zb[m - 1], fr_u64((uint64_t)bit_msb((uint32_t)j, c - k, m - k))));
            for (int t = 0; t < 4; ++t) {
                fr tt = fr_u64((uint64_t)t);
                for (uint32_t x = 0; x < Wn; ++x) {
                    fr lo = T[j * Wn + x], hi = T[(j + h) * Wn + x];
                    row[x] = fr_add(lo, fr_mul(tt, fr_sub(hi, lo)));
                }
                fr S = fr_zero();
                for (uint32_t e = 0; e < cc->ne[i]; ++e) /* entry e weighs w(out e) */
                    S = fr_add(S, fr_mul(omega[cc->out[i][e]],
                                         op_gate(cc->type[i][e], row[cc->in1[i][e]], row[cc->in2[i][e]])));
                fr E = fr_mul(fr_mul(prefix, eq1(zb[k - 1], tt)), suffix);
                part[t] = fr_add(part[t], fr_mul(E, S));
            }
        }
        free(row);
#pragma omp critical
        for (int t = 0; t < 4; ++t) out[t] = fr_add(out[t], part[t]);
    }
}

static void fold_rows(fr *T, size_t n, uint32_t width, fr r) {
    size_t h = n / 2;
#pragma omp parallel for num_threads(g_threads) schedule(static) if (h * width >= 4096)
    for (size_t j = 0; j < h; ++j)
        for (uint32_t x = 0; x < width; ++x) {
            fr lo = T[j * width + x], hi = T[(j + h) * width + x];
            T[j * width + x] = fr_add(lo, fr_mul(r, fr_sub(hi, lo)));
        }
}

/* Phase over one gate input (Libra's phase 1 when which = 1, phase 2 when
 * which = 2), round k of s.  A is the row V~(r_b, .) folded by
 * r_1..r_{k-1} (size 2^(s-k+1)); A0 is the unfolded row; pre[g] holds
 * eq((r_1..r_{k-1}), top k-1 bits of the bound input of entry q) times,
 * in phase 2, eq(r_x, in1 q).  Sums run over the entries q (a plain gate
 * is one entry), each weighted by w of its output gate:
 * Phase 1: g(t) = e sum_q w(out q) pre(q) eq1(t, bit_k(in1 q))
 *                 * op_q(A_t(lo(in1 q)), A0(in2 q))
 * Phase 2: g(t) = e sum_q w(out q) pre(q) eq1(t, bit_k(in2 q))
 *                 * op_q(v_x, A_t(lo(in2 q))). */
static void gate_round(const so_circuit *cc, uint32_t i, int which, const fr *A, const fr *A0,
                       const fr *omega, const fr *pre, fr e, fr vx, uint32_t k, fr out[3]) {
    uint32_t s = cc->s[i + 1];
    size_t m = (size_t)1 << (s - k + 1), h = m / 2;
    uint32_t lomask = (uint32_t)(h - 1);
    for (int t = 0; t < 3; ++t) {
        fr tt = fr_u64((uint64_t)t), S = fr_zero();
        for (uint32_t q = 0; q < cc->ne[i]; ++q) {
            uint8_t ty = cc->type[i][q];
            uint32_t v = which == 1 ? cc->in1[i][q] : cc->in2[i][q];
            uint32_t lo = v & lomask;
            fr at = fr_add(A[lo], fr_mul(tt, fr_sub(A[lo + h], A[lo])));
            fr val = which == 1 ? op_gate(ty, at, A0[cc->in2[i][q]]) : op_gate(ty, vx, at);
            fr coeff = fr_mul(fr_mul(omega[cc->out[i][q]], pre[q]), eq1(tt, fr_u64((uint64_t)bit_msb(v, s, k))));
            S = fr_add(S, fr_mul(coeff, val));
        }
        out[t] = fr_mul(e, S);
    }
}

static void absorb_and_put(transcript *tr, writer *w, uint8_t tag, const fr *e, int n) {
    for (int t = 0; t < n; ++t) put_fr(w, e[t]);
    tr_absorb(tr, tag, e, n);
}

/* A round message: the round polynomial's values at t = 0, 2, ..., n - 1
 * (n = 4 in the copy phase, 3 in the x and y phases).  g(1) is left out:
 * the verifier takes it as claim - g(0), the sumcheck's own relation. */
static void send_round(transcript *tr, writer *w, const fr *g, int n) {
    fr sent[3];
    sent[0] = g[0];
    for (int t = 2; t < n; ++t) sent[t - 1] = g[t];
    absorb_and_put(tr, w, 'R', sent, n - 1);
}

int so_prove(const so_circuit *cc, const uint8_t *inputs, const uint8_t *domain, size_t dlen,
             uint8_t *proof, size_t cap, size_t *len_out) {
    uint32_t d = cc->d, c = cc->c;
    fr *V[SO_MAX_DEPTH + 1];
    int rc = eval_all(cc, inputs, V);
    if (rc != SO_OK) { free_layers(V, d + 1); return rc; }
    uint8_t dig_in[32], dig_out[32];
    table_digest(V[d], (size_t)cc->C * cc->W[d], dig_in);
    table_digest(V[0], (size_t)cc->C * cc->W[0], dig_out);
    transcript tr;
    tr_init(&tr, domain, dlen, d, c, cc->s, cc->wiring_digest, dig_in, dig_out);
    writer w = {proof, 0, cap};
    put_hdr(&w, cc);

    fr zb[32], zg[32], rb[32], rx[32], ry[32], alpha = fr_zero(), beta = fr_zero();
    for (uint32_t k = 0; k < c; ++k) zb[k] = tr_challenge(&tr);
    for (uint32_t k = 0; k < cc->s[0]; ++k) zg[k] = tr_challenge(&tr);

    for (uint32_t i = 0; i < d; ++i) {
        uint32_t W = cc->W[i], Wn = cc->W[i + 1], s = cc->s[i + 1];
        /* w(g): eq(z_g, g) for layer 0, else alpha eq(r_x, g) + beta eq(r_y, g)
         * with the previous layer's r_x, r_y (random combination of the two
         * claims, as in Libra). */
        fr *omega = (fr *)malloc(W * sizeof(fr));
        for (uint32_t g = 0; g < W; ++g)
            omega[g] = i == 0 ? eq_point_index(zg, cc->s[0], g)
                              : fr_add(fr_mul(alpha, eq_point_index(rx, cc->s[i], g)),
                                       fr_mul(beta, eq_point_index(ry, cc->s[i], g)));
        /* copy phase */
        size_t n = cc->C;
        fr *T = (fr *)malloc((size_t)cc->C * Wn * sizeof(fr));
        memcpy(T, V[i + 1], (size_t)cc->C * Wn * sizeof(fr));
        for (uint32_t k = 1; k <= c; ++k) {
            fr g4[4];
            copy_round(cc, i, T, n, omega, zb, rb, k, g4);
            send_round(&tr, &w, g4, 4);
            rb[k - 1] = tr_challenge(&tr);
            fold_rows(T, n, Wn, rb[k - 1]);
            n /= 2;
        }
        fr e = fr_u64(1);
        for (uint32_t m = 0; m < c; ++m) e = fr_mul(e, eq1(zb[m], rb[m]));
        /* A0 = V~(r_b, .), the copy-bound row */
        fr *A0 = (fr *)malloc(Wn * sizeof(fr)), *A = (fr *)malloc(Wn * sizeof(fr));
        uint32_t ne = cc->ne[i];
        fr *pre = (fr *)malloc((ne ? ne : 1) * sizeof(fr)); /* one per entry */
        memcpy(A0, T, Wn * sizeof(fr));
        /* phase over x */
        memcpy(A, A0, Wn * sizeof(fr));
        for (uint32_t q = 0; q < ne; ++q) pre[q] = fr_u64(1);
        for (uint32_t k = 1; k <= s; ++k) {
            fr g3[3];
            gate_round(cc, i, 1, A, A0, omega, pre, e, fr_zero(), k, g3);
            send_round(&tr, &w, g3, 3);
            rx[k - 1] = tr_challenge(&tr);
            fold_rows(A, (size_t)1 << (s - k + 1), 1, rx[k - 1]);
            for (uint32_t q = 0; q < ne; ++q)
                pre[q] = fr_mul(pre[q], eq1(rx[k - 1], fr_u64((uint64_t)bit_msb(cc->in1[i][q], s, k))));
        }
        fr vx = A[0];
        /* phase over y */
        memcpy(A, A0, Wn * sizeof(fr));
        for (uint32_t q = 0; q < ne; ++q) pre[q] = eq_point_index(rx, s, cc->in1[i][q]);
        for (uint32_t k = 1; k <= s; ++k) {
            fr g3[3];
            gate_round(cc, i, 2, A, A0, omega, pre, e, vx, k, g3);
            send_round(&tr, &w, g3, 3);
            ry[k - 1] = tr_challenge(&tr);
            fold_rows(A, (size_t)1 << (s - k + 1), 1, ry[k - 1]);
            for (uint32_t q = 0; q < ne; ++q)
                pre[q] = fr_mul(pre[q], eq1(ry[k - 1], fr_u64((uint64_t)bit_msb(cc->in2[i][q], s, k))));
        }
        fr vy = A[0];
        fr vv[2] = {vx, vy};
        absorb_and_put(&tr, &w, 'V', vv, 2);
        if (i + 1 < d) {
            alpha = tr_challenge(&tr);
            beta = tr_challenge(&tr);
            for (uint32_t k = 0; k < c; ++k) zb[k] = rb[k];
        }
        free(omega); free(T); free(A0); free(A); free(pre);
    }
    free_layers(V, d + 1);
    *len_out = w.len;
    return w.len <= cap ? SO_OK : SO_ERR_ARG;
}

/* ------------------------------------------------------------------ */
/* Verifier.                                                            */

typedef struct {
    const uint8_t *buf;
    size_t len, pos;
    int bad;
} reader;

static fr get_fr(reader *r) {
    fr x = fr_zero();
    if (r->pos + 32 > r->len) { r->bad = 1; return x; }
    if (fr_from_bytes(&x, r->buf + r->pos) != SO_OK) r->bad = 1;
    r->pos += 32;
    return x;
}

static int load_table(const so_circuit *cc, const uint8_t *bytes, uint32_t layer, fr **out) {
    size_t n = (size_t)cc->C * cc->W[layer];
    fr *T = (fr *)calloc(n, sizeof(fr));
    if (!T) return SO_ERR_OOM;
    for (uint32_t b = 0; b < cc->Creal; ++b)
        for (uint32_t x = 0; x < cc->wreal[layer]; ++x)
            if (fr_from_bytes(&T[(size_t)b * cc->W[layer] + x],
                              bytes + 32 * ((size_t)b * cc->wreal[layer] + x)) != SO_OK) {
                free(T);
                return SO_ERR_CANON;
            }
    *out = T;
    return SO_OK;
}

int so_verify(const so_circuit *cc, const uint8_t *inputs, const uint8_t *outputs,
              const uint8_t *proof, size_t len, const uint8_t *domain, size_t dlen) {
    uint32_t d = cc->d, c = cc->c;
    if (len != so_proof_len(cc)) return SO_ERR_REJECT;
    /* header */
    {
        uint8_t hdr[8 + 4 * (SO_MAX_DEPTH + 3)];
        writer w = {hdr, 0, sizeof hdr};
        put_hdr(&w, cc);
        if (memcmp(hdr, proof, w.len) != 0) return SO_ERR_REJECT;
    }
    reader rd = {proof, len, 8 + 4 * ((size_t)d + 3), 0};
    fr *Vin = NULL, *Vout = NULL;
    int rc = load_table(cc, inputs, d, &Vin);
    if (rc != SO_OK) return rc;
    rc = load_table(cc, outputs, 0, &Vout);
    if (rc != SO_OK) { free(Vin); return rc; }
    uint8_t dig_in[32], dig_out[32];
    table_digest(Vin, (size_t)cc->C * cc->W[d], dig_in);
    table_digest(Vout, (size_t)cc->C * cc->W[0], dig_out);
    transcript tr;
    tr_init(&tr, domain, dlen, d, c, cc->s, cc->wiring_digest, dig_in, dig_out);

    fr zb[32], zg[32], rb[32], rx[32], ry[32], prx[32], pry[32];
    fr alpha = fr_zero(), beta = fr_zero();
    fr pt[64];
    for (uint32_t k = 0; k < c; ++k) zb[k] = tr_challenge(&tr);
    for (uint32_t k = 0; k < cc->s[0]; ++k) zg[k] = tr_challenge(&tr);
    /* output claim V~_0(z_b, z_g) from the clear outputs */
    for (uint32_t k = 0; k < c; ++k) pt[k] = zb[k];
    for (uint32_t k = 0; k < cc->s[0]; ++k) pt[c + k] = zg[k];
    fr claim = mle_by_folding(Vout, c + cc->s[0], pt);
    int ok = 1;
    for (uint32_t i = 0; i < d && ok; ++i) {
        uint32_t s = cc->s[i + 1];
        /* each round: g(0), g(2)[, g(3)] from the proof, g(1) = claim - g(0) */
        for (uint32_t k = 0; k < c && ok; ++k) {
            fr g[4], sent[3];
            for (int t = 0; t < 3; ++t) sent[t] = get_fr(&rd);
            if (rd.bad) { ok = 0; break; }
            g[0] = sent[0]; g[2] = sent[1]; g[3] = sent[2];
            g[1] = fr_sub(claim, g[0]);
            tr_absorb(&tr, 'R', sent, 3);
            rb[k] = tr_challenge(&tr);
            claim = interpolate(g, 4, rb[k]);
        }
        for (int phase = 0; phase < 2 && ok; ++phase)
            for (uint32_t k = 0; k < s && ok; ++k) {
                fr g[3], sent[2];
                for (int t = 0; t < 2; ++t) sent[t] = get_fr(&rd);
                if (rd.bad) { ok = 0; break; }
                g[0] = sent[0]; g[2] = sent[1];
                g[1] = fr_sub(claim, g[0]);
                tr_absorb(&tr, 'R', sent, 2);
                fr r = tr_challenge(&tr);
                if (phase == 0) rx[k] = r; else ry[k] = r;
                claim = interpolate(g, 3, r);
            }
        if (!ok) break;
        fr vx = get_fr(&rd), vy = get_fr(&rd);
        if (rd.bad) { ok = 0; break; }
        /* final identity: claim = eq(z_b, r_b) sum_q w(out q) eq(r_x, in1 q)
         *                         eq(r_y, in2 q) op_q(v_x, v_y) over the entries q */
        fr e = fr_u64(1), sum = fr_zero();
        for (uint32_t m = 0; m < c; ++m) e = fr_mul(e, eq1(zb[m], rb[m]));
        for (uint32_t q = 0; q < cc->ne[i]; ++q) {
            uint8_t ty = cc->type[i][q];
            uint32_t g = cc->out[i][q];
            fr om = i == 0 ? eq_point_index(zg, cc->s[0], g)
                           : fr_add(fr_mul(alpha, eq_point_index(prx, cc->s[i], g)),
                                    fr_mul(beta, eq_point_index(pry, cc->s[i], g)));
            fr pred = fr_mul(eq_point_index(rx, s, cc->in1[i][q]), eq_point_index(ry, s, cc->in2[i][q]));
            sum = fr_add(sum, fr_mul(fr_mul(om, pred), op_gate(ty, vx, vy)));
        }
        if (!fr_eq(claim, fr_mul(e, sum))) { ok = 0; break; }
        fr vv[2] = {vx, vy};
        tr_absorb(&tr, 'V', vv, 2);
        if (i + 1 < d) {
            alpha = tr_challenge(&tr);
            beta = tr_challenge(&tr);
            claim = fr_add(fr_mul(alpha, vx), fr_mul(beta, vy));
            for (uint32_t k = 0; k < c; ++k) zb[k] = rb[k];
            for (uint32_t k = 0; k < s; ++k) { prx[k] = rx[k]; pry[k] = ry[k]; }
        } else {
            /* input check: v_x = V~_d(r_b, r_x), v_y = V~_d(r_b, r_y) */
            for (uint32_t k = 0; k < c; ++k) pt[k] = rb[k];
            for (uint32_t k = 0; k < s; ++k) pt[c + k] = rx[k];
            if (!fr_eq(vx, mle_by_folding(Vin, c + s, pt))) { ok = 0; break; }
            for (uint32_t k = 0; k < s; ++k) pt[c + k] = ry[k];
            if (!fr_eq(vy, mle_by_folding(Vin, c + s, pt))) { ok = 0; break; }
        }
    }
    if (rd.pos != rd.len) ok = 0;
    free(Vin);
    free(Vout);
    return ok ? SO_OK : SO_ERR_REJECT;
}

/* ------------------------------------------------------------------ */
/* Exported helpers (canonical 32-byte little-endian elements).         */

static void so_init(void) {
    if (!mu_ready) init_mu();
    if (!sha_ready) sha_init_constants();
}

/* Threads for the parallel loops of the prover (n >= 1); returns the
 * number in effect.  Without OpenMP the oracle stays single-threaded. */
int so_set_threads(int n) {
    so_init();
#ifdef _OPENMP
    g_threads = n < 1 ? 1 : n;
#else
    (void)n;
    g_threads = 1;
#endif
    return g_threads;
}

/* op: 0 add, 1 sub, 2 mul, 3 inverse (of a; 0 maps to 0), 4 eq1(a, b).
 * Returns SO_ERR_CANON if an operand is not below r. */
int so_fr_op(int op, const uint8_t *a, const uint8_t *b, uint8_t *out, size_t n) {
    so_init();
    for (size_t i = 0; i < n; ++i) {
        fr x, y = fr_zero(), z;
        if (fr_from_bytes(&x, a + 32 * i) != SO_OK) return SO_ERR_CANON;
        if (op != 3 && fr_from_bytes(&y, b + 32 * i) != SO_OK) return SO_ERR_CANON;
        switch (op) {
        case 0: z = fr_add(x, y); break;
        case 1: z = fr_sub(x, y); break;
        case 2: z = fr_mul(x, y); break;
        case 3: z = fr_inv(x); break;
        case 4: z = eq1(x, y); break;
        default: return SO_ERR_ARG;
        }
        fr_to_bytes(out + 32 * i, z);
    }
    return SO_OK;
}

/* x mod r of a 512-bit little-endian integer (64 bytes): exposes the
 * Barrett reduction alone for tests. */
void so_reduce512(const uint8_t *x64, uint8_t out[32]) {
    so_init();
    uint64_t x[8];
    for (int i = 0; i < 8; ++i) {
        uint64_t v = 0;
        for (int k = 7; k >= 0; --k) v = (v << 8) | x64[8 * i + k];
        x[i] = v;
    }
    fr_to_bytes(out, fr_reduce512(x));
}

void so_sha256(const uint8_t *msg, size_t n, uint8_t out[32]) {
    so_init();
    sha256(msg, n, out);
}

void so_sha256_constants(uint32_t k[64], uint32_t h0[8]) {
    so_init();
    memcpy(k, SHA_K, sizeof SHA_K);
    memcpy(h0, SHA_H0, sizeof SHA_H0);
}

int so_statement_digest(const uint8_t *data, size_t len, uint8_t out[32]) {
    so_init();
    return statement_digest(data, len, out);
}

/* Multilinear extension of a 2^m table at a point (r_1 binds the top bit). */
int so_mle(const uint8_t *table, uint32_t m, const uint8_t *point, uint8_t out[32]) {
    so_init();
    size_t n = (size_t)1 << m;
    fr *T = (fr *)malloc(n * sizeof(fr)), r[64];
    if (!T || m > 64) { free(T); return SO_ERR_ARG; }
    for (size_t i = 0; i < n; ++i)
        if (fr_from_bytes(&T[i], table + 32 * i) != SO_OK) { free(T); return SO_ERR_CANON; }
    for (uint32_t k = 0; k < m; ++k)
        if (fr_from_bytes(&r[k], point + 32 * k) != SO_OK) { free(T); return SO_ERR_CANON; }
    fr_to_bytes(out, mle_by_folding(T, m, r));
    free(T);
    return SO_OK;
}

/* Values of one layer (padded: 2^c copies x 2^s_layer gates, copy-major). */
int so_eval_layer(const so_circuit *cc, const uint8_t *inputs, uint32_t layer, uint8_t *out) {
    fr *V[SO_MAX_DEPTH + 1];
    if (layer > cc->d) return SO_ERR_ARG;
    int rc = eval_all(cc, inputs, V);
    if (rc == SO_OK) {
        size_t n = (size_t)cc->C * cc->W[layer];
        for (size_t j = 0; j < n; ++j) fr_to_bytes(out + 32 * j, V[layer][j]);
    }
    free_layers(V, cc->d + 1);
    return rc;
}

/* Real (unpadded) outputs, n_copies x widths[0], as the verifier takes them. */
int so_outputs(const so_circuit *cc, const uint8_t *inputs, uint8_t *out) {
    fr *V[SO_MAX_DEPTH + 1];
    int rc = eval_all(cc, inputs, V);
    if (rc == SO_OK)
        for (uint32_t b = 0; b < cc->Creal; ++b)
            for (uint32_t g = 0; g < cc->wreal[0]; ++g)
                fr_to_bytes(out + 32 * ((size_t)b * cc->wreal[0] + g), V[0][(size_t)b * cc->W[0] + g]);
    free_layers(V, cc->d + 1);
    return rc;
}

void so_wiring_digest(const so_circuit *cc, uint8_t out[32]) { memcpy(out, cc->wiring_digest, 32); }

/* ------------------------------------------------------------------ */
/* Associative hash (Sec. 3.4.1, Algorithm 1) and the pairwise-distinct */
/* check (Sec. 3.4.2, Algorithm 2).                                      */

/* Algorithm 1: r = 0, then three times r = (r + e + 4294967295)^3. */
static fr assoc_F(fr e) {
    const fr big = fr_u64(4294967295u);
    fr r = fr_zero();
    for (int i = 0; i < 3; ++i) {
        fr t = fr_add(fr_add(r, e), big);
        r = fr_mul(fr_mul(t, t), t);
    }
    return r;
}

/* F of every element of a list (n canonical elements in, n out). */
int so_assoc_F(const uint8_t *e, size_t n, uint8_t *out) {
    so_init();
    for (size_t i = 0; i < n; ++i) {
        fr x;
        if (fr_from_bytes(&x, e + 32 * i) != SO_OK) return SO_ERR_CANON;
        fr_to_bytes(out + 32 * i, assoc_F(x));
    }
    return SO_OK;
}

/* The associative hash of a list, AH = F(e_1) + ... + F(e_n) (the sum form
 * of Sec. 3.4.1), continued from h_pre (the running value H_pre of
 * Sec. 3.4.2; NULL stands for 0): out = h_pre + AH(list). */
int so_assoc_hash(const uint8_t *e, size_t n, const uint8_t *h_pre, uint8_t out[32]) {
    so_init();
    fr h = fr_zero();
    if (h_pre && fr_from_bytes(&h, h_pre) != SO_OK) return SO_ERR_CANON;
    for (size_t i = 0; i < n; ++i) {
        fr x;
        if (fr_from_bytes(&x, e + 32 * i) != SO_OK) return SO_ERR_CANON;
        h = fr_add(h, assoc_F(x));
    }
    fr_to_bytes(out, h);
    return SO_OK;
}

/* Algorithm 2 on lists A and A* of n elements each: 1 when AH(A) = AH(A*)
 * and A*_i > A*_(i-1) for i = 1 .. n-1 (as integers), else 0;
 * SO_ERR_CANON when an element is not below r. */
int so_pairwise_distinct_check(const uint8_t *A, const uint8_t *As, size_t n) {
    so_init();
    uint8_t h1[32], h2[32];
    int rc = so_assoc_hash(A, n, NULL, h1);
    if (rc != SO_OK) return rc;
    rc = so_assoc_hash(As, n, NULL, h2);
    if (rc != SO_OK) return rc;
    if (memcmp(h1, h2, 32) != 0) return 0;
    for (size_t i = 1; i < n; ++i) {
        fr prev, cur;
        fr_from_bytes(&prev, As + 32 * (i - 1));
        fr_from_bytes(&cur, As + 32 * i);
        if (mw_cmp(cur.w, prev.w, 4) <= 0) return 0;
    }
    return 1;
}

/* ------------------------------------------------------------------ */
/* General circuits (Sec. 2.7).  The second input of a gate of layer i   */
/* may come from any deeper layer j (i + 1 <= j <= d); the first input    */
/* stays in layer i + 1.  Layer i's sumcheck runs over a virtual layer    */
/* X_i: layer i + 1 in full (block 0), then, for each deeper layer j that */
/* layer i reads, only the gates of j it uses, ascending (the "used       */
/* gates" indexing of Sec. 2.7), padded to a power of two.  After the     */
/* rounds the prover sends, for r = r_x and r = r_y, the part of          */
/* X~_i(r_b, r) that each block carries,                                  */
/*     v_beta(r) = sum_{u in block beta} eq(r, u) X~_i(r_b, u),          */
/* a claim on the block's layer.  A layer's claims from every reader are  */
/* combined by random coefficients, each term keeping its own copy point: */
/*     sum_T sum_b eq(z_T, b) sum_g M_T(g) V_j(b, g),                     */
/*     M_T(g) = alpha_x eq(r_x, u(g)) + alpha_y eq(r_y, u(g)),            */
/* which starts the next layer's sumcheck; the copy rounds sum the terms. */
/* The input layer's claims are checked against the clear inputs.  With  */
/* every second input in layer i + 1 this is the layered protocol above.  */

#define SO_MAX_BLOCKS (SO_MAX_DEPTH + 1)

typedef struct so_gcircuit {
    uint32_t d, c, C, Creal;
    uint32_t s[SO_MAX_DEPTH + 1], W[SO_MAX_DEPTH + 1], wreal[SO_MAX_DEPTH + 1];
    uint8_t *type[SO_MAX_DEPTH];            /* one entry per real gate of layer i */
    uint32_t *in1[SO_MAX_DEPTH], *src[SO_MAX_DEPTH], *in2[SO_MAX_DEPTH];
    uint32_t sx[SO_MAX_DEPTH], nb[SO_MAX_DEPTH];     /* X_i: log2 width, blocks */
    uint32_t blayer[SO_MAX_DEPTH][SO_MAX_BLOCKS], bbase[SO_MAX_DEPTH][SO_MAX_BLOCKS];
    uint32_t bcount[SO_MAX_DEPTH][SO_MAX_BLOCKS];
    uint32_t *bys[SO_MAX_DEPTH][SO_MAX_BLOCKS];     /* the block's gates in its layer (block 0: all) */
    uint32_t *u2[SO_MAX_DEPTH];                     /* X_i index of each gate's second input */
    uint8_t wiring_digest[32];
} so_gcircuit;

void so_gcircuit_free(so_gcircuit *gc) {
    if (!gc) return;
    for (uint32_t i = 0; i < gc->d; ++i) {
        free(gc->type[i]); free(gc->in1[i]); free(gc->src[i]); free(gc->in2[i]); free(gc->u2[i]);
        for (uint32_t b = 0; b < gc->nb[i]; ++b) free(gc->bys[i][b]);
    }
    free(gc);
}

/* Wiring bytes: per padded gate of layer i, u8 type || u32le in1 || u32le
 * in2 when its second input is in layer i + 1, u8 (4 + type) || u32le in1
 * || u32le in2 || u32le layer when it is deeper, (2, 0, 0) when padding. */
static int gwiring_digest(so_gcircuit *gc) {
    size_t n = 0;
    for (uint32_t i = 0; i < gc->d; ++i) n += (size_t)gc->W[i] * 13;
    uint8_t *buf = (uint8_t *)malloc(n ? n : 1), *p = buf;
    if (!buf) return SO_ERR_OOM;
    for (uint32_t i = 0; i < gc->d; ++i)
        for (uint32_t g = 0; g < gc->W[i]; ++g) {
            if (g >= gc->wreal[i]) {
                *p++ = 2; put_u32(p, 0); p += 4; put_u32(p, 0); p += 4;
            } else if (gc->src[i][g] == i + 1) {
                *p++ = gc->type[i][g]; put_u32(p, gc->in1[i][g]); p += 4; put_u32(p, gc->in2[i][g]); p += 4;
            } else {
                *p++ = (uint8_t)(4 + gc->type[i][g]); put_u32(p, gc->in1[i][g]); p += 4;
                put_u32(p, gc->in2[i][g]); p += 4; put_u32(p, gc->src[i][g]); p += 4;
            }
        }
    int rc = statement_digest(buf, (size_t)(p - buf), gc->wiring_digest);
    free(buf);
    return rc;
}

so_gcircuit *so_gcircuit_new(uint32_t d, const uint32_t *widths, const uint8_t *types, const uint32_t *in1,
                             const uint32_t *src, const uint32_t *in2, uint32_t n_copies, int *err) {
    so_init();
    *err = SO_ERR_ARG;
    if (d < 1 || d > SO_MAX_DEPTH || n_copies < 1 || !widths || !types || !in1 || !src || !in2) return NULL;
    for (uint32_t i = 0; i <= d; ++i)
        if (widths[i] < 1 || widths[i] > (1u << 24)) return NULL;
    so_gcircuit *gc = (so_gcircuit *)calloc(1, sizeof *gc);
    if (!gc) { *err = SO_ERR_OOM; return NULL; }
    gc->Creal = n_copies;
    gc->c = ceil_log2(n_copies);
    gc->C = 1u << gc->c;
    for (uint32_t i = 0; i <= d; ++i) {
        gc->wreal[i] = widths[i];
        gc->s[i] = ceil_log2(widths[i]);
        gc->W[i] = 1u << gc->s[i];
    }
    size_t off = 0;
    for (uint32_t i = 0; i < d; ++i) {
        uint32_t n = widths[i];
        gc->d = i + 1; /* so that so_gcircuit_free releases what exists */
        gc->type[i] = (uint8_t *)malloc(n);
        gc->in1[i] = (uint32_t *)malloc(4 * (size_t)n);
        gc->src[i] = (uint32_t *)malloc(4 * (size_t)n);
        gc->in2[i] = (uint32_t *)malloc(4 * (size_t)n);
        gc->u2[i] = (uint32_t *)malloc(4 * (size_t)n);
        if (!gc->type[i] || !gc->in1[i] || !gc->src[i] || !gc->in2[i] || !gc->u2[i]) {
            so_gcircuit_free(gc); *err = SO_ERR_OOM; return NULL;
        }
        for (uint32_t g = 0; g < n; ++g) {
            uint8_t t = types[off + g];
            uint32_t a = in1[off + g], j = src[off + g], b = in2[off + g];
            if (t > 1 || a >= widths[i + 1] || j <= i || j > d || b >= widths[j]) { so_gcircuit_free(gc); return NULL; }
            gc->type[i][g] = t; gc->in1[i][g] = a; gc->src[i][g] = j; gc->in2[i][g] = b;
        }
        off += n;
        /* blocks of X_i: layer i + 1 in full, then the used gates of each deeper layer */
        gc->nb[i] = 1;
        gc->blayer[i][0] = i + 1; gc->bbase[i][0] = 0; gc->bcount[i][0] = gc->W[i + 1];
        gc->bys[i][0] = (uint32_t *)malloc(4 * (size_t)gc->W[i + 1]);
        if (!gc->bys[i][0]) { so_gcircuit_free(gc); *err = SO_ERR_OOM; return NULL; }
        for (uint32_t y = 0; y < gc->W[i + 1]; ++y) gc->bys[i][0][y] = y;
        uint32_t base = gc->W[i + 1];
        for (uint32_t j = i + 2; j <= d; ++j) {
            int32_t *pos = (int32_t *)malloc(4 * (size_t)gc->W[j]);
            if (!pos) { so_gcircuit_free(gc); *err = SO_ERR_OOM; return NULL; }
            for (uint32_t y = 0; y < gc->W[j]; ++y) pos[y] = -1;
            for (uint32_t g = 0; g < n; ++g)
                if (gc->src[i][g] == j) pos[gc->in2[i][g]] = 0;
            uint32_t cnt = 0;
            for (uint32_t y = 0; y < gc->W[j]; ++y)
                if (pos[y] == 0) pos[y] = (int32_t)(base + cnt++);
            if (cnt) {
                uint32_t bidx = gc->nb[i]++;
                gc->blayer[i][bidx] = j; gc->bbase[i][bidx] = base; gc->bcount[i][bidx] = cnt;
                gc->bys[i][bidx] = (uint32_t *)malloc(4 * (size_t)cnt);
                if (!gc->bys[i][bidx]) { free(pos); so_gcircuit_free(gc); *err = SO_ERR_OOM; return NULL; }
                for (uint32_t y = 0, k = 0; y < gc->W[j]; ++y)
                    if (pos[y] >= 0) gc->bys[i][bidx][k++] = y;
                for (uint32_t g = 0; g < n; ++g)
                    if (gc->src[i][g] == j) gc->u2[i][g] = (uint32_t)pos[gc->in2[i][g]];
                base += cnt;
            }
            free(pos);
        }
        for (uint32_t g = 0; g < n; ++g)
            if (gc->src[i][g] == i + 1) gc->u2[i][g] = gc->in2[i][g];
        gc->sx[i] = ceil_log2(base);
    }
    gc->d = d;
    if (gwiring_digest(gc) != SO_OK) { so_gcircuit_free(gc); *err = SO_ERR_OOM; return NULL; }
    *err = SO_OK;
    return gc;
}

size_t so_gproof_len(const so_gcircuit *gc) {
    size_t n = 8 + 4 * ((size_t)gc->d + 3);
    for (uint32_t i = 0; i < gc->d; ++i) n += 32 * (3 * (size_t)gc->c + 4 * (size_t)gc->sx[i] + 2 * (size_t)gc->nb[i]);
    return n;
}

uint32_t so_gcircuit_log_xwidth(const so_gcircuit *gc, uint32_t i) { return gc->sx[i]; }
uint32_t so_gcircuit_blocks(const so_gcircuit *gc, uint32_t i) { return gc->nb[i]; }

static int geval_all(const so_gcircuit *gc, const uint8_t *inputs, fr **V) {
    uint32_t d = gc->d;
    for (uint32_t i = 0; i <= d; ++i) V[i] = NULL;
    for (uint32_t i = 0; i <= d; ++i) {
        V[i] = (fr *)calloc((size_t)gc->C * gc->W[i], sizeof(fr));
        if (!V[i]) return SO_ERR_OOM;
    }
    for (uint32_t b = 0; b < gc->Creal; ++b)
        for (uint32_t x = 0; x < gc->wreal[d]; ++x)
            if (fr_from_bytes(&V[d][(size_t)b * gc->W[d] + x], inputs + 32 * ((size_t)b * gc->wreal[d] + x)) != SO_OK)
                return SO_ERR_CANON;
    for (int i = (int)d - 1; i >= 0; --i)
        for (uint32_t b = 0; b < gc->C; ++b)
            for (uint32_t g = 0; g < gc->wreal[i]; ++g) {
                uint32_t j = gc->src[i][g];
                V[i][(size_t)b * gc->W[i] + g] = op_gate(gc->type[i][g], V[i + 1][(size_t)b * gc->W[i + 1] + gc->in1[i][g]],
                                                         V[j][(size_t)b * gc->W[j] + gc->in2[i][g]]);
            }
    return SO_OK;
}

/* The copy-round polynomial g(t), t = 0..3, of one weight term (copy point
 * z, gate weights M) added into out: with T the virtual layer's rows folded
 * by r_1..r_{k-1} (n rows of WX values),
 *   sum_{j < n/2} eq(z, (r_1..r_{k-1}, t, bits(j))) sum_g M(g) op_g(T_t(j, in1 g), T_t(j, u2 g)). */
static void gcopy_round(const so_gcircuit *gc, uint32_t i, const fr *T, size_t n, uint32_t WX, const fr *M,
                        const fr *z, const fr *rb, uint32_t k, fr out[4]) {
    uint32_t c = gc->c;
    size_t h = n / 2;
    fr prefix = fr_u64(1);
    for (uint32_t m = 1; m < k; ++m) prefix = fr_mul(prefix, eq1(z[m - 1], rb[m - 1]));
    fr *row = (fr *)malloc(WX * sizeof(fr));
    for (size_t j = 0; j < h; ++j) {
        fr suffix = fr_u64(1);
        for (uint32_t m = k + 1; m <= c; ++m)
            suffix = fr_mul(suffix, eq1(z[m - 1], fr_u64((uint64_t)bit_msb((uint32_t)j, c - k, m - k))));
        for (int t = 0; t < 4; ++t) {
            fr tt = fr_u64((uint64_t)t);
            for (uint32_t x = 0; x < WX; ++x) {
                fr lo = T[j * WX + x], hi = T[(j + h) * WX + x];
                row[x] = fr_add(lo, fr_mul(fr_sub(hi, lo), tt));
            }
            fr S = fr_zero();
            for (uint32_t g = 0; g < gc->wreal[i]; ++g)
                S = fr_add(S, fr_mul(M[g], op_gate(gc->type[i][g], row[gc->in1[i][g]], row[gc->u2[i][g]])));
            out[t] = fr_add(out[t], fr_mul(fr_mul(fr_mul(prefix, eq1(z[k - 1], tt)), suffix), S));
        }
    }
    free(row);
}

/* Round k of the phase over the first (which = 1) or second (which = 2)
 * input on the virtual layer, with the combined gate weights om (the copy
 * weights folded in): A is the copy-bound row folded by the phase's
 * challenges so far, A0 the unfolded row, pre[g] the eq factor of the bits
 * already bound (and, in phase 2, eq(r_x, in1 g)). */
static void ggate_round(const so_gcircuit *gc, uint32_t i, int which, const fr *A, const fr *A0, const fr *om,
                        const fr *pre, fr vx, uint32_t k, fr out[3]) {
    uint32_t sx = gc->sx[i];
    size_t m = (size_t)1 << (sx - k + 1), h = m / 2;
    uint32_t lomask = (uint32_t)(h - 1);
    for (int t = 0; t < 3; ++t) {
        fr tt = fr_u64((uint64_t)t), S = fr_zero();
        for (uint32_t g = 0; g < gc->wreal[i]; ++g) {
            uint8_t ty = gc->type[i][g];
            uint32_t v = which == 1 ? gc->in1[i][g] : gc->u2[i][g];
            uint32_t lo = v & lomask;
            fr at = fr_add(A[lo], fr_mul(tt, fr_sub(A[lo + h], A[lo])));
            fr val = which == 2 ? op_gate(gc->type[i][g], vx, at) : op_gate(ty, at, A0[gc->u2[i][g]]);
            fr coeff = fr_mul(fr_mul(om[g], pre[g]), eq1(tt, fr_u64((uint64_t)bit_msb(v, sx, k))));
            S = fr_add(S, fr_mul(coeff, val));
        }
        out[t] = S;
    }
}

static void gput_hdr(writer *w, const so_gcircuit *gc) {
    static const char magic[8] = {'S', 'I', 'S', 'U', 'G', 'K', 'R', '2'};
    uint8_t u[4];
    if (w->cap >= 8) memcpy(w->buf, magic, 8);
    w->len = 8;
    put_u32(u, gc->d); if (w->len + 4 <= w->cap) memcpy(w->buf + w->len, u, 4); w->len += 4;
    put_u32(u, gc->c); if (w->len + 4 <= w->cap) memcpy(w->buf + w->len, u, 4); w->len += 4;
    for (uint32_t i = 0; i <= gc->d; ++i) {
        put_u32(u, gc->s[i]);
        if (w->len + 4 <= w->cap) memcpy(w->buf + w->len, u, 4);
        w->len += 4;
    }
}

/* weight terms of a layer's combined claim */
typedef struct {
    uint32_t n;
    fr *z[2 * SO_MAX_DEPTH + 2];  /* copy points (c values each) */
    fr *M[2 * SO_MAX_DEPTH + 2];  /* gate weights (W_j values each) */
} gterms;

static void gterms_free(gterms *t) {
    for (uint32_t k = 0; k < t->n; ++k) { free(t->z[k]); free(t->M[k]); }
    t->n = 0;
}

/* M(g) of the claims of block b of layer i's virtual layer on its layer:
 * ax eq(r_x, u) + ay eq(r_y, u) at the block's gates, 0 elsewhere */
static fr *gblock_weights(const so_gcircuit *gc, uint32_t i, uint32_t b, const fr *rx, const fr *ry, fr ax, fr ay) {
    uint32_t j = gc->blayer[i][b];
    fr *M = (fr *)calloc(gc->W[j], sizeof(fr));
    if (!M) return NULL;
    for (uint32_t k = 0; k < gc->bcount[i][b]; ++k) {
        uint32_t u = gc->bbase[i][b] + k;
        M[gc->bys[i][b][k]] = fr_add(fr_mul(ax, eq_point_index(rx, gc->sx[i], u)),
                                     fr_mul(ay, eq_point_index(ry, gc->sx[i], u)));
    }
    return M;
}

int so_gprove(const so_gcircuit *gc, const uint8_t *inputs, const uint8_t *domain, size_t dlen,
              uint8_t *proof, size_t cap, size_t *len_out) {
    uint32_t d = gc->d, c = gc->c;
    fr *V[SO_MAX_DEPTH + 1];
    int rc = geval_all(gc, inputs, V);
    if (rc != SO_OK) { free_layers(V, d + 1); return rc; }
    uint8_t dig_in[32], dig_out[32];
    table_digest(V[d], (size_t)gc->C * gc->W[d], dig_in);
    table_digest(V[0], (size_t)gc->C * gc->W[0], dig_out);
    transcript tr;
    tr_init(&tr, domain, dlen, d, c, gc->s, gc->wiring_digest, dig_in, dig_out);
    writer w = {proof, 0, cap};
    gput_hdr(&w, gc);
    gterms terms[SO_MAX_DEPTH + 1];
    memset(terms, 0, sizeof terms);
    fr zg[32], rb[32], rx[32], ry[32];
    terms[0].n = 1;
    terms[0].z[0] = (fr *)malloc(32 * sizeof(fr));
    terms[0].M[0] = (fr *)malloc(gc->W[0] * sizeof(fr));
    for (uint32_t k = 0; k < c; ++k) terms[0].z[0][k] = tr_challenge(&tr);
    for (uint32_t k = 0; k < gc->s[0]; ++k) zg[k] = tr_challenge(&tr);
    for (uint32_t g = 0; g < gc->W[0]; ++g) terms[0].M[0][g] = eq_point_index(zg, gc->s[0], g);
    for (uint32_t i = 0; i < d; ++i) {
        uint32_t sx = gc->sx[i], WX = 1u << sx;
        /* the virtual layer's table, folded in place by the copy rounds */
        fr *X = (fr *)calloc((size_t)gc->C * WX, sizeof(fr));
        for (uint32_t b = 0; b < gc->nb[i]; ++b) {
            uint32_t j = gc->blayer[i][b];
            for (uint32_t q = 0; q < gc->C; ++q)
                for (uint32_t k = 0; k < gc->bcount[i][b]; ++k)
                    X[(size_t)q * WX + gc->bbase[i][b] + k] = V[j][(size_t)q * gc->W[j] + gc->bys[i][b][k]];
        }
        size_t n = gc->C;
        for (uint32_t k = 1; k <= c; ++k) {
            fr g4[4] = {fr_zero(), fr_zero(), fr_zero(), fr_zero()};
            for (uint32_t t = 0; t < terms[i].n; ++t) gcopy_round(gc, i, X, n, WX, terms[i].M[t], terms[i].z[t], rb, k, g4);
            send_round(&tr, &w, g4, 4);
            rb[k - 1] = tr_challenge(&tr);
            fold_rows(X, n, WX, rb[k - 1]);
            n /= 2;
        }
        /* the combined gate weights: each term's weights times its copy weight eq(z_T, r_b) */
        fr *om = (fr *)calloc(gc->W[i], sizeof(fr));
        for (uint32_t t = 0; t < terms[i].n; ++t) {
            fr e = fr_u64(1);
            for (uint32_t m = 0; m < c; ++m) e = fr_mul(e, eq1(terms[i].z[t][m], rb[m]));
            for (uint32_t g = 0; g < gc->W[i]; ++g) om[g] = fr_add(om[g], fr_mul(e, terms[i].M[t][g]));
        }
        fr *A0 = (fr *)malloc(WX * sizeof(fr)), *A = (fr *)malloc(WX * sizeof(fr));
        fr *pre = (fr *)malloc((gc->wreal[i] ? gc->wreal[i] : 1) * sizeof(fr));
        memcpy(A0, X, WX * sizeof(fr));
        memcpy(A, A0, WX * sizeof(fr));
        for (uint32_t g = 0; g < gc->wreal[i]; ++g) pre[g] = fr_u64(1);
        for (uint32_t k = 1; k <= sx; ++k) {
            fr g3[3];
            ggate_round(gc, i, 1, A, A0, om, pre, fr_zero(), k, g3);
            send_round(&tr, &w, g3, 3);
            rx[k - 1] = tr_challenge(&tr);
            fold_rows(A, (size_t)1 << (sx - k + 1), 1, rx[k - 1]);
            for (uint32_t g = 0; g < gc->wreal[i]; ++g)
                pre[g] = fr_mul(pre[g], eq1(rx[k - 1], fr_u64((uint64_t)bit_msb(gc->in1[i][g], sx, k))));
        }
        fr vx = A[0];
        memcpy(A, A0, WX * sizeof(fr));
        for (uint32_t g = 0; g < gc->wreal[i]; ++g) pre[g] = eq_point_index(rx, sx, gc->in1[i][g]);
        for (uint32_t k = 1; k <= sx; ++k) {
            fr g3[3];
            ggate_round(gc, i, 2, A, A0, om, pre, vx, k, g3);
            send_round(&tr, &w, g3, 3);
            ry[k - 1] = tr_challenge(&tr);
            fold_rows(A, (size_t)1 << (sx - k + 1), 1, ry[k - 1]);
            for (uint32_t g = 0; g < gc->wreal[i]; ++g)
                pre[g] = fr_mul(pre[g], eq1(ry[k - 1], fr_u64((uint64_t)bit_msb(gc->u2[i][g], sx, k))));
        }
        /* the blocks' parts of X~_i(r_b, r_x) and X~_i(r_b, r_y) */
        fr vb[2 * SO_MAX_BLOCKS];
        uint32_t nb = gc->nb[i];
        for (uint32_t b = 0; b < nb; ++b) {
            vb[b] = fr_zero();
            vb[nb + b] = fr_zero();
            for (uint32_t k = 0; k < gc->bcount[i][b]; ++k) {
                uint32_t u = gc->bbase[i][b] + k;
                vb[b] = fr_add(vb[b], fr_mul(eq_point_index(rx, sx, u), A0[u]));
                vb[nb + b] = fr_add(vb[nb + b], fr_mul(eq_point_index(ry, sx, u), A0[u]));
            }
        }
        absorb_and_put(&tr, &w, 'V', vb, (int)(2 * nb));
        for (uint32_t b = 0; b < nb; ++b) {
            uint32_t j = gc->blayer[i][b];
            if (j == d) continue; /* the input layer: checked by the verifier from the clear inputs */
            fr ax = tr_challenge(&tr), ay = tr_challenge(&tr);
            gterms *T = &terms[j];
            T->z[T->n] = (fr *)malloc(32 * sizeof(fr));
            memcpy(T->z[T->n], rb, 32 * sizeof(fr));
            T->M[T->n] = gblock_weights(gc, i, b, rx, ry, ax, ay);
            T->n++;
        }
        free(X); free(om); free(A0); free(A); free(pre);
    }
    for (uint32_t j = 0; j <= d; ++j) gterms_free(&terms[j]);
    free_layers(V, d + 1);
    *len_out = w.len;
    return w.len <= cap ? SO_OK : SO_ERR_ARG;
}

static int gload_table(const so_gcircuit *gc, const uint8_t *bytes, uint32_t layer, fr **out) {
    fr *T = (fr *)calloc((size_t)gc->C * gc->W[layer], sizeof(fr));
    if (!T) return SO_ERR_OOM;
    for (uint32_t b = 0; b < gc->Creal; ++b)
        for (uint32_t x = 0; x < gc->wreal[layer]; ++x)
            if (fr_from_bytes(&T[(size_t)b * gc->W[layer] + x],
                              bytes + 32 * ((size_t)b * gc->wreal[layer] + x)) != SO_OK) {
                free(T);
                return SO_ERR_CANON;
            }
    *out = T;
    return SO_OK;
}

int so_gverify(const so_gcircuit *gc, const uint8_t *inputs, const uint8_t *outputs, const uint8_t *proof,
               size_t len, const uint8_t *domain, size_t dlen) {
    uint32_t d = gc->d, c = gc->c;
    if (len != so_gproof_len(gc)) return SO_ERR_REJECT;
    {
        uint8_t hdr[8 + 4 * (SO_MAX_DEPTH + 3)];
        writer w = {hdr, 0, sizeof hdr};
        gput_hdr(&w, gc);
        if (memcmp(hdr, proof, w.len) != 0) return SO_ERR_REJECT;
    }
    reader rd = {proof, len, 8 + 4 * ((size_t)d + 3), 0};
    fr *Vin = NULL, *Vout = NULL;
    int rc = gload_table(gc, inputs, d, &Vin);
    if (rc != SO_OK) return rc;
    rc = gload_table(gc, outputs, 0, &Vout);
    if (rc != SO_OK) { free(Vin); return rc; }
    uint8_t dig_in[32], dig_out[32];
    table_digest(Vin, (size_t)gc->C * gc->W[d], dig_in);
    table_digest(Vout, (size_t)gc->C * gc->W[0], dig_out);
    transcript tr;
    tr_init(&tr, domain, dlen, d, c, gc->s, gc->wiring_digest, dig_in, dig_out);
    gterms terms[SO_MAX_DEPTH + 1];
    memset(terms, 0, sizeof terms);
    fr claims[SO_MAX_DEPTH + 1];
    for (uint32_t j = 0; j <= d; ++j) claims[j] = fr_zero();
    fr zg[32], rb[32], rx[32], ry[32], pt[64];
    terms[0].n = 1;
    terms[0].z[0] = (fr *)malloc(32 * sizeof(fr));
    terms[0].M[0] = (fr *)malloc(gc->W[0] * sizeof(fr));
    for (uint32_t k = 0; k < c; ++k) terms[0].z[0][k] = tr_challenge(&tr);
    for (uint32_t k = 0; k < gc->s[0]; ++k) zg[k] = tr_challenge(&tr);
    for (uint32_t g = 0; g < gc->W[0]; ++g) terms[0].M[0][g] = eq_point_index(zg, gc->s[0], g);
    /* output claim V~_0(z_b, z_g) from the clear outputs */
    for (uint32_t k = 0; k < c; ++k) pt[k] = terms[0].z[0][k];
    for (uint32_t k = 0; k < gc->s[0]; ++k) pt[c + k] = zg[k];
    claims[0] = mle_by_folding(Vout, c + gc->s[0], pt);
    int ok = 1;
    for (uint32_t i = 0; i < d && ok; ++i) {
        uint32_t sx = gc->sx[i], nb = gc->nb[i];
        fr claim = claims[i];
        for (uint32_t k = 0; k < c && ok; ++k) {
            fr g[4], sent[3];
            for (int t = 0; t < 3; ++t) sent[t] = get_fr(&rd);
            if (rd.bad) { ok = 0; break; }
            g[0] = sent[0]; g[1] = fr_sub(claim, sent[0]); g[2] = sent[1]; g[3] = sent[2];
            tr_absorb(&tr, 'R', sent, 3);
            rb[k] = tr_challenge(&tr);
            claim = interpolate(g, 4, rb[k]);
        }
        for (int phase = 0; phase < 2 && ok; ++phase)
            for (uint32_t k = 0; k < sx && ok; ++k) {
                fr g[3], sent[2];
                for (int t = 0; t < 2; ++t) sent[t] = get_fr(&rd);
                if (rd.bad) { ok = 0; break; }
                g[0] = sent[0]; g[1] = fr_sub(claim, sent[0]); g[2] = sent[1];
                tr_absorb(&tr, 'R', sent, 2);
                fr r = tr_challenge(&tr);
                if (phase == 0) rx[k] = r; else ry[k] = r;
                claim = interpolate(g, 3, r);
            }
        if (!ok) break;
        fr vb[2 * SO_MAX_BLOCKS], vx = fr_zero(), vy = fr_zero();
        for (uint32_t b = 0; b < 2 * nb; ++b) vb[b] = get_fr(&rd);
        if (rd.bad) { ok = 0; break; }
        for (uint32_t b = 0; b < nb; ++b) { vx = fr_add(vx, vb[b]); vy = fr_add(vy, vb[nb + b]); }
        /* final identity: claim = sum_T eq(z_T, r_b) sum_g M_T(g) eq(r_x, in1 g) eq(r_y, u2 g) op_g(v_x, v_y) */
        fr sum = fr_zero();
        for (uint32_t t = 0; t < terms[i].n; ++t) {
            fr e = fr_u64(1), part = fr_zero();
            for (uint32_t m = 0; m < c; ++m) e = fr_mul(e, eq1(terms[i].z[t][m], rb[m]));
            for (uint32_t g = 0; g < gc->wreal[i]; ++g) {
                fr pred = fr_mul(eq_point_index(rx, sx, gc->in1[i][g]), eq_point_index(ry, sx, gc->u2[i][g]));
                part = fr_add(part, fr_mul(fr_mul(terms[i].M[t][g], pred), op_gate(gc->type[i][g], vx, vy)));
            }
            sum = fr_add(sum, fr_mul(e, part));
        }
        if (!fr_eq(claim, sum)) { ok = 0; break; }
        tr_absorb(&tr, 'V', vb, (int)(2 * nb));
        for (uint32_t b = 0; b < nb && ok; ++b) {
            uint32_t j = gc->blayer[i][b];
            if (j == d) {
                /* input check: v(r) = sum_{u in block} eq(r, u) V~_d(r_b, y_u), from the clear inputs */
                for (int which = 0; which < 2 && ok; ++which) {
                    const fr *r = which == 0 ? rx : ry;
                    fr want = fr_zero();
                    for (uint32_t k = 0; k < gc->bcount[i][b]; ++k) {
                        fr col = fr_zero();
                        for (uint32_t q = 0; q < gc->C; ++q)
                            col = fr_add(col, fr_mul(eq_point_index(rb, c, q),
                                                     Vin[(size_t)q * gc->W[d] + gc->bys[i][b][k]]));
                        want = fr_add(want, fr_mul(eq_point_index(r, sx, gc->bbase[i][b] + k), col));
                    }
                    if (!fr_eq(want, vb[which * nb + b])) ok = 0;
                }
                continue;
            }
            fr ax = tr_challenge(&tr), ay = tr_challenge(&tr);
            gterms *T = &terms[j];
            T->z[T->n] = (fr *)malloc(32 * sizeof(fr));
            memcpy(T->z[T->n], rb, 32 * sizeof(fr));
            T->M[T->n] = gblock_weights(gc, i, b, rx, ry, ax, ay);
            T->n++;
            claims[j] = fr_add(claims[j], fr_add(fr_mul(ax, vb[b]), fr_mul(ay, vb[nb + b])));
        }
    }
    if (rd.pos != rd.len) ok = 0;
    for (uint32_t j = 0; j <= d; ++j) gterms_free(&terms[j]);
    free(Vin);
    free(Vout);
    return ok ? SO_OK : SO_ERR_REJECT;
}

int so_goutputs(const so_gcircuit *gc, const uint8_t *inputs, uint8_t *out) {
    fr *V[SO_MAX_DEPTH + 1];
    int rc = geval_all(gc, inputs, V);
    if (rc == SO_OK)
        for (uint32_t b = 0; b < gc->Creal; ++b)
            for (uint32_t g = 0; g < gc->wreal[0]; ++g)
                fr_to_bytes(out + 32 * ((size_t)b * gc->wreal[0] + g), V[0][(size_t)b * gc->W[0] + g]);
    free_layers(V, gc->d + 1);
    return rc;
}
