// Host verifier of the data-parallel GKR proof, and host Merkle digests.
//
// Field arithmetic here is 4 x 64-bit Montgomery (CIOS with 128-bit
// products), fully reduced to [0, r).  The verifier replays the transcript
// and checks, layer by layer (GKR, Sec. 2.2):
//   - every round: g(0) + g(1) = claim (the sumcheck round check of
//     Sec. 3.2.1), then claim = g(r) by Lagrange interpolation;
//   - the layer's final identity
//       claim = eq(z_b, r_b) sum_g w(g) eq(r_x, in1 g) eq(r_y, in2 g) op_g(v_x, v_y);
//   - the output claim V~_0(z_b, z_g) from the clear outputs and, after the
//     last layer, v_x = V~_d(r_b, r_x), v_y = V~_d(r_b, r_y) from the inputs.
#include <cstring>
#include <vector>

#include "../../include/sisu.h"
#include "internal.h"
#include "sha256.cuh"

namespace sisu {
namespace {

typedef unsigned __int128 u128;

struct HF {
  uint64_t w[4];
};

const uint64_t kMod[4] = {0x43e1f593f0000001ull, 0x2833e84879b97091ull, 0xb85045b68181585dull,
                          0x30644e72e131a029ull};
const uint64_t kNp = 0xc2e1f593efffffffull;
const HF kOne = {{0xac96341c4ffffffbull, 0x36fc76959f60cd29ull, 0x666ea36f7879462eull, 0x0e0a77c19a07df2full}};
const HF kR2 = {{0x1bb8e645ae216da7ull, 0x53fe3ab1e35c59e3ull, 0x8c49833d53bb8085ull, 0x0216d0b17f4e44a5ull}};
const HF kZero = {{0, 0, 0, 0}};

bool geq_mod(const uint64_t* a) {
  for (int i = 3; i >= 0; --i)
    if (a[i] != kMod[i]) return a[i] > kMod[i];
  return true;
}

void sub_mod(uint64_t* a) {
  uint64_t br = 0;
  for (int i = 0; i < 4; ++i) {
    u128 d = (u128)a[i] - kMod[i] - br;
    a[i] = (uint64_t)d;
    br = (uint64_t)(d >> 64) & 1;
  }
}

HF add(const HF& a, const HF& b) {
  HF s;
  uint64_t c = 0;
  for (int i = 0; i < 4; ++i) {
    u128 t = (u128)a.w[i] + b.w[i] + c;
    s.w[i] = (uint64_t)t;
    c = (uint64_t)(t >> 64);
  }
  if (geq_mod(s.w)) sub_mod(s.w);
  return s;
}

HF sub(const HF& a, const HF& b) {
  HF d;
  uint64_t br = 0;
  for (int i = 0; i < 4; ++i) {
    u128 t = (u128)a.w[i] - b.w[i] - br;
    d.w[i] = (uint64_t)t;
    br = (uint64_t)(t >> 64) & 1;
  }
  if (br) {
    uint64_t c = 0;
    for (int i = 0; i < 4; ++i) {
      u128 t = (u128)d.w[i] + kMod[i] + c;
      d.w[i] = (uint64_t)t;
      c = (uint64_t)(t >> 64);
    }
  }
  return d;
}

HF mul(const HF& a, const HF& b) {
  uint64_t t[6] = {0, 0, 0, 0, 0, 0};
  for (int i = 0; i < 4; ++i) {
    uint64_t c = 0;
    for (int j = 0; j < 4; ++j) {
      u128 x = (u128)a.w[j] * b.w[i] + t[j] + c;
      t[j] = (uint64_t)x;
      c = (uint64_t)(x >> 64);
    }
    u128 x = (u128)t[4] + c;
    t[4] = (uint64_t)x;
    t[5] = (uint64_t)(x >> 64);
    uint64_t m = t[0] * kNp;
    x = (u128)m * kMod[0] + t[0];
    c = (uint64_t)(x >> 64);
    for (int j = 1; j < 4; ++j) {
      x = (u128)m * kMod[j] + t[j] + c;
      t[j - 1] = (uint64_t)x;
      c = (uint64_t)(x >> 64);
    }
    x = (u128)t[4] + c;
    t[3] = (uint64_t)x;
    t[4] = t[5] + (uint64_t)(x >> 64);
  }
  HF r = {{t[0], t[1], t[2], t[3]}};
  if (t[4] || geq_mod(r.w)) sub_mod(r.w);
  return r;
}

bool eq(const HF& a, const HF& b) { return memcmp(a.w, b.w, 32) == 0; }

HF from_u64(uint64_t v) { return mul(HF{{v, 0, 0, 0}}, kR2); }

// canonical 32 little-endian bytes -> Montgomery; false if not below r
bool load(const uint8_t* p, HF* out) {
  HF x;
  for (int i = 0; i < 4; ++i) {
    uint64_t v = 0;
    for (int k = 7; k >= 0; --k) v = (v << 8) | p[8 * i + k];
    x.w[i] = v;
  }
  if (geq_mod(x.w)) return false;
  *out = mul(x, kR2);
  return true;
}

void store(uint8_t* p, const HF& a) {
  HF x = mul(a, HF{{1, 0, 0, 0}});
  for (int i = 0; i < 4; ++i)
    for (int k = 0; k < 8; ++k) p[8 * i + k] = (uint8_t)(x.w[i] >> (8 * k));
}

HF pow(HF a, const uint64_t* e) {
  HF acc = kOne;
  for (int i = 255; i >= 0; --i) {
    acc = mul(acc, acc);
    if ((e[i / 64] >> (i % 64)) & 1) acc = mul(acc, a);
  }
  return acc;
}

HF inv(const HF& a) {
  uint64_t e[4] = {kMod[0] - 2, kMod[1], kMod[2], kMod[3]};
  return pow(a, e);
}

HF one_minus(const HF& a) { return sub(kOne, a); }

// EQ(r_1..r_m) over 2^m indices, r_1 <-> most significant bit
std::vector<HF> eq_table(const std::vector<HF>& r) {
  std::vector<HF> t(1, kOne);
  for (const HF& rk : r) {
    std::vector<HF> u(t.size() * 2);
    for (size_t j = 0; j < t.size(); ++j) {
      u[2 * j] = mul(t[j], one_minus(rk));
      u[2 * j + 1] = mul(t[j], rk);
    }
    t.swap(u);
  }
  return t;
}

HF eq_point(const std::vector<HF>& a, const std::vector<HF>& b) {
  HF acc = kOne;
  for (size_t k = 0; k < a.size(); ++k) acc = mul(acc, add(mul(a[k], b[k]), mul(one_minus(a[k]), one_minus(b[k]))));
  return acc;
}

// multilinear extension by folding the top variable first
HF mle(std::vector<HF> t, const std::vector<HF>& r) {
  size_t n = t.size();
  for (const HF& rk : r) {
    n /= 2;
    for (size_t j = 0; j < n; ++j) t[j] = add(t[j], mul(rk, sub(t[j + n], t[j])));
  }
  return t[0];
}

struct Lagrange {
  HF inv_den[4][4];  // unused slots zero
  Lagrange() {
    for (int n = 3; n <= 4; ++n)
      for (int i = 0; i < n; ++i) {
        HF den = kOne;
        for (int j = 0; j < n; ++j)
          if (j != i) den = mul(den, sub(from_u64(i), from_u64(j)));
        inv_den[n - 1][i] = inv(den);
      }
  }
  HF at(const HF* g, int n, const HF& x) const {
    HF acc = kZero;
    for (int i = 0; i < n; ++i) {
      HF num = inv_den[n - 1][i];
      for (int j = 0; j < n; ++j)
        if (j != i) num = mul(num, sub(x, from_u64(j)));
      acc = add(acc, mul(g[i], num));
    }
    return acc;
  }
};

// Fiat-Shamir transcript on the SHA-256 compression function: absorb
// tweaks word 7 of the state with 256 tag + n and compresses the elements'
// canonical LE bytes 64 at a time (zero-padded); the first challenge after
// an absorb or the initial hash reads the state, later ones first compress
// Q(ctr) = 'C' || u32le ctr || 0^59; a challenge is the element whose
// Montgomery form is LE(st) mod 2^254 (squeezed again while >= r).
struct Transcript {
  uint32_t st[8];
  bool fresh = true;
  void absorb(uint8_t tag, const HF* e, int n) {
    std::vector<uint8_t> msg((size_t)64 * ((32 * n + 63) / 64), 0);
    const int nb = (32 * n + 63) / 64;
    for (int i = 0; i < n; ++i) store(msg.data() + 32 * i, e[i]);
    st[7] ^= ((uint32_t)tag << 8) | (uint32_t)n;
    for (int b = 0; b < nb; ++b) {
      uint32_t blk[16];
      const uint8_t* p = msg.data() + 64 * b;
      for (int k = 0; k < 16; ++k)
        blk[k] = ((uint32_t)p[4 * k] << 24) | ((uint32_t)p[4 * k + 1] << 16) | ((uint32_t)p[4 * k + 2] << 8) | p[4 * k + 3];
      sha256_compress(st, blk);
    }
    fresh = true;
  }
  void squeeze(uint32_t ctr) {
    uint32_t q[16] = {0};
    q[0] = (uint32_t('C') << 24) | ((ctr & 0xffu) << 16) | (((ctr >> 8) & 0xffu) << 8) | ((ctr >> 16) & 0xffu);
    q[1] = (ctr >> 24) << 24;
    sha256_compress(st, q);
  }
  HF challenge() {
    uint32_t ctr = 0;
    if (!fresh) squeeze(ctr++);
    fresh = false;
    for (;; squeeze(ctr++)) {
      uint8_t b[32];
      for (int i = 0; i < 8; ++i) {
        b[4 * i] = (uint8_t)(st[i] >> 24); b[4 * i + 1] = (uint8_t)(st[i] >> 16);
        b[4 * i + 2] = (uint8_t)(st[i] >> 8); b[4 * i + 3] = (uint8_t)st[i];
      }
      b[31] &= 0x3f;
      HF x;
      for (int i = 0; i < 4; ++i) {
        uint64_t v = 0;
        for (int k = 7; k >= 0; --k) v = (v << 8) | b[8 * i + k];
        x.w[i] = v;
      }
      if (!geq_mod(x.w)) return x;  // x is the Montgomery form
    }
  }
};

// padded canonical table bytes (C x W) from unpadded rows (Creal x wreal)
std::vector<uint8_t> padded_bytes(const uint8_t* src, uint32_t C, uint32_t W, uint32_t Creal, uint32_t wreal) {
  std::vector<uint8_t> out((size_t)C * W * 32, 0);
  for (uint32_t b = 0; b < Creal; ++b) memcpy(&out[(size_t)b * W * 32], src + (size_t)b * wreal * 32, (size_t)wreal * 32);
  return out;
}

bool load_table(const std::vector<uint8_t>& bytes, std::vector<HF>* out) {
  size_t n = bytes.size() / 32;
  out->resize(n);
  for (size_t i = 0; i < n; ++i)
    if (!load(&bytes[32 * i], &(*out)[i])) return false;
  return true;
}

}  // namespace

void host_statement_digest(const uint8_t* data, size_t len, uint32_t out[8]) {
  std::vector<uint32_t> level;
  uint32_t root[8];
  if (len == 0) {
    Sha256Stream h;
    h.begin();
    h.byte(0x02);
    h.end(root);
  } else {
    size_t nleaf = (len + 1023) / 1024;
    level.resize(nleaf * 8);
    for (size_t L = 0; L < nleaf; ++L) {
      size_t off = L * 1024, m = std::min((size_t)1024, len - off);
      uint32_t h[8];
      sha256_init(h);
      size_t full = m / 64;
      uint32_t blk[16];
      for (size_t b = 0; b < full; ++b) {
        const uint8_t* p = data + off + 64 * b;
        for (int k = 0; k < 16; ++k)
          blk[k] = ((uint32_t)p[4 * k] << 24) | ((uint32_t)p[4 * k + 1] << 16) | ((uint32_t)p[4 * k + 2] << 8) | p[4 * k + 3];
        sha256_compress(h, blk);
      }
      // tail bytes, tag 0x00, padding
      Sha256Stream s;
      memcpy(s.h, h, 32);
      s.fill = 0;
      s.total = full * 64;
      for (int k = 0; k < 16; ++k) s.blk[k] = 0;
      s.bytes(data + off + 64 * full, m - 64 * full);
      s.byte(0x00);
      s.end(&level[8 * L]);
    }
    size_t n = nleaf;
    while (n > 1) {
      size_t m = 0;
      for (size_t j = 0; j + 1 < n; j += 2) {
        Sha256Stream s;
        s.begin();
        s.digest_words(&level[8 * j]);
        s.digest_words(&level[8 * (j + 1)]);
        s.byte(0x01);
        uint32_t o[8];
        s.end(o);
        memcpy(&level[8 * m], o, 32);
        ++m;
      }
      if (n % 2) {
        memmove(&level[8 * m], &level[8 * (n - 1)], 32);
        ++m;
      }
      n = m;
    }
    memcpy(root, level.data(), 32);
  }
  Sha256Stream s;
  s.begin();
  s.digest_words(root);
  for (int i = 0; i < 8; ++i) s.byte((uint8_t)((uint64_t)len >> (8 * i)));
  s.byte(0x03);
  s.end(out);
}

static int host_verify_general(const HostCircuit& hc, const uint8_t* inputs, const uint8_t* outputs,
                               const uint8_t* proof, size_t proof_len, const uint8_t* domain, size_t dlen);

int host_verify(const HostCircuit& hc, const uint8_t* inputs, const uint8_t* outputs, const uint8_t* proof,
                size_t proof_len, const uint8_t* domain, size_t dlen) {
  if (hc.general) return host_verify_general(hc, inputs, outputs, proof, proof_len, domain, dlen);
  const uint32_t d = hc.d, c = hc.c;
  if (proof_len != hc.proof_len()) return SISU_ERR_REJECT;
  // header
  {
    std::vector<uint8_t> hdr(8 + 4 * ((size_t)d + 3));
    memcpy(hdr.data(), "SISUGKR2", 8);
    auto put = [&](size_t at, uint32_t v) {
      for (int k = 0; k < 4; ++k) hdr[at + k] = (uint8_t)(v >> (8 * k));
    };
    put(8, d);
    put(12, c);
    for (uint32_t i = 0; i <= d; ++i) put(16 + 4 * (size_t)i, hc.s[i]);
    if (memcmp(hdr.data(), proof, hdr.size()) != 0) return SISU_ERR_REJECT;
  }
  size_t pos = 8 + 4 * ((size_t)d + 3);
  auto next = [&](HF* x) -> bool {
    if (pos + 32 > proof_len) return false;
    bool ok = load(proof + pos, x);
    pos += 32;
    return ok;
  };
  std::vector<uint8_t> in_b = padded_bytes(inputs, hc.C, hc.W[d], hc.Creal, hc.wreal[d]);
  std::vector<uint8_t> out_b = padded_bytes(outputs, hc.C, hc.W[0], hc.Creal, hc.wreal[0]);
  std::vector<HF> Vin, Vout;
  if (!load_table(in_b, &Vin) || !load_table(out_b, &Vout)) return SISU_ERR_NOT_CANONICAL;
  uint32_t dig_in[8], dig_out[8];
  host_statement_digest(in_b.data(), in_b.size(), dig_in);
  host_statement_digest(out_b.data(), out_b.size(), dig_out);

  Transcript tr;
  {
    Sha256Stream h;
    h.begin();
    h.bytes(domain, dlen);
    h.byte(0);
    h.u32le(d);
    h.u32le(c);
    for (uint32_t i = 0; i <= d; ++i) h.u32le(hc.s[i]);
    h.digest_words(hc.wiring_digest);
    h.digest_words(dig_in);
    h.digest_words(dig_out);
    h.end(tr.st);
  }
  std::vector<HF> zb(c), zg(hc.s[0]);
  for (auto& z : zb) z = tr.challenge();
  for (auto& z : zg) z = tr.challenge();
  std::vector<HF> pt(zb);
  pt.insert(pt.end(), zg.begin(), zg.end());
  HF claim = mle(Vout, pt);
  static const Lagrange lag;
  HF alpha = kZero, beta = kZero;
  std::vector<HF> prx, pry;
  for (uint32_t i = 0; i < d; ++i) {
    const uint32_t s = hc.s[i + 1], W = hc.W[i];
    std::vector<HF> rb(c), rx(s), ry(s);
    // each round sends g(0), g(2)[, g(3)]; g(1) = claim - g(0)
    for (uint32_t k = 0; k < c; ++k) {
      HF g[4], sent[3];
      for (auto& v : sent)
        if (!next(&v)) return SISU_ERR_REJECT;
      g[0] = sent[0]; g[2] = sent[1]; g[3] = sent[2];
      g[1] = sub(claim, g[0]);
      tr.absorb('R', sent, 3);
      rb[k] = tr.challenge();
      claim = lag.at(g, 4, rb[k]);
    }
    for (int phase = 0; phase < 2; ++phase)
      for (uint32_t k = 0; k < s; ++k) {
        HF g[3], sent[2];
        for (auto& v : sent)
          if (!next(&v)) return SISU_ERR_REJECT;
        g[0] = sent[0]; g[2] = sent[1];
        g[1] = sub(claim, g[0]);
        tr.absorb('R', sent, 2);
        HF r = tr.challenge();
        (phase == 0 ? rx : ry)[k] = r;
        claim = lag.at(g, 3, r);
      }
    HF vx, vy;
    if (!next(&vx) || !next(&vy)) return SISU_ERR_REJECT;
    // final identity of the layer
    std::vector<HF> qx = eq_table(rx), qy = eq_table(ry);
    std::vector<HF> om;
    if (i == 0) {
      om = eq_table(zg);
    } else {
      std::vector<HF> ex = eq_table(prx), ey = eq_table(pry);
      om.resize(W);
      for (uint32_t g = 0; g < W; ++g) om[g] = add(mul(alpha, ex[g]), mul(beta, ey[g]));
    }
    HF sum = kZero;
    const HF vsum = add(vx, vy), vprod = mul(vx, vy);
    for (size_t e = 0; e < hc.out[i].size(); ++e) {  // entries, each weighed by w of its gate
      const uint8_t t = hc.type[i][e];
      HF term = mul(om[hc.out[i][e]], mul(qx[hc.in1[i][e]], qy[hc.in2[i][e]]));
      sum = add(sum, mul(term, t == 0 ? vsum : vprod));
    }
    if (!eq(claim, mul(eq_point(zb, rb), sum))) return SISU_ERR_REJECT;
    HF vv[2] = {vx, vy};
    tr.absorb('V', vv, 2);
    if (i + 1 < d) {
      alpha = tr.challenge();
      beta = tr.challenge();
      claim = add(mul(alpha, vx), mul(beta, vy));
      zb = rb;
      prx = rx;
      pry = ry;
    } else {
      std::vector<HF> p1(rb), p2(rb);
      p1.insert(p1.end(), rx.begin(), rx.end());
      p2.insert(p2.end(), ry.begin(), ry.end());
      if (!eq(vx, mle(Vin, p1)) || !eq(vy, mle(Vin, p2))) return SISU_ERR_REJECT;
    }
  }
  if (pos != proof_len) return SISU_ERR_REJECT;
  return SISU_OK;
}

// General circuits (Sec. 2.7): layer i's rounds run over its virtual layer
// X_i (2^sx positions); the layer ends with every block's part of
// X~_i(r_b, r_x) and X~_i(r_b, r_y).  The final identity sums the weight
// terms of the layer's claims, each with its own copy point; a block on the
// input layer is checked against the clear inputs, any other becomes a term
// of its layer's claim with two fresh coefficients.
static int host_verify_general(const HostCircuit& hc, const uint8_t* inputs, const uint8_t* outputs,
                               const uint8_t* proof, size_t proof_len, const uint8_t* domain, size_t dlen) {
  const uint32_t d = hc.d, c = hc.c;
  if (proof_len != hc.proof_len()) return SISU_ERR_REJECT;
  {
    std::vector<uint8_t> hdr(8 + 4 * ((size_t)d + 3));
    memcpy(hdr.data(), "SISUGKR2", 8);
    auto put = [&](size_t at, uint32_t v) {
      for (int k = 0; k < 4; ++k) hdr[at + k] = (uint8_t)(v >> (8 * k));
    };
    put(8, d);
    put(12, c);
    for (uint32_t i = 0; i <= d; ++i) put(16 + 4 * (size_t)i, hc.s[i]);
    if (memcmp(hdr.data(), proof, hdr.size()) != 0) return SISU_ERR_REJECT;
  }
  size_t pos = 8 + 4 * ((size_t)d + 3);
  auto next = [&](HF* x) -> bool {
    if (pos + 32 > proof_len) return false;
    bool ok = load(proof + pos, x);
    pos += 32;
    return ok;
  };
  std::vector<uint8_t> in_b = padded_bytes(inputs, hc.C, hc.W[d], hc.Creal, hc.wreal[d]);
  std::vector<uint8_t> out_b = padded_bytes(outputs, hc.C, hc.W[0], hc.Creal, hc.wreal[0]);
  std::vector<HF> Vin, Vout;
  if (!load_table(in_b, &Vin) || !load_table(out_b, &Vout)) return SISU_ERR_NOT_CANONICAL;
  uint32_t dig_in[8], dig_out[8];
  host_statement_digest(in_b.data(), in_b.size(), dig_in);
  host_statement_digest(out_b.data(), out_b.size(), dig_out);
  Transcript tr;
  {
    Sha256Stream h;
    h.begin();
    h.bytes(domain, dlen);
    h.byte(0);
    h.u32le(d);
    h.u32le(c);
    for (uint32_t i = 0; i <= d; ++i) h.u32le(hc.s[i]);
    h.digest_words(hc.wiring_digest);
    h.digest_words(dig_in);
    h.digest_words(dig_out);
    h.end(tr.st);
  }
  struct Term {
    std::vector<HF> z, M;
  };
  std::vector<std::vector<Term>> terms(d + 1);
  std::vector<HF> claims(d + 1, kZero);
  std::vector<HF> zb(c), zg(hc.s[0]);
  for (auto& z : zb) z = tr.challenge();
  for (auto& z : zg) z = tr.challenge();
  terms[0].push_back({zb, eq_table(zg)});
  {
    std::vector<HF> pt(zb);
    pt.insert(pt.end(), zg.begin(), zg.end());
    claims[0] = mle(Vout, pt);
  }
  static const Lagrange lag;
  for (uint32_t i = 0; i < d; ++i) {
    const uint32_t sx = hc.sx[i], nb = (uint32_t)hc.blocks[i].size();
    HF claim = claims[i];
    std::vector<HF> rb(c), rx(sx), ry(sx);
    for (uint32_t k = 0; k < c; ++k) {
      HF g[4], sent[3];
      for (auto& v : sent)
        if (!next(&v)) return SISU_ERR_REJECT;
      g[0] = sent[0]; g[1] = sub(claim, sent[0]); g[2] = sent[1]; g[3] = sent[2];
      tr.absorb('R', sent, 3);
      rb[k] = tr.challenge();
      claim = lag.at(g, 4, rb[k]);
    }
    for (int phase = 0; phase < 2; ++phase)
      for (uint32_t k = 0; k < sx; ++k) {
        HF g[3], sent[2];
        for (auto& v : sent)
          if (!next(&v)) return SISU_ERR_REJECT;
        g[0] = sent[0]; g[1] = sub(claim, sent[0]); g[2] = sent[1];
        tr.absorb('R', sent, 2);
        HF r = tr.challenge();
        (phase == 0 ? rx : ry)[k] = r;
        claim = lag.at(g, 3, r);
      }
    std::vector<HF> vb(2 * (size_t)nb);
    HF vx = kZero, vy = kZero;
    for (uint32_t b = 0; b < 2 * nb; ++b)
      if (!next(&vb[b])) return SISU_ERR_REJECT;
    for (uint32_t b = 0; b < nb; ++b) {
      vx = add(vx, vb[b]);
      vy = add(vy, vb[nb + b]);
    }
    // final identity over the layer's weight terms
    const std::vector<HF> qx = eq_table(rx), qy = eq_table(ry);
    const HF vsum = add(vx, vy), vprod = mul(vx, vy);
    HF sum = kZero;
    for (const Term& T : terms[i]) {
      HF part = kZero;
      for (size_t e = 0; e < hc.out[i].size(); ++e) {
        HF term = mul(T.M[hc.out[i][e]], mul(qx[hc.in1[i][e]], qy[hc.u2[i][e]]));
        part = add(part, mul(term, hc.type[i][e] == 0 ? vsum : vprod));
      }
      sum = add(sum, mul(eq_point(T.z, rb), part));
    }
    if (!eq(claim, sum)) return SISU_ERR_REJECT;
    tr.absorb('V', vb.data(), (int)vb.size());
    const std::vector<HF> erb = eq_table(rb);
    for (uint32_t b = 0; b < nb; ++b) {
      const HostCircuit::Block& B = hc.blocks[i][b];
      auto gate = [&](uint32_t k) { return b == 0 ? k : B.ys[k]; };
      if (B.layer == d) {  // against the clear inputs
        HF wx = kZero, wy = kZero;
        for (uint32_t k = 0; k < B.count; ++k) {
          HF col = kZero;
          for (uint32_t q = 0; q < hc.C; ++q) col = add(col, mul(erb[q], Vin[(size_t)q * hc.W[d] + gate(k)]));
          wx = add(wx, mul(qx[B.base + k], col));
          wy = add(wy, mul(qy[B.base + k], col));
        }
        if (!eq(wx, vb[b]) || !eq(wy, vb[nb + b])) return SISU_ERR_REJECT;
        continue;
      }
      const HF ax = tr.challenge(), ay = tr.challenge();
      Term T{rb, std::vector<HF>(hc.W[B.layer], kZero)};
      for (uint32_t k = 0; k < B.count; ++k) T.M[gate(k)] = add(mul(ax, qx[B.base + k]), mul(ay, qy[B.base + k]));
      terms[B.layer].push_back(std::move(T));
      claims[B.layer] = add(claims[B.layer], add(mul(ax, vb[b]), mul(ay, vb[nb + b])));
    }
  }
  if (pos != proof_len) return SISU_ERR_REJECT;
  return SISU_OK;
}

}  // namespace sisu
