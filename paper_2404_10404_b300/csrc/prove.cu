// Prover kernels: the device transcript, layer initialisation, the copy
// phase and Libra's two phases of the GKR layer sumcheck.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "fr_wide.cuh"
#include "internal.h"
#include "launch.cuh"
#include "sha256.cuh"

namespace sisu {

// ---------------------------------------------------------------------------
// small device helpers

__device__ __forceinline__ Fr fr_one_minus(const Fr& z) { return fr_sub(fr_one(), z); }

// eq(r_1..r_s, v) = prod_k (bit_k(v) ? r_k : 1 - r_k), bit 1 = most significant
__device__ __forceinline__ Fr eq_index(const Fr* r, uint32_t s, uint32_t v) {
  Fr acc = fr_one();
  for (uint32_t k = 0; k < s; ++k) {
    uint32_t bit = (v >> (s - 1 - k)) & 1u;
    acc = fr_mul(acc, bit ? r[k] : fr_one_minus(r[k]));
  }
  return acc;
}

// x + r (y - x): the multilinear line through two table entries
__device__ __forceinline__ Fr fold2(const Fr& x, const Fr& y, const Fr& r) {
  return fr_add(x, fr_mul(r, fr_sub(y, x)));
}

__device__ __forceinline__ void store_words(uint8_t* base, size_t off, const Fr& canon) {
  uint32_t* p = reinterpret_cast<uint32_t*>(base + off);
#pragma unroll
  for (int i = 0; i < 8; ++i) p[i] = canon.v[i];
}

// ---------------------------------------------------------------------------
// Fiat-Shamir transcript on the SHA-256 compression function F (the paper
// fixes no hash; this convention is the project's own):
//   absorb:    h = st with word 7 xor (256 tag + n); h = F(h, B) for every
//              64-byte block B of the n canonical LE elements (zero-padded
//              to whole blocks); st = h.
//   challenge: unless the state is fresh from an absorb (or from the
//              initial hash), st = F(st, Q(ctr++)) first; then while
//              x = LE(st) mod 2^254 >= r, st = F(st, Q(ctr++)).  The
//              challenge is the field element whose Montgomery form is x
//              (x 2^-256 mod r), so it needs no conversion.
//              Q(c) = 'C' || u32le c || 59 zero bytes.
// A round thus costs two compressions (absorb of three or four elements)
// where a full SHA-256 of the message and a separate challenge hash took
// four, and the hash runs on the critical path of every round.

// The compression runs out of line in one of two forms: the compact loop
// (kSmall) for the single-thread kernels that run it once, cold (transcript
// init, layer end of wide layers); the unrolled form everywhere it is warm:
// the cluster kernel of Libra's phases, and the round kernels, which warm it
// at their start (warm_transcript_code).
template <bool kSmall>
__device__ __forceinline__ ShaWords8 tr_compress(const ShaWords8& h, const ShaWords16& blk) {
  return kSmall ? sha256_compress_small_v(h, blk) : sha256_compress_v(h, blk);
}

// absorb of N canonical elements (N <= 4)
template <int N, bool kSmall>
__device__ __noinline__ void tr_absorb_n(uint32_t* st, uint32_t tag, const Fr* canon) {
  constexpr int NB = (8 * N + 15) / 16;  // blocks
  ShaWords8 h;
#pragma unroll
  for (int i = 0; i < 8; ++i) h.w[i] = st[i];
  h.w[7] ^= (tag << 8) | (uint32_t)N;
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    ShaWords16 blk;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const int w = 16 * b + k;  // message word: limb w % 8 of element w / 8, byte-swapped
      blk.w[k] = w < 8 * N ? bswap32(canon[w >> 3].v[w & 7]) : 0u;
    }
    h = tr_compress<kSmall>(h, blk);
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) st[i] = h.w[i];
}

template <bool kSmall>
__device__ __forceinline__ ShaWords8 tr_squeeze(const ShaWords8& h, uint32_t ctr) {
  ShaWords16 q;
#pragma unroll
  for (int k = 0; k < 16; ++k) q.w[k] = 0;
  q.w[0] = (uint32_t('C') << 24) | ((ctr & 0xffu) << 16) | (((ctr >> 8) & 0xffu) << 8) | ((ctr >> 16) & 0xffu);
  q.w[1] = (ctr >> 24) << 24;
  return tr_compress<kSmall>(h, q);
}

// next challenge (Montgomery form) from the state st; `fresh`: the state
// comes straight from an absorb or the initial hash.  A bounded number of
// tries (each rejected with probability below 1/4), then the error flag.
template <bool kSmall>
__device__ __noinline__ Fr tr_challenge_st(uint32_t* st, uint32_t* error, bool fresh) {
  ShaWords8 h;
#pragma unroll
  for (int i = 0; i < 8; ++i) h.w[i] = st[i];
  uint32_t ctr = 0;
  if (!fresh) h = tr_squeeze<kSmall>(h, ctr++);
  for (; ctr < 4096u; h = tr_squeeze<kSmall>(h, ctr++)) {
    Fr x;
#pragma unroll
    for (int k = 0; k < 8; ++k) x.v[k] = bswap32(h.w[k]);
    x.v[7] &= 0x3fffffffu;
    if (fr_lt_modulus(x)) {
#pragma unroll
      for (int i = 0; i < 8; ++i) st[i] = h.w[i];
      return x;
    }
  }
  atomicOr(error, 2u);
  return fr_zero();
}

// One lane of a round kernel runs the unrolled compression once on scratch
// words at the start, so that its code is in the SM's instruction caches when
// the last CTA runs the round's transcript at the end.  Cold, the unrolled
// form was slower there than the compact loop; warm, it is faster (medium
// step 19.64 -> 19.35 ms).
__device__ __forceinline__ void warm_transcript_code(uint32_t a, uint32_t b) {
  ShaWords8 hw;
  ShaWords16 bw;
#pragma unroll
  for (int i = 0; i < 8; ++i) hw.w[i] = a + i;
#pragma unroll
  for (int i = 0; i < 16; ++i) bw.w[i] = b + i;
  hw = tr_compress<false>(hw, bw);
  asm volatile("" ::"r"(hw.w[0]));
}

// the transcripts of the single-thread kernels (transcript init, layer end)
__device__ __forceinline__ Fr tr_challenge(DevState* S, bool fresh) {
  return tr_challenge_st<true>(S->st, &S->error, fresh);
}

// The last block of a round, called by the lanes of its warp 0 with the
// grid-wide sums g(0..NV-1) in lane 0: the round message g(0), g(2), ...,
// g(NV-1) (g(1) is left out: the verifier takes it as the claim minus g(0))
// as canonical values into the proof, one lane each, then absorb 'R' and
// squeeze the round's challenge.  The sums are plain (not Montgomery)
// values below 2r: the copy weights E and the Libra tables H, K are kept
// plain, so one conditional subtraction makes them canonical.
template <int NV>
__device__ __forceinline__ void round_finalize(DevState* S, const Fr (&v)[NV], uint8_t* proof, size_t off,
                                               Fr* rslot) {
  __shared__ Fr sh[NV];
  const int lane = threadIdx.x & 31;
  if (lane == 0) {
    sh[0] = v[0];
#pragma unroll
    for (int t = 2; t < NV; ++t) sh[t - 1] = v[t];
  }
  __syncwarp();
  if (lane < NV - 1) {
    Fr c = fr_reduce_once(sh[lane]);
    store_words(proof, off + 32 * (size_t)lane, c);
    sh[lane] = c;
  }
  __syncwarp();
  if (lane == 0) {
    Fr canon[NV - 1];
#pragma unroll
    for (int t = 0; t < NV - 1; ++t) canon[t] = sh[t];
    tr_absorb_n<NV - 1, false>(S->st, 'R', canon);
    *rslot = tr_challenge_st<false>(S->st, &S->error, true);
  }
}

// Block-wide sum of NV field elements per thread; result in thread 0.
template <int BD, int NV>
__device__ __forceinline__ void block_sum(Fr (&v)[NV]) {
  __shared__ Fr red[NV][BD / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int t = 0; t < NV; ++t) v[t] = fr_warp_sum(v[t]);
  if (BD > 32) {
    if (lane == 0)
#pragma unroll
      for (int t = 0; t < NV; ++t) red[t][warp] = v[t];
    __syncthreads();
    if (warp == 0) {
#pragma unroll
      for (int t = 0; t < NV; ++t) {
        Fr x = lane < BD / 32 ? red[t][lane] : fr_zero();
        v[t] = fr_warp_sum(x);
      }
    }
    __syncthreads();
  }
}

// Writes this block's partial sums; returns true in the last block to
// finish, which then holds the grid-wide sums in thread 0's v.  With
// kInThread0 the block's sums are already in thread 0 (the other threads'
// v are ignored), so the block reduction is skipped.  The last block sums
// the partials with one warp per value (NV <= BD / 32).
template <int BD, int NV, bool kInThread0 = false>
__device__ __forceinline__ bool grid_sum_last_block(Fr (&v)[NV], uint32_t* partials, DevState* S) {
  static_assert(NV <= BD / 32, "one warp per value");
  __shared__ bool is_last;
  __shared__ Fr tot[NV];
  const uint32_t nblk = gridDim.x * gridDim.y;
  const uint32_t bid = blockIdx.y * gridDim.x + blockIdx.x;
  if (!kInThread0) block_sum<BD, NV>(v);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int t = 0; t < NV; ++t) fr_store_cg(partials, (size_t)bid * NV + t, v[t]);
    __threadfence();
    uint32_t prev = atomicAdd(&S->counter, 1u);
    is_last = (prev == nblk - 1);
  }
  __syncthreads();
  if (!is_last) return false;
  __threadfence();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (warp < NV) {  // warp t sums value t over every block's partial
    Fr x = fr_zero();
    for (uint32_t p = lane; p < nblk; p += 32) x = fr_add(x, fr_load_cg(partials, (size_t)p * NV + warp));
    x = fr_warp_sum(x);
    if (lane == 0) tot[warp] = x;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int t = 0; t < NV; ++t) v[t] = tot[t];
    S->counter = 0;
  }
  return true;
}

// ---------------------------------------------------------------------------
// transcript initialisation and the initial claim point z = (z_b, z_g)
//   st = SHA256(domain || 0x00 || u32le d || u32le c || u32le s_0..s_d ||
//               Dig(wiring) || Dig(inputs) || Dig(outputs))

__global__ void k_transcript_init(InitParams p, DevState* S) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  Sha256Stream h;
  h.begin();
  h.bytes(p.domain, p.dlen);
  h.byte(0);
  h.u32le(p.d);
  h.u32le(p.c);
  for (uint32_t i = 0; i <= p.d; ++i) h.u32le(p.s[i]);
  h.digest_words(p.wiring);
  h.digest_words(S->dig_in);
  h.digest_words(S->dig_out);
  uint32_t o[8];
  h.end(o);
  for (int i = 0; i < 8; ++i) S->st[i] = o[i];
  S->counter = 0;
  S->error = 0;
  // the first challenge reads the fresh initial state
  for (uint32_t k = 0; k < p.c; ++k) S->zb[k] = tr_challenge(S, k == 0);
  for (uint32_t k = 0; k < p.s[0]; ++k) S->zg[k] = tr_challenge(S, p.c == 0 && k == 0);
}

int launch_transcript_init(const InitParams& p, DevState* S, void* stream) {
  k_transcript_init<<<1, 32, 0, (cudaStream_t)stream>>>(p, S);
  return post_launch();
}

// ---------------------------------------------------------------------------
// layer initialisation: E = EQ(copy point) over the 2^c copies and the gate
// weights w(g) over the layer's present gates (in the sorted order):
//   layer 0:  w(g) = eq(z_g, g)
//   layer i:  w(g) = alpha eq(r_x, g) + beta eq(r_y, g)   (previous layer's r_x, r_y)
//
// Each eq over n bits is the product of two half tables, over the high
// n - n/2 and the low n/2 bits of the index (bit 1 of the point binds the
// most significant index bit).  A first launch builds the half tables (at
// most n/2 + 1 products an entry, alpha and beta folded into the high
// halves), a second combines them: one product per E entry, one or two per
// gate weight, where a direct product over all bits took n.

__host__ __device__ inline uint32_t eq_half_entries(uint32_t n) { return (1u << (n - n / 2)) + (1u << (n / 2)); }

// entry v of the table over bits k0 .. k0 + nb - 1 of point P, started from init
__device__ __forceinline__ Fr eq_half_entry(const Fr* P, uint32_t k0, uint32_t nb, uint32_t v, Fr acc) {
  for (uint32_t b = 0; b < nb; ++b) {
    const Fr pk = P[k0 + b];
    acc = fr_mul(acc, ((v >> (nb - 1 - b)) & 1u) ? pk : fr_one_minus(pk));
  }
  return acc;
}

// Half tables, in order: E high (plain: started from the integer 1), E low;
// then layer 0: z_g high, low; layer i: alpha r_x high, r_x low, beta r_y
// high, r_y low.
//
// With cq > 0 the copies are those of one rank of 2^cq holding the copies
// b = j 2^cq + q (Sec. 3.2.1: the machine index as the low copy bits): E
// runs over the c high bits of b only, and its high half starts from the
// rank's factor eq(point bits c .. c + cq - 1, q), so that E(j) is the
// weight of global copy j 2^cq + q.
__global__ void k_eq_halves(DevState* S, uint32_t layer, uint32_t c, uint32_t si, uint32_t* __restrict__ tab,
                            uint32_t cq, uint32_t q) {
  pdl_wait();
  const uint32_t nE = eq_half_entries(c), nW = eq_half_entries(si);
  const uint32_t total = nE + (layer == 0 ? nW : 2 * nW);
  for (uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
    const bool isE = idx < nE;
    const uint32_t n = isE ? c : si;
    uint32_t u = isE ? idx : (idx - nE) % nW;
    const uint32_t which = isE ? 0 : (idx - nE) / nW;  // 0: z_g or r_x, 1: r_y
    const uint32_t nh = n - n / 2, hsize = 1u << nh;
    const bool hi = u < hsize;
    if (!hi) u -= hsize;
    const Fr* P = isE ? (layer == 0 ? S->zb : S->rb) : layer == 0 ? S->zg : which == 0 ? S->rx : S->ry;
    Fr init = fr_one();
    // the copy weights come out plain and scaled by 2^32 (see the copy round)
    if (hi) init = isE ? fr_int_2_32() : layer == 0 ? fr_one() : which == 0 ? S->alpha : S->beta;
    if (hi && isE && cq) init = eq_half_entry(P, c, cq, q, init);  // the rank's factor
    fr_store(tab, idx, eq_half_entry(P, hi ? 0 : nh, hi ? nh : n / 2, u, init));
  }
}

// om: the gate weights in entry order (om[q] = w(gate of entry q)); omo (not
// null; nsg = the entries of sg): also in gate order, 0 for a gate with no
// entry (a gate's several entries all write its one weight).
__global__ void k_layer_init(uint32_t layer, uint32_t c, uint32_t si, const uint4* __restrict__ sg, uint32_t ntot,
                             const uint32_t* __restrict__ tab, uint32_t* __restrict__ E, uint32_t* __restrict__ om,
                             uint32_t* __restrict__ omo, uint32_t nsg) {
  pdl_wait();
  const uint32_t C = 1u << c;
  const size_t total = (size_t)C + (omo ? nsg : ntot);
  const uint32_t nE = eq_half_entries(c), nW = eq_half_entries(si);
  const uint32_t cl = c / 2, sl = si / 2;
  const uint32_t* Eh = tab;
  const uint32_t* El = tab + 8 * ((size_t)1 << (c - cl));
  const uint32_t* Xh = tab + 8 * (size_t)nE;
  const uint32_t* Xl = Xh + 8 * ((size_t)1 << (si - sl));
  const uint32_t* Yh = Xh + 8 * (size_t)nW;
  const uint32_t* Yl = Yh + 8 * ((size_t)1 << (si - sl));
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    if (idx < C) {
      const uint32_t v = (uint32_t)idx;
      fr_store(E, idx, fr_mul(fr_load(Eh, v >> cl), fr_load(El, v & ((1u << cl) - 1))));  // plain, times 2^32
    } else {
      const uint32_t q = (uint32_t)(idx - C), g = sg[q].z, gh = g >> sl, gl = g & ((1u << sl) - 1);
      if (q >= ntot) {  // a gate with no entry (omo only)
        fr_store(omo, g, fr_zero());
        continue;
      }
      Fr w = fr_mul(fr_load(Xh, gh), fr_load(Xl, gl));
      if (layer != 0) w = fr_add(w, fr_mul(fr_load(Yh, gh), fr_load(Yl, gl)));
      fr_store(om, q, w);
      if (omo) fr_store(omo, g, w);
    }
  }
}

size_t eq_half_words(uint32_t c, uint32_t smax) { return 8 * ((size_t)eq_half_entries(c) + 2 * eq_half_entries(smax)); }

int launch_layer_init(DevState* S, uint32_t layer, uint32_t c, uint32_t s_i, const DevLayer& L, uint32_t* E,
                      uint32_t* omega_s, uint32_t* eqh, void* stream, uint32_t cq, uint32_t q, uint32_t* omega_o) {
  cudaStream_t st = (cudaStream_t)stream;
  const uint32_t nh = eq_half_entries(c) + (layer == 0 ? 1 : 2) * eq_half_entries(s_i);
  const int rc = launch_pdl(k_eq_halves, grid_for(nh, 128), 128, st, S, layer, c, s_i, eqh, cq, q);
  if (rc) return rc;
  size_t n = ((size_t)1 << c) + (omega_o ? L.nsg : L.ntot);
  return launch_pdl(k_layer_init, grid_for(n, 128), 128, st, layer, c, s_i, L.sgate, L.ntot, (const uint32_t*)eqh, E,
                    omega_s, omega_o, L.nsg);
}

// ---------------------------------------------------------------------------
// copy-phase round (degree 3 in the bound copy variable):
//   g(t) = sum_{j < h} E_t(j) sum_g w(g) op_g(T_t(j, in1 g), T_t(j, in2 g)),  t = 0..3
// with X_t(j) = X(j) + t (X(j + h) - X(j)).  Per pair the gate sum S_j(t)
// is quadratic in t, S_j(t) = S_j(0) + (S_j(1) - S_j(0) - c_j) t + c_j t^2,
// so S_j(0), S_j(1) and the t^2 coefficient c_j fix it:
//   S_j(2) = 2 S_j(1) - S_j(0) + 2 c_j,  S_j(3) = 3 S_j(1) - 2 S_j(0) + 6 c_j.
// A mul gate w x_t y_t adds w x_0 y_0, w x_1 y_1 and (w x_1 - w x_0)(y_1 - y_0)
// (its t^2 coefficient); an add gate w (x_t + y_t) is affine in t and adds
// only to the first two.  The three sums are lazily reduced: each thread
// adds full 512-bit products (fracc_mac) and reduces once per pair segment,
// so a mul gate costs two Montgomery products and three full products, an
// add gate two full products.  The reduction leaves a factor 2^-32 in every
// sum; the copy weights E are kept scaled by 2^32 (from the layer init on,
// the folds being linear), so the weighted sums come out exact with no
// product to undo it.  Consumers of E(r_b) itself multiply by 2^-32 once.
//
// Work split: the (pair, gate) items, pair-major, are cut into ranges of
// equal cost (gates are sorted mul first, so equal item counts would leave
// some CTAs twice the work of others).  The weights kCostMul : kCostAdd are
// the measured times of the two kinds of item on B300 (a mul item, two
// Montgomery and three full products, takes about 2.2 times an add item,
// two full products).  With more pairs than CTAs each CTA takes one contiguous
// range and walks it one pair segment at a time; with fewer (the late,
// latency-bound rounds) each pair gets m CTAs and every range lies inside
// one pair, so no CTA pays the per-segment reduction twice.  After each
// segment the CTA sums S_j(t) over the block and four lanes of warp 0 apply
// the weights E_t(j) (plain form, so the weighted sums are plain); the two
// weights are fetched with cp.async while the segment's items run.

constexpr uint64_t kCostMul = 9, kCostAdd = 4;

__host__ __device__ __forceinline__ uint64_t copy_pair_cost(uint32_t nmul, uint32_t ntot) {
  return kCostMul * nmul + kCostAdd * (ntot - nmul);
}

// item position of cost position X (rounded up to a gate boundary)
// gate position inside a pair of cost position r (0 <= r <= pair cost)
__device__ __forceinline__ uint64_t item_in_pair(uint64_t r, uint32_t nmul, uint32_t ntot) {
  const uint64_t mc = kCostMul * nmul;
  const uint64_t g = r < mc ? (r + kCostMul - 1) / kCostMul : nmul + (r - mc + kCostAdd - 1) / kCostAdd;
  return min(g, (uint64_t)ntot);
}

__device__ __forceinline__ uint64_t item_at_cost(uint64_t X, uint32_t nmul, uint32_t ntot, uint64_t pair_cost) {
  const uint64_t j = X / pair_cost;
  return j * ntot + item_in_pair(X - j * pair_cost, nmul, ntot);
}

// The split of a round's items over nc CTAs (at most ncmax, and no more than
// one CTA per `min_items` items): with h <= nc, m CTAs per pair and ranges of
// per_cta cost units inside a pair; otherwise one contiguous range of per_cta
// units per CTA (m = 0).
struct CopySplit {
  uint32_t nc, m;
  uint64_t per_cta;
};

__host__ __device__ __forceinline__ CopySplit copy_split(uint32_t h, uint32_t nmul, uint32_t ntot, uint32_t ncmax,
                                                         uint32_t min_items) {
  const uint64_t total = (uint64_t)h * ntot;
  const uint64_t pair_cost = copy_pair_cost(nmul, ntot);
  uint64_t nc = (total + min_items - 1) / min_items;
  if (nc > ncmax) nc = ncmax;
  if (nc < 1) nc = 1;
  CopySplit sp;
  if (h <= nc) {
    sp.m = (uint32_t)(nc / h);
    sp.per_cta = (pair_cost + sp.m - 1) / sp.m;
    sp.nc = h * sp.m;
  } else {
    const uint64_t total_cost = (uint64_t)h * pair_cost;
    sp.m = 0;
    sp.per_cta = (total_cost + nc - 1) / nc;
    sp.nc = (uint32_t)((total_cost + sp.per_cta - 1) / sp.per_cta);
  }
  return sp;
}

// The items of CTA `bid` of a round split by (per_cta, m): returns, in lanes
// t < 4 of warp 0, the CTA's share of g(t) (plain, below 2r).  Called by
// every thread of the block.
template <int BD>
__device__ __forceinline__ Fr copy_items(const uint32_t* __restrict__ T, uint32_t sn, uint32_t h,
                                         const uint32_t* __restrict__ E, const uint32_t* __restrict__ om,
                                         const uint4* __restrict__ sg, uint32_t nmul, uint32_t ntot,
                                         uint64_t per_cta, uint32_t m, uint32_t bid, uint32_t* sh_e) {
  const uint64_t pair_cost = copy_pair_cost(nmul, ntot);
  uint64_t q0, q1;  // the CTA's item range
  uint32_t j;       // the pair of its first item
  if (m) {  // a range inside pair j: no 64-bit division on the (latency-bound) late rounds
    j = bid / m;
    const uint32_t sub = bid - j * m;
    const uint64_t base = (uint64_t)j * ntot;
    q0 = base + item_in_pair(min(pair_cost, (uint64_t)sub * per_cta), nmul, ntot);
    q1 = base + item_in_pair(min(pair_cost, (uint64_t)(sub + 1) * per_cta), nmul, ntot);
  } else {
    const uint64_t total_cost = (uint64_t)h * pair_cost;
    q0 = item_at_cost(min(total_cost, (uint64_t)bid * per_cta), nmul, ntot, pair_cost);
    q1 = item_at_cost(min(total_cost, (uint64_t)(bid + 1) * per_cta), nmul, ntot, pair_cost);
    j = (uint32_t)(q0 / ntot);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  Fr tot = fr_zero();  // lane t < 4 of warp 0: sum over segments of E_t(j) S_j(t)
  for (uint64_t seg = q0; seg < q1; ++j) {  // one segment per pair, pairs in order
    const uint64_t segend = min(q1, (uint64_t)(j + 1) * ntot);
    if (threadIdx.x < 4) {  // E(j) -> sh_e[0..7], E(j + h) -> sh_e[8..15], 16 bytes a thread
      __syncwarp(0xfu);     // the previous segment's reads of sh_e are done
      const uint32_t* src = E + 8 * (size_t)(threadIdx.x < 2 ? j : j + h) + 4 * (threadIdx.x & 1);
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n\tcp.async.commit_group;" ::"r"(
                       (uint32_t)__cvta_generic_to_shared(sh_e + 4 * threadIdx.x)),
                   "l"(src)
                   : "memory");
    }
    const uint32_t g0 = (uint32_t)(seg - (uint64_t)j * ntot), g1 = (uint32_t)(segend - (uint64_t)j * ntot);
    const uint32_t* lo = T + (((size_t)j << sn) << 3);
    const uint32_t* hi = T + (((size_t)(j + h) << sn) << 3);
    FrAcc a0 = fracc_zero(), a1 = fracc_zero(), ac = fracc_zero();
    for (uint32_t q = g0 + threadIdx.x; q < g1; q += BD) {
      const uint4 gi = sg[q];
      const Fr w = fr_load(om, q);
      const Fr x0 = fr_load(lo, gi.x), x1 = fr_load(hi, gi.x);
      const Fr y0 = fr_load(lo, gi.y), y1 = fr_load(hi, gi.y);
      if (q < nmul) {
        const Fr wx0 = fr_mul(w, x0), wx1 = fr_mul(w, x1);
        fracc_mac(a0, wx0, y0);
        fracc_mac(a1, wx1, y1);
        fracc_mac(ac, fr_sub(wx1, wx0), fr_sub(y1, y0));
      } else {
        fracc_mac(a0, w, fr_add(x0, y0));
        fracc_mac(a1, w, fr_add(x1, y1));
      }
    }
    Fr s[3] = {fr_redc288(a0), fr_redc288(a1), fr_redc288(ac)};
    block_sum<BD, 3>(s);  // thread 0 holds 2^-32 (S_j(0), S_j(1), c_j) for this segment
    if (warp == 0) {
      Fr sj[3];
#pragma unroll
      for (int t = 0; t < 3; ++t)
#pragma unroll
        for (int i = 0; i < 8; ++i) sj[t].v[i] = __shfl_sync(0xffffffffu, s[t].v[i], 0);
      if (lane < 4) {
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        __syncwarp(0xfu);  // every lane sees all four copies
        Fr e0, e1;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          e0.v[i] = sh_e[i];
          e1.v[i] = sh_e[8 + i];
        }
        const Fr de = fr_sub(e1, e0);
        Fr et = e0, st;
        const Fr d = fr_sub(sj[1], sj[0]);
        if (lane == 2) {
          st = fr_add(fr_add(sj[1], d), fr_dbl(sj[2]));  // S(1) + (S(1) - S(0)) + 2c
        } else if (lane == 3) {
          st = fr_add(sj[1], fr_dbl(fr_add(d, fr_add(sj[2], fr_dbl(sj[2])))));  // S(1) + 2 (S(1) - S(0) + 3c)
        } else {
          st = lane == 0 ? sj[0] : sj[1];
        }
        for (int t = 0; t < lane; ++t) et = fr_add(et, de);
        tot = fr_add(tot, fr_mul(et, st));
      }
    }
    seg = segend;
  }
  return tot;  // E's factor 2^32 has cancelled the reductions' 2^-32
}

// Gathers of the per-warp item loop staged through shared memory: each
// lane copies its next item's five elements (w, x0, x1, y0, y1) there with
// 16-byte cp.async while it computes the current one, so the products never
// wait on an L2 or DRAM gather.  A warp's area holds two stages of five
// elements a lane, each element as two 16-byte halves in lane-contiguous
// rows (conflict-free 16-byte accesses).
constexpr uint32_t kStageWords4 = 2 * 5 * 2 * 32;  // 16-byte words a warp (10 KiB)

__device__ __forceinline__ uint4* stage_slot(uint4* stg, int st, int f, int half, int lane) {
  return stg + ((st * 5 + f) * 2 + half) * 32 + lane;
}

__device__ __forceinline__ void stage_issue(uint4* stg, int st, int lane, const uint32_t* w,
                                            const uint32_t* x0, const uint32_t* x1, const uint32_t* y0,
                                            const uint32_t* y1) {
  const uint32_t* src[5] = {w, x0, x1, y0, y1};
#pragma unroll
  for (int f = 0; f < 5; ++f)
#pragma unroll
    for (int half = 0; half < 2; ++half)
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                       (uint32_t)__cvta_generic_to_shared(stage_slot(stg, st, f, half, lane))),
                   "l"(src[f] + 4 * half)
                   : "memory");
}

__device__ __forceinline__ Fr stage_read(uint4* stg, int st, int f, int lane) {
  const uint4 a = *stage_slot(stg, st, f, 0, lane), b = *stage_slot(stg, st, f, 1, lane);
  Fr x;
  x.v[0] = a.x; x.v[1] = a.y; x.v[2] = a.z; x.v[3] = a.w;
  x.v[4] = b.x; x.v[5] = b.y; x.v[6] = b.z; x.v[7] = b.w;
  return x;
}

// The round's items of the big rounds (more pairs than CTAs, m = 0), split
// further: each warp of CTA `bid` owns a contiguous 1/NW of the CTA's cost
// range, sums every pair segment it touches with warp shuffles and weights
// it by E_t(j) itself, so the CTA meets no block barrier per segment (in
// the CTA-wide form every segment ended in a block reduction, where warps
// that finished early waited).  Returns, in lanes t < 4 of every warp, the
// warp's share of g(t) (plain, below 2r); sh_e: this warp's 16 words.
template <int BD>
__device__ __forceinline__ Fr copy_items_warp(const uint32_t* __restrict__ T, uint32_t sn, uint32_t h,
                                              const uint32_t* __restrict__ E, const uint32_t* __restrict__ om,
                                              const uint4* __restrict__ sg, uint32_t nmul, uint32_t ntot,
                                              uint64_t per_cta, uint32_t m, uint32_t bid, uint32_t* sh_e,
                                              uint4* stg) {
  constexpr int NW = BD / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint64_t pair_cost = copy_pair_cost(nmul, ntot);
  uint64_t c0, c1;  // the CTA's cost range
  if (m) {  // range `sub` of the m inside pair j
    const uint32_t j = bid / m, sub = bid - j * m;
    c0 = (uint64_t)j * pair_cost + min(pair_cost, (uint64_t)sub * per_cta);
    c1 = (uint64_t)j * pair_cost + min(pair_cost, (uint64_t)(sub + 1) * per_cta);
  } else {
    const uint64_t total_cost = (uint64_t)h * pair_cost;
    c0 = min(total_cost, (uint64_t)bid * per_cta);
    c1 = min(total_cost, c0 + per_cta);
  }
  const uint64_t q0 = item_at_cost(c0 + (c1 - c0) * warp / NW, nmul, ntot, pair_cost);
  const uint64_t q1 = item_at_cost(c0 + (c1 - c0) * (warp + 1) / NW, nmul, ntot, pair_cost);
  uint32_t j = (uint32_t)(q0 / ntot);
  Fr tot = fr_zero();  // lane t < 4: sum over segments of E_t(j) S_j(t)
  for (uint64_t seg = q0; seg < q1; ++j) {  // one segment per pair, pairs in order
    const uint64_t segend = min(q1, (uint64_t)(j + 1) * ntot);
    if (lane < 4) {  // E(j) -> sh_e[0..7], E(j + h) -> sh_e[8..15], 16 bytes a lane
      __syncwarp(0xfu);  // the previous segment's reads of sh_e are done
      const uint32_t* src = E + 8 * (size_t)(lane < 2 ? j : j + h) + 4 * (lane & 1);
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n\tcp.async.commit_group;" ::"r"(
                       (uint32_t)__cvta_generic_to_shared(sh_e + 4 * lane)),
                   "l"(src)
                   : "memory");
    }
    const uint32_t g0 = (uint32_t)(seg - (uint64_t)j * ntot), g1 = (uint32_t)(segend - (uint64_t)j * ntot);
    const uint32_t* lo = T + (((size_t)j << sn) << 3);
    const uint32_t* hi = T + (((size_t)(j + h) << sn) << 3);
    FrAcc a0 = fracc_zero(), a1 = fracc_zero(), ac = fracc_zero();
    // two-stage pipeline: item q + 32's gathers are in flight while item q
    // is computed (one cp.async group a lane and item)
    uint32_t q = g0 + lane;
    int st = 0;
    if (q < g1) {
      const uint4 gi = sg[q];
      stage_issue(stg, 0, lane, om + 8 * (size_t)q, lo + 8 * (size_t)gi.x, hi + 8 * (size_t)gi.x,
                  lo + 8 * (size_t)gi.y, hi + 8 * (size_t)gi.y);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
    for (; q < g1; q += 32, st ^= 1) {
      const uint32_t qn = q + 32;
      if (qn < g1) {
        const uint4 gi = sg[qn];
        stage_issue(stg, st ^ 1, lane, om + 8 * (size_t)qn, lo + 8 * (size_t)gi.x, hi + 8 * (size_t)gi.x,
                    lo + 8 * (size_t)gi.y, hi + 8 * (size_t)gi.y);
      }
      asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 1;" ::: "memory");
      const Fr w = stage_read(stg, st, 0, lane);
      const Fr x0 = stage_read(stg, st, 1, lane), x1 = stage_read(stg, st, 2, lane);
      const Fr y0 = stage_read(stg, st, 3, lane), y1 = stage_read(stg, st, 4, lane);
      if (q < nmul) {
        const Fr wx0 = fr_mul(w, x0), wx1 = fr_mul(w, x1);
        fracc_mac(a0, wx0, y0);
        fracc_mac(a1, wx1, y1);
        fracc_mac(ac, fr_sub(wx1, wx0), fr_sub(y1, y0));
      } else {
        fracc_mac(a0, w, fr_add(x0, y0));
        fracc_mac(a1, w, fr_add(x1, y1));
      }
    }
    Fr sj[3] = {fr_redc288(a0), fr_redc288(a1), fr_redc288(ac)};
#pragma unroll
    for (int t = 0; t < 3; ++t) {
      sj[t] = fr_warp_sum(sj[t]);  // lane 0: 2^-32 (S_j(0), S_j(1), c_j) over this warp's items
#pragma unroll
      for (int i = 0; i < 8; ++i) sj[t].v[i] = __shfl_sync(0xffffffffu, sj[t].v[i], 0);
    }
    if (lane < 4) {
      asm volatile("cp.async.wait_group 0;" ::: "memory");
      __syncwarp(0xfu);  // every lane sees all four copies
      Fr e0, e1;
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        e0.v[i] = sh_e[i];
        e1.v[i] = sh_e[8 + i];
      }
      const Fr de = fr_sub(e1, e0);
      Fr et = e0, st;
      const Fr d = fr_sub(sj[1], sj[0]);
      if (lane == 2) {
        st = fr_add(fr_add(sj[1], d), fr_dbl(sj[2]));  // S(1) + (S(1) - S(0)) + 2c
      } else if (lane == 3) {
        st = fr_add(sj[1], fr_dbl(fr_add(d, fr_add(sj[2], fr_dbl(sj[2])))));  // S(1) + 2 (S(1) - S(0) + 3c)
      } else {
        st = lane == 0 ? sj[0] : sj[1];
      }
      for (int t = 0; t < lane; ++t) et = fr_add(et, de);
      tot = fr_add(tot, fr_mul(et, st));
    }
    seg = segend;
  }
  return tot;  // E's factor 2^32 has cancelled the reductions' 2^-32
}

// kWarp: the big rounds' form (m = 0, segments per warp); else the CTA-wide
// form (any split; used for m > 0).
// sums_out: null for a whole proof; for one rank of a copy-sharded proof
// the rank's round sums g(0..3) (plain, below 2r) go there instead of the
// round message and the transcript, which wait for every rank's sums.
template <int BD, bool kWarp>
__global__ void __launch_bounds__(BD) k_copy_round(const uint32_t* __restrict__ T, uint32_t sn, uint32_t h,
                                                   const uint32_t* __restrict__ E, const uint32_t* __restrict__ om,
                                                   const uint4* __restrict__ sg, uint32_t nmul, uint32_t ntot,
                                                   uint64_t per_cta, uint32_t m, uint32_t* partials, DevState* S,
                                                   uint8_t* proof, size_t off, uint32_t k, uint32_t* sums_out) {
  pdl_wait();
  __shared__ __align__(16) uint32_t sh_e[BD / 32][16];  // E(j), E(j + h) of a warp's current segment
  if (threadIdx.x == BD - 32) warm_transcript_code(k, h);
  Fr acc[4];  // thread 0: the CTA's share of g(0..3)
  if (!kWarp) {  // the CTA-wide form: lanes t < 4 of warp 0
    const Fr tot = copy_items<BD>(T, sn, h, E, om, sg, nmul, ntot, per_cta, m, blockIdx.x, sh_e[0]);
#pragma unroll
    for (int t = 0; t < 4; ++t) {
#pragma unroll
      for (int i = 0; i < 8; ++i) acc[t].v[i] = __shfl_sync(0xffffffffu, tot.v[i], t);
      if (threadIdx.x != 0) acc[t] = fr_zero();
    }
  } else {  // segments per warp, then the warps' sums by a shuffle tree in warp 0
    __shared__ Fr wtot[BD / 32][4];
    extern __shared__ uint4 cr_stage[];  // kStageWords4 a warp
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const Fr tot = copy_items_warp<BD>(T, sn, h, E, om, sg, nmul, ntot, per_cta, m, blockIdx.x, sh_e[warp],
                                       cr_stage + warp * kStageWords4);
    if (lane < 4) wtot[warp][lane] = tot;
    __syncthreads();
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      acc[t] = warp == 0 && lane < BD / 32 ? wtot[lane][t] : fr_zero();
      if (warp == 0) acc[t] = fr_warp_sum(acc[t]);
      if (threadIdx.x != 0) acc[t] = fr_zero();
    }
  }
  if (grid_sum_last_block<BD, 4, true>(acc, partials, S) && threadIdx.x < 32) {
    if (sums_out) {
      if (threadIdx.x == 0)
#pragma unroll
        for (int t = 0; t < 4; ++t) fr_store(sums_out, t, acc[t]);
    } else {
      round_finalize<4>(S, acc, proof, off, &S->rb[k]);
    }
  }
}

// A launch shape of a copy round: the CTA width (128, 256 or 384 threads),
// the form and the CTA count's granularity (min_items).  The tuning table
// (sisu_tune_copy_round; unset entries keep the default), per (log2 W_{i+1},
// log2 pairs), is k_copy_c's, the layered circuits' copy round.  This
// general form (general circuits, copy-sharded ranks) runs its default: 384
// threads (at 168 registers one CTA fills the register file with 12 warps;
// 256 threads left a third of it idle: round 1 of a medium layer 224 -> 206
// us), per-warp pair segments while pairs outnumber CTAs (else CTA-wide
// segments), about one (pair, gate) item a thread.
struct CopyTune {
  uint16_t bd;        // 0: unset
  uint8_t form;       // general form: 0 per-warp segments iff more pairs than CTAs, 1 CTA-wide, 2 per-warp
  uint32_t min_items;
};
constexpr uint32_t kTuneLog = 25;
static CopyTune g_copy_c_tune[kTuneLog][kTuneLog];

template <int BD>
static int copy_round_per_sm() {
  static int per_sm = 0;
  if (per_sm == 0) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_copy_round<BD, false>, BD, 0) != cudaSuccess || n < 1)
      n = 1;
    per_sm = n;
  }
  return per_sm;
}

template <int BD>
static int launch_copy_round_bd(int form, uint32_t min_items, const uint32_t* T, uint32_t sn, uint32_t h,
                                const uint32_t* E, const uint32_t* omega_s, const DevLayer& L, uint32_t* partials,
                                DevState* S, uint8_t* proof, size_t off, uint32_t k, cudaStream_t st,
                                uint32_t* sums_out) {
  const uint32_t ncmax = std::min<uint32_t>(kSMs * copy_round_per_sm<BD>(), kMaxPartials);
  // contiguous ranges of equal cost: one wave of CTAs, and for small rounds
  // about min_items items a CTA (short serial chains)
  const CopySplit sp = copy_split(h, L.nmul, L.ntot, ncmax, min_items ? min_items : BD);
  const bool warp = form == 2 || (form == 0 && sp.m == 0);
  if (warp) {
    const size_t smem = (size_t)(BD / 32) * kStageWords4 * sizeof(uint4);
    static bool attr = false;
    if (!attr) {
      const cudaError_t e = cudaFuncSetAttribute(k_copy_round<BD, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)smem);
      if (e != cudaSuccess) return (int)e;
      attr = true;
    }
    return launch_pdl_smem(k_copy_round<BD, true>, sp.nc, BD, smem, st, T, sn, h, E, omega_s, L.sgate, L.nmul,
                           L.ntot, sp.per_cta, sp.m, partials, S, proof, off, k, sums_out);
  }
  return launch_pdl(k_copy_round<BD, false>, sp.nc, BD, st, T, sn, h, E, omega_s, L.sgate, L.nmul, L.ntot,
                    sp.per_cta, sp.m, partials, S, proof, off, k, sums_out);
}

int launch_copy_round(const uint32_t* T, uint32_t sn, uint32_t h, const uint32_t* E, const uint32_t* omega_s,
                      const DevLayer& L, uint32_t* partials, DevState* S, uint8_t* proof, size_t off, uint32_t k,
                      void* stream, uint32_t* sums_out) {
  cudaStream_t st = (cudaStream_t)stream;
  const CopyTune t = {384, 0, 0};
  if (t.bd == 128)
    return launch_copy_round_bd<128>(t.form, t.min_items, T, sn, h, E, omega_s, L, partials, S, proof, off, k, st,
                                     sums_out);
  if (t.bd == 256)
    return launch_copy_round_bd<256>(t.form, t.min_items, T, sn, h, E, omega_s, L, partials, S, proof, off, k, st,
                                     sums_out);
  return launch_copy_round_bd<384>(t.form, t.min_items, T, sn, h, E, omega_s, L, partials, S, proof, off, k, st,
                                   sums_out);
}

int set_copy_tune(uint32_t sn, uint32_t log_pairs, uint32_t bd, uint32_t form, uint32_t min_items) {
  if (sn >= kTuneLog || log_pairs >= kTuneLog) return -1;
  if (bd != 0 && bd != 128 && bd != 256 && bd != 384) return -1;
  if (form > 2) return -1;
  g_copy_c_tune[sn][log_pairs] = CopyTune{(uint16_t)bd, (uint8_t)form, min_items};
  return 0;
}

// ---------------------------------------------------------------------------
// The copy phase by the recurrence of its linear part.
//
// Write U_k(j) = sum_g w(g) op_g(T_k(j, in1 g), T_k(j, in2 g)) for the gate
// sum of row j of round k's table (n_k = 2 h_k rows).  A pair's sums are
// S_j(0) = U_k(j) and S_j(1) = U_k(j + h_k), and the fold by r_k gives row j
// of the next table, whose gate sum is
//   U_{k+1}(j) = (1 - r_k) U_k(j) + r_k U_k(j + h_k) + (r_k^2 - r_k) c_j,
// c_j = sum over the mul entries of w (x1 - x0)(y1 - y0), the pair's t^2
// coefficient: an add gate's value folds linearly, and the product x' y' of
// two folded inputs is (1 - r) x0 y0 + r x1 y1 + (r^2 - r)(x1 - x0)(y1 - y0).
// So the first round's U_0(b) are the dot products of layer i's rows with
// the gate weights (k_rowdot), every round's items are the mul entries' t^2
// terms alone (one Montgomery and one full product a mul item, nothing for
// an add item), and U_{k+1} follows from U_k and the c_j of round k with
// two products a row.  The messages and the proof bytes are those of the
// item-by-item form; only the work changes.  U and c are kept as the lazy
// sums' reductions leave them (Montgomery form times 2^-32), which the copy
// weights' factor 2^32 cancels in the message.

constexpr uint32_t kRowDotThreads = 256;

// U(b) = sum_g w(g) V(b, g) for the C rows of layer i's values (2^sv a row),
// w in gate order.  A row goes to tpr = 2^lt consecutive threads (a power
// of two up to a CTA, chosen so that few rows still fill the GPU); each
// sums every tpr-th element of it, two a step with inlined full
// products into two accumulators (independent chains), the next step's row
// elements copied into shared memory by cp.async meanwhile (two stages; the
// weights, the same for every row, come through L1), and the row's threads
// add their sums by shuffles (and shared memory across warps).
__global__ void __launch_bounds__(kRowDotThreads) k_rowdot(const uint32_t* __restrict__ V, uint32_t sv,
                                                           const uint32_t* __restrict__ omo, uint32_t C,
                                                           uint32_t lt, uint32_t* __restrict__ U) {
  pdl_wait();
  __shared__ uint4 rd_stage[kRowDotThreads / 32][2 * 2 * 2 * 32];  // [warp][stage, element, half, lane]
  const uint32_t W = 1u << sv, tpr = 1u << lt;
  const uint32_t lane = threadIdx.x & 31, sub = threadIdx.x & (tpr - 1);
  uint4* stg = rd_stage[threadIdx.x >> 5];
  auto slot = [&](int st, int e, int half) { return stg + ((st * 2 + e) * 2 + half) * 32 + lane; };
  const size_t nthreads = (size_t)gridDim.x * kRowDotThreads;
  const size_t first = (size_t)blockIdx.x * kRowDotThreads + threadIdx.x;
  // every thread of a warp runs the same number of rows (for the shuffles)
  const size_t rows_per_pass = nthreads >> lt;
  const size_t passes = ((size_t)C + rows_per_pass - 1) / rows_per_pass;
  for (size_t pass = 0; pass < passes; ++pass) {
    const size_t b = pass * rows_per_pass + (first >> lt);
    FrAcc a0 = fracc_zero(), a1 = fracc_zero();
    if (b < C) {
      const uint32_t* row = V + ((b << sv) << 3);
      // step g: elements g and g + tpr (the second only while below W)
      auto issue = [&](int st, uint32_t g) {
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          if (e == 1 && g + tpr >= W) break;
          const uint32_t* src = row + 8 * (size_t)(g + e * tpr);
#pragma unroll
          for (int half = 0; half < 2; ++half)
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                             (uint32_t)__cvta_generic_to_shared(slot(st, e, half))),
                         "l"(src + 4 * half)
                         : "memory");
        }
      };
      auto staged = [&](int st, int e) {
        const uint4 lo = *slot(st, e, 0), hi = *slot(st, e, 1);
        Fr x;
        x.v[0] = lo.x; x.v[1] = lo.y; x.v[2] = lo.z; x.v[3] = lo.w;
        x.v[4] = hi.x; x.v[5] = hi.y; x.v[6] = hi.z; x.v[7] = hi.w;
        return x;
      };
      uint32_t g = sub;
      int st = 0;
      if (g < W) issue(0, g);
      asm volatile("cp.async.commit_group;" ::: "memory");
      for (; g < W; g += 2 * tpr, st ^= 1) {
        if (g + 2 * tpr < W) issue(st ^ 1, g + 2 * tpr);
        asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 1;" ::: "memory");
        fracc_mac_kara_inl(a0, fr_load(omo, g), staged(st, 0));
        if (g + tpr < W) fracc_mac_kara_inl(a1, fr_load(omo, g + tpr), staged(st, 1));
      }
    }
    fracc_add(a0, a1);
    Fr u = fr_redc288(a0);
    for (uint32_t o = min(tpr, 32u) >> 1; o > 0; o >>= 1) {
      Fr v;
#pragma unroll
      for (int i = 0; i < 8; ++i) v.v[i] = __shfl_down_sync(0xffffffffu, u.v[i], o);
      u = fr_add(u, v);
    }
    if (tpr > 32) {  // a row over several warps of the CTA: their sums through shared memory
      __shared__ Fr wsum[kRowDotThreads / 32];
      if (lane == 0) wsum[threadIdx.x >> 5] = u;
      __syncthreads();
      if (sub == 0)
        for (uint32_t w = 1; w < tpr / 32; ++w) u = fr_add(u, wsum[(threadIdx.x >> 5) + w]);
      __syncthreads();
    }
    if (b < C && sub == 0) fr_store(U, b, u);
  }
}

int launch_rowdot(const uint32_t* V, uint32_t sv, const uint32_t* omo, uint32_t C, uint32_t* U, void* stream) {
  // threads a row: enough that the C rows give at least 2048 threads an
  // SM, with at least 16 elements a thread and at most a CTA a row
  uint32_t lt = 0;
  while ((1u << lt) < kRowDotThreads && sv > lt + 4 && ((size_t)C << lt) < (size_t)kSMs * 2048) ++lt;
  const size_t threads = (size_t)C << lt;
  const unsigned grid = (unsigned)std::max<size_t>(1, std::min<size_t>((threads + kRowDotThreads - 1) / kRowDotThreads,
                                                                       (size_t)kSMs * 8));
  return launch_pdl(k_rowdot, grid, kRowDotThreads, (cudaStream_t)stream, V, sv, omo, C, lt, U);
}

// The work of pair j after its c_j is known, by the four lanes t = 0..3 of
// a group (mask: the group's lanes, which all call this): round k's gate
// sums U_k(j), U_k(j + h), formed from the previous round's (k > 0; the
// four products split over the lanes and stored to Ucur for the next
// round) or as k_rowdot left them in Ucur; then lane t's message term
// E_t(j) S_j(t), S_j(t) = U0 + t (U1 - U0) + (t^2 - t) c, added to its
// running sum.  withU false: the c term alone (t = 2, 3), for a share of
// c_j whose U terms come from the pair's first share.  rp, qp: r_{k-1} and
// r_{k-1}^2 - r_{k-1} (Montgomery form).
__device__ __forceinline__ void pair_group(uint32_t j, uint32_t h, uint32_t t, uint32_t mask, bool upd, bool withU,
                                           const uint32_t* Uprev, const uint32_t* cprev, uint32_t* Ucur,
                                           const uint32_t* E, const Fr& rp, const Fr& qp, const Fr& c, Fr& macc) {
  const uint32_t src0 = (threadIdx.x & 31) & ~3u;  // the group's lane 0
  Fr U0 = fr_zero(), U1 = fr_zero();
  if (withU) {
    Fr u;  // lanes 0, 2: U0, U1 once the shares of the update are in
    if (upd) {
      // lane t: rp (hi - lo) of row j + (t >> 1) h (t even), qp c of that row (t odd)
      const size_t row = j + (size_t)(t >> 1) * h;
      const Fr lo = fr_load(Uprev, row);
      const Fr a = (t & 1) ? fr_mul(qp, fr_load(cprev, row)) : fr_mul(rp, fr_sub(fr_load(Uprev, row + 2 * (size_t)h), lo));
      Fr o;
#pragma unroll
      for (int i = 0; i < 8; ++i) o.v[i] = __shfl_xor_sync(mask, a.v[i], 1);
      u = fr_add(fr_add(lo, a), o);
      if ((t & 1) == 0) fr_store(Ucur, row, u);
    } else {
      u = fr_load(Ucur, j + (size_t)(t >> 1) * h);
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      U0.v[i] = __shfl_sync(mask, u.v[i], src0);
      U1.v[i] = __shfl_sync(mask, u.v[i], src0 + 2);
    }
  }
  if (!withU && t < 2) return;
  const Fr e0 = fr_load(E, j), e1 = fr_load(E, j + (size_t)h);
  const Fr de = fr_sub(e1, e0);
  Fr et = t == 0 ? e0 : t == 1 ? e1 : fr_add(e1, de);
  if (t == 3) et = fr_add(et, de);
  const Fr d = fr_sub(U1, U0);
  const Fr c2 = fr_dbl(c);
  Fr st;
  if (t == 0) {
    st = U0;
  } else if (t == 1) {
    st = U1;
  } else if (t == 2) {
    st = fr_add(fr_add(U1, d), c2);  // U0 + 2 d + 2 c
  } else {
    st = fr_add(fr_add(U1, fr_dbl(d)), fr_dbl(fr_add(c2, c)));  // U0 + 3 d + 6 c
  }
  macc = fr_add(macc, fr_mul(et, st));
}

// One round of the copy phase over its mul entries (pairs j < h of the
// table T, 2^sn positions a row).  m = 0 (h at least the CTA count): CTA b
// takes the whole pairs [b h / nc, (b + 1) h / nc), in chunks of at most
// kCChunk pairs; its warps split a chunk's items evenly, stage each item's
// gathers in shared memory (as the per-warp copy round does), and sum the
// t^2 terms of every pair segment; a pair split between warps is combined
// from their two boundary records.  Then one thread a pair forms U_k from
// U_{k-1} (k > 0), stores c_j and adds the pair's message terms.  m > 0 (h
// below the CTA count): CTA b takes a share `sub` of the mul entries of pair
// j = b / m; it adds the c terms of its share and, for sub = 0, the U terms;
// the last block sums the shares into c_j.  The grid's sums go to the
// transcript as a copy round's do.
constexpr uint32_t kCChunk = 128;

template <int BD>
__global__ void __launch_bounds__(BD) k_copy_c(const uint32_t* __restrict__ T, uint32_t sn, uint32_t h,
                                               const uint32_t* __restrict__ E, const uint32_t* __restrict__ om,
                                               const uint4* __restrict__ sg, uint32_t nmul, uint32_t m,
                                               uint32_t per, const uint32_t* Uprev, const uint32_t* cprev,
                                               uint32_t* Ucur, uint32_t* ccur, uint32_t* cpart, uint32_t* partials,
                                               DevState* S, uint8_t* proof, size_t off, uint32_t k) {
  pdl_wait();
  constexpr int NW = BD / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == BD - 32) warm_transcript_code(k, h);
  const bool upd = k > 0;
  Fr rp = fr_zero(), qp = fr_zero();
  if (upd) {
    rp = S->rb[k - 1];
    qp = fr_sub(fr_mul(rp, rp), rp);
  }
  Fr acc[4] = {fr_zero(), fr_zero(), fr_zero(), fr_zero()};
  if (m == 0) {
    __shared__ Fr cpair[kCChunk];
    __shared__ Fr rec_val[NW][2];
    __shared__ uint32_t rec_pair[NW][2];
    extern __shared__ uint4 cc_stage[];  // kStageWords4 a warp
    uint4* stg = cc_stage + warp * kStageWords4;
    const uint32_t pb0 = (uint32_t)((uint64_t)blockIdx.x * h / gridDim.x);
    const uint32_t pb1 = (uint32_t)((uint64_t)(blockIdx.x + 1) * h / gridDim.x);
    for (uint32_t cb = pb0; cb < pb1; cb += kCChunk) {
      const uint32_t np = min(pb1 - cb, kCChunk);
      for (uint32_t p = threadIdx.x; p < np; p += BD) cpair[p] = fr_zero();
      if (lane < 2) rec_pair[warp][lane] = 0xffffffffu;
      __syncthreads();
      const uint64_t ni = (uint64_t)np * nmul;
      const uint64_t i0 = ni * warp / NW, i1 = ni * (warp + 1) / NW;
      for (uint64_t seg = i0; seg < i1;) {
        const uint32_t p = (uint32_t)(seg / nmul);
        const uint64_t segend = min(i1, (uint64_t)(p + 1) * nmul);
        const uint32_t g0 = (uint32_t)(seg - (uint64_t)p * nmul), g1 = (uint32_t)(segend - (uint64_t)p * nmul);
        const uint32_t j = cb + p;
        const uint32_t* lo = T + (((size_t)j << sn) << 3);
        const uint32_t* hi = T + (((size_t)(j + h) << sn) << 3);
        FrAcc ac = fracc_zero();
        // two-stage pipeline as in the per-warp copy round
        uint32_t q = g0 + lane;
        int st = 0;
        auto issue = [&](int stage, uint32_t qq) {
          const uint4 gi = sg[qq];
          stage_issue(stg, stage, lane, om + 8 * (size_t)qq, lo + 8 * (size_t)gi.x, hi + 8 * (size_t)gi.x,
                      lo + 8 * (size_t)gi.y, hi + 8 * (size_t)gi.y);
        };
        if (q < g1) issue(0, q);
        asm volatile("cp.async.commit_group;" ::: "memory");
        for (; q < g1; q += 32, st ^= 1) {
          if (q + 32 < g1) issue(st ^ 1, q + 32);
          asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 1;" ::: "memory");
          const Fr w = stage_read(stg, st, 0, lane);
          const Fr x0 = stage_read(stg, st, 1, lane), x1 = stage_read(stg, st, 2, lane);
          const Fr y0 = stage_read(stg, st, 3, lane), y1 = stage_read(stg, st, 4, lane);
          fracc_mac(ac, fr_mul(w, fr_sub(x1, x0)), fr_sub(y1, y0));
        }
        const Fr cs = fr_warp_sum(fr_redc288(ac));
        if (lane == 0) {
          if (g0 == 0 && g1 == nmul) {
            cpair[p] = cs;
          } else {
            const int slot = seg == i0 ? 0 : 1;  // only a warp's first and last segments can be partial
            rec_pair[warp][slot] = p;
            rec_val[warp][slot] = cs;
          }
        }
        seg = segend;
      }
      __syncthreads();
      for (uint32_t p = threadIdx.x; p < np; p += BD) {
        Fr c = cpair[p];
        for (int w2 = 0; w2 < NW; ++w2)
#pragma unroll
          for (int s2 = 0; s2 < 2; ++s2)
            if (rec_pair[w2][s2] == p) c = fr_add(c, rec_val[w2][s2]);
        fr_store(ccur, cb + p, c);
      }
      __syncthreads();  // the chunk's shared records are read before the next chunk's
    }
    // the message terms of the CTA's pairs, a group of four lanes a pair
    // (their c_j from this block's stores above, visible after the barrier)
    const uint32_t t = threadIdx.x & 3, mask = 0xfu << ((threadIdx.x & 31) & ~3u);
    Fr macc = fr_zero();
    for (uint32_t j = pb0 + (threadIdx.x >> 2); j < pb1; j += BD / 4)
      pair_group(j, h, t, mask, upd, true, Uprev, cprev, Ucur, E, rp, qp, fr_load(ccur, j), macc);
#pragma unroll
    for (int tt = 0; tt < 4; ++tt) acc[tt] = t == (uint32_t)tt ? macc : fr_zero();
    block_sum<BD, 4>(acc);  // thread 0
  } else {
    const uint32_t j = blockIdx.x / m, sub = blockIdx.x - j * m;
    const uint32_t q0 = min(nmul, sub * per), q1 = min(nmul, q0 + per);
    const uint32_t* lo = T + (((size_t)j << sn) << 3);
    const uint32_t* hi = T + (((size_t)(j + h) << sn) << 3);
    FrAcc ac = fracc_zero();
    for (uint32_t q = q0 + threadIdx.x; q < q1; q += BD) {
      const uint4 gi = sg[q];
      const Fr w = fr_load(om, q);
      const Fr x0 = fr_load(lo, gi.x), x1 = fr_load(hi, gi.x);
      const Fr y0 = fr_load(lo, gi.y), y1 = fr_load(hi, gi.y);
      fracc_mac(ac, fr_mul(w, fr_sub(x1, x0)), fr_sub(y1, y0));
    }
    Fr cs[1] = {fr_redc288(ac)};
    block_sum<BD, 1>(cs);  // thread 0
    __shared__ Fr cshare;
    if (threadIdx.x == 0) {
      fr_store_cg(cpart, blockIdx.x, cs[0]);
      cshare = cs[0];
    }
    __syncthreads();
    Fr macc = fr_zero();
    if (threadIdx.x < 4)
      pair_group(j, h, threadIdx.x, 0xfu, upd, sub == 0, Uprev, cprev, Ucur, E, rp, qp, cshare, macc);
    // the four lanes' terms to thread 0 (grid_sum_last_block takes thread 0's)
    __shared__ Fr mterm[4];
    if (threadIdx.x < 4) mterm[threadIdx.x] = macc;
    __syncthreads();
    if (threadIdx.x == 0)
#pragma unroll
      for (int tt = 0; tt < 4; ++tt) acc[tt] = mterm[tt];
  }
  const bool last = grid_sum_last_block<BD, 4, true>(acc, partials, S);
  if (!last) return;
  if (m > 0) {  // c_j from the shares of every pair, for the next round's U
    for (uint32_t jj = threadIdx.x; jj < h; jj += BD) {
      Fr c = fr_zero();
      for (uint32_t s2 = 0; s2 < m; ++s2) c = fr_add(c, fr_load_cg(cpart, (size_t)jj * m + s2));
      fr_store(ccur, jj, c);
    }
  }
  if (threadIdx.x < 32) round_finalize<4>(S, acc, proof, off, &S->rb[k]);
}

// Launch shapes of k_copy_c, from the copy round's tuning table (the same
// (log2 W, log2 pairs) classes): the CTA width (128, 256 or 384 threads;
// default 256), the split (form 0: whole pairs a CTA while pairs are at
// least the CTAs, shares of a pair otherwise; 1: shares whenever the pairs
// fit the shares' scratch; 2: whole pairs always) and the items a share
// takes at least (default half a CTA's threads).
template <int BD>
static int copy_c_per_sm() {
  static int per_sm = 0;
  if (per_sm == 0) {
    const size_t smem = (size_t)(BD / 32) * kStageWords4 * sizeof(uint4);
    if (cudaFuncSetAttribute(k_copy_c<BD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
      return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_copy_c<BD>, BD, smem) != cudaSuccess || n < 1) n = 1;
    per_sm = n;
  }
  return per_sm;
}

template <int BD>
static int launch_copy_c_bd(int form, uint32_t min_items, const uint32_t* T, uint32_t sn, uint32_t h,
                            const uint32_t* E, const uint32_t* omega_s, const DevLayer& L, const uint32_t* Uprev,
                            const uint32_t* cprev, uint32_t* Ucur, uint32_t* ccur, uint32_t* cpart,
                            uint32_t* partials, DevState* S, uint8_t* proof, size_t off, uint32_t k,
                            cudaStream_t st) {
  const int per_sm = copy_c_per_sm<BD>();
  if (per_sm == 0) return (int)cudaErrorInvalidValue;
  const uint32_t nc = std::min<uint32_t>(kSMs * per_sm, kMaxPartials / 2);  // the shares use the upper half
  const size_t smem = (size_t)(BD / 32) * kStageWords4 * sizeof(uint4);
  uint32_t m = 0, per = 0, grid = nc;
  const bool shares = form == 2 ? false : form == 1 ? h <= kMaxPartials / 2 : h < nc;
  if (shares) {  // shares of a pair's mul entries, each at least min_items of them
    const uint32_t mi = min_items ? min_items : BD / 2;
    const uint32_t by_items = std::max<uint32_t>(1, (L.nmul + mi - 1) / mi);
    m = std::max<uint32_t>(1, std::min<uint32_t>(std::max<uint32_t>(1, nc / h), by_items));
    per = (L.nmul + m - 1) / m;
    grid = h * m;
  } else if (h < nc) {
    grid = h;  // whole pairs, one a CTA
  }
  return launch_pdl_smem(k_copy_c<BD>, grid, BD, m ? 0 : smem, st, T, sn, h, E, omega_s, L.sgate, L.nmul, m, per,
                         Uprev, cprev, Ucur, ccur, cpart, partials, S, proof, off, k);
}

int launch_copy_c(const uint32_t* T, uint32_t sn, uint32_t h, const uint32_t* E, const uint32_t* omega_s,
                  const DevLayer& L, const uint32_t* Uprev, const uint32_t* cprev, uint32_t* Ucur, uint32_t* ccur,
                  uint32_t* cpart, uint32_t* partials, DevState* S, uint8_t* proof, size_t off, uint32_t k,
                  void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  uint32_t lh = 0;
  while ((2u << lh) <= h) ++lh;
  CopyTune t = {256, 0, 0};
  if (sn < kTuneLog && lh < kTuneLog && g_copy_c_tune[sn][lh].bd) t = g_copy_c_tune[sn][lh];
  if (t.bd == 128)
    return launch_copy_c_bd<128>(t.form, t.min_items, T, sn, h, E, omega_s, L, Uprev, cprev, Ucur, ccur, cpart,
                                 partials, S, proof, off, k, st);
  if (t.bd == 384)
    return launch_copy_c_bd<384>(t.form, t.min_items, T, sn, h, E, omega_s, L, Uprev, cprev, Ucur, ccur, cpart,
                                 partials, S, proof, off, k, st);
  return launch_copy_c_bd<256>(t.form, t.min_items, T, sn, h, E, omega_s, L, Uprev, cprev, Ucur, ccur, cpart,
                               partials, S, proof, off, k, st);
}

// ---------------------------------------------------------------------------
// copy-sharded proofs (Sec. 3.2.1: the machine index is the low part of the
// copy index, so every rank binds its own copy bits first and the round
// polynomial of a copy round is the sum of the ranks' polynomials)

// After the ranks' sums of round k are gathered (world x 4 values, rank by
// rank, plain and below 2r): their sum is the round polynomial, which goes
// into the proof and the transcript as in a whole proof (every rank runs
// this, so every rank draws the same challenge).
__global__ void k_shard_absorb(const uint32_t* __restrict__ sums_all, uint32_t world, DevState* S, uint8_t* proof,
                               size_t off, uint32_t k) {
  Fr v[4] = {fr_zero(), fr_zero(), fr_zero(), fr_zero()};
  if (threadIdx.x == 0)
#pragma unroll
    for (int t = 0; t < 4; ++t)
      for (uint32_t q = 0; q < world; ++q) v[t] = fr_add(v[t], fr_load(sums_all, 4 * (size_t)q + t));
  round_finalize<4>(S, v, proof, off, &S->rb[k]);
}

int launch_shard_absorb(const uint32_t* sums_all, uint32_t world, DevState* S, uint8_t* proof, size_t off,
                        uint32_t k, void* stream) {
  k_shard_absorb<<<1, 32, 0, (cudaStream_t)stream>>>(sums_all, world, S, proof, off, k);
  return post_launch();
}

// the rank's copy-bound row A (Wn values) and its copy weight E[0] into one
// message of Wn + 1 values
__global__ void k_shard_row(const uint32_t* __restrict__ A, const uint32_t* __restrict__ E, uint32_t Wn,
                            uint32_t* __restrict__ out) {
  for (uint32_t x = blockIdx.x * blockDim.x + threadIdx.x; x <= Wn; x += gridDim.x * blockDim.x)
    fr_store(out, x, fr_load(x < Wn ? A : E, x < Wn ? x : 0));
}

int launch_shard_row(const uint32_t* A, const uint32_t* E, uint32_t Wn, uint32_t* out, void* stream) {
  k_shard_row<<<grid_for(Wn + 1, 128), 128, 0, (cudaStream_t)stream>>>(A, E, Wn, out);
  return post_launch();
}

// rank 0: the gathered messages (rank q's at q * stride values) as the
// table of world rows (row q = rank q's row: the rank is the copy index's
// low part, the one still unbound) and its copy weights
__global__ void k_shard_table(const uint32_t* __restrict__ rows, uint32_t world, uint32_t Wn, uint32_t stride,
                              uint32_t* __restrict__ T, uint32_t* __restrict__ E) {
  const size_t total = (size_t)world * (Wn + 1);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const size_t q = i / (Wn + 1), x = i - q * (Wn + 1);
    const Fr v = fr_load(rows, q * stride + x);
    if (x < Wn) fr_store(T, q * Wn + x, v);
    else fr_store(E, q, v);
  }
}

int launch_shard_table(const uint32_t* rows, uint32_t world, uint32_t Wn, uint32_t stride, uint32_t* T, uint32_t* E,
                       void* stream) {
  k_shard_table<<<grid_for((size_t)world * (Wn + 1), 128), 128, 0, (cudaStream_t)stream>>>(rows, world, Wn, stride,
                                                                                          T, E);
  return post_launch();
}

// fold of the copy rows and of E by the round's challenge r = r_b[k]:
//   dst(j, x) = src(j, x) + r (src(j + h, x) - src(j, x)),  j < h
// (in place when src == dst: each thread writes only the entry it read).
// Every entry is multiplied by the same r, so the product is the
// fixed-multiplier form (fr_mul_fixed: eight row products and a two-word
// reduction, 40% fewer multiply-adds than a Montgomery product), with the
// eight coefficients built once per CTA in shared memory (read by broadcast
// loads, so the kernel fits four CTAs per SM: the fold streams HBM and
// needs the warps to keep loads in flight).
__global__ void __launch_bounds__(256, 4) k_copy_fold(const uint32_t* src, uint32_t* dst, uint32_t sn, uint32_t h,
                                                   uint32_t* E, const DevState* S, uint32_t k) {
  pdl_wait();
  __shared__ __align__(16) uint32_t shK[64];
  if (threadIdx.x < 8) fr_store(shK, threadIdx.x, fr_fixed_coeff(S->rb[k], (int)threadIdx.x));
  __syncthreads();
  const size_t nel = (size_t)h << sn;
  const size_t total = nel + h;
  // two entries a thread per step, their four loads issued before either
  // product (more bytes in flight for the HBM half of this balanced kernel)
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total; idx += 2 * stride) {
    const size_t idy = idx + stride;
    const bool rowa = idx < nel, rowb = idy < nel, hasb = idy < total;
    const uint32_t* ba = rowa ? src : E;
    const uint32_t* bb = rowb ? src : E;
    const size_t a0 = rowa ? idx : idx - nel, a1 = rowa ? idx + nel : idx - nel + h;
    const size_t b0 = rowb ? idy : idy - nel, b1 = rowb ? idy + nel : idy - nel + h;
    const Fr xa = fr_load(ba, a0), ya = fr_load(ba, a1);
    Fr xb = fr_zero(), yb = fr_zero();
    if (hasb) {
      xb = fr_load(bb, b0);
      yb = fr_load(bb, b1);
    }
    fr_store(rowa ? dst : E, a0, fr_add(xa, fr_mul_fixed(fr_sub(ya, xa), shK)));
    if (hasb) fr_store(rowb ? dst : E, b0, fr_add(xb, fr_mul_fixed(fr_sub(yb, xb), shK)));
  }
}

int launch_copy_fold(const uint32_t* src, uint32_t* dst, uint32_t sn, uint32_t h, uint32_t* E, DevState* S,
                     uint32_t k, void* stream) {
  size_t n = ((size_t)h << sn) + h;
  // one resident wave (four CTAs per SM), so each CTA builds the eight
  // coefficients once for many entries
  return launch_pdl(k_copy_fold, grid_for(n, 256, 4), 256, (cudaStream_t)stream, src, dst, sn, h, E,
                    (const DevState*)S, k);
}

// ---------------------------------------------------------------------------
// Libra phase 1 (over x) bookkeeping, from the row A = V~(r_b, .) and
// e = E(r_b):  H1(x) = e sum_{g: in1 g = x} w(g) (mul ? A(in2 g) : 1)
//              H2(x) = e sum_{g: in1 g = x, add} w(g) A(in2 g)
// so that sum_y P(r_b, x, y) = A(x) H1(x) + H2(x).

__global__ void k_xinit(const uint32_t* __restrict__ A, const uint32_t* __restrict__ E,
                        const uint32_t* __restrict__ om, const uint4* __restrict__ sg, uint32_t nmul,
                        const uint32_t* __restrict__ off1, const uint32_t* __restrict__ pos1, uint32_t Wn,
                        uint32_t* __restrict__ At, uint32_t* __restrict__ H1, uint32_t* __restrict__ H2,
                        uint32_t* __restrict__ Ay) {
  const Fr e = fr_mul(fr_load(E, 0), fr_mont_2_neg32());  // E carries a factor 2^32
  for (uint32_t x = blockIdx.x * blockDim.x + threadIdx.x; x < Wn; x += gridDim.x * blockDim.x) {
    Fr a1 = fr_zero(), a2 = fr_zero();
    for (uint32_t p = off1[x], pe = off1[x + 1]; p < pe; ++p) {
      uint32_t q = pos1[p];
      uint4 gi = sg[q];
      Fr w = fr_load(om, q);
      Fr wa = fr_mul(w, fr_load(A, gi.y));
      if (q < nmul) {
        a1 = fr_add(a1, wa);
      } else {
        a1 = fr_add(a1, w);
        a2 = fr_add(a2, wa);
      }
    }
    fr_store(H1, x, fr_mul(e, a1));
    fr_store(H2, x, fr_mul(e, a2));
    Fr a = fr_load(A, x);
    fr_store(At, x, a);
    fr_store(Ay, x, a);
  }
}

int launch_xinit(const uint32_t* Arow, const uint32_t* E, const uint32_t* omega_s, const DevLayer& L, uint32_t Wn,
                 uint32_t* At, uint32_t* H1, uint32_t* H2, uint32_t* Ay, void* stream) {
  k_xinit<<<grid_for(Wn, 64), 64, 0, (cudaStream_t)stream>>>(Arow, E, omega_s, L.sgate, L.nmul, L.off1, L.pos1,
                                                             Wn, At, H1, H2, Ay);
  return post_launch();
}

// Libra phase 2 (over y): Q = EQ(r_x); v_x = A(r_x) from the size-2 table.
__global__ void k_eq_rx(DevState* S, uint32_t s, uint32_t W, uint32_t* __restrict__ Q, const uint32_t* __restrict__ At) {
  const size_t gid = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  for (size_t x = gid; x < W; x += (size_t)gridDim.x * blockDim.x) fr_store(Q, x, eq_index(S->rx, s, (uint32_t)x));
  if (gid == 0) S->vx = s == 0 ? fr_load(At, 0) : fold2(fr_load(At, 0), fr_load(At, 1), S->rx[s - 1]);
}

int launch_eq_rx(DevState* S, uint32_t s, uint32_t W, uint32_t* Q, const uint32_t* At, void* stream) {
  k_eq_rx<<<grid_for(W, 128), 128, 0, (cudaStream_t)stream>>>(S, s, W, Q, At);
  return post_launch();
}

//   K1(y) = e sum_{g: in2 g = y} w(g) Q(in1 g) (mul ? v_x : 1)
//   K2(y) = e sum_{g: in2 g = y, add} w(g) Q(in1 g) v_x
// so that sum over boolean x of P(r_b, r_x, y) = A(y) K1(y) + K2(y).
__global__ void k_yinit(const uint32_t* __restrict__ E, const uint32_t* __restrict__ om, const uint32_t* __restrict__ Q,
                        const uint4* __restrict__ sg, uint32_t nmul, const uint32_t* __restrict__ off2,
                        const uint32_t* __restrict__ pos2, uint32_t Wn, uint32_t* __restrict__ K1,
                        uint32_t* __restrict__ K2, const DevState* S) {
  const Fr e = fr_mul(fr_load(E, 0), fr_mont_2_neg32());  // E carries a factor 2^32
  const Fr ev = fr_mul(e, S->vx);
  for (uint32_t y = blockIdx.x * blockDim.x + threadIdx.x; y < Wn; y += gridDim.x * blockDim.x) {
    Fr m = fr_zero(), a = fr_zero();
    for (uint32_t p = off2[y], pe = off2[y + 1]; p < pe; ++p) {
      uint32_t q = pos2[p];
      Fr wq = fr_mul(fr_load(om, q), fr_load(Q, sg[q].x));
      if (q < nmul) m = fr_add(m, wq);
      else a = fr_add(a, wq);
    }
    fr_store(K1, y, fr_add(fr_mul(e, a), fr_mul(ev, m)));
    fr_store(K2, y, fr_mul(ev, a));
  }
}

int launch_yinit(const uint32_t* E, const uint32_t* omega_s, const uint32_t* Q, const DevLayer& L, uint32_t Wn,
                 uint32_t* K1, uint32_t* K2, DevState* S, void* stream) {
  k_yinit<<<grid_for(Wn, 64), 64, 0, (cudaStream_t)stream>>>(E, omega_s, Q, L.sgate, L.nmul, L.off2, L.pos2, Wn,
                                                             K1, K2, S);
  return post_launch();
}

// One round of a Libra phase over tables (A, B1, B2) of size m after the
// fold of the previous round's challenge (when k > 0):
//   g(t) = sum_{j < m/2} A_t(j) B1_t(j) + B2_t(j),  t = 0, 1, 2.
template <int BD>
__global__ void __launch_bounds__(BD) k_gate_round(uint32_t* A, uint32_t* B1, uint32_t* B2, uint32_t m, int phase,
                                                   uint32_t k, uint32_t* partials, DevState* S, uint8_t* proof,
                                                   size_t off) {
  if (threadIdx.x == BD - 32) warm_transcript_code(k, m);
  const uint32_t hq = m / 2;
  Fr* rs = phase == 0 ? S->rx : S->ry;
  const bool fold = k > 0;
  Fr r = fr_zero();
  if (fold) r = rs[k - 1];
  Fr acc[3] = {fr_zero(), fr_zero(), fr_zero()};
  for (uint32_t j = blockIdx.x * BD + threadIdx.x; j < hq; j += gridDim.x * BD) {
    Fr a0, a1, p0, p1, q0, q1;
    if (fold) {
      a0 = fold2(fr_load(A, j), fr_load(A, j + m), r);
      a1 = fold2(fr_load(A, j + hq), fr_load(A, j + hq + m), r);
      p0 = fold2(fr_load(B1, j), fr_load(B1, j + m), r);
      p1 = fold2(fr_load(B1, j + hq), fr_load(B1, j + hq + m), r);
      q0 = fold2(fr_load(B2, j), fr_load(B2, j + m), r);
      q1 = fold2(fr_load(B2, j + hq), fr_load(B2, j + hq + m), r);
      fr_store(A, j, a0); fr_store(A, j + hq, a1);
      fr_store(B1, j, p0); fr_store(B1, j + hq, p1);
      fr_store(B2, j, q0); fr_store(B2, j + hq, q1);
    } else {
      a0 = fr_load(A, j); a1 = fr_load(A, j + hq);
      p0 = fr_load(B1, j); p1 = fr_load(B1, j + hq);
      q0 = fr_load(B2, j); q1 = fr_load(B2, j + hq);
    }
    const Fr a2 = fr_sub(fr_dbl(a1), a0), p2 = fr_sub(fr_dbl(p1), p0), q2 = fr_sub(fr_dbl(q1), q0);
    acc[0] = fr_add(acc[0], fr_add(fr_mul(a0, p0), q0));
    acc[1] = fr_add(acc[1], fr_add(fr_mul(a1, p1), q1));
    acc[2] = fr_add(acc[2], fr_add(fr_mul(a2, p2), q2));
  }
  if (grid_sum_last_block<BD, 3>(acc, partials, S) && threadIdx.x < 32) round_finalize<3>(S, acc, proof, off, &rs[k]);
}

int launch_gate_round(uint32_t* A, uint32_t* B1, uint32_t* B2, uint32_t m, int phase, uint32_t k, uint32_t* partials,
                      DevState* S, uint8_t* proof, size_t off, void* stream) {
  const uint32_t hq = m / 2;
  unsigned g = grid_for(hq, 128, 8);
  k_gate_round<128><<<g, 128, 0, (cudaStream_t)stream>>>(A, B1, B2, m, phase, k, partials, S, proof, off);
  return post_launch();
}

// end of a layer: v_y, the proof's (v_x, v_y), absorb 'V', next alpha, beta
__global__ void k_layer_end(DevState* S, const uint32_t* Ay, uint32_t s, uint8_t* proof, size_t off, int last) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  Fr vy = s == 0 ? fr_load(Ay, 0) : fold2(fr_load(Ay, 0), fr_load(Ay, 1), S->ry[s - 1]);
  S->vy = vy;
  Fr canon[2] = {fr_to_canonical(S->vx), fr_to_canonical(vy)};
  store_words(proof, off, canon[0]);
  store_words(proof, off + 32, canon[1]);
  tr_absorb_n<2, true>(S->st, 'V', canon);
  if (!last) {
    S->alpha = tr_challenge(S, true);
    S->beta = tr_challenge(S, false);
  }
}

int launch_layer_end(DevState* S, const uint32_t* Ay, uint32_t s, uint8_t* proof, size_t off, int last,
                     void* stream) {
  k_layer_end<<<1, 32, 0, (cudaStream_t)stream>>>(S, Ay, s, proof, off, last);
  return post_launch();
}

// ---------------------------------------------------------------------------
// Libra's two phases of one layer in one launch of a thread-block cluster.
//
// Each round is latency-bound (tables of at most a few thousand entries),
// so a separate launch per round cost more than the round's arithmetic.
// The cluster's CTAs share every round: each folds and evaluates its pairs,
// sends its partial sums to CTA 0 through distributed shared memory, CTA 0
// runs the transcript, and the challenge comes back the same way.  Tables
// live in global memory and are read through L2 (__ldcg): entries written
// by another CTA in the previous round are ordered by the cluster barrier.

namespace cg = cooperative_groups;
constexpr int kTailCTAs = 8;
constexpr int kTailThreads = 256;

constexpr uint32_t kSoloMax = 256;  // table entries at which CTA 0 finishes a phase alone

struct TailShared {
  Fr part[kTailCTAs][2];  // partial sums g(0), g(2) of every CTA (each CTA sends its own to all)
  Fr canon[3];            // canonical round values
  Fr bcast;               // the round's challenge, for every thread of the CTA
  Fr vx;                  // CTA 0: v_x, read by every CTA
  uint32_t st[8];         // this CTA's copy of the transcript state
  Fr red[3][kTailThreads / 32];
  Fr rx[2][16];           // r_x,k and 1 - r_x,k
  Fr eqh[256], eql[256];  // eq(r_x, x) = eqh[x >> sl] eql[x mod 2^sl]
  Fr solo[3][kSoloMax];   // CTA 0: the tables of a phase's last rounds
};

// One round over tables (A, B1, B2) of size m (after the fold of `rprev`
// when k > 0): g(t) = sum_{j < m/2} A_t(j) B1_t(j) + B2_t(j) for t = 0 and
// t = 2, the round message (g(1) is the claim minus g(0), for the verifier).
// A is in Montgomery form and B1, B2 are plain, so the products and the
// sums are plain.  The round runs in two cluster-wide steps, each thread
// doing at most a few products: the fold (one product per new table
// entry), then one product per (pair, t).  Every CTA sends its partial sums
// to every CTA and then runs the transcript on its own copy of the state,
// so the challenge needs no further barrier; CTA 0 alone writes the proof
// bytes and the challenge (rslot).  Returns the round's challenge
// (Montgomery form) in every thread.
__device__ Fr tail_round(cg::cluster_group& cl, TailShared& sh, uint32_t* A, uint32_t* B1, uint32_t* B2,
                         uint32_t m, uint32_t k, const Fr& rprev, DevState* S, uint8_t* proof, size_t off,
                         Fr* rslot) {
  const uint32_t rank = cl.block_rank();
  const uint32_t gtid = rank * kTailThreads + threadIdx.x, gstride = kTailCTAs * kTailThreads;
  if (k > 0) {
    // fold of the three tables from 2m to m entries (in place: entry q < m
    // is written only by the thread that reads q and q + m)
    for (uint32_t q = gtid; q < 3 * m; q += gstride) {
      const uint32_t tab = q / m, idx = q - tab * m;
      uint32_t* T = tab == 0 ? A : tab == 1 ? B1 : B2;
      fr_store(T, idx, fold2(fr_load_cg(T, idx), fr_load_cg(T, idx + m), rprev));
    }
    cl.sync();
  }
  const uint32_t hq = m / 2;
  Fr acc0 = fr_zero(), acc2 = fr_zero();
  for (uint32_t q = gtid; q < 2 * hq; q += gstride) {
    const uint32_t j = q >> 1;
    Fr a = fr_load_cg(A, j), p = fr_load_cg(B1, j), c = fr_load_cg(B2, j);
    if (q & 1) {  // t = 2: X_2 = 2 X(j + m/2) - X(j)
      a = fr_sub(fr_dbl(fr_load_cg(A, j + hq)), a);
      p = fr_sub(fr_dbl(fr_load_cg(B1, j + hq)), p);
      c = fr_sub(fr_dbl(fr_load_cg(B2, j + hq)), c);
    }
    const Fr v = fr_add(fr_mul(a, p), c);
    if (q & 1) acc2 = fr_add(acc2, v);
    else acc0 = fr_add(acc0, v);
  }
  Fr acc[2] = {acc0, acc2};
  // CTA sum, then to every CTA's shared memory
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int t = 0; t < 2; ++t) acc[t] = fr_warp_sum(acc[t]);
  if (lane == 0)
#pragma unroll
    for (int t = 0; t < 2; ++t) sh.red[t][warp] = acc[t];
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      acc[t] = fr_warp_sum(lane < kTailThreads / 32 ? sh.red[t][lane] : fr_zero());
#pragma unroll
      for (int i = 0; i < 8; ++i) acc[t].v[i] = __shfl_sync(0xffffffffu, acc[t].v[i], 0);
    }
    if (lane < kTailCTAs) {  // lane d sends this CTA's sums to CTA d
      Fr* dst = cl.map_shared_rank(&sh.part[0][0], lane);
#pragma unroll
      for (int t = 0; t < 2; ++t) dst[rank * 2 + t] = acc[t];
    }
  }
  cl.sync();
  if (warp == 0) {
    if (lane < 2) {  // the message g(0), g(2)
      Fr v = fr_zero();
#pragma unroll
      for (int c = 0; c < kTailCTAs; ++c) v = fr_add(v, sh.part[c][lane]);
      v = fr_reduce_once(v);  // plain and below 2r: now canonical
      if (rank == 0) store_words(proof, off + 32 * (size_t)lane, v);
      sh.canon[lane] = v;
    }
    __syncwarp();
    if (lane == 0) {
      Fr canon[2] = {sh.canon[0], sh.canon[1]};
      tr_absorb_n<2, false>(sh.st, 'R', canon);
      const Fr r = tr_challenge_st<false>(sh.st, &S->error, true);
      if (rank == 0) *rslot = r;
      sh.bcast = r;
    }
  }
  __syncthreads();
  return sh.bcast;
}

// The last rounds of a phase, k = k0 .. s-1, by CTA 0 alone (call it from
// CTA 0 only): once the tables have at most kSoloMax entries the cluster's
// barriers and partial-sum exchange cost more than the work, so the tables
// move to CTA 0's shared memory and its threads fold, evaluate and reduce
// with block barriers.  On entry the tables as round k0 - 1 left them (or
// as the phase's bookkeeping wrote them, k0 = 0) are in global memory and
// r is r_{k0-1}.  Records every challenge in rslot[k] and in the slot
// rhist[k] of shared memory (when not null), and returns the last one; the
// final two entries of the first table stay in sh.solo[0][0..1].
__device__ Fr tail_solo(TailShared& sh, const uint32_t* A, const uint32_t* B1, const uint32_t* B2, uint32_t Wn,
                        uint32_t s, uint32_t k0, Fr r, DevState* S, uint8_t* proof, size_t off, Fr* rslot,
                        Fr (*rhist)[16]) {
  const uint32_t n0 = k0 == 0 ? Wn : Wn >> (k0 - 1);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (uint32_t e = threadIdx.x; e < 3 * n0; e += kTailThreads) {
    const uint32_t tab = e / n0, idx = e - tab * n0;
    sh.solo[tab][idx] = fr_load_cg(tab == 0 ? A : tab == 1 ? B1 : B2, idx);
  }
  __syncthreads();
  for (uint32_t k = k0; k < s; ++k) {
    const uint32_t m = Wn >> k, hq = m / 2;
    if (k > 0) {  // fold from 2m to m entries in place (entry idx < m: read and written by one thread)
      for (uint32_t e = threadIdx.x; e < 3 * m; e += kTailThreads) {
        const uint32_t tab = e / m, idx = e - tab * m;
        sh.solo[tab][idx] = fold2(sh.solo[tab][idx], sh.solo[tab][idx + m], r);
      }
      __syncthreads();
    }
    Fr acc[2] = {fr_zero(), fr_zero()};
    for (uint32_t q = threadIdx.x; q < 2 * hq; q += kTailThreads) {
      const uint32_t j = q >> 1;
      Fr a = sh.solo[0][j], pp = sh.solo[1][j], c = sh.solo[2][j];
      if (q & 1) {  // t = 2
        a = fr_sub(fr_dbl(sh.solo[0][j + hq]), a);
        pp = fr_sub(fr_dbl(sh.solo[1][j + hq]), pp);
        c = fr_sub(fr_dbl(sh.solo[2][j + hq]), c);
      }
      acc[q & 1] = fr_add(acc[q & 1], fr_add(fr_mul(a, pp), c));
    }
#pragma unroll
    for (int t = 0; t < 2; ++t) acc[t] = fr_warp_sum(acc[t]);
    if (lane == 0)
#pragma unroll
      for (int t = 0; t < 2; ++t) sh.red[t][warp] = acc[t];
    __syncthreads();
    if (warp == 0) {
#pragma unroll
      for (int t = 0; t < 2; ++t) acc[t] = fr_warp_sum(lane < kTailThreads / 32 ? sh.red[t][lane] : fr_zero());
      if (lane == 0) {
        Fr canon[2] = {fr_reduce_once(acc[0]), fr_reduce_once(acc[1])};  // plain, below 2r
        store_words(proof, off + 64 * (size_t)k, canon[0]);
        store_words(proof, off + 64 * (size_t)k + 32, canon[1]);
        tr_absorb_n<2, false>(sh.st, 'R', canon);
        const Fr rk = tr_challenge_st<false>(sh.st, &S->error, true);
        rslot[k] = rk;
        if (rhist) {
          rhist[1][k] = rk;
          rhist[0][k] = fr_sub(fr_one(), rk);
        }
        sh.bcast = rk;
      }
    }
    __syncthreads();
    r = sh.bcast;
  }
  return r;
}

__global__ void __cluster_dims__(kTailCTAs, 1, 1) __launch_bounds__(kTailThreads) k_layer_tail(TailParams p) {
  pdl_wait();
  cg::cluster_group cl = cg::this_cluster();
  __shared__ TailShared sh;
  const uint32_t rank = cl.block_rank();
  const uint32_t gtid = rank * kTailThreads + threadIdx.x, gstride = kTailCTAs * kTailThreads;
  DevState* S = p.S;
  const Fr e = fr_mul(fr_load(p.E, 0), fr_mont_2_neg32());  // E carries a factor 2^32
  if (threadIdx.x < 8) sh.st[threadIdx.x] = S->st[threadIdx.x];  // ordered by the cluster barrier below
  // Libra phase 1 bookkeeping: H1(x) = e sum_{in1 g = x} w(g) (mul ? A(in2 g) : 1),
  // H2(x) = e sum_{in1 g = x, add} w(g) A(in2 g).  The per-entry terms are
  // formed entry-parallel first (one product each, all at once), so that the
  // sums over the in1 lists are additions only: the lists are a few entries
  // long, and a product per list step put their longest one on the critical
  // path.
  uint32_t* P1 = p.P;
  uint32_t* P2 = p.P + 8 * (size_t)p.ntot;
  for (uint32_t g = gtid; g < p.ntot; g += gstride) {
    const Fr w = fr_load(p.om, g);
    const Fr wa = fr_mul(w, fr_load(p.A, p.sg[g].y));
    const bool mul = g < p.nmul;
    fr_store(P1, g, mul ? wa : w);
    fr_store(P2, g, mul ? fr_zero() : wa);
  }
  cl.sync();  // the terms, for every CTA of the cluster
  for (uint32_t x = gtid; x < p.Wn; x += gstride) {
    Fr a1 = fr_zero(), a2 = fr_zero();
    for (uint32_t q = p.off1[x], qe = p.off1[x + 1]; q < qe; ++q) {
      const uint32_t g = p.pos1[q];
      a1 = fr_add(a1, fr_load_cg(P1, g));
      a2 = fr_add(a2, fr_load_cg(P2, g));
    }
    fr_store(p.H1, x, fr_mul(e, a1));
    fr_store(p.H2, x, fr_mul(e, a2));
    Fr a = fr_load(p.A, x);
    fr_store(p.At, x, a);
    fr_store(p.Ay, x, a);
  }
  cl.sync();
  // rounds k < k0 over the cluster, k >= k0 by CTA 0 alone (tables of at
  // most kSoloMax entries)
  uint32_t k0 = 0;
  while (k0 < p.s && (p.Wn >> (k0 == 0 ? 0 : k0 - 1)) > kSoloMax) ++k0;
  Fr r = fr_zero();
  for (uint32_t k = 0; k < k0; ++k) {
    r = tail_round(cl, sh, p.At, p.H1, p.H2, p.Wn >> k, k, r, S, p.proof, p.offx + 64 * (size_t)k, &S->rx[k]);
    if (threadIdx.x == 0) {  // r_x,k and 1 - r_x,k for eq(r_x, .)
      sh.rx[1][k] = r;
      sh.rx[0][k] = fr_sub(fr_one(), r);
    }
  }
  if (rank == 0) {
    r = tail_solo(sh, p.At, p.H1, p.H2, p.Wn, p.s, k0, r, S, p.proof, p.offx, S->rx, sh.rx);
    if (threadIdx.x == 0) {  // v_x = A(r_x)
      const Fr vx = p.s == 0 ? sh.solo[0][0] : fold2(sh.solo[0][0], sh.solo[0][1], r);
      S->vx = vx;
      sh.vx = vx;
    }
  }
  cl.sync();  // CTA 0's late challenges and transcript state, for every CTA
  if (rank != 0) {
    const TailShared* s0 = cl.map_shared_rank(&sh, 0);
    for (uint32_t k = k0 + threadIdx.x; k < p.s; k += kTailThreads) {
      sh.rx[0][k] = s0->rx[0][k];
      sh.rx[1][k] = s0->rx[1][k];
    }
    if (threadIdx.x < 8) sh.st[threadIdx.x] = s0->st[threadIdx.x];
    r = s0->bcast;
  }
  // eq(r_x, x) over the Wn positions of layer i+1, as the product of two
  // half tables over the high sh and the low sl bits of x (r_x,0 binds the
  // most significant bit), which every CTA builds in its own shared memory
  const uint32_t sl = p.s / 2, shb = p.s - sl, lmask = (1u << sl) - 1;
  __syncthreads();
  for (uint32_t u = threadIdx.x; u < (1u << shb) + (1u << sl); u += kTailThreads) {
    const bool hi = u < (1u << shb);
    const uint32_t v = hi ? u : u - (1u << shb), nb = hi ? shb : sl, k0 = hi ? 0 : shb;
    Fr acc = fr_one();
    for (uint32_t b = 0; b < nb; ++b) acc = fr_mul(acc, sh.rx[(v >> (nb - 1 - b)) & 1u][k0 + b]);
    (hi ? sh.eqh : sh.eql)[v] = acc;
  }
  cl.sync();  // the half tables, and v_x from CTA 0
  const Fr vx = *cl.map_shared_rank(&sh.vx, 0);
  // Libra phase 2 bookkeeping: K1(y) = e sum_{in2 g = y} w(g) Q(in1 g) (mul ? v_x : 1),
  // K2(y) = e sum_{in2 g = y, add} w(g) Q(in1 g) v_x,  Q = eq(r_x, .)
  const Fr ev = fr_mul(e, vx);
  // per-entry terms w(g) Q(in1 g), entry-parallel as in phase 1 (P1: mul
  // entries, P2: add entries)
  for (uint32_t g = gtid; g < p.ntot; g += gstride) {
    const uint32_t x1 = p.sg[g].x;
    const Fr wq = fr_mul(fr_load(p.om, g), fr_mul(sh.eqh[x1 >> sl], sh.eql[x1 & lmask]));
    const bool mul = g < p.nmul;
    fr_store(P1, g, mul ? wq : fr_zero());
    fr_store(P2, g, mul ? fr_zero() : wq);
  }
  cl.sync();
  for (uint32_t y = gtid; y < p.Wn; y += gstride) {
    Fr mu = fr_zero(), ad = fr_zero();
    for (uint32_t q = p.off2[y], qe = p.off2[y + 1]; q < qe; ++q) {
      const uint32_t g = p.pos2[q];
      mu = fr_add(mu, fr_load_cg(P1, g));
      ad = fr_add(ad, fr_load_cg(P2, g));
    }
    fr_store(p.H1, y, fr_add(fr_mul(e, ad), fr_mul(ev, mu)));
    fr_store(p.H2, y, fr_mul(ev, ad));
  }
  cl.sync();
  for (uint32_t k = 0; k < k0; ++k)
    r = tail_round(cl, sh, p.Ay, p.H1, p.H2, p.Wn >> k, k, r, S, p.proof, p.offy + 64 * (size_t)k, &S->ry[k]);
  if (rank == 0) r = tail_solo(sh, p.Ay, p.H1, p.H2, p.Wn, p.s, k0, r, S, p.proof, p.offy, S->ry, nullptr);
  // end of the layer: v_y, (v_x, v_y) into the proof, absorb 'V', alpha, beta
  if (rank == 0 && threadIdx.x < 32) {
    const int lane = threadIdx.x;
    if (lane < 2) {
      Fr v = lane == 0 ? vx : (p.s == 0 ? sh.solo[0][0] : fold2(sh.solo[0][0], sh.solo[0][1], r));
      if (lane == 1) S->vy = v;
      Fr c = fr_to_canonical(v);
      if (!p.no_end) store_words(p.proof, p.offv + 32 * (size_t)lane, c);
      sh.canon[lane] = c;
    }
    __syncwarp();
    if (lane == 0) {
      if (!p.no_end) {
        Fr canon[2] = {sh.canon[0], sh.canon[1]};
        tr_absorb_n<2, false>(sh.st, 'V', canon);
        if (!p.last) {
          S->alpha = tr_challenge_st<false>(sh.st, &S->error, true);
          S->beta = tr_challenge_st<false>(sh.st, &S->error, false);
        }
      }
#pragma unroll
      for (int i = 0; i < 8; ++i) S->st[i] = sh.st[i];
    }
  }
  cl.sync();  // no CTA leaves while another may still read its shared memory
}

int launch_layer_tail(const TailParams& p, void* stream) {
  return launch_pdl(k_layer_tail, kTailCTAs, kTailThreads, (cudaStream_t)stream, p);
}

// ---------------------------------------------------------------------------
// General circuits (Sec. 2.7): layer i's sumcheck runs over a virtual layer
// X_i (layer i + 1, then the used gates of deeper layers); the claims on a
// layer from all its readers are weight terms sum_t eq(z_t, b) M_t(g), each
// with its own copy point z_t, summed round by round in the copy phase.

// the terms' copy weights E_t(b) = 2^32 eq(z_t, b) (plain) over 2^c copies
// and gate weights om_t(q) = M_t(g_q) = alpha_x eq(r_x, u) + alpha_y eq(r_y,
// u) at the reading layer's X position u of gate g_q (0 when not used)
__global__ void k_general_terms(const GeneralTerm* __restrict__ terms, uint32_t nt, uint32_t c,
                                const uint4* __restrict__ sg, uint32_t ntot, uint32_t* __restrict__ Et,
                                uint32_t* __restrict__ omt) {
  const uint32_t C = 1u << c;
  const size_t per = (size_t)C + ntot, total = per * nt;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const uint32_t t = (uint32_t)(idx / per);
    const size_t rest = idx - (size_t)t * per;
    const GeneralTerm tm = terms[t];
    if (rest < C) {
      fr_store(Et, (size_t)t * C + rest, eq_half_entry(tm.rb, 0, c, (uint32_t)rest, fr_int_2_32()));
    } else {
      const uint32_t q = (uint32_t)(rest - C), u = tm.pos[sg[q].z];
      Fr w = fr_zero();
      if (u != 0xffffffffu)
        w = fr_add(fr_mul(tm.alpha[0], eq_index(tm.rx, tm.sxr, u)), fr_mul(tm.alpha[1], eq_index(tm.ry, tm.sxr, u)));
      fr_store(omt, (size_t)t * ntot + q, w);
    }
  }
}

int launch_general_terms(const GeneralTerm* terms_dev, uint32_t nt, uint32_t c, const uint4* sg, uint32_t ntot,
                         uint32_t* Et, uint32_t* omt, void* stream) {
  const size_t n = ((size_t)(1u << c) + ntot) * nt;
  k_general_terms<<<grid_for(n, 128), 128, 0, (cudaStream_t)stream>>>(terms_dev, nt, c, sg, ntot, Et, omt);
  return post_launch();
}

// the fold of a copy-weight table alone by the round's challenge r_b[k]
__global__ void k_fold_e(uint32_t* E, uint32_t h, const DevState* S, uint32_t k) {
  const Fr r = S->rb[k];
  for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < h; j += gridDim.x * blockDim.x)
    fr_store(E, j, fold2(fr_load(E, j), fr_load(E, j + h), r));
}

int launch_fold_e(uint32_t* E, uint32_t h, const DevState* S, uint32_t k, void* stream) {
  k_fold_e<<<grid_for(h, 128), 128, 0, (cudaStream_t)stream>>>(E, h, S, k);
  return post_launch();
}

// om_c(q) = sum_t e_t om_t(q), with e_t (Montgomery) from E_t[0] = 2^32 e_t
// (plain): E_t[0] times 2^-32 R^2 is e_t R.  E_c[0] = 2^32, so that the
// phases' copy weight is 1.
__global__ void k_combine_terms(const uint32_t* __restrict__ Et, uint32_t C, const uint32_t* __restrict__ omt,
                                uint32_t ntot, uint32_t nt, uint32_t* __restrict__ omc, uint32_t* __restrict__ Ec) {
  const Fr scale = fr_mul(fr_mont_2_neg32(), fr_r2());
  for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < ntot; q += gridDim.x * blockDim.x) {
    Fr w = fr_zero();
    for (uint32_t t = 0; t < nt; ++t)
      w = fr_add(w, fr_mul(fr_mul(fr_load(Et, (size_t)t * C), scale), fr_load(omt, (size_t)t * ntot + q)));
    fr_store(omc, q, w);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) fr_store(Ec, 0, fr_int_2_32());
}

int launch_combine_terms(const uint32_t* Et, uint32_t C, const uint32_t* omt, uint32_t ntot, uint32_t nt,
                         uint32_t* omc, uint32_t* Ec, void* stream) {
  k_combine_terms<<<grid_for(ntot ? ntot : 1, 128), 128, 0, (cudaStream_t)stream>>>(Et, C, omt, ntot, nt, omc, Ec);
  return post_launch();
}

// CTA 2 b + p sums block b of the row A against eq(r, .), r = r_x (p = 0)
// or r_y (p = 1): eq(r, u) = hi[u >> sl] lo[u mod 2^sl] from half tables in
// shared memory (sx <= 16)
constexpr uint32_t kBlockThreads = 256;
__global__ void __launch_bounds__(kBlockThreads) k_block_values(const uint32_t* __restrict__ A, uint32_t sx,
                                                                const uint2* __restrict__ blocks, uint32_t nb,
                                                                const DevState* S, uint32_t* __restrict__ vals) {
  __shared__ Fr hi[256], lo[256];
  __shared__ Fr red[kBlockThreads / 32];
  const uint32_t b = blockIdx.x >> 1, p = blockIdx.x & 1;
  const Fr* r = p == 0 ? S->rx : S->ry;
  const uint32_t sl = sx / 2, sh = sx - sl;
  for (uint32_t e = threadIdx.x; e < (1u << sh) + (1u << sl); e += kBlockThreads) {
    const bool h = e < (1u << sh);
    const uint32_t v = h ? e : e - (1u << sh);
    (h ? hi : lo)[v] = eq_half_entry(r, h ? 0 : sh, h ? sh : sl, v, fr_one());
  }
  __syncthreads();
  const uint2 blk = blocks[b];
  Fr acc = fr_zero();
  for (uint32_t u = blk.x + threadIdx.x; u < blk.x + blk.y; u += kBlockThreads)
    acc = fr_add(acc, fr_mul(fr_mul(hi[u >> sl], lo[u & ((1u << sl) - 1)]), fr_load(A, u)));
  acc = fr_warp_sum(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    Fr x = threadIdx.x < kBlockThreads / 32 ? red[threadIdx.x] : fr_zero();
    x = fr_warp_sum(x);
    if (threadIdx.x == 0) fr_store(vals, (size_t)p * nb + b, x);
  }
}

int launch_block_values(const uint32_t* A, uint32_t sx, const uint2* blocks, uint32_t nb, const DevState* S,
                        uint32_t* vals, void* stream) {
  k_block_values<<<2 * nb, kBlockThreads, 0, (cudaStream_t)stream>>>(A, sx, blocks, nb, S, vals);
  return post_launch();
}

// absorb of n canonical elements (any n), the transcript's absorb step
__device__ void tr_absorb_var(uint32_t* st, uint32_t tag, const uint32_t* canon_words, uint32_t n) {
  ShaWords8 h;
  for (int i = 0; i < 8; ++i) h.w[i] = st[i];
  h.w[7] ^= (tag << 8) | n;
  for (uint32_t b = 0; 16 * b < 8 * n; ++b) {
    ShaWords16 blk;
    for (int k = 0; k < 16; ++k) {
      const uint32_t w = 16 * b + k;
      blk.w[k] = w < 8 * n ? bswap32(canon_words[w]) : 0u;
    }
    h = tr_compress<true>(h, blk);
  }
  for (int i = 0; i < 8; ++i) st[i] = h.w[i];
}

__global__ void k_block_absorb(const uint32_t* __restrict__ vals, uint32_t nb, uint64_t squeeze_mask, DevState* S,
                               uint8_t* proof, size_t off, uint32_t c, uint32_t sx, uint32_t* __restrict__ hist) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  uint32_t canon[8 * 2 * 64];
  for (uint32_t k = 0; k < 2 * nb; ++k) {
    const Fr v = fr_to_canonical(fr_load(vals, k));
    store_words(proof, off + 32 * (size_t)k, v);
    for (int i = 0; i < 8; ++i) canon[8 * k + i] = v.v[i];
  }
  tr_absorb_var(S->st, 'V', canon, 2 * nb);
  // the layer's challenges, then the blocks' alphas
  for (uint32_t k = 0; k < c; ++k) fr_store(hist, k, S->rb[k]);
  for (uint32_t k = 0; k < sx; ++k) {
    fr_store(hist, c + k, S->rx[k]);
    fr_store(hist, c + sx + k, S->ry[k]);
  }
  bool fresh = true;
  for (uint32_t b = 0; b < nb; ++b) {
    if (!((squeeze_mask >> b) & 1u)) continue;
    const Fr ax = tr_challenge_st<true>(S->st, &S->error, fresh);
    const Fr ay = tr_challenge_st<true>(S->st, &S->error, false);
    fresh = false;
    fr_store(hist, c + 2 * sx + 2 * b, ax);
    fr_store(hist, c + 2 * sx + 2 * b + 1, ay);
  }
}

int launch_block_absorb(const uint32_t* vals, uint32_t nb, uint64_t squeeze_mask, DevState* S, uint8_t* proof,
                        size_t off, uint32_t c, uint32_t sx, uint32_t* hist, void* stream) {
  k_block_absorb<<<1, 32, 0, (cudaStream_t)stream>>>(vals, nb, squeeze_mask, S, proof, off, c, sx, hist);
  return post_launch();
}

}  // namespace sisu
