// Internal declarations shared by the library's translation units.
#pragma once
#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "fr.cuh"

#ifndef __CUDACC__
// CUDA's vector types, for translation units built by the host compiler
struct uint2 {
  uint32_t x, y;
};
struct uint4 {
  uint32_t x, y, z, w;
};
#endif

namespace sisu {

constexpr uint32_t kMaxLog = 32;         // bound on c and s_i (sizes <= 2^24 in practice)
constexpr uint32_t kMaxDomain = 256;     // transcript domain bytes
constexpr uint32_t kMaxPartials = 8192;  // blocks whose partial sums one round reduces
// host inputs of at least kEvalChunkMin bytes are copied in kEvalChunks
// chunks of copies, each evaluated while the next one is in transfer
constexpr uint32_t kEvalChunks = 8;
constexpr size_t kEvalChunkMin = (size_t)32 << 20;

// Device-resident prover state: the transcript and every challenge, so that
// no host round trip is needed inside a proof.  Challenges are stored in
// Montgomery form.
struct DevState {
  uint32_t st[8];       // transcript state, 32 bytes as big-endian words
  uint32_t dig_in[8];   // statement digest of the inputs
  uint32_t dig_out[8];  // statement digest of the outputs
  uint32_t counter;     // last-block-done counter of the running round
  uint32_t error;       // nonzero: a device-side check failed
  uint32_t pad[6];
  Fr zb[kMaxLog], zg[kMaxLog];             // initial claim point (copy bits, gate bits)
  Fr rb[kMaxLog], rx[kMaxLog], ry[kMaxLog];  // challenges of the running layer
  Fr alpha, beta, vx, vy;
};

struct InitParams {
  uint8_t domain[kMaxDomain];
  uint32_t dlen;
  uint32_t d, c;
  uint32_t s[65];
  uint32_t wiring[8];  // statement digest of the wiring (big-endian words)
};

// Per-layer device views of the circuit.
struct DevLayer {
  // accumulation layers (some gate has several entries): per gate g its
  // entries eo[offo[g] .. offo[g+1]) as {in1 | type << 30, in2}; null otherwise
  const uint32_t* offo;
  const uint2* eo;
  const uint4* sgate;    // entries, mul first then add, each sorted by in1: {in1, in2, out gate, 0};
                         // then the gates with no entry {0, 0, g, 0}
  const uint32_t* off1;  // CSR over layer i+1 positions x: sgate positions with in1 == x
  const uint32_t* pos1;
  const uint32_t* off2;  // same for in2
  const uint32_t* pos2;
  uint32_t nmul, ntot;   // number of mul entries, of entries
  uint32_t nsg;          // entries of sgate: the entries, then one for each gate with no entry
};

// Host copy of the padded circuit (the verifier and the digests use it).
struct HostCircuit {
  uint32_t d = 0, c = 0, C = 0, Creal = 0;
  std::vector<uint32_t> s, W, wreal;
  // gate layer i as fan-in-2 entries sorted by output gate (stable): gate
  // g's value is the sum of its entries (Sec. 3.4.3); a plain gate has one
  // entry, a padding gate none
  std::vector<std::vector<uint32_t>> out;
  std::vector<std::vector<uint8_t>> type;
  std::vector<std::vector<uint32_t>> in1, in2;
  uint32_t wiring_digest[8];
  // General circuits (Sec. 2.7): entry e's second input is gate in2 of
  // layer src[i][e] (i + 1 .. d).  Layer i's sumcheck runs over a virtual
  // layer X_i of 2^sx[i] positions: layer i + 1 in full (block 0), then for
  // each deeper layer it reads the gates it uses, ascending; u2[i][e] is the
  // X_i position of entry e's second input.
  bool general = false;
  struct Block {
    uint32_t layer, base, count;
    std::vector<uint32_t> ys;  // the block's gates in its layer (block 0: all of layer i + 1)
  };
  std::vector<std::vector<uint32_t>> src, u2;
  std::vector<uint32_t> sx;
  std::vector<std::vector<Block>> blocks;
  size_t proof_len() const;
};

// ---------------------------------------------------------------------------
// kernel launch wrappers (kernels.cu); all return cudaError_t as int

uint64_t launches_add(uint64_t n);
// per-kernel event timing (sisu_profile_enable): the index of the record
// opened for a launch of `kind` (-1 when the kind is off), closed after it
long prof_begin(uint32_t kind, double work, void* stream);
void prof_end(long idx, void* stream);
constexpr uint32_t kProfAssocHash = 9, kProfAssocPair = 10;
// sets the calling thread's sisu_last_error() message, returns code
int report_error(int code, const char* msg);
// SISU_OK when p is device (or managed) memory that kernels may read and
// write, else SISU_ERR_INVALID_ARG naming `what`: a host address handed to
// a kernel would fault the GPU.  cudaPointerGetAttributes allocates nothing
// and does not synchronise; ordinary and page-locked host memory are both
// refused.
int require_device(const void* p, const char* what);

// the input conversion and the layer evaluation of copies b0 .. b0 + nb - 1
// (each copy evaluates independently of the others)
int launch_inputs_to_mont(const uint32_t* in, uint32_t* V, uint32_t b0, uint32_t nb, uint32_t s, uint32_t Creal,
                          uint32_t wreal, uint32_t* err, void* stream);
int launch_eval_layer(const uint32_t* Vn, uint32_t* V, const DevLayer& L, uint32_t b0, uint32_t nb, uint32_t s,
                      uint32_t sn, void* stream);
int launch_layer_to_canonical(const uint32_t* V, uint32_t* out, uint32_t c, uint32_t s, uint32_t Creal,
                              uint32_t wreal, void* stream);
// Merkle statement digests (8 words each): of two Montgomery tables at
// once, elements converted to canonical bytes on the fly, the launches
// shared by both trees (scratch: digest_scratch_words(na * 32) +
// digest_scratch_words(nb * 32) words); or of raw device bytes.
int launch_digest_tables2(const uint32_t* ta, size_t na, const uint32_t* tb, size_t nb, uint32_t* scratch,
                          uint32_t* out_a, uint32_t* out_b, void* stream);
int launch_digest_bytes(const uint8_t* data, size_t len, uint32_t* scratch, uint32_t* out_words,
                        void* stream);
size_t digest_scratch_words(size_t len_bytes);

int launch_transcript_init(const InitParams& p, DevState* S, void* stream);
// cq, q: the copies are rank q's of 2^cq (copies j 2^cq + q, j < 2^c); 0, 0
// for all copies.  omega_o (not null): the gate weights in gate order as
// well, 2^s_i values (0 for a gate with no entry).
int launch_layer_init(DevState* S, uint32_t layer, uint32_t c, uint32_t s_i, const DevLayer& L, uint32_t* E,
                      uint32_t* omega_s, uint32_t* eqh, void* stream, uint32_t cq = 0, uint32_t q = 0,
                      uint32_t* omega_o = nullptr);
// words of the eq half-table scratch of launch_layer_init (copy bits c,
// largest layer log-width smax)
size_t eq_half_words(uint32_t c, uint32_t smax);
// the copy round's launch shape for layers of 2^sn positions and rounds of
// 2^log_pairs pairs (bd 0: the default); -1 for a value out of range
int set_copy_tune(uint32_t sn, uint32_t log_pairs, uint32_t bd, uint32_t form, uint32_t min_items);
// sums_out (not null): the round's sums g(0..3) go there (one rank of a
// copy-sharded proof) instead of the message and transcript
int launch_copy_round(const uint32_t* T, uint32_t sn, uint32_t h, const uint32_t* E, const uint32_t* omega_s,
                      const DevLayer& L, uint32_t* partials, DevState* S, uint8_t* proof, size_t off,
                      uint32_t k, void* stream, uint32_t* sums_out = nullptr);
// The copy phase by its linear recurrence: the rows' gate sums U(b) of
// layer i's values (rows of 2^sv, gate weights omo in gate order), and one
// round over the mul entries (U and c of the previous round in, of this
// round out; cpart: kMaxPartials / 2 values of scratch).
int launch_rowdot(const uint32_t* V, uint32_t sv, const uint32_t* omo, uint32_t C, uint32_t* U, void* stream);
int launch_copy_c(const uint32_t* T, uint32_t sn, uint32_t h, const uint32_t* E, const uint32_t* omega_s,
                  const DevLayer& L, const uint32_t* Uprev, const uint32_t* cprev, uint32_t* Ucur, uint32_t* ccur,
                  uint32_t* cpart, uint32_t* partials, DevState* S, uint8_t* proof, size_t off, uint32_t k,
                  void* stream);
int launch_copy_fold(const uint32_t* src, uint32_t* dst, uint32_t sn, uint32_t h, uint32_t* E,
                     DevState* S, uint32_t k, void* stream);
// copy-sharded proofs: the round message from the gathered sums of every
// rank; a rank's copy-bound row and weight as one message; rank 0's table
// of the gathered rows (stride values apart) and weights
int launch_shard_absorb(const uint32_t* sums_all, uint32_t world, DevState* S, uint8_t* proof, size_t off,
                        uint32_t k, void* stream);
int launch_shard_row(const uint32_t* A, const uint32_t* E, uint32_t Wn, uint32_t* out, void* stream);
int launch_shard_table(const uint32_t* rows, uint32_t world, uint32_t Wn, uint32_t stride, uint32_t* T, uint32_t* E,
                       void* stream);
// per-copy Merkle subtree roots of two tables of nc copies (row widths of at
// least 32 elements), and the two statement digests from every rank's roots
int launch_digest_copy_roots(const uint32_t* ta, uint32_t wa, const uint32_t* tb, uint32_t wb, uint32_t nc,
                             uint32_t* scratch, uint32_t* roots_a, uint32_t* roots_b, void* stream);
int launch_digest_from_roots(const uint32_t* all, uint32_t nc, uint32_t world, uint32_t wa, uint32_t wb,
                             uint32_t* scratch, uint32_t* out_a, uint32_t* out_b, void* stream);
int launch_xinit(const uint32_t* Arow, const uint32_t* E, const uint32_t* omega_s, const DevLayer& L,
                 uint32_t Wn, uint32_t* At, uint32_t* H1, uint32_t* H2, uint32_t* Ay, void* stream);
int launch_gate_round(uint32_t* A, uint32_t* B1, uint32_t* B2, uint32_t m, int phase, uint32_t k,
                      uint32_t* partials, DevState* S, uint8_t* proof, size_t off, void* stream);
int launch_eq_rx(DevState* S, uint32_t s, uint32_t W, uint32_t* Q, const uint32_t* At, void* stream);
int launch_yinit(const uint32_t* E, const uint32_t* omega_s, const uint32_t* Q, const DevLayer& L,
                 uint32_t Wn, uint32_t* K1, uint32_t* K2, DevState* S, void* stream);
int launch_layer_end(DevState* S, const uint32_t* Ay, uint32_t s, uint8_t* proof, size_t off, int last,
                     void* stream);

// General circuits: X_i[b][u] for every copy b and position u of the
// virtual layer (u < wn: layer i + 1; then the used gates of deeper
// layers, map[u - wn] = {layer, gate}; zero padding up to 2^sx)
struct GatherLayers {
  const uint32_t* V[65];
  uint32_t s[65];
};
int launch_gather_x(const GatherLayers& gl, uint32_t next, const uint2* map, uint32_t nmap, uint32_t* X,
                    uint32_t C, uint32_t sn, uint32_t sx, void* stream);
// the weight terms of a general layer's claims: E_t (2^32 eq(z_t, b), plain)
// and om_t (M_t of the gate of each sorted entry), t < nt
struct GeneralTerm {
  const Fr* rb;        // the reading layer's copy challenges (c)
  const Fr* rx;        // and its x and y challenges (sxr)
  const Fr* ry;
  const Fr* alpha;     // alpha_x, alpha_y of the reading layer's block
  const uint32_t* pos; // X position in the reading layer of each gate of this layer (~0: not used)
  uint32_t sxr;
};
int launch_general_terms(const GeneralTerm* terms_dev, uint32_t nt, uint32_t c, const uint4* sg, uint32_t ntot,
                         uint32_t* Et, uint32_t* omt, void* stream);
int launch_fold_e(uint32_t* E, uint32_t h, const DevState* S, uint32_t k, void* stream);
// om_c = sum_t e_t om_t (e_t = E_t[0] 2^-32, the copy weight at r_b), E_c[0] = 2^32
int launch_combine_terms(const uint32_t* Et, uint32_t C, const uint32_t* omt, uint32_t ntot, uint32_t nt,
                         uint32_t* omc, uint32_t* Ec, void* stream);
// v_b(r) = sum_{u in block b} eq(r, u) A(u) for r = r_x (vals[b]) and r_y
// (vals[nb + b]); blocks given as base/count pairs
int launch_block_values(const uint32_t* A, uint32_t sx, const uint2* blocks, uint32_t nb, const DevState* S,
                        uint32_t* vals, void* stream);
// the block values into the proof and the transcript ('V'), then alpha_x,
// alpha_y of every block whose layer is not the input layer (flags bit b),
// and the layer's challenges, into the history record hist (rb: c values,
// rx, ry: sx values each, then 2 nb alphas)
int launch_block_absorb(const uint32_t* vals, uint32_t nb, uint64_t squeeze_mask, DevState* S, uint8_t* proof,
                        size_t off, uint32_t c, uint32_t sx, uint32_t* hist, void* stream);

// Libra's two phases of one layer in a single thread-block-cluster launch
// (tables up to kTailMaxWidth entries): phase-1 init, the x rounds,
// EQ(r_x), phase-2 init, the y rounds and the end of the layer.
constexpr uint32_t kTailMaxWidth = 1u << 16;
struct TailParams {
  const uint32_t* A;  // row V~(r_b, .) after the copy phase
  const uint32_t* E;  // E[0] = 2^32 eq(z_b, r_b) (the copy weights carry a factor 2^32)
  const uint32_t* om; // gate weights, sorted order
  const uint4* sg;
  const uint32_t *off1, *pos1, *off2, *pos2;
  uint32_t nmul, ntot, Wn, s;
  uint32_t *At, *H1, *H2, *Ay;
  uint32_t* P;        // scratch: two values per entry (per-entry terms of the bookkeeping sums)
  DevState* S;
  uint8_t* proof;
  size_t offx, offy, offv;
  int last;
  int no_end;         // general layers: the block values end the layer instead (v_x, v_y and the state kept)
};
int launch_layer_tail(const TailParams& p, void* stream);

int launch_fr_batch(int op, const uint32_t* a, const uint32_t* b, uint32_t* out, size_t n,
                    uint32_t* flags, void* stream);
int run_microbench(int kind, uint32_t blocks, uint32_t threads, uint32_t iters, void* stream, double* ms,
                   double* ops);

// host verifier (verify.cpp)
int host_verify(const HostCircuit& hc, const uint8_t* inputs, const uint8_t* outputs, const uint8_t* proof,
                size_t proof_len, const uint8_t* domain, size_t dlen);
// host Merkle statement digest of bytes (big-endian words out)
void host_statement_digest(const uint8_t* data, size_t len, uint32_t out[8]);

}  // namespace sisu
