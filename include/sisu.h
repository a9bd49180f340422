/*
 * sisu.h - C ABI of the B300-native data-parallel GKR prover.
 *
 * The library proves the evaluation of a layered arithmetic circuit made of
 * many identical sub-circuit copies (data-parallel GKR, paper Sec. 2.2; the
 * workload of Sec. 3.2 and Sec. 4.1: one copy per validator check) over the
 * BN254 scalar field r (Sec. 4.1).  Each layer is reduced to the next by the
 * GKR layer sumcheck (Sec. 2.2) with Libra's linear-time two-phase prover
 * (Sec. 2.3), preceded by a phase over the copy variables; Fiat-Shamir
 * challenges come from a SHA-256 transcript.
 *
 * Conventions shared by every call
 *   - Field elements cross the boundary as 32-byte little-endian canonical
 *     integers in [0, r), r = 0x30644e72e131a029b85045b68181585d
 *                             2833e84879b9709143e1f593f0000001.
 *     An element >= r is rejected with SISU_ERR_NOT_CANONICAL.
 *   - Layer 0 holds the outputs, layer d the inputs (Sec. 2.2).  Gate g of
 *     gate layer i (0 <= i < d) reads gates in1[g] and in2[g] of layer i+1
 *     and adds (type 0) or multiplies (type 1) them.  All copies share the
 *     wiring.  Widths and the copy count need not be powers of two: they are
 *     padded with absent gates of value 0 and zero inputs (Sec. 2.2).
 *   - Tables of values are copy-major: element (b, g) at index b*width + g.
 *   - "stream" is a cudaStream_t (NULL = the legacy default stream).  Device
 *     pointers must be 16-byte aligned.  Every buffer that a call hands to
 *     its kernels as device memory (inputs or outputs flagged on_device,
 *     sisu_fr_batch's arrays, sisu_statement_digest's data, the shard
 *     exchange buffers) is checked with cudaPointerGetAttributes before
 *     anything is launched: host memory there, pageable or page-locked, is
 *     refused with SISU_ERR_INVALID_ARG instead of reaching a kernel.
 *   - Every call returns SISU_OK (0) or a negative SISU_ERR_* code; the
 *     calling thread's last error message is sisu_last_error().  No call
 *     aborts or exits.  Handles are not thread-safe: one thread (or one
 *     stream) at a time per handle.
 */
#ifndef SISU_H
#define SISU_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SISU_OK 0
#define SISU_ERR_INVALID_ARG (-1)  /* null pointer, zero size, bad gate type */
#define SISU_ERR_INDEX_OOB (-2)    /* in1/in2 not below the next layer's width, or an entry's gate not below its layer's */
#define SISU_ERR_NOT_CANONICAL (-3) /* a field element >= r */
#define SISU_ERR_OOM (-4)          /* device or host allocation failed */
#define SISU_ERR_CUDA (-5)         /* a CUDA runtime call failed */
#define SISU_ERR_TIMEOUT (-6)      /* a bounded device wait gave up */
#define SISU_ERR_REJECT (-7)       /* sisu_gkr_verify: the proof is invalid */
#define SISU_ERR_ZERO_INVERSE (-8) /* sisu_fr_batch inverse: a zero input */
#define SISU_ERR_TOO_LARGE (-9)    /* sizes beyond the library's limits */
#define SISU_ERR_BUFFER (-10)      /* caller buffer too small */

/* Limits: d <= 64 gate layers, widths <= 2^24, copies <= 2^24,
 * copies x width <= 2^32 per layer (padded sizes). */
#define SISU_MAX_LAYERS 64u
#define SISU_MAX_WIDTH (1u << 24)
#define SISU_MAX_COPIES (1u << 24)

typedef struct sisu_circuit sisu_circuit;       /* device wiring + gate lists */
typedef struct sisu_eval sisu_eval;             /* resident values of all layers */
typedef struct sisu_transcript sisu_transcript; /* Fiat-Shamir domain */

/* One gate layer i: `width` gates; type[g] in {0 add, 1 mul}; in1[g],
 * in2[g] index gates of layer i+1 (Sec. 2.2, the add_i / mult_i wiring). */
typedef struct {
  uint32_t width;
  const uint8_t* type;
  const uint32_t* in1;
  const uint32_t* in2;
} sisu_layer;

/* ---- circuits (Sec. 2.2: layered circuit, identical copies) ---------------
 * Copies the wiring (the caller may free its arrays afterwards), validates
 * it, uploads it to the current device and builds the per-layer gate lists
 * the prover uses (gates grouped by type, and indexed by in1 and by in2).
 * layers[0..n_gate_layers-1] are gate layers 0..d-1; input_width is the
 * width of layer d.  Errors: INVALID_ARG, INDEX_OOB, TOO_LARGE, OOM, CUDA. */
int sisu_circuit_create(const sisu_layer* layers, uint32_t n_gate_layers, uint32_t input_width,
                        uint32_t n_copies, sisu_circuit** out);
/* The same circuit held on the host only, for sisu_gkr_verify and
 * sisu_circuit_info on machines without a GPU (no CUDA call is made);
 * sisu_circuit_eval on such a handle returns INVALID_ARG. */
int sisu_circuit_create_host(const sisu_layer* layers, uint32_t n_gate_layers, uint32_t input_width,
                             uint32_t n_copies, sisu_circuit** out);

/* Accumulation gates (Sec. 3.4.3): gate layer i given as `n_entries`
 * fan-in-2 entries; entry e adds op_e(V_{i+1}(in1[e]), V_{i+1}(in2[e]))
 * (type[e] in {0 add, 1 mul}) to gate out[e] < width.  A gate's value is
 * the sum of its entries, 0 when it has none; entries of one gate may mix
 * types.  The order of a gate's entries is kept (it is part of the wiring
 * the transcript binds).  A circuit whose every gate has exactly one entry
 * is the same circuit as through sisu_circuit_create: same proofs. */
typedef struct {
  uint32_t width;      /* gates of the layer */
  uint32_t n_entries;  /* entries of the layer */
  const uint32_t* out; /* gate of each entry */
  const uint8_t* type;
  const uint32_t* in1;
  const uint32_t* in2;
} sisu_acc_layer;

/* As sisu_circuit_create / sisu_circuit_create_host, from entry lists.
 * Errors: INVALID_ARG, INDEX_OOB, TOO_LARGE, OOM, CUDA. */
int sisu_circuit_create_acc(const sisu_acc_layer* layers, uint32_t n_gate_layers, uint32_t input_width,
                            uint32_t n_copies, sisu_circuit** out);
int sisu_circuit_create_acc_host(const sisu_acc_layer* layers, uint32_t n_gate_layers, uint32_t input_width,
                                 uint32_t n_copies, sisu_circuit** out);

/* General circuits (Sec. 2.7): a gate of layer i takes its first input
 * from layer i + 1 and its second from any deeper layer src (i + 1 .. d),
 * so values skip layers instead of being forwarded gate by gate.  One
 * entry per gate: type (0 add, 1 mul), in1 (a gate of layer i + 1), src,
 * in2 (a gate of layer src).  Layer i is proven over a virtual layer X_i:
 * layer i + 1 in full, then for each deeper layer it reads only the gates
 * it uses, ascending (the paper's used-gates indexing), padded to a power
 * of two of at most 2^16 positions.  Its round messages run over X_i's
 * bits, and it ends with, for r = r_x and r = r_y, each block's part
 * v(r) = sum_{u in block} eq(r, u) X~_i(r_b, u) (layer i + 1's block
 * first): claims on the blocks' layers.  A layer's claims from all its
 * readers are combined with random coefficients, each keeping its own copy
 * point, and summed round by round in its copy phase.  A circuit whose
 * second inputs all come from layer i + 1 gives the layered proof, byte
 * for byte.  Proof: per layer c x 3, sx_i x 2, sx_i x 2 elements, then 2 x
 * (blocks of layer i) block values.  Not supported by the server or by
 * copy-sharded proving.
 * Errors: INVALID_ARG, INDEX_OOB (an input beyond its layer, or a src not
 * below the gate's layer), TOO_LARGE (a virtual layer above 2^16), OOM,
 * CUDA. */
typedef struct {
  uint32_t width;
  const uint8_t* type;
  const uint32_t* in1;
  const uint32_t* src;
  const uint32_t* in2;
} sisu_general_layer;
int sisu_circuit_create_general(const sisu_general_layer* layers, uint32_t n_gate_layers, uint32_t input_width,
                                uint32_t n_copies, sisu_circuit** out);
int sisu_circuit_create_general_host(const sisu_general_layer* layers, uint32_t n_gate_layers,
                                     uint32_t input_width, uint32_t n_copies, sisu_circuit** out);
void sisu_circuit_destroy(sisu_circuit* circ);

/* Padded shape: log2 of the copy count, log2 widths of layers 0..d (array
 * of d+1), proof length in bytes, and the device bytes one sisu_eval holds.
 * Any output pointer may be NULL. */
int sisu_circuit_info(const sisu_circuit* circ, uint32_t* depth, uint32_t* log_copies,
                      uint32_t* log_widths, size_t* proof_len, size_t* eval_bytes);

/* ---- forward evaluation (the layer relation of Sec. 2.2) -------------------
 * inputs: n_copies x input_width elements (32 B each), host or device
 * memory (inputs_on_device != 0).  Every layer's values stay resident on
 * the device in the returned handle.  The call returns once the work is
 * enqueued on `stream` and the inputs were found canonical (one wait).
 * Host inputs of at least 32 MiB (unpadded circuits) are copied in eight
 * chunks of copies on a stream of the handle while the chunks already
 * copied are evaluated on `stream` (each copy evaluates independently);
 * the ordering seen by `stream` is unchanged, and pinned host memory lets
 * the copies run asynchronously.  The statement digest of the inputs is
 * formed on another stream of the handle while the layers evaluate; a
 * proof on this handle waits for it (the handle also holds its scratch,
 * about 1/16 of the input layer's bytes).
 * Errors: INVALID_ARG, NOT_CANONICAL, OOM, CUDA. */
int sisu_circuit_eval(const sisu_circuit* circ, const uint8_t* inputs, int inputs_on_device,
                      void* stream, sisu_eval** out);
/* Re-evaluate into an existing handle (no allocation); same rules. */
int sisu_eval_update(sisu_eval* ev, const uint8_t* inputs, int inputs_on_device, void* stream);
/* Outputs (layer 0), n_copies x width_0 elements, to host memory (blocks)
 * or device memory (out_on_device != 0, enqueued on `stream`).
 * Errors: INVALID_ARG, BUFFER (cap too small), CUDA. */
int sisu_eval_outputs(const sisu_eval* ev, uint8_t* out, size_t cap, int out_on_device,
                      void* stream);
/* One whole padded layer (2^c x 2^s_layer elements, canonical) to host
 * memory; for tests and inspection.  Blocks. */
int sisu_eval_layer(const sisu_eval* ev, uint32_t layer, uint8_t* out, size_t cap, void* stream);
void sisu_eval_destroy(sisu_eval* ev);

/* ---- transcript domain ----------------------------------------------------
 * The Fiat-Shamir domain string (<= 256 bytes); NULL/0 selects the default
 * "SISU-GKR-v1".  Errors: INVALID_ARG, OOM. */
int sisu_transcript_create(const uint8_t* domain, size_t len, sisu_transcript** out);
void sisu_transcript_destroy(sisu_transcript* tr);

/* ---- proving (Sec. 2.2 GKR, Sec. 2.3 Libra two-phase sumcheck) -----------
 * Proves that `ev` holds the evaluation of `circ`.  Every step runs on the
 * device, enqueued on `stream`, with challenges kept in device memory; the
 * call blocks once at the end to copy the proof out.  Deterministic: the
 * same (circuit, inputs, domain) give the same bytes.
 * Proof layout: "SISUGKR2" || u32le d || u32le c || u32le s_0..s_d, then for
 * each layer i = 0..d-1: c x 3 elements (copy rounds: the round
 * polynomial at t = 0, 2, 3) || s_{i+1} x 2 (x rounds, t = 0, 2) ||
 * s_{i+1} x 2 (y rounds) || v_x || v_y.  A round leaves out g(1): the
 * verifier takes it as the running claim minus g(0).
 * sisu_gkr_prove allocates *proof (free it with sisu_free);
 * sisu_gkr_prove_into writes into the caller's buffer of `cap` bytes.
 * The first proof on an eval handle allocates the prover's workspace
 * (about copies/2 x max width x 32 bytes), kept until sisu_eval_destroy.
 * Errors: INVALID_ARG, BUFFER, OOM, CUDA. */
int sisu_gkr_prove(const sisu_circuit* circ, sisu_eval* ev, const sisu_transcript* tr, void* stream,
                   uint8_t** proof, size_t* proof_len);
int sisu_gkr_prove_into(const sisu_circuit* circ, sisu_eval* ev, const sisu_transcript* tr,
                        void* stream, uint8_t* proof, size_t cap, size_t* proof_len);

/* Batched proving (many independent instances): proves every
 * (circs[i], evals[i]) with one transcript domain, spreading the instances
 * over `concurrency` library-owned streams (0 = 4) so that one instance's
 * latency-bound phases overlap the others' arithmetic.  The work starts
 * after the caller's prior work on `stream`, and the call returns when
 * every proof is in proofs[i] (caps[i] bytes each; lens[i] = length, may be
 * NULL).  Each eval handle may appear once.  Proof bytes are identical to
 * sisu_gkr_prove_into's.  From the second proof on a handle, its launch
 * sequence is replayed from a CUDA graph (also for sisu_gkr_prove_into),
 * unless per-kernel profiling is on or SISU_NO_GRAPHS is set.
 * Errors: as sisu_gkr_prove_into, INVALID_ARG for a repeated handle. */
int sisu_gkr_prove_batch(const sisu_circuit* const* circs, sisu_eval* const* evals, uint32_t n,
                         const sisu_transcript* tr, void* stream, uint32_t concurrency, uint8_t* const* proofs,
                         const size_t* caps, size_t* lens);

/* ---- serving (continuous batching of proof jobs) --------------------------
 * A server owns one device allocation of `budget_bytes` (its memory budget),
 * `max_active` slots (two streams, three events and a 1 MiB pinned proof
 * buffer each, made once) and a worker thread.  Jobs queue in arrival
 * order.  Whenever a slot is free the worker admits the oldest queued job
 * whose footprint (all layer values plus the prover workspace, see
 * sisu_circuit_info) fits in the free part of the budget, lays the job out
 * there, and enqueues its evaluation and proof on the slot's stream.  A job
 * at the head that does not fit is passed by at most 16 admissions; then
 * nothing else is admitted until it fits (at the latest when the running
 * jobs finish), so no job starves.  Admitted jobs run concurrently, so
 * their rounds interleave on the device; a finished job frees its slot and
 * memory, which admits the next.  Every proof is byte
 * for byte the proof sisu_gkr_prove_into gives for the same inputs and
 * domain (NULL/0 = the default domain).  The server works on the device
 * that is current at creation.  Per-kernel profiling must be off while a
 * server runs.
 * submit: the circuit must outlive the job and the inputs (host or device,
 *   n_copies x input_width elements) must stay unchanged until the job is
 *   done; pinned host inputs let the input copy run asynchronously.
 *   Errors: TOO_LARGE when the footprint exceeds the whole budget.
 * poll: *status = 0 queued, 1 running, 2 done (the proof is copied out and
 *   the ticket released), or a negative SISU_ERR_* (e.g. NOT_CANONICAL
 *   inputs; the ticket is released).  *latency_ms = completion - submission;
 *   *admit_order (may be NULL) = the number of jobs admitted before this
 *   one (UINT64_MAX for a job dropped unadmitted).
 * pause: paused != 0 stops admissions (running jobs continue, submissions
 *   queue), 0 resumes them.
 * pending: queued and running job counts.
 * destroy: waits for running jobs; queued jobs are dropped. */
typedef struct sisu_server sisu_server;
int sisu_server_create(size_t budget_bytes, uint32_t max_active, const uint8_t* domain, size_t dlen,
                       sisu_server** out);
int sisu_server_submit(sisu_server* s, const sisu_circuit* circ, const uint8_t* inputs, int inputs_on_device,
                       uint64_t* ticket);
int sisu_server_poll(sisu_server* s, uint64_t ticket, int* status, uint8_t* proof, size_t cap, size_t* len,
                     double* latency_ms, uint64_t* admit_order);
int sisu_server_pause(sisu_server* s, int paused);
/* The device bytes a server job of this circuit takes from the budget
 * (layer values, input staging when host inputs need padding, digest
 * scratch and the prover workspace).  Errors: INVALID_ARG. */
int sisu_job_footprint(const sisu_circuit* circ, int inputs_on_device, size_t* bytes);
int sisu_server_pending(sisu_server* s, uint32_t* queued, uint32_t* running);
void sisu_server_destroy(sisu_server* s);

/* Host verifier: replays the transcript, checks g(0) + g(1) = claim in
 * every round (Sec. 3.2.1), the final identity of every layer by summing
 * the wiring predicates, the output claim from `outputs` and the input
 * claims from `inputs` (both host memory, unpadded, copy-major).
 * Returns SISU_OK or SISU_ERR_REJECT (or INVALID_ARG / NOT_CANONICAL). */
int sisu_gkr_verify(const sisu_circuit* circ, const uint8_t* inputs, const uint8_t* outputs,
                    const uint8_t* proof, size_t proof_len, const uint8_t* domain, size_t dlen);

/* ---- copy-sharded proving (Sec. 3.2.1, distributed GKR) -------------------
 * The paper spreads the sumcheck over machines: the variables split into
 * machine bits and local bits, the machines' partial round polynomials are
 * summed at a master, and after the local rounds the master continues on a
 * table of one entry per machine.  Here the machine index is the low part
 * of the copy index: rank q of `world` (a power of two) holds copies
 * b = j * world + q, j < 2^c_loc.  Copy bits are bound most significant
 * first, so rounds 0 .. c_loc - 1 of a layer's copy phase bind rank-local
 * bits only, and the proof is byte for byte the one-GPU proof of all
 * world * 2^c_loc copies.
 *
 * A rank's evaluation is sisu_circuit_eval of a circuit with the same
 * wiring and 2^c_loc copies (no padded copies; output and input widths of
 * at least 32, so that each copy's rows are whole 1 KiB digest chunks) on
 * its copies' inputs, in the order j = 0, 1, ....  The exchanges between
 * the calls are the caller's (for example NCCL all-gathers, or device
 * copies between ranks that share a GPU); every call only enqueues work on
 * `stream` and reads or writes the device buffers given at creation, each
 * 16-byte aligned, of the sizes sisu_shard_buffer_sizes reports:
 *   roots_send  -> all-gather -> roots_recv   (every rank's copy digests)
 *   sums_send   -> all-gather -> sums_recv    (a copy round's 4 sums)
 *   row_send    -> gather to rank 0 -> row_recv (rank 0 only; the rank's
 *                                               copy-bound row and weight)
 *   state       <- broadcast from rank 0      (transcript and challenges)
 * "all-gather" puts rank q's send buffer at q * (send size) in recv.
 * One proof, every rank in step:
 *   roots; exchange; begin;
 *   for each layer i < depth:
 *     layer_begin(i);
 *     for k < local_rounds: copy_round(i, k); exchange sums; absorb(i, k);
 *     row(i); gather rows; rank 0: finish(i); broadcast state;
 *   rank 0: proof.
 * Errors: INVALID_ARG (shapes, buffers, a layer or round out of range), OOM,
 * CUDA, TOO_LARGE. */
typedef struct sisu_shard sisu_shard;
typedef struct {
  void* roots_send;
  void* roots_recv;
  void* sums_send;
  void* sums_recv;
  void* row_send;
  void* row_recv;  /* rank 0; may be NULL on other ranks */
  void* state;
} sisu_shard_buffers;
/* sizes[7]: bytes of roots_send, roots_recv, sums_send, sums_recv, row_send,
 * row_recv, state for this rank's evaluation in a world of `world` ranks. */
int sisu_shard_buffer_sizes(const sisu_eval* local, uint32_t world, size_t* sizes);
/* Allocates the rank's workspace (the evaluation must outlive the shard).
 * tr: transcript domain, NULL for the default. */
int sisu_shard_create(sisu_eval* local, uint32_t rank, uint32_t world, const sisu_transcript* tr,
                      const sisu_shard_buffers* bufs, sisu_shard** out);
void sisu_shard_destroy(sisu_shard* sh);
/* local_rounds = c_loc (copy rounds a rank runs alone each layer),
 * copy_bits = c_loc + log2(world), proof_len = the whole proof's bytes. */
int sisu_shard_info(const sisu_shard* sh, uint32_t* local_rounds, uint32_t* copy_bits, size_t* proof_len);
/* roots_send = the Merkle subtree roots of the rank's input rows, then of
 * its output rows (the statement digests' trees are perfect: a copy's rows
 * are a subtree). */
int sisu_shard_roots(sisu_shard* sh, void* stream);
/* From roots_recv: the statement digests, the initial transcript state and
 * the claim point (every rank alike). */
int sisu_shard_begin(sisu_shard* sh, void* stream);
/* The rank's copy weights eq(z, j world + q) and the layer's gate weights. */
int sisu_shard_layer_begin(sisu_shard* sh, uint32_t layer, void* stream);
/* sums_send = the rank's part g_q(0..3) of copy round k (k < local_rounds). */
int sisu_shard_copy_round(sisu_shard* sh, uint32_t layer, uint32_t k, void* stream);
/* From sums_recv: the round message (their sum), its transcript step and
 * challenge, then the fold of the rank's rows and weights. */
int sisu_shard_absorb(sisu_shard* sh, uint32_t layer, uint32_t k, void* stream);
/* row_send = the rank's copy-bound row (W_{layer+1} values) and its weight. */
int sisu_shard_row(sisu_shard* sh, uint32_t layer, void* stream);
/* Rank 0, from row_recv: the last log2(world) copy rounds on the table of
 * one row a rank, Libra's two phases and the end of the layer (into state). */
int sisu_shard_finish(sisu_shard* sh, uint32_t layer, void* stream);
/* Waits for `stream`; rank 0's buffer then holds the whole proof. */
int sisu_shard_proof(sisu_shard* sh, void* stream, uint8_t* proof, size_t cap, size_t* proof_len);

/* ---- associative hash (Sec. 3.4.1, Algorithm 1) and the pairwise-distinct
 * check (Sec. 3.4.2, Algorithm 2) ---------------------------------------------
 * F(e): r = 0, then three times r = (r + e + 2^32 - 1)^3 in the BN254 scalar
 * field; the hash of a list is h_pre + F(e_1) + ... + F(e_n), which does not
 * depend on the order of the list and continues from the hash h_pre of an
 * earlier list (the running value H_pre of Sec. 3.4.2; NULL stands for 0).
 *
 * Elements are 32-byte canonical little-endian values, `elems` holding
 * offsets[n_segments] of them back to back: host memory (on_device = 0,
 * copied in by the call) or device memory (on_device != 0, 16-byte
 * aligned).  Segment g is elements [offsets[g], offsets[g+1]) (host array
 * of n_segments + 1 values, offsets[0] = 0, not decreasing; empty segments
 * allowed) and gets out[32 g .. 32 g + 31] (host) = h_pre[g] + sum of F over
 * it, h_pre a host array of n_segments canonical values or NULL.  The work
 * is enqueued on `stream` (a cudaStream_t or NULL); the call blocks until
 * the results are copied out.
 * Errors: INVALID_ARG (NULL arrays, offsets, misaligned device array),
 * NOT_CANONICAL (an element or h_pre value not below r), CUDA. */
int sisu_assoc_hash_segments(const uint8_t* elems, const uint64_t* offsets, uint32_t n_segments,
                             const uint8_t* h_pre, int on_device, void* stream, uint8_t* out);
/* One segment of n elements; h_pre: one canonical value or NULL. */
int sisu_assoc_hash(const uint8_t* elems, uint64_t n, const uint8_t* h_pre, int on_device, void* stream,
                    uint8_t* out);
/* Algorithm 2 on lists a and a_sorted of n elements each (same memory kind,
 * as above): *result = 1 when the two hashes are equal and a_sorted is
 * strictly ascending as integers (a_sorted[i] > a_sorted[i-1]), else 0.
 * With a_sorted the sorted permutation of a that the prover supplies, 1
 * means the elements of a are pairwise distinct.  h_a, h_sorted (host, 32
 * bytes, may be NULL) receive the two hashes.  n = 0 gives 1.
 * Errors: INVALID_ARG, NOT_CANONICAL, CUDA. */
int sisu_pairwise_distinct_check(const uint8_t* a, const uint8_t* a_sorted, uint64_t n, int on_device, void* stream,
                                 int* result, uint8_t* h_a, uint8_t* h_sorted);
/* Algorithm 2 on every segment g (elements [offsets[g], offsets[g+1]) of
 * both arrays; offsets as for sisu_assoc_hash_segments): results[g] (host,
 * n_segments ints) as above; h_a, h_sorted (host, 32 n_segments bytes each,
 * may be NULL) receive the segments' hashes.  A segment's order check does
 * not look across its first element. */
int sisu_pairwise_distinct_check_segments(const uint8_t* a, const uint8_t* a_sorted, const uint64_t* offsets,
                                          uint32_t n_segments, int on_device, void* stream, int* results,
                                          uint8_t* h_a, uint8_t* h_sorted);
/* Slot hashes and Algorithm 2 per epoch in one call (Sec. 3.4.1-3.4.2):
 * every slot g (elements [slot_offsets[g], slot_offsets[g+1]) of a) is
 * hashed by Algorithm 1 into slot_hashes (host, 32 n_slots bytes), and
 * every epoch e (slots e*slots_per_epoch .. (e+1)*slots_per_epoch - 1, and
 * the same element range of a_sorted) gets Algorithm 2's answer in
 * results[e] (host, n_slots / slots_per_epoch ints).  Because AH is a sum
 * of F over the elements, the epoch's hash of a is the sum (mod r) of its
 * slots' hashes: a is read once, for the slot hashes, and only a_sorted is
 * hashed again (with its order check).  The answers equal those of
 * sisu_pairwise_distinct_check_segments on the epochs.  h_a, h_sorted
 * (host, 32 bytes an epoch, may be NULL) receive the epoch hashes.  Arrays
 * and memory kinds as for sisu_assoc_hash_segments; slots_per_epoch must
 * divide n_slots.  Blocks until done.
 * Errors: INVALID_ARG, NOT_CANONICAL, CUDA. */
int sisu_assoc_epochs(const uint8_t* a, const uint8_t* a_sorted, const uint64_t* slot_offsets, uint32_t n_slots,
                      uint32_t slots_per_epoch, int on_device, void* stream, uint8_t* slot_hashes, int* results,
                      uint8_t* h_a, uint8_t* h_sorted);
/* The prover's side of Algorithm 2: `out` receives the n canonical elements
 * of `in` in ascending order (as integers), equal values kept.  in and out
 * are both host or both device memory (on_device; device arrays 16-byte
 * aligned; in == out allowed).  A least-significant-digit radix sort over
 * the bytes on which the elements differ; *passes (may be NULL) receives
 * the number of byte passes run (3 for values below 2^24, up to 32).
 * Blocks until done.  Errors: INVALID_ARG, NOT_CANONICAL, TOO_LARGE
 * (n >= 2^32), CUDA. */
int sisu_sort_elements(const uint8_t* in, uint64_t n, int on_device, void* stream, uint8_t* out, uint32_t* passes);

/* ---- field core (Sec. 4.1, BN254 scalar field) ----------------------------
 * Elementwise on device arrays of n canonical elements, enqueued on
 * `stream` and awaited: op 0 a+b, 1 a-b, 2 a*b, 3 a^-1 (batched inversion:
 * Montgomery's trick per thread, one Fermat exponentiation per batch; a
 * zero input yields 0 and SISU_ERR_ZERO_INVERSE), 4 a*b + (1-a)(1-b),
 * 5 out[i] = sum of a[j]*b[j] for j from 64*floor(i/64) to i (the lazily
 * reduced dot product the copy-phase rounds use: full 512-bit products
 * summed exactly, one reduction per sum), 6 a[i]*b[0] (the product by
 * one fixed multiplier that folds a table by a challenge: eight 32x256-bit
 * rows and a two-word reduction), 7 a^2 by the squaring routine (28
 * doubled off-diagonal and 8 diagonal partial products, then the
 * reduction), 8 the same square taken of the representative a R + r of a's
 * Montgomery form (exercises inputs in [r, 2r)).  b is ignored for ops 3, 7
 * and 8.  Errors: INVALID_ARG, NOT_CANONICAL, ZERO_INVERSE. */
int sisu_fr_batch(int op, const uint8_t* a, const uint8_t* b, uint8_t* out, size_t n, void* stream);

/* Merkle statement digest of device bytes (the transcript's digest of
 * wiring, inputs and outputs): SHA-256 tree over 1024-byte chunks, leaf =
 * H(chunk || 0x00), node = H(left || right || 0x01), odd last node moved
 * up, digest = H(root || u64le len || 0x03).  out: 32 host bytes. */
int sisu_statement_digest(const uint8_t* data, size_t len, uint8_t* out, void* stream);

/* The same digest without any allocation, for callers that must not let a
 * library allocate device memory: a serving loop or framework that owns
 * all device memory through its own pool (cudaMalloc can synchronise the
 * device and fragments the pool) or code running while that pool's lock is
 * held.  (The paper has no counterpart: this is a property of the library.)
 *   data: device bytes, len <= 67108864 (64 MiB); larger inputs return
 *         SISU_ERR_TOO_LARGE with a message naming the limit.
 *   out:  32 device bytes the caller provides, written by work enqueued on
 *         `stream` (the call does not wait).
 * Scratch: a fixed 4 MiB array in the library's device memory, which every
 * GPU that loads the library holds until the process exits.  The first call
 * on a device looks up that array's device address (cudaGetSymbolAddress)
 * and caches it for later calls.  All calls share the array: calls that overlap on the GPU (on
 * different streams, or from different threads) race and must be ordered
 * by the caller.  Nothing in the array needs to start at zero.  No
 * cudaMalloc, cudaFree or other allocating routine is called.
 * Both buffers are checked with cudaPointerGetAttributes (which allocates
 * nothing) before any launch: host memory, pinned or not, is refused.
 * Errors: INVALID_ARG (NULL, or data / out not device memory), TOO_LARGE,
 * CUDA (with the runtime's error string). */
int sisu_statement_digest_noalloc(const uint8_t* data, size_t len, uint8_t* out, void* stream);

/* Launch shape of a layered circuit's copy-round kernel for layers whose
 * next layer has 2^log_width positions, in rounds of 2^log_pairs pairs
 * (both < 25), as an autotuner picks it: cta_threads 128, 256 or 384 (0
 * restores the default, 256), form 0 = whole pairs a CTA while pairs are
 * at least the CTAs and shares of a pair's mul entries otherwise (the
 * default), 1 = shares whenever there are at most 4096 pairs, 2 = whole
 * pairs always; min_items = mul entries a share at least (0: half a CTA's
 * threads).  General circuits and copy-sharded ranks keep their own fixed
 * shape.  Proof bytes do not depend on it.  Process-wide; set it before the
 * first proof of an eval handle (a handle replays the launches it
 * captured).  Errors: INVALID_ARG. */
int sisu_tune_copy_round(uint32_t log_width, uint32_t log_pairs, uint32_t cta_threads, uint32_t form,
                         uint32_t min_items);

/* Integer-pipe microbenchmarks used for the roofline: kind 0 = independent
 * 32-bit multiply-add chains (mad.lo), kind 1 = mad.hi chains, kind 2 =
 * Montgomery products as the kernels call them, kind 3 = the same products
 * inlined, kind 4 = 32x32+64-bit mad.wide chains, kind 5 = Montgomery
 * products built from 64-bit partial products (mul.wide), kind 6 = kinds 2
 * and 5 run side by side on the same operands, kind 7 = full 512-bit
 * products added into one 544-bit accumulator (no reduction), kind 8 =
 * Montgomery squares by the squaring routine, kind 9 = kind 7 with each
 * product by one level of Karatsuba, kind 10 = kinds 7 and 9 on the same
 * arbitrary 256-bit operands (all-ones words included), kind 11 =
 * Montgomery products as a Karatsuba product and a separate reduction,
 * kind 12 = kinds 2 and 11 on the same operands, kind 13 = Montgomery
 * products two a call with their steps interleaved, kind 14 = kind 13
 * against kind 2 on the same operands, kind 15 = Montgomery products with
 * the reduction's products by the low limb of r as multiply-adds (kind 2
 * forms them by shifts and subtractions), kind 16 = kind 15 against kind 2
 * on the same operands.  Reports the elapsed milliseconds and the number of
 * operations (multiply-adds, or field products for kinds 2, 3, 5, 7, 8, 9,
 * 11, 13 and 15); for kinds 6, 10, 12, 14 and 16, *ops is minus the number
 * of threads whose two results disagreed (0 when they all agree). */
int sisu_microbench(int kind, uint32_t blocks, uint32_t threads, uint32_t iters, void* stream,
                    double* ms, double* ops);

/* Per-kernel timing with CUDA events on the launching stream.  Bit k of
 * kind_mask enables kind k: 0 copy-phase round, 1 copy-phase fold, 2 layer
 * evaluation, 3 x/y-phase round, 4 statement digests, 5 layer init, 6 x/y
 * phase init, 7 transcript-only kernels, 8 input conversion, 9 associative
 * hash sums, 10 pairwise-distinct sums (for 9 and 10 the work counted is
 * evaluations of F, not field products), 11 the copy phase's row sums of a
 * layer; 0 disables.
 * sisu_profile_read waits for the recorded events of one kind and returns
 * their summed milliseconds, the launch count and the algorithmic field
 * products of those launches, in Montgomery products (264 multiply-adds; a
 * full 512-bit product counts 128/264 of one): a layered circuit's copy
 * round forms one Montgomery and one full product per mul entry and pair,
 * and 4 (first round) or 8 Montgomery products per pair; its row sums one
 * full product per copy and gate; a general circuit's copy round 2 + 4 f
 * products per pair and gate (6 per mul gate, 2 per add gate); then forgets
 * them. */
int sisu_profile_enable(uint32_t kind_mask);
int sisu_profile_read(uint32_t kind, double* ms, uint64_t* launches, double* fr_mults);
/* The recorded launches of one kind one by one, oldest first, without
 * forgetting them: up to `cap` milliseconds and field-product counts; *n =
 * the number recorded. */
int sisu_profile_launches(uint32_t kind, double* ms, double* fr_mults, size_t cap, size_t* n);

/* Number of kernels this library launched so far in this process (a CUDA
 * graph replay counts the kernels it runs). */
uint64_t sisu_kernel_launches(void);

void sisu_free(void* p);
const char* sisu_last_error(void);
const char* sisu_version(void);

#ifdef __cplusplus
}
#endif
#endif /* SISU_H */
