// Copy-sharded proving: one rank's part of a proof whose copies are spread
// over `world` ranks (the paper's distributed GKR, Sec. 3.2.1).
//
// The paper splits the variables of the layer polynomial into machine bits
// and local bits; the machine's partial round polynomials are summed at a
// master, and after the local rounds the master rebuilds a table of one
// entry per machine and runs the remaining rounds itself.  Here the machine
// index is the low part of the copy index: rank q holds copies b = j world +
// q.  Copy variables are bound most significant first, so a rank's copy
// rounds 1 .. c - log2(world) bind only its own bits; each is the sum over
// the ranks of their round polynomials (all-gather of 4 values a rank, then
// every rank sums them and runs the same transcript).  Then each rank's
// table is one row, rank 0 gathers the rows and their copy weights as a
// table of world rows, runs the last log2(world) copy rounds and Libra's
// phases on it, and its transcript state goes back to every rank for the
// next layer.  The proof bytes equal a one-GPU proof of all the copies.
//
// The exchanges themselves are the caller's (NCCL, or device copies between
// ranks that share one GPU); every call here only enqueues kernels on the
// caller's stream, reading and writing the exchange buffers it was given.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <memory>
#include <new>
#include <vector>

#include "handles.h"

using namespace sisu;

namespace {
constexpr int kBufs = 7;  // roots send/recv, sums send/recv, row send/recv, state

size_t al(size_t b) { return (b + 255) & ~(size_t)255; }

uint32_t log2_exact(uint32_t v) {
  uint32_t s = 0;
  while ((1u << s) < v) ++s;
  return s;
}

uint32_t max_next_width(const HostCircuit& hc) {
  uint32_t w = 1;
  for (uint32_t i = 0; i < hc.d; ++i) w = std::max(w, hc.W[i + 1]);
  return w;
}

void buffer_sizes(const HostCircuit& hc, uint32_t world, size_t out[kBufs]) {
  const size_t roots = 2 * (size_t)hc.C * 32, sums = 4 * 32, row = ((size_t)max_next_width(hc) + 1) * 32;
  const size_t v[kBufs] = {roots, roots * world, sums, sums * world, row, row * world, sizeof(DevState)};
  for (int k = 0; k < kBufs; ++k) out[k] = v[k];
}
}  // namespace

struct sisu_shard {
  sisu_eval* ev = nullptr;  // the rank's evaluation: its circuit holds this rank's copies
  uint32_t rank = 0, world = 1, cq = 0, c_loc = 0, c_full = 0;
  Workspace w;              // laid out in dev (not owned by w)
  uint32_t *T0 = nullptr, *E0 = nullptr, *top = nullptr;
  void* dev = nullptr;
  uint8_t* host = nullptr;  // pinned: proof bytes, then the error word
  sisu_shard_buffers b{};
  sisu_transcript tr{};
  std::vector<size_t> layer_off;  // proof offset of each layer's first message
  ~sisu_shard() {
    if (dev) cudaFree(dev);
    if (host) cudaFreeHost(host);
  }
};

extern "C" int sisu_shard_buffer_sizes(const sisu_eval* local, uint32_t world, size_t* sizes) {
  if (!local || !sizes) return report_error(SISU_ERR_INVALID_ARG, "NULL eval or sizes");
  if (world == 0 || (world & (world - 1)) != 0) return report_error(SISU_ERR_INVALID_ARG, "world must be a power of two");
  buffer_sizes(local->circ->hc, world, sizes);
  return SISU_OK;
}

extern "C" int sisu_shard_create(sisu_eval* local, uint32_t rank, uint32_t world, const sisu_transcript* tr,
                                 const sisu_shard_buffers* bufs, sisu_shard** out) {
  if (!out) return report_error(SISU_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!local || !bufs) return report_error(SISU_ERR_INVALID_ARG, "NULL eval or buffers");
  if (world == 0 || (world & (world - 1)) != 0 || world > (1u << 20))
    return report_error(SISU_ERR_INVALID_ARG, "world must be a power of two, at most 2^20");
  if (rank >= world) return report_error(SISU_ERR_INVALID_ARG, "rank beyond world");
  const HostCircuit& hc = local->circ->hc;
  if (hc.general) return report_error(SISU_ERR_INVALID_ARG, "copy-sharded proving of general circuits is not supported");
  if (hc.Creal != hc.C)
    return report_error(SISU_ERR_INVALID_ARG, "a rank's copy count must be a power of two (no padded copies)");
  if (hc.W[0] < 32 || hc.W[hc.d] < 32)
    return report_error(SISU_ERR_INVALID_ARG, "sharding needs output and input widths of at least 32 (1 KiB rows)");
  const uint32_t cq = log2_exact(world);
  if (hc.c + cq + hc.s[0] > 32 || hc.c + cq >= kMaxLog)
    return report_error(SISU_ERR_TOO_LARGE, "copies x width above 2^32");
  if (!bufs->roots_send || !bufs->roots_recv || !bufs->sums_send || !bufs->sums_recv || !bufs->row_send ||
      !bufs->state || (rank == 0 && !bufs->row_recv))
    return report_error(SISU_ERR_INVALID_ARG, "an exchange buffer is NULL");
  const void* ptrs[kBufs] = {bufs->roots_send, bufs->roots_recv, bufs->sums_send, bufs->sums_recv,
                             bufs->row_send, bufs->row_recv, bufs->state};
  for (const void* p : ptrs)
    if (((uintptr_t)p & 15) != 0) return report_error(SISU_ERR_INVALID_ARG, "exchange buffers must be 16-byte aligned");
  for (const void* p : ptrs)
    if (p)
      if (int rc = require_device(p, "exchange buffer")) return rc;
  std::unique_ptr<sisu_shard> sh(new (std::nothrow) sisu_shard());
  if (!sh) return report_error(SISU_ERR_OOM, "host allocation");
  sh->ev = local;
  sh->rank = rank;
  sh->world = world;
  sh->cq = cq;
  sh->c_loc = hc.c;
  sh->c_full = hc.c + cq;
  sh->b = *bufs;
  if (tr) {
    sh->tr = *tr;
  } else {
    const char* d = "SISU-GKR-v1";
    sh->tr.len = (uint32_t)strlen(d);
    memcpy(sh->tr.domain, d, sh->tr.len);
  }
  const uint32_t wmax = max_next_width(hc);
  const size_t C = (size_t)hc.C * world;
  const size_t ws = workspace_footprint_c(local->circ, sh->c_full);
  const size_t t0 = al((size_t)world * wmax * 32), e0 = al((size_t)world * 32);
  const size_t top = al(2 * digest_scratch_words(C * 1024) * 4);
  if (cudaMalloc(&sh->dev, ws + t0 + e0 + top) != cudaSuccess)
    return report_error(SISU_ERR_OOM, "device allocation of the shard's workspace");
  uint8_t* base = (uint8_t*)sh->dev;
  sh->T0 = (uint32_t*)(base + ws);
  sh->E0 = (uint32_t*)(base + ws + t0);
  sh->top = (uint32_t*)(base + ws + t0 + e0);
  size_t off = 8 + 4 * ((size_t)hc.d + 3);
  for (uint32_t i = 0; i < hc.d; ++i) {
    sh->layer_off.push_back(off);
    off += 32 * (3 * (size_t)sh->c_full + 4 * (size_t)hc.s[i + 1] + 2);
  }
  if (cudaMallocHost(&sh->host, off + 16) != cudaSuccess) return report_error(SISU_ERR_OOM, "pinned host allocation");
  sh->w.owns_host = false;
  if (int rc = workspace_layout(local->circ, &sh->w, base, sh->host, sh->c_full, 0)) return rc;
  sh->w.S = (DevState*)bufs->state;  // the state is the caller's: it is broadcast from rank 0 in place
  if (cudaStreamSynchronize(0) != cudaSuccess) return report_error(SISU_ERR_CUDA, "shard set-up");
  *out = sh.release();
  return SISU_OK;
}

extern "C" void sisu_shard_destroy(sisu_shard* sh) { delete sh; }

extern "C" int sisu_shard_info(const sisu_shard* sh, uint32_t* local_rounds, uint32_t* copy_bits, size_t* proof_len) {
  if (!sh) return report_error(SISU_ERR_INVALID_ARG, "NULL shard");
  if (local_rounds) *local_rounds = sh->c_loc;
  if (copy_bits) *copy_bits = sh->c_full;
  if (proof_len) *proof_len = sh->w.proof_len;
  return SISU_OK;
}

static int cuda_err(int e, const char* what) {
  if (e == 0) return SISU_OK;
  char msg[256];
  snprintf(msg, sizeof msg, "%s: %s", what, cudaGetErrorString((cudaError_t)e));
  return report_error(SISU_ERR_CUDA, msg);
}

extern "C" int sisu_shard_roots(sisu_shard* sh, void* stream) {
  if (!sh) return report_error(SISU_ERR_INVALID_ARG, "NULL shard");
  const HostCircuit& hc = sh->ev->circ->hc;
  uint32_t* send = (uint32_t*)sh->b.roots_send;
  return cuda_err(launch_digest_copy_roots(sh->ev->V[hc.d], hc.W[hc.d], sh->ev->V[0], hc.W[0], hc.C, sh->w.dscratch,
                                           send, send + 8 * (size_t)hc.C, stream),
                  "digest roots");
}

extern "C" int sisu_shard_begin(sisu_shard* sh, void* stream) {
  if (!sh) return report_error(SISU_ERR_INVALID_ARG, "NULL shard");
  const HostCircuit& hc = sh->ev->circ->hc;
  cudaStream_t st = (cudaStream_t)stream;
  DevState* S = sh->w.S;
  if (cudaMemsetAsync(S, 0, sizeof(DevState), st) != cudaSuccess) return report_error(SISU_ERR_CUDA, "memset");
  int rc = launch_digest_from_roots((const uint32_t*)sh->b.roots_recv, hc.C, sh->world, hc.W[hc.d], hc.W[0], sh->top,
                                    S->dig_in, S->dig_out, st);
  if (rc) return cuda_err(rc, "statement digests");
  InitParams ip;
  memset(&ip, 0, sizeof ip);
  memcpy(ip.domain, sh->tr.domain, sh->tr.len);
  ip.dlen = sh->tr.len;
  ip.d = hc.d;
  ip.c = sh->c_full;
  for (uint32_t i = 0; i <= hc.d; ++i) ip.s[i] = hc.s[i];
  memcpy(ip.wiring, hc.wiring_digest, 32);
  return cuda_err(launch_transcript_init(ip, S, st), "transcript init");
}

extern "C" int sisu_shard_layer_begin(sisu_shard* sh, uint32_t layer, void* stream) {
  if (!sh) return report_error(SISU_ERR_INVALID_ARG, "NULL shard");
  const HostCircuit& hc = sh->ev->circ->hc;
  if (layer >= hc.d) return report_error(SISU_ERR_INVALID_ARG, "layer beyond depth");
  return cuda_err(launch_layer_init(sh->w.S, layer, sh->c_loc, hc.s[layer], sh->ev->circ->L[layer], sh->w.E,
                                    sh->w.om, sh->w.eqh, stream, sh->cq, sh->rank),
                  "layer init");
}

static const uint32_t* round_table(const sisu_shard* sh, uint32_t layer, uint32_t k) {
  return k == 0 ? sh->ev->V[layer + 1] : sh->w.T;
}

extern "C" int sisu_shard_copy_round(sisu_shard* sh, uint32_t layer, uint32_t k, void* stream) {
  if (!sh) return report_error(SISU_ERR_INVALID_ARG, "NULL shard");
  const HostCircuit& hc = sh->ev->circ->hc;
  if (layer >= hc.d || k >= sh->c_loc) return report_error(SISU_ERR_INVALID_ARG, "layer or round out of range");
  Workspace& w = sh->w;
  const uint32_t h = hc.C >> (k + 1);
  return cuda_err(launch_copy_round(round_table(sh, layer, k), hc.s[layer + 1], h, w.E, w.om, sh->ev->circ->L[layer],
                                    w.partials, w.S, w.proof, sh->layer_off[layer] + 96 * (size_t)k, k, stream,
                                    (uint32_t*)sh->b.sums_send),
                  "copy round");
}

extern "C" int sisu_shard_absorb(sisu_shard* sh, uint32_t layer, uint32_t k, void* stream) {
  if (!sh) return report_error(SISU_ERR_INVALID_ARG, "NULL shard");
  const HostCircuit& hc = sh->ev->circ->hc;
  if (layer >= hc.d || k >= sh->c_loc) return report_error(SISU_ERR_INVALID_ARG, "layer or round out of range");
  Workspace& w = sh->w;
  int rc = launch_shard_absorb((const uint32_t*)sh->b.sums_recv, sh->world, w.S, w.proof,
                               sh->layer_off[layer] + 96 * (size_t)k, k, stream);
  if (rc) return cuda_err(rc, "round message");
  const uint32_t h = hc.C >> (k + 1);
  return cuda_err(launch_copy_fold(round_table(sh, layer, k), w.T, hc.s[layer + 1], h, w.E, w.S, k, stream),
                  "copy fold");
}

extern "C" int sisu_shard_row(sisu_shard* sh, uint32_t layer, void* stream) {
  if (!sh) return report_error(SISU_ERR_INVALID_ARG, "NULL shard");
  const HostCircuit& hc = sh->ev->circ->hc;
  if (layer >= hc.d) return report_error(SISU_ERR_INVALID_ARG, "layer beyond depth");
  const uint32_t* A = sh->c_loc == 0 ? sh->ev->V[layer + 1] : sh->w.T;
  return cuda_err(launch_shard_row(A, sh->w.E, hc.W[layer + 1], (uint32_t*)sh->b.row_send, stream), "row");
}

extern "C" int sisu_shard_finish(sisu_shard* sh, uint32_t layer, void* stream) {
  if (!sh) return report_error(SISU_ERR_INVALID_ARG, "NULL shard");
  if (sh->rank != 0) return report_error(SISU_ERR_INVALID_ARG, "only rank 0 finishes a layer");
  const HostCircuit& hc = sh->ev->circ->hc;
  if (layer >= hc.d) return report_error(SISU_ERR_INVALID_ARG, "layer beyond depth");
  cudaStream_t st = (cudaStream_t)stream;
  Workspace& w = sh->w;
  const DevLayer& L = sh->ev->circ->L[layer];
  const uint32_t sn = hc.s[layer + 1], Wn = hc.W[layer + 1];
  int rc = launch_shard_table((const uint32_t*)sh->b.row_recv, sh->world, Wn, max_next_width(hc) + 1, sh->T0, sh->E0,
                              st);
  if (rc) return cuda_err(rc, "gathered table");
  // the last log2(world) copy rounds, over the table of one row a rank
  for (uint32_t k = sh->c_loc; k < sh->c_full; ++k) {
    const uint32_t h = sh->world >> (k - sh->c_loc + 1);
    rc = launch_copy_round(sh->T0, sn, h, sh->E0, w.om, L, w.partials, w.S, w.proof,
                           sh->layer_off[layer] + 96 * (size_t)k, k, st);
    if (rc) return cuda_err(rc, "copy round");
    rc = launch_copy_fold(sh->T0, sh->T0, sn, h, sh->E0, w.S, k, st);
    if (rc) return cuda_err(rc, "copy fold");
  }
  return enqueue_layer_phases(hc, L, w, layer, sh->T0, sh->E0, w.om, hc.s[layer + 1],
                              sh->layer_off[layer] + 96 * (size_t)sh->c_full, false, st);
}

extern "C" int sisu_shard_proof(sisu_shard* sh, void* stream, uint8_t* proof, size_t cap, size_t* proof_len) {
  if (!sh || !proof) return report_error(SISU_ERR_INVALID_ARG, "NULL shard or proof buffer");
  const size_t n = sh->w.proof_len;
  if (proof_len) *proof_len = n;
  if (cap < n) return report_error(SISU_ERR_BUFFER, "proof buffer too small");
  cudaStream_t st = (cudaStream_t)stream;
  const size_t eoff = (n + 3) & ~(size_t)3;
  if (cudaMemcpyAsync(sh->host, sh->w.proof, n, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaMemcpyAsync(sh->host + eoff, &sh->w.S->error, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return report_error(SISU_ERR_CUDA, "proof copy");
  if (cudaError_t e = cudaStreamSynchronize(st)) return cuda_err((int)e, "shard proof");
  uint32_t err;
  memcpy(&err, sh->host + eoff, 4);
  if (err) return report_error(SISU_ERR_CUDA, "device-side check failed");
  memcpy(proof, sh->host, n);
  return SISU_OK;
}
