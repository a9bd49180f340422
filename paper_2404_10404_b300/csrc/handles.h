// Handle types of the C ABI and the internal entry points that the prover,
// the batch call and the server share.
#pragma once
#include <cuda_runtime.h>

#include <memory>
#include <vector>

#include "../../include/sisu.h"
#include "internal.h"

using sisu::DevLayer;
using sisu::DevState;
using sisu::HostCircuit;
using sisu::kMaxDomain;

struct sisu_circuit {
  HostCircuit hc;
  std::vector<DevLayer> L;  // device views, gate layers 0..d-1 (general: over the virtual layers)
  void* dev = nullptr;      // one allocation holding every device array
  int device = 0;
  // general circuits: per layer the gather map of X_i past layer i + 1
  // ({layer, gate} per position), the blocks' {base, count}, and per block
  // the X position of each gate of the block's layer (~0: not used)
  std::vector<const uint2*> gmap, blk;
  std::vector<std::vector<const uint32_t*>> pmap;
  ~sisu_circuit() {
    if (dev) cudaFree(dev);
  }
};

struct Workspace {
  void* dev = nullptr;  // owned allocation (null when placed in caller memory)
  uint32_t *T = nullptr, *E = nullptr, *om = nullptr, *At = nullptr, *H1 = nullptr, *H2 = nullptr,
           *Ay = nullptr, *Q = nullptr, *partials = nullptr, *dscratch = nullptr, *eqh = nullptr, *P = nullptr;
  uint32_t* omo = nullptr;  // the gate weights in gate order (first copy rounds), after om
  // the copy phase by its linear recurrence: the rows' gate sums of two
  // rounds (C values each), the pairs' t^2 coefficients of two rounds (C/2
  // each), after E in its region, and the shares of a pair's coefficient
  // (rounds with few pairs), in the upper half of the partial sums
  uint32_t *Ub[2] = {nullptr, nullptr}, *cb[2] = {nullptr, nullptr}, *cpart = nullptr;
  // general circuits: the claim terms' copy and gate weights, their round
  // sums, the combined weights, every layer's challenges and alphas
  // (hstride values a layer), the block values, the term descriptors
  uint32_t *Et = nullptr, *omt = nullptr, *sums = nullptr, *omc = nullptr, *Ec = nullptr, *hist = nullptr,
           *vals = nullptr;
  void* gterms = nullptr;
  uint32_t hstride = 0;
  std::vector<uint32_t> term_off;  // first descriptor of each layer's terms (d + 1 entries)
  DevState* S = nullptr;
  uint8_t* proof = nullptr;
  uint8_t* host = nullptr;  // pinned: proof bytes followed by the error word
  bool owns_host = true;    // false when the pinned bytes belong to the caller
  size_t proof_len = 0;
  // the proof's launch sequence captured as a CUDA graph (same circuit,
  // workspace and transcript domain give the same launches every time)
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t exec = nullptr;
  uint8_t gdomain[kMaxDomain];
  uint32_t gdlen = 0;
  bool gvalid = false;
  uint64_t graph_kernels = 0;  // kernel nodes in the captured graph
  int proofs = 0;              // proofs enqueued so far on this workspace
  ~Workspace() {
    if (exec) cudaGraphExecDestroy(exec);
    if (cap_stream) cudaStreamDestroy(cap_stream);
    if (dev) cudaFree(dev);
    if (host && owns_host) cudaFreeHost(host);
  }
};

struct sisu_eval {
  const sisu_circuit* circ = nullptr;
  std::vector<uint32_t*> V;  // layers 0..d, Montgomery, padded
  std::vector<uint32_t*> X;  // general circuits: the virtual layer of each gate layer (V[i + 1] when it is only that)
  void* dev = nullptr;        // owned allocation (null when placed in caller memory)
  uint32_t* stage = nullptr;  // padded-input staging (only when padding is needed)
  uint32_t* flag = nullptr;   // device error word
  uint32_t* host_flag = nullptr;
  std::unique_ptr<Workspace> ws;
  bool placed = false;         // layers, flag and staging live in caller memory
  // chunked transfer of host inputs (created on first use): the copy stream
  // and one event per chunk, plus one for the start
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t chunk_ev[sisu::kEvalChunks + 1] = {};
  // the inputs' statement digest, formed on its own stream while the layers
  // evaluate: dig (device, 24 words: the digest, then two unused second
  // outputs of the two-table digest launches), its scratch, the stream and
  // two events (inputs converted; digest done, which a proof waits for)
  uint32_t* dig = nullptr;
  uint32_t* dscratch = nullptr;
  cudaStream_t dig_stream = nullptr;
  cudaEvent_t in_ready = nullptr, dig_ev = nullptr;
  bool dig_recorded = false;
  bool owns_dig = true;  // false when the digest stream and events belong to a server slot
  ~sisu_eval() {
    if (copy_stream) cudaStreamSynchronize(copy_stream);
    if (dig_stream) cudaStreamSynchronize(dig_stream);
    for (cudaEvent_t e : chunk_ev)
      if (e) cudaEventDestroy(e);
    if (owns_dig) {
      if (in_ready) cudaEventDestroy(in_ready);
      if (dig_ev) cudaEventDestroy(dig_ev);
      if (dig_stream) cudaStreamDestroy(dig_stream);
    }
    if (copy_stream) cudaStreamDestroy(copy_stream);
    ws.reset();
    if (stage && !placed) cudaFree(stage);
    if (dev) cudaFree(dev);
    if (host_flag && !placed) cudaFreeHost(host_flag);
  }
};

struct sisu_transcript {
  uint8_t domain[kMaxDomain];
  uint32_t len;
};


namespace sisu {
// device bytes of one evaluation (layers, flag, staging for padded host
// inputs) and of one prover workspace
size_t eval_footprint(const sisu_circuit* cc, bool host_inputs);
size_t workspace_footprint(const sisu_circuit* cc);
// lay out an evaluation / a workspace in caller memory (256-byte aligned)
void eval_place(sisu_eval* ev, const sisu_circuit* cc, uint8_t* dev, bool host_inputs, uint32_t* host_flag);
int workspace_place(sisu_eval* ev, uint8_t* dev, uint8_t* host_pinned, cudaStream_t st);
// enqueue the evaluation (no wait; the canonicity flag is checked later)
int eval_enqueue(sisu_eval* ev, const uint8_t* inputs, int on_device, cudaStream_t st);
// enqueue one proof plus the copies of its bytes and error word to host
int proof_enqueue(const sisu_circuit* cc, sisu_eval* ev, const sisu_transcript* tr, cudaStream_t st);
// after the stream work: check the error word, copy the proof out
int proof_finish(const sisu_circuit* cc, sisu_eval* ev, uint8_t* proof);
int report_error(int code, const char* msg);
// Libra's phases and the end of gate layer i from the copy-bound row A (of
// 2^s values), gate weights om and the copy weight E[0], messages from
// proof offset offx (enqueued on st); no_end leaves the layer's end out
int enqueue_layer_phases(const HostCircuit& hc, const DevLayer& L, Workspace& w, uint32_t i, const uint32_t* A,
                         const uint32_t* E, const uint32_t* om, uint32_t s, size_t offx, bool no_end, cudaStream_t st);
// the workspace's regions (kWsRegions of them) in `dev`, the proof header
// (copy count 2^c_proof) and a zeroed state, set on st
int workspace_layout(const sisu_circuit* cc, Workspace* ws, uint8_t* dev, uint8_t* host, uint32_t c_proof,
                     cudaStream_t st);
size_t workspace_footprint_c(const sisu_circuit* cc, uint32_t c_proof);
}  // namespace sisu
