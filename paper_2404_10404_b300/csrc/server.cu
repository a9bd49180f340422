// Proof server: continuous batching of independent proof jobs on one GPU.
//
// Jobs (circuit + inputs) queue in arrival order.  A worker thread admits
// queued jobs as soon as a slot and enough device memory are free: the
// job's evaluation and prover workspace are laid out in one device arena
// (the memory budget, allocated once), and its evaluation and proof are
// enqueued on the slot's own stream.  Admitted jobs run concurrently, so
// their rounds interleave on the device.  A finished job (its event has
// completed) releases its slot and memory, which admits the next.
//
// Admission takes the oldest queued job that fits in the free memory, so a
// large job at the head does not hold back smaller ones behind it (jobs of
// one size keep their arrival order).  To keep the large job from starving,
// at most kMaxBypass admissions may pass the job at the head; after that
// nothing else is admitted until it fits, which it does at the latest when
// the running jobs have finished (its footprint is within the budget).
#include <cuda_runtime.h>

#include <chrono>
#include <climits>
#include <cstdint>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "handles.h"

using namespace sisu;

namespace {

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

// First-fit allocator over [0, size) in 256-byte units, coalescing on release.
struct Arena {
  std::map<size_t, size_t> free_;  // offset -> length
  explicit Arena(size_t size = 0) {
    if (size) free_[0] = size;
  }
  bool alloc(size_t n, size_t* off) {
    n = (n + 255) & ~(size_t)255;
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < n) continue;
      *off = it->first;
      const size_t rest = it->second - n, at = it->first + n;
      free_.erase(it);
      if (rest) free_[at] = rest;
      return true;
    }
    return false;
  }
  void release(size_t off, size_t n) {
    n = (n + 255) & ~(size_t)255;
    auto it = free_.emplace(off, n).first;
    auto next = std::next(it);
    if (next != free_.end() && it->first + it->second == next->first) {
      it->second += next->second;
      free_.erase(next);
    }
    if (it != free_.begin()) {
      auto prev = std::prev(it);
      if (prev->first + prev->second == it->first) {
        prev->second += it->second;
        free_.erase(it);
      }
    }
  }
};

constexpr size_t kSlotPinned = 1u << 20;  // proof bytes + error word per slot (proofs are below 600 KB)
constexpr uint32_t kMaxBypass = 16;       // admissions that may pass the job at the head of the queue

struct Job {
  uint64_t ticket = 0;
  const sisu_circuit* circ = nullptr;
  const uint8_t* inputs = nullptr;
  int on_device = 0;
  int status = 0;  // 0 queued, 1 running, 2 done, < 0 error code
  double t_submit = 0, t_start = 0, t_done = 0;
  size_t off = 0, bytes = 0, eval_bytes = 0;
  int slot = -1;
  uint64_t admit_order = 0;  // jobs admitted before this one
  std::unique_ptr<sisu_eval> ev;
  std::vector<uint8_t> proof;
};

}  // namespace

struct sisu_server {
  int device = 0;
  size_t budget = 0;
  uint32_t max_active = 0;
  uint8_t* arena_mem = nullptr;
  Arena arena;
  sisu_transcript domain{};
  // per slot: the job's stream and completion event, the stream and two
  // events of its inputs' digest (lent to the job's eval handle, so that no
  // job creates or destroys a stream), and pinned memory for the proof bytes,
  // then at +kSlotPinned-256 the evaluation flag
  std::vector<cudaStream_t> streams, dig_streams;
  std::vector<cudaEvent_t> done, in_ready, dig_done;
  std::vector<uint8_t*> pinned;
  std::vector<char> busy;
  uint64_t admitted = 0;          // jobs admitted so far
  uint64_t head = 0;              // ticket of the job at the head of the queue when last looked at
  uint32_t head_bypass = 0;       // admissions that passed it
  std::mutex mu;
  std::condition_variable cv;
  bool stop = false;
  bool paused = false;  // no admissions while set (running jobs continue)
  std::deque<Job*> queue;
  std::vector<Job*> active;
  std::map<uint64_t, std::unique_ptr<Job>> jobs;
  uint64_t next_ticket = 1;
  std::thread worker;

  size_t footprint(const sisu_circuit* cc, bool host_inputs, size_t* eval_bytes) const {
    *eval_bytes = (eval_footprint(cc, host_inputs) + 255) & ~(size_t)255;
    return *eval_bytes + workspace_footprint(cc);
  }

  // admit and start the oldest queued job that fits, if a slot is free
  bool admit_one() {
    Job* j = nullptr;
    {
      std::lock_guard<std::mutex> lock(mu);
      if (paused || queue.empty() || active.size() >= max_active) return false;
      int slot = -1;
      for (uint32_t k = 0; k < max_active; ++k)
        if (!busy[k]) {
          slot = (int)k;
          break;
        }
      if (slot < 0) return false;
      if (queue.front()->ticket != head) {
        head = queue.front()->ticket;
        head_bypass = 0;
      }
      size_t off = 0, failed = SIZE_MAX;  // smallest footprint that did not fit
      size_t at = queue.size();
      for (size_t k = 0; k < queue.size(); ++k) {
        if (k > 0 && head_bypass >= kMaxBypass) break;  // the head waits for memory, nobody passes it
        if (queue[k]->bytes >= failed) continue;
        if (arena.alloc(queue[k]->bytes, &off)) {
          at = k;
          break;
        }
        failed = queue[k]->bytes;
      }
      if (at == queue.size()) return false;
      Job* h = queue[at];
      queue.erase(queue.begin() + (long)at);
      if (at > 0) ++head_bypass;
      busy[slot] = 1;
      h->off = off;
      h->slot = slot;
      h->status = 1;
      h->t_start = now_s();
      h->admit_order = admitted++;
      active.push_back(h);
      j = h;
    }
    cudaStream_t st = streams[j->slot];
    uint8_t* base = arena_mem + j->off;
    uint32_t* host_flag = (uint32_t*)(pinned[j->slot] + kSlotPinned - 256);
    *host_flag = 0;
    j->ev.reset(new sisu_eval());
    j->ev->dig_stream = dig_streams[j->slot];
    j->ev->in_ready = in_ready[j->slot];
    j->ev->dig_ev = dig_done[j->slot];
    j->ev->owns_dig = false;
    eval_place(j->ev.get(), j->circ, base, !j->on_device, host_flag);
    int rc = workspace_place(j->ev.get(), base + j->eval_bytes, pinned[j->slot], st);
    if (!rc) rc = eval_enqueue(j->ev.get(), j->inputs, j->on_device, st);
    if (!rc) rc = proof_enqueue(j->circ, j->ev.get(), &domain, st);
    if (!rc && cudaEventRecord(done[j->slot], st) != cudaSuccess) rc = SISU_ERR_CUDA;
    if (rc) {
      cudaStreamSynchronize(st);
      finish(j, rc);
    }
    return true;
  }

  void finish(Job* j, int rc) {
    j->ev.reset();
    std::lock_guard<std::mutex> lock(mu);
    arena.release(j->off, j->bytes);
    busy[j->slot] = 0;
    j->status = rc ? rc : 2;
    j->t_done = now_s();
    for (size_t k = 0; k < active.size(); ++k)
      if (active[k] == j) {
        active.erase(active.begin() + (long)k);
        break;
      }
    cv.notify_all();
  }

  // complete every running job whose stream work is done
  bool reap() {
    std::vector<Job*> act;
    {
      std::lock_guard<std::mutex> lock(mu);
      act = active;
    }
    bool any = false;
    for (Job* j : act) {
      cudaError_t q = cudaEventQuery(done[j->slot]);
      if (q == cudaErrorNotReady) continue;
      int rc = SISU_OK;
      if (q != cudaSuccess) {
        rc = SISU_ERR_CUDA;
      } else if (*j->ev->host_flag & 1u) {
        rc = SISU_ERR_NOT_CANONICAL;
      } else {
        j->proof.resize(j->circ->hc.proof_len());
        rc = proof_finish(j->circ, j->ev.get(), j->proof.data());
      }
      finish(j, rc);
      any = true;
    }
    return any;
  }

  void run() {
    cudaSetDevice(device);
    for (;;) {
      bool progress = reap();
      while (admit_one()) progress = true;
      std::unique_lock<std::mutex> lock(mu);
      if (stop && active.empty()) break;
      if (!progress) cv.wait_for(lock, std::chrono::microseconds(50));
    }
  }

  // frees whatever exists, also after a failed create (the worker, when it
  // was started, has been joined by sisu_server_destroy)
  ~sisu_server() {
    for (size_t k = 0; k < streams.size(); ++k) {
      if (streams[k]) cudaStreamSynchronize(streams[k]);
      if (dig_streams[k]) cudaStreamSynchronize(dig_streams[k]);
    }
    for (size_t k = 0; k < streams.size(); ++k) {
      if (streams[k]) cudaStreamDestroy(streams[k]);
      if (dig_streams[k]) cudaStreamDestroy(dig_streams[k]);
      if (done[k]) cudaEventDestroy(done[k]);
      if (in_ready[k]) cudaEventDestroy(in_ready[k]);
      if (dig_done[k]) cudaEventDestroy(dig_done[k]);
      if (pinned[k]) cudaFreeHost(pinned[k]);
    }
    if (arena_mem) cudaFree(arena_mem);
  }
};

extern "C" int sisu_server_create(size_t budget_bytes, uint32_t max_active, const uint8_t* domain, size_t dlen,
                                  sisu_server** out) {
  if (!out) return report_error(SISU_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (budget_bytes < (1u << 20) || max_active == 0 || max_active > 256)
    return report_error(SISU_ERR_INVALID_ARG, "budget below 1 MiB or slots not in 1..256");
  if (dlen > kMaxDomain || (dlen && !domain)) return report_error(SISU_ERR_INVALID_ARG, "bad domain");
  std::unique_ptr<sisu_server> s(new (std::nothrow) sisu_server());
  if (!s) return report_error(SISU_ERR_OOM, "host allocation");
  if (cudaGetDevice(&s->device) != cudaSuccess) return report_error(SISU_ERR_CUDA, "no current CUDA device");
  s->budget = (budget_bytes + 255) & ~(size_t)255;
  s->max_active = max_active;
  if (dlen) {
    memcpy(s->domain.domain, domain, dlen);
    s->domain.len = (uint32_t)dlen;
  } else {
    const char* d = "SISU-GKR-v1";
    s->domain.len = (uint32_t)strlen(d);
    memcpy(s->domain.domain, d, s->domain.len);
  }
  if (cudaMalloc(&s->arena_mem, s->budget) != cudaSuccess)
    return report_error(SISU_ERR_OOM, "device allocation of the server's memory budget failed");
  s->arena = Arena(s->budget);
  s->streams.assign(max_active, nullptr);
  s->dig_streams.assign(max_active, nullptr);
  s->done.assign(max_active, nullptr);
  s->in_ready.assign(max_active, nullptr);
  s->dig_done.assign(max_active, nullptr);
  s->pinned.assign(max_active, nullptr);
  s->busy.assign(max_active, 0);
  for (uint32_t k = 0; k < max_active; ++k) {
    // on failure the unique_ptr's destructor frees what was made so far
    if (cudaStreamCreateWithFlags(&s->streams[k], cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&s->dig_streams[k], cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&s->done[k], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&s->in_ready[k], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&s->dig_done[k], cudaEventDisableTiming) != cudaSuccess ||
        cudaMallocHost(&s->pinned[k], kSlotPinned) != cudaSuccess)
      return report_error(SISU_ERR_CUDA, "server stream, event or pinned buffer");
  }
  sisu_server* raw = s.get();
  s->worker = std::thread([raw] { raw->run(); });
  *out = s.release();
  return SISU_OK;
}

extern "C" int sisu_job_footprint(const sisu_circuit* circ, int inputs_on_device, size_t* bytes) {
  if (!circ || !bytes) return report_error(SISU_ERR_INVALID_ARG, "NULL argument");
  if (!circ->dev) return report_error(SISU_ERR_INVALID_ARG, "circuit was created for host verification only");
  if (circ->hc.general) return report_error(SISU_ERR_INVALID_ARG, "the server does not take general circuits");
  *bytes = ((eval_footprint(circ, !inputs_on_device) + 255) & ~(size_t)255) + workspace_footprint(circ);
  return SISU_OK;
}

extern "C" int sisu_server_submit(sisu_server* s, const sisu_circuit* circ, const uint8_t* inputs,
                                  int inputs_on_device, uint64_t* ticket) {
  if (!s || !circ || !inputs || !ticket) return report_error(SISU_ERR_INVALID_ARG, "NULL argument");
  if (!circ->dev) return report_error(SISU_ERR_INVALID_ARG, "circuit was created for host verification only");
  if (circ->hc.general) return report_error(SISU_ERR_INVALID_ARG, "the server does not take general circuits");
  if (inputs_on_device)
    if (int rc = require_device(inputs, "inputs")) return rc;
  std::unique_ptr<Job> j(new (std::nothrow) Job());
  if (!j) return report_error(SISU_ERR_OOM, "host allocation");
  j->circ = circ;
  j->inputs = inputs;
  j->on_device = inputs_on_device;
  j->bytes = s->footprint(circ, !inputs_on_device, &j->eval_bytes);
  if (j->bytes > s->budget) return report_error(SISU_ERR_TOO_LARGE, "job footprint exceeds the server's memory budget");
  if (circ->hc.proof_len() + 512 > kSlotPinned) return report_error(SISU_ERR_TOO_LARGE, "proof larger than a slot");
  std::lock_guard<std::mutex> lock(s->mu);
  if (s->stop) return report_error(SISU_ERR_INVALID_ARG, "server is shutting down");
  j->ticket = s->next_ticket++;
  j->t_submit = now_s();
  *ticket = j->ticket;
  s->queue.push_back(j.get());
  s->jobs[j->ticket] = std::move(j);
  s->cv.notify_all();
  return SISU_OK;
}

extern "C" int sisu_server_poll(sisu_server* s, uint64_t ticket, int* status, uint8_t* proof, size_t cap,
                                size_t* len, double* latency_ms, uint64_t* admit_order) {
  if (!s || !status) return report_error(SISU_ERR_INVALID_ARG, "NULL argument");
  std::lock_guard<std::mutex> lock(s->mu);
  auto it = s->jobs.find(ticket);
  if (it == s->jobs.end()) return report_error(SISU_ERR_INVALID_ARG, "unknown ticket");
  Job* j = it->second.get();
  *status = j->status;
  if (j->status == 0 || j->status == 1) return SISU_OK;
  if (latency_ms) *latency_ms = 1e3 * (j->t_done - j->t_submit);
  if (admit_order) *admit_order = j->status == 2 || j->t_start > 0 ? j->admit_order : UINT64_MAX;
  if (j->status == 2) {
    if (len) *len = j->proof.size();
    if (!proof || cap < j->proof.size()) return report_error(SISU_ERR_BUFFER, "proof buffer too small");
    memcpy(proof, j->proof.data(), j->proof.size());
  }
  s->jobs.erase(it);
  return SISU_OK;
}

extern "C" int sisu_server_pause(sisu_server* s, int paused) {
  if (!s) return report_error(SISU_ERR_INVALID_ARG, "NULL server");
  std::lock_guard<std::mutex> lock(s->mu);
  s->paused = paused != 0;
  s->cv.notify_all();
  return SISU_OK;
}

extern "C" int sisu_server_pending(sisu_server* s, uint32_t* queued, uint32_t* running) {
  if (!s) return report_error(SISU_ERR_INVALID_ARG, "NULL server");
  std::lock_guard<std::mutex> lock(s->mu);
  if (queued) *queued = (uint32_t)s->queue.size();
  if (running) *running = (uint32_t)s->active.size();
  return SISU_OK;
}

extern "C" void sisu_server_destroy(sisu_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    s->stop = true;
    for (Job* j : s->queue) {
      j->status = SISU_ERR_INVALID_ARG;
      j->t_done = now_s();
    }
    s->queue.clear();
    s->cv.notify_all();
  }
  if (s->worker.joinable()) s->worker.join();
  delete s;
}
