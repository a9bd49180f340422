// C ABI of the data-parallel GKR prover: handles, evaluation and the
// prover's launch sequence.  Everything in a proof runs on the device,
// stream-ordered, with challenges in device memory; the host waits once,
// for the proof bytes.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <mutex>
#include <new>

#include "handles.h"

using namespace sisu;

namespace sisu {
static std::atomic<uint64_t> g_launches{0};
uint64_t launches_add(uint64_t n) { return g_launches.fetch_add(n) + n; }
}  // namespace sisu

// ---------------------------------------------------------------------------
// errors

static thread_local char g_err[512] = "";

static int fail(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof g_err, fmt, ap);
  va_end(ap);
  return code;
}

namespace sisu {
int report_error(int code, const char* msg) { return fail(code, "%s", msg); }
}  // namespace sisu

static int cuda_fail(cudaError_t e, const char* what) {
  return fail(SISU_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

namespace sisu {
int require_device(const void* p, const char* what) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();  // not a sticky error: clear it
    return fail(SISU_ERR_INVALID_ARG, "%s: not an address the CUDA runtime knows", what);
  }
  if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)
    return fail(SISU_ERR_INVALID_ARG, "%s is not device memory", what);
  return SISU_OK;
}
}  // namespace sisu

#define CK(call, what)                                   \
  do {                                                   \
    cudaError_t e_ = (cudaError_t)(call);                \
    if (e_ != cudaSuccess) return cuda_fail(e_, what);   \
  } while (0)

static uint32_t ceil_log2(uint64_t v) {
  uint32_t s = 0;
  while ((1ull << s) < v) ++s;
  return s;
}

namespace sisu {
size_t HostCircuit::proof_len() const {
  size_t n = 8 + 4 * ((size_t)d + 3);
  for (uint32_t i = 0; i < d; ++i)
    n += general ? 32 * (3 * (size_t)c + 4 * (size_t)sx[i] + 2 * blocks[i].size())
                 : 32 * (3 * (size_t)c + 4 * (size_t)s[i + 1] + 2);
  return n;
}
}  // namespace sisu

// ---------------------------------------------------------------------------
// per-kernel timing with CUDA events (diagnostics; off unless enabled)

namespace {
struct ProfRec {
  cudaEvent_t a, b;
  double work;
  uint32_t kind;
};
uint32_t g_prof_mask = 0;
std::vector<ProfRec> g_prof;
std::vector<cudaEvent_t> g_event_pool;

cudaEvent_t pool_event() {
  if (!g_event_pool.empty()) {
    cudaEvent_t e = g_event_pool.back();
    g_event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Times one launch when its kind is enabled.
struct ProfScope {
  long idx = -1;
  cudaStream_t st;
  ProfScope(uint32_t kind, double work, cudaStream_t s) : st(s) { idx = sisu::prof_begin(kind, work, s); }
  ~ProfScope() { sisu::prof_end(idx, st); }
};
}  // namespace

long sisu::prof_begin(uint32_t kind, double work, void* stream) {
  if (!(g_prof_mask & (1u << kind))) return -1;
  ProfRec r{pool_event(), pool_event(), work, kind};
  cudaEventRecord(r.a, (cudaStream_t)stream);
  g_prof.push_back(r);
  return (long)g_prof.size() - 1;
}

void sisu::prof_end(long idx, void* stream) {
  if (idx >= 0) cudaEventRecord(g_prof[idx].b, (cudaStream_t)stream);
}

enum : uint32_t {
  kProfCopyRound = 0, kProfCopyFold = 1, kProfEval = 2, kProfGateRound = 3, kProfDigest = 4,
  kProfLayerInit = 5, kProfPhaseInit = 6, kProfTranscript = 7, kProfInputs = 8, kProfRowSums = 11
};

extern "C" int sisu_profile_enable(uint32_t kind_mask) {
  g_prof_mask = kind_mask;
  return SISU_OK;
}

extern "C" int sisu_profile_launches(uint32_t kind, double* ms, double* fr_mults, size_t cap, size_t* n) {
  size_t k = 0;
  for (ProfRec& r : g_prof) {
    if (r.kind != kind) continue;
    cudaError_t e = cudaEventSynchronize(r.b);
    if (e != cudaSuccess) return cuda_fail(e, "profile events");
    if (k < cap) {
      float x = 0;
      cudaEventElapsedTime(&x, r.a, r.b);
      if (ms) ms[k] = x;
      if (fr_mults) fr_mults[k] = r.work;
    }
    ++k;
  }
  if (n) *n = k;
  return SISU_OK;
}

extern "C" int sisu_profile_read(uint32_t kind, double* ms, uint64_t* launches, double* fr_mults) {
  double t = 0, w = 0;
  uint64_t n = 0;
  std::vector<ProfRec> keep;
  for (ProfRec& r : g_prof) {
    if (r.kind != kind) {
      keep.push_back(r);
      continue;
    }
    cudaError_t e = cudaEventSynchronize(r.b);
    if (e != cudaSuccess) return cuda_fail(e, "profile events");
    float x = 0;
    cudaEventElapsedTime(&x, r.a, r.b);
    t += x;
    w += r.work;
    ++n;
    g_event_pool.push_back(r.a);
    g_event_pool.push_back(r.b);
  }
  g_prof.swap(keep);
  if (ms) *ms = t;
  if (launches) *launches = n;
  if (fr_mults) *fr_mults = w;
  return SISU_OK;
}

// ---------------------------------------------------------------------------
// handles

static const char kDefaultDomain[] = "SISU-GKR-v1";

// ---------------------------------------------------------------------------
// circuit creation

// Wiring bytes: for each gate layer i and padded gate g in turn,
//   one entry:   u8 type || u32le in1 || u32le in2
//   no entry:    u8 2 || u32le 0 || u32le 0          (a padding gate)
//   k >= 2:      u8 3 || u32le k, then k times u8 type || u32le in1 || u32le in2
// (a plain circuit, one entry a gate, keeps the one-record-a-gate bytes)
static void wiring_digest(const HostCircuit& hc, uint32_t out[8]) {
  size_t n = 0;
  for (uint32_t i = 0; i < hc.d; ++i) n += ((size_t)hc.W[i] + hc.out[i].size()) * 13;
  std::vector<uint8_t> buf(n);
  uint8_t* p = buf.data();
  auto put = [&](uint32_t v) {
    p[0] = (uint8_t)v; p[1] = (uint8_t)(v >> 8); p[2] = (uint8_t)(v >> 16); p[3] = (uint8_t)(v >> 24);
    p += 4;
  };
  for (uint32_t i = 0; i < hc.d; ++i) {
    size_t e = 0;
    const size_t ne = hc.out[i].size();
    for (uint32_t g = 0; g < hc.W[i]; ++g) {
      size_t e1 = e;
      while (e1 < ne && hc.out[i][e1] == g) ++e1;
      if (e1 - e == 0) {
        *p++ = 2; put(0); put(0);
      } else if (e1 - e == 1) {
        // a general circuit's gate reading a deeper layer (Sec. 2.7):
        // u8 4 + type || u32le in1 || u32le in2 || u32le layer
        const bool far = hc.general && hc.src[i][e] != i + 1;
        *p++ = (uint8_t)(far ? 4 + hc.type[i][e] : hc.type[i][e]); put(hc.in1[i][e]); put(hc.in2[i][e]);
        if (far) put(hc.src[i][e]);
      } else {
        *p++ = 3; put((uint32_t)(e1 - e));
        for (size_t q = e; q < e1; ++q) {
          *p++ = hc.type[i][q]; put(hc.in1[i][q]); put(hc.in2[i][q]);
        }
      }
      e = e1;
    }
  }
  host_statement_digest(buf.data(), (size_t)(p - buf.data()), out);
}

// the padded shape of a circuit from its d + 1 widths (layer d = inputs)
static int circuit_shape(const uint32_t* widths, uint32_t d, uint32_t n_copies, HostCircuit& hc) {
  if (d == 0) return fail(SISU_ERR_INVALID_ARG, "need at least one gate layer");
  if (d > SISU_MAX_LAYERS) return fail(SISU_ERR_TOO_LARGE, "more than %u layers", SISU_MAX_LAYERS);
  if (n_copies == 0) return fail(SISU_ERR_INVALID_ARG, "zero copies");
  if (n_copies > SISU_MAX_COPIES) return fail(SISU_ERR_TOO_LARGE, "more than 2^24 copies");
  hc.d = d;
  hc.Creal = n_copies;
  hc.c = ceil_log2(n_copies);
  hc.C = 1u << hc.c;
  hc.s.resize(d + 1);
  hc.W.resize(d + 1);
  hc.wreal.resize(d + 1);
  for (uint32_t i = 0; i <= d; ++i) {
    const uint32_t w = widths[i];
    if (w == 0) return fail(SISU_ERR_INVALID_ARG, "layer %u has zero width", i);
    if (w > SISU_MAX_WIDTH) return fail(SISU_ERR_TOO_LARGE, "layer %u wider than 2^24", i);
    hc.wreal[i] = w;
    hc.s[i] = ceil_log2(w);
    hc.W[i] = 1u << hc.s[i];
    if (hc.c + hc.s[i] > 32) return fail(SISU_ERR_TOO_LARGE, "copies x width of layer %u above 2^32", i);
  }
  hc.out.assign(d, {});
  hc.type.assign(d, {});
  hc.in1.assign(d, {});
  hc.in2.assign(d, {});
  return SISU_OK;
}

// one entry of layer i, validated; entries must arrive in order of gate
static int add_entry(HostCircuit& hc, uint32_t i, uint32_t g, uint8_t t, uint32_t a, uint32_t b) {
  if (t > 1) return fail(SISU_ERR_INVALID_ARG, "layer %u gate %u: type %u", i, g, t);
  if (a >= hc.wreal[i + 1] || b >= hc.wreal[i + 1])
    return fail(SISU_ERR_INDEX_OOB, "layer %u gate %u: input index beyond width %u", i, g, hc.wreal[i + 1]);
  hc.out[i].push_back(g);
  hc.type[i].push_back(t);
  hc.in1[i].push_back(a);
  hc.in2[i].push_back(b);
  return SISU_OK;
}

// Digest, then (on_device) the device arrays of every layer: the entries
// grouped by type (mul first), each group sorted by in1, followed by the
// gates with no entry; the CSR of the entries by in1 and by in2; and for
// layers where some gate has several entries, the entries by gate.
static int circuit_finish(std::unique_ptr<sisu_circuit>& cc, bool on_device, sisu_circuit** out) {
  HostCircuit& hc = cc->hc;
  const uint32_t d = hc.d;
  for (uint32_t i = 0; i < d; ++i)
    if ((uint64_t)hc.C * hc.out[i].size() > (1ull << 32) || hc.out[i].size() > (1ull << 28))
      return fail(SISU_ERR_TOO_LARGE, "layer %u: copies x entries above 2^32", i);
  wiring_digest(hc, hc.wiring_digest);
  if (!on_device) {
    *out = cc.release();
    return SISU_OK;
  }
  struct Lay {
    std::vector<uint4> sg;
    std::vector<uint32_t> off1, pos1, off2, pos2, offo;
    std::vector<uint2> eo;
    uint32_t nmul, ntot;
  };
  std::vector<Lay> H(d);
  size_t bytes = 0;
  auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
  for (uint32_t i = 0; i < d; ++i) {
    Lay& l = H[i];
    // a general layer's wiring reads its virtual layer: second inputs at their X positions
    const uint32_t W = hc.W[i], Wn = hc.general ? (1u << hc.sx[i]) : hc.W[i + 1];
    const std::vector<uint32_t>& IN2 = hc.general ? hc.u2[i] : hc.in2[i];
    const uint32_t ne = (uint32_t)hc.out[i].size();
    std::vector<uint32_t> muls, adds, count(W, 0);
    for (uint32_t e = 0; e < ne; ++e) {
      (hc.type[i][e] == 1 ? muls : adds).push_back(e);
      ++count[hc.out[i][e]];
    }
    // each type group sorted by in1 (then entry) for locality of the row gathers
    auto by_in1 = [&](uint32_t a, uint32_t b) {
      return hc.in1[i][a] != hc.in1[i][b] ? hc.in1[i][a] < hc.in1[i][b] : a < b;
    };
    std::sort(muls.begin(), muls.end(), by_in1);
    std::sort(adds.begin(), adds.end(), by_in1);
    l.nmul = (uint32_t)muls.size();
    l.ntot = ne;
    bool acc = false;
    uint32_t empty = 0;
    for (uint32_t g = 0; g < W; ++g) {
      acc |= count[g] > 1;
      empty += count[g] == 0;
    }
    l.sg.resize((size_t)ne + empty);
    for (uint32_t q = 0; q < ne; ++q) {
      const uint32_t e = q < l.nmul ? muls[q] : adds[q - l.nmul];
      l.sg[q] = make_uint4(hc.in1[i][e], IN2[e], hc.out[i][e], 0);
    }
    for (uint32_t g = 0, q = ne; g < W; ++g)
      if (count[g] == 0) l.sg[q++] = make_uint4(0, 0, g, 0);
    auto csr = [&](int which, std::vector<uint32_t>& off, std::vector<uint32_t>& pos) {
      off.assign(Wn + 1, 0);
      pos.resize(l.ntot);
      for (uint32_t q = 0; q < l.ntot; ++q) ++off[(which ? l.sg[q].y : l.sg[q].x) + 1];
      for (uint32_t x = 0; x < Wn; ++x) off[x + 1] += off[x];
      std::vector<uint32_t> fill(off.begin(), off.end() - 1);
      for (uint32_t q = 0; q < l.ntot; ++q) pos[fill[which ? l.sg[q].y : l.sg[q].x]++] = q;
    };
    csr(0, l.off1, l.pos1);
    csr(1, l.off2, l.pos2);
    if (acc) {  // entries by gate (hc's order is by gate already)
      l.offo.assign(W + 1, 0);
      for (uint32_t g = 0; g < W; ++g) l.offo[g + 1] = l.offo[g] + count[g];
      l.eo.resize(ne);
      for (uint32_t e = 0; e < ne; ++e) l.eo[e] = make_uint2(hc.in1[i][e] | ((uint32_t)hc.type[i][e] << 30), IN2[e]);
    }
    bytes += al(l.sg.size() * 16 + 16) + 2 * al(l.off1.size() * 4) + 2 * al(l.pos1.size() * 4 + 4) +
             al(l.offo.size() * 4) + al(l.eo.size() * 8);
  }
  // general circuits: per layer the gather map of X_i past layer i + 1, the
  // blocks' (base, count), and per block the X position of each gate of its
  // layer (~0 when not used)
  std::vector<std::vector<uint2>> gmap(d), blk(d);
  std::vector<std::vector<std::vector<uint32_t>>> pmap(d);
  if (hc.general) {
    for (uint32_t i = 0; i < d; ++i) {
      for (size_t b = 0; b < hc.blocks[i].size(); ++b) {
        const HostCircuit::Block& B = hc.blocks[i][b];
        blk[i].push_back(make_uint2(B.base, B.count));
        std::vector<uint32_t> pm(hc.W[B.layer], 0xffffffffu);
        for (uint32_t k = 0; k < B.count; ++k) pm[b == 0 ? k : B.ys[k]] = B.base + k;
        if (b > 0)
          for (uint32_t k = 0; k < B.count; ++k) gmap[i].push_back(make_uint2(B.layer, B.ys[k]));
        pmap[i].push_back(std::move(pm));
      }
      bytes += al(gmap[i].size() * 8 + 8) + al(blk[i].size() * 8);
      for (auto& pm : pmap[i]) bytes += al(pm.size() * 4);
    }
  }
  CK(cudaGetDevice(&cc->device), "cudaGetDevice");
  cudaError_t e = cudaMalloc(&cc->dev, bytes);
  if (e != cudaSuccess) return fail(SISU_ERR_OOM, "device allocation of %zu bytes for the wiring", bytes);
  uint8_t* p = (uint8_t*)cc->dev;
  cc->L.resize(d);
  auto up = [&](const void* src, size_t n, size_t reserve) -> void* {
    void* dst = p;
    if (n) {
      cudaError_t e2 = cudaMemcpy(dst, src, n, cudaMemcpyHostToDevice);
      if (e2 != cudaSuccess) return nullptr;
    }
    p += al(reserve);
    return dst;
  };
  for (uint32_t i = 0; i < d; ++i) {
    Lay& l = H[i];
    DevLayer& D = cc->L[i];
    D.sgate = (const uint4*)up(l.sg.data(), l.sg.size() * 16, l.sg.size() * 16 + 16);
    D.off1 = (const uint32_t*)up(l.off1.data(), l.off1.size() * 4, l.off1.size() * 4);
    D.pos1 = (const uint32_t*)up(l.pos1.data(), l.pos1.size() * 4, l.pos1.size() * 4 + 4);
    D.off2 = (const uint32_t*)up(l.off2.data(), l.off2.size() * 4, l.off2.size() * 4);
    D.pos2 = (const uint32_t*)up(l.pos2.data(), l.pos2.size() * 4, l.pos2.size() * 4 + 4);
    D.offo = l.offo.empty() ? nullptr : (const uint32_t*)up(l.offo.data(), l.offo.size() * 4, l.offo.size() * 4);
    D.eo = l.eo.empty() ? nullptr : (const uint2*)up(l.eo.data(), l.eo.size() * 8, l.eo.size() * 8);
    if (!D.sgate || !D.off1 || !D.pos1 || !D.off2 || !D.pos2 || (!l.offo.empty() && (!D.offo || !D.eo)))
      return fail(SISU_ERR_CUDA, "upload of the wiring failed");
    D.nmul = l.nmul;
    D.ntot = l.ntot;
    D.nsg = (uint32_t)l.sg.size();
  }
  if (hc.general) {
    cc->gmap.resize(d);
    cc->blk.resize(d);
    cc->pmap.resize(d);
    for (uint32_t i = 0; i < d; ++i) {
      cc->gmap[i] = (const uint2*)up(gmap[i].data(), gmap[i].size() * 8, gmap[i].size() * 8 + 8);
      cc->blk[i] = (const uint2*)up(blk[i].data(), blk[i].size() * 8, blk[i].size() * 8);
      for (auto& pm : pmap[i]) cc->pmap[i].push_back((const uint32_t*)up(pm.data(), pm.size() * 4, pm.size() * 4));
      if (!cc->gmap[i] || !cc->blk[i]) return fail(SISU_ERR_CUDA, "upload of the general wiring failed");
      for (auto* q : cc->pmap[i])
        if (!q) return fail(SISU_ERR_CUDA, "upload of the general wiring failed");
    }
  }
  *out = cc.release();
  return SISU_OK;
}

static int circuit_create(const sisu_layer* layers, uint32_t n_gate_layers, uint32_t input_width,
                          uint32_t n_copies, bool on_device, sisu_circuit** out) {
  if (!out) return fail(SISU_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!layers || n_gate_layers == 0) return fail(SISU_ERR_INVALID_ARG, "need at least one gate layer");
  if (n_gate_layers > SISU_MAX_LAYERS) return fail(SISU_ERR_TOO_LARGE, "more than %u layers", SISU_MAX_LAYERS);
  std::unique_ptr<sisu_circuit> cc(new (std::nothrow) sisu_circuit());
  if (!cc) return fail(SISU_ERR_OOM, "host allocation");
  std::vector<uint32_t> widths(n_gate_layers + 1);
  for (uint32_t i = 0; i < n_gate_layers; ++i) widths[i] = layers[i].width;
  widths[n_gate_layers] = input_width;
  if (int rc = circuit_shape(widths.data(), n_gate_layers, n_copies, cc->hc)) return rc;
  for (uint32_t i = 0; i < n_gate_layers; ++i) {
    const sisu_layer& ly = layers[i];
    if (!ly.type || !ly.in1 || !ly.in2) return fail(SISU_ERR_INVALID_ARG, "layer %u: NULL wiring array", i);
    for (uint32_t g = 0; g < ly.width; ++g)
      if (int rc = add_entry(cc->hc, i, g, ly.type[g], ly.in1[g], ly.in2[g])) return rc;
  }
  return circuit_finish(cc, on_device, out);
}

static int circuit_create_acc(const sisu_acc_layer* layers, uint32_t n_gate_layers, uint32_t input_width,
                              uint32_t n_copies, bool on_device, sisu_circuit** out) {
  if (!out) return fail(SISU_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!layers || n_gate_layers == 0) return fail(SISU_ERR_INVALID_ARG, "need at least one gate layer");
  if (n_gate_layers > SISU_MAX_LAYERS) return fail(SISU_ERR_TOO_LARGE, "more than %u layers", SISU_MAX_LAYERS);
  std::unique_ptr<sisu_circuit> cc(new (std::nothrow) sisu_circuit());
  if (!cc) return fail(SISU_ERR_OOM, "host allocation");
  std::vector<uint32_t> widths(n_gate_layers + 1);
  for (uint32_t i = 0; i < n_gate_layers; ++i) widths[i] = layers[i].width;
  widths[n_gate_layers] = input_width;
  if (int rc = circuit_shape(widths.data(), n_gate_layers, n_copies, cc->hc)) return rc;
  for (uint32_t i = 0; i < n_gate_layers; ++i) {
    const sisu_acc_layer& ly = layers[i];
    if (ly.n_entries && (!ly.out || !ly.type || !ly.in1 || !ly.in2))
      return fail(SISU_ERR_INVALID_ARG, "layer %u: NULL entry array", i);
    if (ly.n_entries > (1u << 28)) return fail(SISU_ERR_TOO_LARGE, "layer %u: more than 2^28 entries", i);
    // stable counting sort of the entries by gate
    std::vector<uint32_t> start(ly.width + 1, 0);
    for (uint32_t e = 0; e < ly.n_entries; ++e) {
      if (ly.out[e] >= ly.width) return fail(SISU_ERR_INDEX_OOB, "layer %u entry %u: gate beyond width", i, e);
      ++start[ly.out[e] + 1];
    }
    for (uint32_t g = 0; g < ly.width; ++g) start[g + 1] += start[g];
    std::vector<uint32_t> order(ly.n_entries);
    for (uint32_t e = 0; e < ly.n_entries; ++e) order[start[ly.out[e]]++] = e;
    for (uint32_t e : order)
      if (int rc = add_entry(cc->hc, i, ly.out[e], ly.type[e], ly.in1[e], ly.in2[e])) return rc;
  }
  return circuit_finish(cc, on_device, out);
}

// General circuits (Sec. 2.7): one entry per gate, its second input from
// layer src (i + 1 .. d); the virtual layers X_i and their blocks.
static int circuit_create_general(const sisu_general_layer* layers, uint32_t n_gate_layers, uint32_t input_width,
                                  uint32_t n_copies, bool on_device, sisu_circuit** out) {
  if (!out) return fail(SISU_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!layers || n_gate_layers == 0) return fail(SISU_ERR_INVALID_ARG, "need at least one gate layer");
  if (n_gate_layers > SISU_MAX_LAYERS) return fail(SISU_ERR_TOO_LARGE, "more than %u layers", SISU_MAX_LAYERS);
  std::unique_ptr<sisu_circuit> cc(new (std::nothrow) sisu_circuit());
  if (!cc) return fail(SISU_ERR_OOM, "host allocation");
  std::vector<uint32_t> widths(n_gate_layers + 1);
  for (uint32_t i = 0; i < n_gate_layers; ++i) widths[i] = layers[i].width;
  widths[n_gate_layers] = input_width;
  HostCircuit& hc = cc->hc;
  if (int rc = circuit_shape(widths.data(), n_gate_layers, n_copies, hc)) return rc;
  const uint32_t d = n_gate_layers;
  hc.general = true;
  hc.src.assign(d, {});
  hc.u2.assign(d, {});
  hc.sx.assign(d, 0);
  hc.blocks.assign(d, {});
  for (uint32_t i = 0; i < d; ++i) {
    const sisu_general_layer& ly = layers[i];
    if (!ly.type || !ly.in1 || !ly.src || !ly.in2) return fail(SISU_ERR_INVALID_ARG, "layer %u: NULL wiring array", i);
    for (uint32_t g = 0; g < ly.width; ++g) {
      const uint32_t j = ly.src[g];
      if (j <= i || j > d) return fail(SISU_ERR_INDEX_OOB, "layer %u gate %u: second input's layer %u", i, g, j);
      if (ly.type[g] > 1) return fail(SISU_ERR_INVALID_ARG, "layer %u gate %u: type %u", i, g, ly.type[g]);
      if (ly.in1[g] >= hc.wreal[i + 1] || ly.in2[g] >= hc.wreal[j])
        return fail(SISU_ERR_INDEX_OOB, "layer %u gate %u: input index beyond its layer's width", i, g);
      hc.out[i].push_back(g);
      hc.type[i].push_back(ly.type[g]);
      hc.in1[i].push_back(ly.in1[g]);
      hc.in2[i].push_back(ly.in2[g]);
      hc.src[i].push_back(j);
    }
    // X_i: layer i + 1 in full, then the used gates of each deeper layer, ascending
    HostCircuit::Block b0{i + 1, 0, hc.W[i + 1], {}};
    hc.blocks[i].push_back(b0);
    uint32_t base = hc.W[i + 1];
    std::vector<uint32_t> u2(ly.width);
    for (uint32_t g = 0; g < ly.width; ++g)
      if (hc.src[i][g] == i + 1) u2[g] = hc.in2[i][g];
    for (uint32_t j = i + 2; j <= d; ++j) {
      std::vector<uint32_t> pos(hc.W[j], 0xffffffffu);
      for (uint32_t g = 0; g < ly.width; ++g)
        if (hc.src[i][g] == j) pos[hc.in2[i][g]] = 0;
      HostCircuit::Block B{j, base, 0, {}};
      for (uint32_t y = 0; y < hc.W[j]; ++y)
        if (pos[y] == 0) {
          pos[y] = base + B.count++;
          B.ys.push_back(y);
        }
      if (!B.count) continue;
      for (uint32_t g = 0; g < ly.width; ++g)
        if (hc.src[i][g] == j) u2[g] = pos[hc.in2[i][g]];
      base += B.count;
      hc.blocks[i].push_back(std::move(B));
    }
    hc.u2[i] = std::move(u2);
    hc.sx[i] = ceil_log2(base);
    if (hc.sx[i] > 16)
      return fail(SISU_ERR_TOO_LARGE, "layer %u: virtual layer wider than 2^16 (general circuits)", i);
    if (hc.c + hc.sx[i] > 32) return fail(SISU_ERR_TOO_LARGE, "copies x virtual width of layer %u above 2^32", i);
  }
  return circuit_finish(cc, on_device, out);
}

extern "C" int sisu_circuit_create_general(const sisu_general_layer* layers, uint32_t n_gate_layers,
                                           uint32_t input_width, uint32_t n_copies, sisu_circuit** out) {
  return circuit_create_general(layers, n_gate_layers, input_width, n_copies, true, out);
}

extern "C" int sisu_circuit_create_general_host(const sisu_general_layer* layers, uint32_t n_gate_layers,
                                                uint32_t input_width, uint32_t n_copies, sisu_circuit** out) {
  return circuit_create_general(layers, n_gate_layers, input_width, n_copies, false, out);
}

extern "C" int sisu_circuit_create(const sisu_layer* layers, uint32_t n_gate_layers, uint32_t input_width,
                                   uint32_t n_copies, sisu_circuit** out) {
  return circuit_create(layers, n_gate_layers, input_width, n_copies, true, out);
}

extern "C" int sisu_circuit_create_host(const sisu_layer* layers, uint32_t n_gate_layers, uint32_t input_width,
                                        uint32_t n_copies, sisu_circuit** out) {
  return circuit_create(layers, n_gate_layers, input_width, n_copies, false, out);
}

extern "C" int sisu_circuit_create_acc(const sisu_acc_layer* layers, uint32_t n_gate_layers, uint32_t input_width,
                                       uint32_t n_copies, sisu_circuit** out) {
  return circuit_create_acc(layers, n_gate_layers, input_width, n_copies, true, out);
}

extern "C" int sisu_circuit_create_acc_host(const sisu_acc_layer* layers, uint32_t n_gate_layers,
                                            uint32_t input_width, uint32_t n_copies, sisu_circuit** out) {
  return circuit_create_acc(layers, n_gate_layers, input_width, n_copies, false, out);
}

static bool has_device(const sisu_circuit* circ) { return circ && circ->dev; }

extern "C" void sisu_circuit_destroy(sisu_circuit* circ) { delete circ; }

extern "C" int sisu_circuit_info(const sisu_circuit* circ, uint32_t* depth, uint32_t* log_copies,
                                 uint32_t* log_widths, size_t* proof_len, size_t* eval_bytes) {
  if (!circ) return fail(SISU_ERR_INVALID_ARG, "circuit is NULL");
  const HostCircuit& hc = circ->hc;
  if (depth) *depth = hc.d;
  if (log_copies) *log_copies = hc.c;
  if (log_widths)
    for (uint32_t i = 0; i <= hc.d; ++i) log_widths[i] = hc.s[i];
  if (proof_len) *proof_len = hc.proof_len();
  if (eval_bytes) {
    size_t n = 0;
    for (uint32_t i = 0; i <= hc.d; ++i) n += ((size_t)hc.C << hc.s[i]) * 32;
    *eval_bytes = n;
  }
  return SISU_OK;
}

// ---------------------------------------------------------------------------
// evaluation

namespace sisu {
// general circuits: positions of X_i past layer i + 1 (the used gates of
// deeper layers), and whether X_i needs a table of its own
static uint32_t gather_count(const HostCircuit& hc, uint32_t i) {
  uint32_t n = 0;
  for (size_t b = 1; b < hc.blocks[i].size(); ++b) n += hc.blocks[i][b].count;
  return n;
}
static bool own_x(const HostCircuit& hc, uint32_t i) {
  return hc.general && (hc.blocks[i].size() > 1 || hc.sx[i] != hc.s[i + 1]);
}

// device bytes of the inputs' digest scratch (the two-table launch with an
// empty second table)
static size_t eval_digest_scratch_bytes(const HostCircuit& hc) {
  const size_t words = digest_scratch_words(((size_t)hc.C << hc.s[hc.d]) * 32) + digest_scratch_words(0);
  return (words * 4 + 255) & ~(size_t)255;
}

int eval_enqueue(sisu_eval* ev, const uint8_t* inputs, int on_device, cudaStream_t st) {
  const sisu_circuit* cc = ev->circ;
  const HostCircuit& hc = cc->hc;
  const uint32_t d = hc.d;
  const size_t in_bytes = (size_t)hc.Creal * hc.wreal[d] * 32;
  const bool padded = hc.Creal != hc.C || hc.wreal[d] != hc.W[d];
  // Host inputs of an unpadded circuit arrive in chunks of copies on the
  // handle's copy stream while the copies already in are converted and
  // evaluated on `st`: every copy evaluates on its own rows (the circuits
  // are data-parallel), so the evaluation of chunk k overlaps the transfer
  // of chunk k + 1 and only the last chunk's evaluation follows the copy.
  const uint32_t nchunk =
      (!on_device && !padded && !hc.general && hc.C >= kEvalChunks && in_bytes >= kEvalChunkMin) ? kEvalChunks : 1;
  // new inputs land only after the previous inputs' digest has read them
  if (ev->dig_recorded) CK(cudaStreamWaitEvent(st, ev->dig_ev, 0), "stream wait");
  const uint32_t* src;
  if (on_device) {
    if (((uintptr_t)inputs & 15) != 0) return fail(SISU_ERR_INVALID_ARG, "device inputs not 16-byte aligned");
    src = (const uint32_t*)inputs;
  } else if (nchunk > 1) {
    if (!ev->copy_stream) {
      CK(cudaStreamCreateWithFlags(&ev->copy_stream, cudaStreamNonBlocking), "stream create");
      for (cudaEvent_t& e : ev->chunk_ev) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "event create");
    }
    // the copies overwrite the input layer only after the work queued on st
    // before this call (a proof may still read it)
    CK(cudaEventRecord(ev->chunk_ev[kEvalChunks], st), "event record");
    CK(cudaStreamWaitEvent(ev->copy_stream, ev->chunk_ev[kEvalChunks], 0), "stream wait");
    const size_t row = (size_t)hc.W[d] * 32;
    for (uint32_t k = 0; k < nchunk; ++k) {
      const size_t b0 = (size_t)hc.C * k / nchunk, b1 = (size_t)hc.C * (k + 1) / nchunk;
      CK(cudaMemcpyAsync((uint8_t*)ev->V[d] + b0 * row, inputs + b0 * row, (b1 - b0) * row, cudaMemcpyHostToDevice,
                         ev->copy_stream),
         "input copy");
      CK(cudaEventRecord(ev->chunk_ev[k], ev->copy_stream), "event record");
    }
    src = ev->V[d];
  } else {
    uint32_t* dst = padded ? ev->stage : ev->V[d];
    CK(cudaMemcpyAsync(dst, inputs, in_bytes, cudaMemcpyHostToDevice, st), "input copy");
    src = dst;
  }
  CK(cudaMemsetAsync(ev->flag, 0, 4, st), "memset");
  if (!ev->dig_stream) {
    CK(cudaStreamCreateWithFlags(&ev->dig_stream, cudaStreamNonBlocking), "stream create");
    CK(cudaEventCreateWithFlags(&ev->in_ready, cudaEventDisableTiming), "event create");
    CK(cudaEventCreateWithFlags(&ev->dig_ev, cudaEventDisableTiming), "event create");
  }
  for (uint32_t k = 0; k < nchunk; ++k) {
    const uint32_t b0 = (uint32_t)((uint64_t)hc.C * k / nchunk), b1 = (uint32_t)((uint64_t)hc.C * (k + 1) / nchunk);
    if (nchunk > 1) CK(cudaStreamWaitEvent(st, ev->chunk_ev[k], 0), "stream wait");
    {
      ProfScope ps(kProfInputs, (double)((size_t)(b1 - b0) << hc.s[d]), st);
      CK(launch_inputs_to_mont(src, ev->V[d], b0, b1 - b0, hc.s[d], hc.Creal, hc.wreal[d], ev->flag, st),
         "input conversion");
    }
    if (k + 1 == nchunk) {  // the input layer is complete: its digest on the side stream
      CK(cudaEventRecord(ev->in_ready, st), "event record");
      CK(cudaStreamWaitEvent(ev->dig_stream, ev->in_ready, 0), "stream wait");
      CK(launch_digest_tables2(ev->V[d], (size_t)hc.C << hc.s[d], nullptr, 0, ev->dscratch, ev->dig, ev->dig + 8,
                               ev->dig_stream),
         "input digest");
      CK(cudaEventRecord(ev->dig_ev, ev->dig_stream), "event record");
      ev->dig_recorded = true;
    }
    for (int i = (int)d - 1; i >= 0; --i) {
      ProfScope ps(kProfEval, (double)(b1 - b0) * cc->L[i].nmul, st);
      const uint32_t* from = ev->V[i + 1];
      uint32_t sn = hc.s[i + 1];
      if (hc.general) {  // a general layer reads its virtual layer, gathered first
        if (ev->X[i] != ev->V[i + 1]) {
          GatherLayers gl;
          for (uint32_t l = 0; l <= d; ++l) {
            gl.V[l] = ev->V[l];
            gl.s[l] = hc.s[l];
          }
          CK(launch_gather_x(gl, i + 1, cc->gmap[i], gather_count(hc, i), ev->X[i], hc.C, hc.s[i + 1], hc.sx[i], st),
             "virtual layer");
        }
        from = ev->X[i];
        sn = hc.sx[i];
      }
      CK(launch_eval_layer(from, ev->V[i], cc->L[i], b0, b1 - b0, hc.s[i], sn, st), "eval layer");
    }
  }
  CK(cudaMemcpyAsync(ev->host_flag, ev->flag, 4, cudaMemcpyDeviceToHost, st), "flag copy");
  return SISU_OK;
}

size_t eval_footprint(const sisu_circuit* cc, bool host_inputs) {
  const HostCircuit& hc = cc->hc;
  size_t total = 0;
  for (uint32_t i = 0; i <= hc.d; ++i) total += ((size_t)hc.C << hc.s[i]) * 32;
  total += 256;  // flag and the inputs' digest
  const bool padded = hc.Creal != hc.C || hc.wreal[hc.d] != hc.W[hc.d];
  if (padded && host_inputs) total += ((size_t)hc.Creal * hc.wreal[hc.d] * 32 + 255) & ~(size_t)255;
  total += eval_digest_scratch_bytes(hc);
  return total;
}

void eval_place(sisu_eval* ev, const sisu_circuit* cc, uint8_t* dev, bool host_inputs, uint32_t* host_flag) {
  const HostCircuit& hc = cc->hc;
  ev->circ = cc;
  ev->placed = true;
  ev->V.resize(hc.d + 1);
  size_t off = 0;
  for (uint32_t i = 0; i <= hc.d; ++i) {
    ev->V[i] = (uint32_t*)(dev + off);
    off += ((size_t)hc.C << hc.s[i]) * 32;
  }
  ev->flag = (uint32_t*)(dev + off);
  ev->dig = ev->flag + 16;
  off += 256;
  const bool padded = hc.Creal != hc.C || hc.wreal[hc.d] != hc.W[hc.d];
  ev->stage = (padded && host_inputs) ? (uint32_t*)(dev + off) : nullptr;
  if (padded && host_inputs) off += ((size_t)hc.Creal * hc.wreal[hc.d] * 32 + 255) & ~(size_t)255;
  ev->dscratch = (uint32_t*)(dev + off);
  ev->host_flag = host_flag;
}
}  // namespace sisu

static int eval_run(sisu_eval* ev, const uint8_t* inputs, int on_device, cudaStream_t st) {
  int rc = eval_enqueue(ev, inputs, on_device, st);
  if (rc) return rc;
  CK(cudaStreamSynchronize(st), "eval");
  if (*ev->host_flag & 1u) return fail(SISU_ERR_NOT_CANONICAL, "an input element is not below r");
  return SISU_OK;
}

extern "C" int sisu_circuit_eval(const sisu_circuit* circ, const uint8_t* inputs, int inputs_on_device,
                                 void* stream, sisu_eval** out) {
  if (!out) return fail(SISU_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!circ || !inputs) return fail(SISU_ERR_INVALID_ARG, "NULL circuit or inputs");
  if (!has_device(circ)) return fail(SISU_ERR_INVALID_ARG, "circuit was created for host verification only");
  if (inputs_on_device)
    if (int rc = require_device(inputs, "inputs")) return rc;
  const HostCircuit& hc = circ->hc;
  std::unique_ptr<sisu_eval> ev(new (std::nothrow) sisu_eval());
  if (!ev) return fail(SISU_ERR_OOM, "host allocation");
  ev->circ = circ;
  size_t total = 0;
  std::vector<size_t> offs(hc.d + 1), xoffs(hc.d, 0);
  for (uint32_t i = 0; i <= hc.d; ++i) {
    offs[i] = total;
    total += ((size_t)hc.C << hc.s[i]) * 32;
  }
  for (uint32_t i = 0; i < hc.d; ++i)
    if (own_x(hc, i)) {
      xoffs[i] = total;
      total += ((size_t)hc.C << hc.sx[i]) * 32;
    }
  if (cudaMalloc(&ev->dev, total + 256 + eval_digest_scratch_bytes(hc)) != cudaSuccess)
    return fail(SISU_ERR_OOM, "device allocation of %zu bytes for the layer values", total);
  ev->V.resize(hc.d + 1);
  for (uint32_t i = 0; i <= hc.d; ++i) ev->V[i] = (uint32_t*)((uint8_t*)ev->dev + offs[i]);
  if (hc.general) {
    ev->X.resize(hc.d);
    for (uint32_t i = 0; i < hc.d; ++i)
      ev->X[i] = own_x(hc, i) ? (uint32_t*)((uint8_t*)ev->dev + xoffs[i]) : ev->V[i + 1];
  }
  ev->flag = (uint32_t*)((uint8_t*)ev->dev + total);
  ev->dig = ev->flag + 16;
  ev->dscratch = (uint32_t*)((uint8_t*)ev->dev + total + 256);
  const bool padded = hc.Creal != hc.C || hc.wreal[hc.d] != hc.W[hc.d];
  if (padded && !inputs_on_device) {
    if (cudaMalloc(&ev->stage, (size_t)hc.Creal * hc.wreal[hc.d] * 32) != cudaSuccess)
      return fail(SISU_ERR_OOM, "device allocation for the input staging");
  }
  CK(cudaMallocHost(&ev->host_flag, 4), "cudaMallocHost");
  int rc = eval_run(ev.get(), inputs, inputs_on_device, (cudaStream_t)stream);
  if (rc != SISU_OK) return rc;
  *out = ev.release();
  return SISU_OK;
}

extern "C" int sisu_eval_update(sisu_eval* ev, const uint8_t* inputs, int inputs_on_device, void* stream) {
  if (!ev || !inputs) return fail(SISU_ERR_INVALID_ARG, "NULL eval or inputs");
  if (inputs_on_device)
    if (int rc = require_device(inputs, "inputs")) return rc;
  const HostCircuit& hc = ev->circ->hc;
  const bool padded = hc.Creal != hc.C || hc.wreal[hc.d] != hc.W[hc.d];
  if (padded && !inputs_on_device && !ev->stage) {
    if (cudaMalloc(&ev->stage, (size_t)hc.Creal * hc.wreal[hc.d] * 32) != cudaSuccess)
      return fail(SISU_ERR_OOM, "device allocation for the input staging");
  }
  return eval_run(ev, inputs, inputs_on_device, (cudaStream_t)stream);
}

extern "C" int sisu_eval_outputs(const sisu_eval* ev, uint8_t* out, size_t cap, int out_on_device, void* stream) {
  if (!ev || !out) return fail(SISU_ERR_INVALID_ARG, "NULL eval or output");
  const HostCircuit& hc = ev->circ->hc;
  const size_t n = (size_t)hc.Creal * hc.wreal[0] * 32;
  if (cap < n) return fail(SISU_ERR_BUFFER, "output buffer of %zu bytes, need %zu", cap, n);
  cudaStream_t st = (cudaStream_t)stream;
  if (out_on_device) {
    if (((uintptr_t)out & 15) != 0) return fail(SISU_ERR_INVALID_ARG, "device output not 16-byte aligned");
    if (int rc = require_device(out, "out")) return rc;
    CK(launch_layer_to_canonical(ev->V[0], (uint32_t*)out, hc.c, hc.s[0], hc.Creal, hc.wreal[0], st), "outputs");
    return SISU_OK;
  }
  uint32_t* tmp = nullptr;
  CK(cudaMallocAsync(&tmp, n, st), "cudaMallocAsync");
  int rc = launch_layer_to_canonical(ev->V[0], tmp, hc.c, hc.s[0], hc.Creal, hc.wreal[0], st);
  if (rc == 0) rc = cudaMemcpyAsync(out, tmp, n, cudaMemcpyDeviceToHost, st);
  cudaFreeAsync(tmp, st);
  cudaError_t e = cudaStreamSynchronize(st);
  if (rc) return cuda_fail((cudaError_t)rc, "outputs");
  if (e) return cuda_fail(e, "outputs");
  return SISU_OK;
}

extern "C" int sisu_eval_layer(const sisu_eval* ev, uint32_t layer, uint8_t* out, size_t cap, void* stream) {
  if (!ev || !out) return fail(SISU_ERR_INVALID_ARG, "NULL eval or output");
  const HostCircuit& hc = ev->circ->hc;
  if (layer > hc.d) return fail(SISU_ERR_INVALID_ARG, "layer %u beyond depth %u", layer, hc.d);
  const size_t n = ((size_t)hc.C << hc.s[layer]) * 32;
  if (cap < n) return fail(SISU_ERR_BUFFER, "buffer of %zu bytes, need %zu", cap, n);
  cudaStream_t st = (cudaStream_t)stream;
  uint32_t* tmp = nullptr;
  CK(cudaMallocAsync(&tmp, n, st), "cudaMallocAsync");
  int rc = launch_layer_to_canonical(ev->V[layer], tmp, hc.c, hc.s[layer], hc.C, hc.W[layer], st);
  if (rc == 0) rc = cudaMemcpyAsync(out, tmp, n, cudaMemcpyDeviceToHost, st);
  cudaFreeAsync(tmp, st);
  cudaError_t e = cudaStreamSynchronize(st);
  if (rc) return cuda_fail((cudaError_t)rc, "layer copy");
  if (e) return cuda_fail(e, "layer copy");
  return SISU_OK;
}

extern "C" void sisu_eval_destroy(sisu_eval* ev) { delete ev; }

// ---------------------------------------------------------------------------
// transcript domain

extern "C" int sisu_transcript_create(const uint8_t* domain, size_t len, sisu_transcript** out) {
  if (!out) return fail(SISU_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (len > kMaxDomain) return fail(SISU_ERR_INVALID_ARG, "domain longer than %u bytes", kMaxDomain);
  if (len && !domain) return fail(SISU_ERR_INVALID_ARG, "NULL domain with nonzero length");
  sisu_transcript* t = new (std::nothrow) sisu_transcript();
  if (!t) return fail(SISU_ERR_OOM, "host allocation");
  if (!domain || len == 0) {
    t->len = (uint32_t)strlen(kDefaultDomain);
    memcpy(t->domain, kDefaultDomain, t->len);
  } else {
    t->len = (uint32_t)len;
    memcpy(t->domain, domain, len);
  }
  *out = t;
  return SISU_OK;
}

extern "C" void sisu_transcript_destroy(sisu_transcript* tr) { delete tr; }

// ---------------------------------------------------------------------------
// proving

constexpr int kWsRegions = 22;

// proof bytes of a circuit's shape with 2^c copies
static size_t proof_len_c(const HostCircuit& hc, uint32_t c) {
  if (hc.general) return hc.proof_len();
  size_t n = 8 + 4 * ((size_t)hc.d + 3);
  for (uint32_t i = 0; i < hc.d; ++i) n += 32 * (3 * (size_t)c + 4 * (size_t)hc.s[i + 1] + 2);
  return n;
}

// general circuits: the readers (layer i, block b) of each layer's claims,
// in the order the prover meets them (the input layer's are checked by the
// verifier, so it has none)
static std::vector<std::vector<std::pair<uint32_t, uint32_t>>> general_readers(const HostCircuit& hc) {
  std::vector<std::vector<std::pair<uint32_t, uint32_t>>> r(hc.d + 1);
  if (!hc.general) return r;
  for (uint32_t i = 0; i < hc.d; ++i)
    for (uint32_t b = 0; b < hc.blocks[i].size(); ++b)
      if (hc.blocks[i][b].layer < hc.d) r[hc.blocks[i][b].layer].push_back({i, b});
  return r;
}

static void workspace_sizes(const sisu_circuit* cc, size_t sizes[kWsRegions], uint32_t c_proof) {
  const HostCircuit& hc = cc->hc;
  uint32_t wmax_next = 1, wmax = 1, nmax = 1, sxmax = 0, nbmax = 0, lmax = 0, nterms = 0;
  for (uint32_t i = 0; i < hc.d; ++i) {
    wmax_next = std::max(wmax_next, hc.general ? 1u << hc.sx[i] : hc.W[i + 1]);
    nmax = std::max(nmax, cc->L[i].ntot);
    if (hc.general) {
      sxmax = std::max(sxmax, hc.sx[i]);
      nbmax = std::max(nbmax, (uint32_t)hc.blocks[i].size());
    }
  }
  for (const auto& rd : general_readers(hc)) {
    lmax = std::max(lmax, (uint32_t)rd.size());
    nterms += (uint32_t)rd.size();
  }
  for (uint32_t i = 0; i <= hc.d; ++i) wmax = std::max(wmax, hc.W[i]);
  const size_t half = hc.C >= 2 ? (size_t)(hc.C / 2) * wmax_next * 32 : 32;
  const size_t dig = (digest_scratch_words((size_t)hc.C * hc.W[hc.d] * 32) +
                      digest_scratch_words((size_t)hc.C * hc.W[0] * 32)) * 4;
  uint32_t smax = 0;
  for (uint32_t i = 0; i < hc.d; ++i) smax = std::max(smax, hc.s[i]);
  const size_t hstride = hc.c + 2 * (size_t)sxmax + 2 * (size_t)nbmax;
  const bool g = hc.general;
  const size_t v[kWsRegions] = {half, (size_t)hc.C * 4 * 32, ((size_t)nmax + wmax) * 32,
                                (size_t)wmax_next * 32,
                                (size_t)wmax_next * 32, (size_t)wmax_next * 32, (size_t)wmax_next * 32,
                                (size_t)wmax * 32, (size_t)kMaxPartials * 4 * 32, dig, sizeof(DevState),
                                proof_len_c(hc, c_proof), eq_half_words(hc.c, smax) * 4, (size_t)nmax * 2 * 32,
                                g ? (size_t)lmax * hc.C * 32 : 0, g ? (size_t)lmax * nmax * 32 : 0,
                                g ? (size_t)lmax * 128 : 0, g ? (size_t)nmax * 32 : 0, g ? (size_t)32 : 0,
                                g ? (size_t)hc.d * hstride * 32 : 0, g ? (size_t)2 * nbmax * 32 : 0,
                                g ? (size_t)nterms * sizeof(GeneralTerm) : 0};
  for (int k = 0; k < kWsRegions; ++k) sizes[k] = v[k];
}

static size_t al256(size_t b) { return (b + 255) & ~(size_t)255; }

namespace sisu {
size_t workspace_footprint(const sisu_circuit* cc) {
  size_t sizes[kWsRegions], total = 0;
  workspace_sizes(cc, sizes, cc->hc.c);
  for (size_t x : sizes) total += al256(x);
  return total;
}

size_t workspace_footprint_c(const sisu_circuit* cc, uint32_t c_proof) {
  size_t sizes[kWsRegions], total = 0;
  workspace_sizes(cc, sizes, c_proof);
  for (size_t x : sizes) total += al256(x);
  return total;
}

// Lay out the workspace in `dev` (workspace_footprint_c bytes) with the
// pinned proof bytes at `host` (proof bytes + 16), the header of a proof
// over 2^c_proof copies and a zeroed state set on `st`.
int workspace_layout(const sisu_circuit* cc, Workspace* ws, uint8_t* dev, uint8_t* host, uint32_t c_proof,
                     cudaStream_t st) {
  const HostCircuit& hc = cc->hc;
  size_t sizes[kWsRegions];
  workspace_sizes(cc, sizes, c_proof);
  uint8_t* p = dev;
  void* ptrs[kWsRegions];
  for (int k = 0; k < kWsRegions; ++k) {
    ptrs[k] = p;
    p += al256(sizes[k]);
  }
  ws->T = (uint32_t*)ptrs[0];
  ws->E = (uint32_t*)ptrs[1];
  ws->Ub[0] = ws->E + 8 * (size_t)hc.C;
  ws->Ub[1] = ws->Ub[0] + 8 * (size_t)hc.C;
  ws->cb[0] = ws->Ub[1] + 8 * (size_t)hc.C;
  ws->cb[1] = ws->cb[0] + 4 * (size_t)hc.C;

  ws->om = (uint32_t*)ptrs[2];
  {
    uint32_t nmax = 1;
    for (uint32_t i = 0; i < hc.d; ++i) nmax = std::max(nmax, cc->L[i].ntot);
    ws->omo = ws->om + 8 * (size_t)nmax;
  }
  ws->At = (uint32_t*)ptrs[3];
  ws->H1 = (uint32_t*)ptrs[4];
  ws->H2 = (uint32_t*)ptrs[5];
  ws->Ay = (uint32_t*)ptrs[6];
  ws->Q = (uint32_t*)ptrs[7];
  ws->partials = (uint32_t*)ptrs[8];
  // a round's grid sums use at most kMaxPartials / 2 blocks' four values; the
  // upper half of the region holds the shares of the pairs' coefficients
  ws->cpart = ws->partials + 8 * 2 * (size_t)kMaxPartials;
  ws->dscratch = (uint32_t*)ptrs[9];
  ws->S = (DevState*)ptrs[10];
  ws->proof = (uint8_t*)ptrs[11];
  ws->eqh = (uint32_t*)ptrs[12];
  ws->P = (uint32_t*)ptrs[13];
  if (hc.general) {
    ws->Et = (uint32_t*)ptrs[14];
    ws->omt = (uint32_t*)ptrs[15];
    ws->sums = (uint32_t*)ptrs[16];
    ws->omc = (uint32_t*)ptrs[17];
    ws->Ec = (uint32_t*)ptrs[18];
    ws->hist = (uint32_t*)ptrs[19];
    ws->vals = (uint32_t*)ptrs[20];
    ws->gterms = ptrs[21];
    uint32_t sxmax = 0, nbmax = 0;
    for (uint32_t i = 0; i < hc.d; ++i) {
      sxmax = std::max(sxmax, hc.sx[i]);
      nbmax = std::max(nbmax, (uint32_t)hc.blocks[i].size());
    }
    ws->hstride = hc.c + 2 * sxmax + 2 * nbmax;
    // the terms of every layer's claims: their challenges in the reading
    // layer's history record, their alphas, the gate positions
    std::vector<GeneralTerm> terms;
    ws->term_off.assign(hc.d + 1, 0);
    const auto readers = general_readers(hc);
    for (uint32_t j = 0; j <= hc.d; ++j) {
      ws->term_off[j] = (uint32_t)terms.size();
      if (j == hc.d) break;
      for (auto [i, b] : readers[j]) {
        const Fr* h = (const Fr*)(ws->hist + 8 * (size_t)i * ws->hstride);
        GeneralTerm t;
        t.rb = h;
        t.rx = h + hc.c;
        t.ry = h + hc.c + hc.sx[i];
        t.alpha = h + hc.c + 2 * hc.sx[i] + 2 * b;
        t.pos = cc->pmap[i][b];
        t.sxr = hc.sx[i];
        terms.push_back(t);
      }
    }
    if (!terms.empty())
      CK(cudaMemcpy(ws->gterms, terms.data(), terms.size() * sizeof(GeneralTerm), cudaMemcpyHostToDevice),
         "term descriptors");
  }
  ws->proof_len = proof_len_c(hc, c_proof);
  ws->host = host;
  // the proof header is fixed by the circuit
  std::vector<uint8_t> hdr(8 + 4 * ((size_t)hc.d + 3));
  memcpy(hdr.data(), "SISUGKR2", 8);
  auto put = [&](size_t at, uint32_t v) {
    hdr[at] = (uint8_t)v; hdr[at + 1] = (uint8_t)(v >> 8); hdr[at + 2] = (uint8_t)(v >> 16); hdr[at + 3] = (uint8_t)(v >> 24);
  };
  put(8, hc.d);
  put(12, c_proof);
  for (uint32_t i = 0; i <= hc.d; ++i) put(16 + 4 * (size_t)i, hc.s[i]);
  // staged through the pinned proof buffer so that the copy can stay asynchronous
  memcpy(host, hdr.data(), hdr.size());
  CK(cudaMemcpyAsync(ws->proof, host, hdr.size(), cudaMemcpyHostToDevice, st), "header upload");
  CK(cudaMemsetAsync(ws->S, 0, sizeof(DevState), st), "memset");
  return SISU_OK;
}

static int workspace_init(sisu_eval* ev, Workspace* ws, uint8_t* dev, uint8_t* host, cudaStream_t st) {
  return workspace_layout(ev->circ, ws, dev, host, ev->circ->hc.c, st);
}

int workspace_place(sisu_eval* ev, uint8_t* dev, uint8_t* host_pinned, cudaStream_t st) {
  std::unique_ptr<Workspace> ws(new (std::nothrow) Workspace());
  if (!ws) return fail(SISU_ERR_OOM, "host allocation");
  ws->owns_host = false;
  int rc = workspace_init(ev, ws.get(), dev, host_pinned, st);
  if (rc) return rc;
  ev->ws = std::move(ws);
  return SISU_OK;
}
}  // namespace sisu

static int workspace_alloc(sisu_eval* ev) {
  const sisu_circuit* cc = ev->circ;
  std::unique_ptr<Workspace> ws(new (std::nothrow) Workspace());
  if (!ws) return fail(SISU_ERR_OOM, "host allocation");
  const size_t total = workspace_footprint(cc);
  if (cudaMalloc(&ws->dev, total) != cudaSuccess)
    return fail(SISU_ERR_OOM, "device allocation of %zu bytes for the prover workspace", total);
  uint8_t* host = nullptr;
  if (cudaMallocHost(&host, cc->hc.proof_len() + 16) != cudaSuccess)
    return fail(SISU_ERR_OOM, "pinned host allocation");
  ws->owns_host = true;
  int rc = workspace_init(ev, ws.get(), (uint8_t*)ws->dev, host, 0);
  if (rc) return rc;
  CK(cudaStreamSynchronize(0), "workspace init");
  ev->ws = std::move(ws);
  return SISU_OK;
}

static int enqueue_general_layer(const sisu_circuit* cc, sisu_eval* ev, uint32_t i, size_t& off, cudaStream_t st);

// a full 512-bit product (128 multiply-adds) in units of a Montgomery
// product (264), for the copy phase's work counts
constexpr double kFullProduct = 128.0 / 264.0;

// Enqueue one whole proof on `st` (no host synchronisation).
static int enqueue_prove(const sisu_circuit* cc, sisu_eval* ev, const sisu_transcript* tr, cudaStream_t st) {
  const HostCircuit& hc = cc->hc;
  Workspace& w = *ev->ws;
  const uint32_t d = hc.d, c = hc.c;
  // statement digests: the outputs' here, the inputs' formed by the
  // evaluation on its side stream (the proof's stream waits for it before
  // this work is enqueued or replayed); the wiring's is cached
  {
    ProfScope ps(kProfDigest, 0, st);
    CK(launch_digest_tables2(ev->V[0], (size_t)hc.C << hc.s[0], nullptr, 0, w.dscratch, w.S->dig_out, ev->dig + 16,
                             st),
       "statement digests");
    CK(cudaMemcpyAsync(w.S->dig_in, ev->dig, 32, cudaMemcpyDeviceToDevice, st), "digest copy");
  }
  InitParams ip;
  memset(&ip, 0, sizeof ip);
  if (tr) {
    memcpy(ip.domain, tr->domain, tr->len);
    ip.dlen = tr->len;
  } else {
    ip.dlen = (uint32_t)strlen(kDefaultDomain);
    memcpy(ip.domain, kDefaultDomain, ip.dlen);
  }
  ip.d = d;
  ip.c = c;
  for (uint32_t i = 0; i <= d; ++i) ip.s[i] = hc.s[i];
  memcpy(ip.wiring, hc.wiring_digest, 32);
  {
    ProfScope ps(kProfTranscript, 0, st);
    CK(launch_transcript_init(ip, w.S, st), "transcript init");
  }

  size_t off = 8 + 4 * ((size_t)d + 3);
  for (uint32_t i = 0; i < d; ++i) {
    if (hc.general) {
      if (int rc = enqueue_general_layer(cc, ev, i, off, st)) return rc;
      continue;
    }
    const DevLayer& L = cc->L[i];
    const uint32_t s = hc.s[i + 1], Wn = hc.W[i + 1], sn = hc.s[i + 1];
    {
      ProfScope ps(kProfLayerInit, (double)hc.C * c + (double)L.ntot * (i == 0 ? hc.s[0] : 2.0 * hc.s[i] + 2), st);
      // gate weights in gate order too, for the rows' gate sums
      CK(launch_layer_init(w.S, i, c, hc.s[i], L, w.E, w.om, w.eqh, st, 0, 0, w.omo), "layer init");
    }
    // copy phase: c rounds, each followed by the fold of its challenge
    const uint32_t* A = ev->V[i + 1];

    // the copy phase by the recurrence of its linear part: the rows' gate
    // sums from layer i's values, then the mul entries' t^2 terms a round.
    // Work counted in Montgomery-product units of 264 multiply-adds: a full
    // 512-bit product is 128 of them (kFullProduct of a unit)
    {
      ProfScope ps(kProfRowSums, kFullProduct * hc.C * hc.W[i], st);
      CK(launch_rowdot(ev->V[i], hc.s[i], w.omo, hc.C, w.Ub[0], st), "row sums");
    }
    for (uint32_t k = 0; k < c; ++k) {
      const uint32_t* tab = k == 0 ? ev->V[i + 1] : w.T;
      const uint32_t h = hc.C >> (k + 1);
      {
        // a mul entry of a pair: one Montgomery and one full product; a pair:
        // its four message terms and (after the first round) the four
        // products of its two rows' update
        ProfScope ps(kProfCopyRound, ((1.0 + kFullProduct) * L.nmul + (k ? 8.0 : 4.0)) * h, st);
        CK(launch_copy_c(tab, sn, h, w.E, w.om, L, w.Ub[(k + 1) & 1], w.cb[(k + 1) & 1], w.Ub[k & 1], w.cb[k & 1],
                         w.cpart, w.partials, w.S, w.proof, off + 32 * 3 * (size_t)k, k, st),
           "copy round");
      }
      {
        ProfScope ps(kProfCopyFold, (double)h * Wn + h, st);
        CK(launch_copy_fold(tab, w.T, sn, h, w.E, w.S, k, st), "copy fold");
      }
      A = w.T;
    }
    const size_t offx = off + 32 * 3 * (size_t)c;  // a copy round sends 3 values, an x/y round 2
    if (int rc = sisu::enqueue_layer_phases(hc, L, w, i, A, w.E, w.om, hc.s[i + 1], offx, false, st)) return rc;
    off = offx + 32 * 4 * (size_t)s + 64;
  }
  return SISU_OK;
}

// Gate layer i of a general circuit (Sec. 2.7), over its virtual layer X_i
// (2^sx positions): layer 0 starts from the claim point (z_b, z_g) as in a
// layered proof; a deeper layer from the terms of its readers' claims (each
// with its own copy point), whose round sums are added in every copy round
// and whose weights, times their copy weights at r_b, are the phases' gate
// weights.  The layer ends with the blocks' values, their transcript step
// and the alphas of the blocks' claims.
static int enqueue_general_layer(const sisu_circuit* cc, sisu_eval* ev, uint32_t i, size_t& off, cudaStream_t st) {
  const HostCircuit& hc = cc->hc;
  Workspace& w = *ev->ws;
  const DevLayer& L = cc->L[i];
  const uint32_t c = hc.c, sx = hc.sx[i], WX = 1u << sx;
  const uint32_t nt = i == 0 ? 1 : w.term_off[i + 1] - w.term_off[i];
  const size_t Cw = 8 * (size_t)hc.C, Nw = 8 * (size_t)L.ntot;
  uint32_t *E = w.E, *om = w.om;
  if (i == 0) {
    CK(launch_layer_init(w.S, 0, c, hc.s[0], L, w.E, w.om, w.eqh, st), "layer init");
  } else {
    CK(launch_general_terms((const GeneralTerm*)w.gterms + w.term_off[i], nt, c, L.sgate, L.ntot, w.Et, w.omt, st),
       "claim terms");
    E = w.Et;
    om = w.omt;
  }
  const double per_pair = 2.0 * L.ntot + 4.0 * L.nmul;
  const uint32_t* A = ev->X[i];
  for (uint32_t k = 0; k < c; ++k) {
    const uint32_t* tab = k == 0 ? ev->X[i] : w.T;
    const uint32_t h = hc.C >> (k + 1);
    const size_t offk = off + 96 * (size_t)k;
    {
      ProfScope ps(kProfCopyRound, per_pair * h * nt, st);
      if (nt == 1) {
        CK(launch_copy_round(tab, sx, h, E, om, L, w.partials, w.S, w.proof, offk, k, st), "copy round");
      } else {  // each term's sums, then their sum is the round message
        for (uint32_t t = 0; t < nt; ++t)
          CK(launch_copy_round(tab, sx, h, E + t * Cw, om + t * Nw, L, w.partials, w.S, w.proof, offk, k, st,
                               w.sums + 32 * (size_t)t),
             "copy round");
        CK(launch_shard_absorb(w.sums, nt, w.S, w.proof, offk, k, st), "round message");
      }
    }
    {
      ProfScope ps(kProfCopyFold, (double)h * WX + h * nt, st);
      CK(launch_copy_fold(tab, w.T, sx, h, E, w.S, k, st), "copy fold");
      for (uint32_t t = 1; t < nt; ++t) CK(launch_fold_e(E + t * Cw, h, w.S, k, st), "weight fold");
    }
    A = w.T;
  }
  if (nt > 1) {  // the phases' gate weights: every term's, times its copy weight at r_b
    CK(launch_combine_terms(E, hc.C, om, L.ntot, nt, w.omc, w.Ec, st), "combined weights");
    E = w.Ec;
    om = w.omc;
  }
  const size_t offx = off + 96 * (size_t)c, offv = offx + 128 * (size_t)sx;
  if (int rc = sisu::enqueue_layer_phases(hc, L, w, i, A, E, om, sx, offx, true, st)) return rc;
  const uint32_t nb = (uint32_t)hc.blocks[i].size();
  uint64_t mask = 0;
  for (uint32_t b = 0; b < nb; ++b)
    if (hc.blocks[i][b].layer < hc.d) mask |= 1ull << b;
  CK(launch_block_values(A, sx, cc->blk[i], nb, w.S, w.vals, st), "block values");
  CK(launch_block_absorb(w.vals, nb, mask, w.S, w.proof, offv, c, sx, w.hist + 8 * (size_t)i * w.hstride, st),
     "block absorb");
  off = offv + 64 * (size_t)nb;
  return SISU_OK;
}

// Libra's two phases (x, then y) and the end of gate layer i, from the
// copy-bound row A = V~_{i+1}(r_b, .) (general circuits: of the virtual
// layer) with gate weights om, the copy weight E[0] = 2^32 eq(z_b, r_b)
// and s = log2 of the row; the phases' messages start at proof offset offx.
// no_end: the layer's end (v_x, v_y, their transcript step, alpha, beta) is
// left to the caller.
int sisu::enqueue_layer_phases(const HostCircuit& hc, const DevLayer& L, Workspace& w, uint32_t i,
                               const uint32_t* A, const uint32_t* E, const uint32_t* om, uint32_t s, size_t offx,
                               bool no_end, cudaStream_t st) {
  const uint32_t d = hc.d, Wn = 1u << s;
  const size_t offy = offx + 32 * 2 * (size_t)s;
  const size_t offv = offy + 32 * 2 * (size_t)s;
  if (Wn <= kTailMaxWidth) {
    // Libra's two phases and the end of the layer in one cluster launch
    TailParams tp;
    tp.A = A; tp.E = E; tp.om = om; tp.sg = L.sgate;
    tp.off1 = L.off1; tp.pos1 = L.pos1; tp.off2 = L.off2; tp.pos2 = L.pos2;
    tp.nmul = L.nmul; tp.ntot = L.ntot; tp.Wn = Wn; tp.s = s; tp.P = w.P;
    tp.At = w.At; tp.H1 = w.H1; tp.H2 = w.H2; tp.Ay = w.Ay;
    tp.S = w.S; tp.proof = w.proof; tp.offx = offx; tp.offy = offy; tp.offv = offv; tp.last = i + 1 == d;
    tp.no_end = no_end;
    ProfScope ps(kProfGateRound, (double)Wn * (6.0 + s) + 2.0 * L.ntot, st);
    CK(launch_layer_tail(tp, st), "layer tail");
    return SISU_OK;
  }
  if (no_end) return fail(SISU_ERR_TOO_LARGE, "general layers wider than 2^16");
  // wide layers: one launch per round over the whole GPU
  {
    ProfScope ps(kProfPhaseInit, (double)L.ntot + 2.0 * Wn, st);
    CK(launch_xinit(A, E, om, L, Wn, w.At, w.H1, w.H2, w.Ay, st), "x init");
  }
  for (uint32_t k = 0; k < s; ++k) {
    ProfScope ps(kProfGateRound, (double)(Wn >> k) / 2 * (k ? 9.0 : 3.0), st);
    CK(launch_gate_round(w.At, w.H1, w.H2, Wn >> k, 0, k, w.partials, w.S, w.proof, offx + 64 * (size_t)k, st),
       "x round");
  }
  {
    ProfScope ps(kProfPhaseInit, (double)Wn * s + L.ntot + 3.0 * Wn, st);
    CK(launch_eq_rx(w.S, s, Wn, w.Q, w.At, st), "eq(r_x)");
    CK(launch_yinit(E, om, w.Q, L, Wn, w.H1, w.H2, w.S, st), "y init");
  }
  for (uint32_t k = 0; k < s; ++k) {
    ProfScope ps(kProfGateRound, (double)(Wn >> k) / 2 * (k ? 9.0 : 3.0), st);
    CK(launch_gate_round(w.Ay, w.H1, w.H2, Wn >> k, 1, k, w.partials, w.S, w.proof, offy + 64 * (size_t)k, st),
       "y round");
  }
  {
    ProfScope ps(kProfTranscript, 0, st);
    CK(launch_layer_end(w.S, w.Ay, s, w.proof, offv, i + 1 == d, st), "layer end");
  }
  return SISU_OK;
}

// One whole proof and the copies of its bytes and error word to pinned host
// memory, enqueued on `st` (no host wait).
int sisu::proof_enqueue(const sisu_circuit* cc, sisu_eval* ev, const sisu_transcript* tr, cudaStream_t st);
static int enqueue_proof_and_copy(const sisu_circuit* cc, sisu_eval* ev, const sisu_transcript* tr, cudaStream_t st) {
  Workspace& w = *ev->ws;
  const size_t n = cc->hc.proof_len();
  // the inputs' digest (outside a capture: launch_proof waits before the replay)
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  CK(cudaStreamIsCapturing(st, &cs), "capture status");
  if (cs == cudaStreamCaptureStatusNone && ev->dig_recorded) CK(cudaStreamWaitEvent(st, ev->dig_ev, 0), "stream wait");
  int rc = enqueue_prove(cc, ev, tr, st);
  if (rc) return rc;
  CK(cudaMemcpyAsync(w.host, w.proof, n, cudaMemcpyDeviceToHost, st), "proof copy");
  CK(cudaMemcpyAsync(w.host + ((n + 3) & ~(size_t)3), &w.S->error, 4, cudaMemcpyDeviceToHost, st), "flag copy");
  return SISU_OK;
}

static bool graphs_enabled() {
  static int on = -1;
  if (on < 0) {
    const char* e = getenv("SISU_NO_GRAPHS");
    on = (e && e[0] && e[0] != '0') ? 0 : 1;
  }
  return on == 1;
}

// Enqueue a proof on `st`: replay the workspace's graph (captured on the
// second proof of a handle, when every lazily initialised launch parameter
// is settled), or launch kernel by kernel while profiling or on the first
// proof.
static int launch_proof(const sisu_circuit* cc, sisu_eval* ev, const sisu_transcript* tr, cudaStream_t st) {
  Workspace& w = *ev->ws;
  const uint8_t* dom = tr ? tr->domain : (const uint8_t*)kDefaultDomain;
  const uint32_t dlen = tr ? tr->len : (uint32_t)strlen(kDefaultDomain);
  if (!graphs_enabled() || g_prof_mask != 0 || w.proofs++ == 0) return enqueue_proof_and_copy(cc, ev, tr, st);
  if (!w.gvalid || w.gdlen != dlen || memcmp(w.gdomain, dom, dlen) != 0) {
    if (w.exec) {
      cudaGraphExecDestroy(w.exec);
      w.exec = nullptr;
    }
    w.gvalid = false;
    if (!w.cap_stream) CK(cudaStreamCreateWithFlags(&w.cap_stream, cudaStreamNonBlocking), "stream create");
    CK(cudaStreamBeginCapture(w.cap_stream, cudaStreamCaptureModeThreadLocal), "graph capture");
    const uint64_t before = launches_add(0);
    int rc = enqueue_proof_and_copy(cc, ev, tr, w.cap_stream);
    // captured kernels are launched by each replay, not now
    w.graph_kernels = launches_add(0) - before;
    launches_add((uint64_t)0 - w.graph_kernels);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(w.cap_stream, &g);
    if (rc) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    if (e != cudaSuccess) return cuda_fail(e, "graph capture");
    e = cudaGraphInstantiate(&w.exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(e, "graph instantiate");
    memcpy(w.gdomain, dom, dlen);
    w.gdlen = dlen;
    w.gvalid = true;
  }
  if (ev->dig_recorded) CK(cudaStreamWaitEvent(st, ev->dig_ev, 0), "stream wait");
  CK(cudaGraphLaunch(w.exec, st), "graph launch");
  launches_add(w.graph_kernels);
  return SISU_OK;
}

int sisu::proof_enqueue(const sisu_circuit* cc, sisu_eval* ev, const sisu_transcript* tr, cudaStream_t st) {
  return enqueue_proof_and_copy(cc, ev, tr, st);
}

// After the proof's stream work completed: check the device error word and
// copy the bytes out.
static int finish_proof(const sisu_circuit* cc, sisu_eval* ev, uint8_t* proof) {
  Workspace& w = *ev->ws;
  const size_t n = cc->hc.proof_len();
  uint32_t err;
  memcpy(&err, w.host + ((n + 3) & ~(size_t)3), 4);
  if (err) return fail(SISU_ERR_CUDA, "device-side check failed (code %u)", err);
  memcpy(proof, w.host, n);
  return SISU_OK;
}

int sisu::proof_finish(const sisu_circuit* cc, sisu_eval* ev, uint8_t* proof) { return finish_proof(cc, ev, proof); }

static int prepare_proof(const sisu_circuit* circ, sisu_eval* ev, uint8_t* proof, size_t cap, size_t* proof_len) {
  if (!circ || !ev || !proof) return fail(SISU_ERR_INVALID_ARG, "NULL circuit, eval or proof buffer");
  if (ev->circ != circ) return fail(SISU_ERR_INVALID_ARG, "eval handle belongs to another circuit");
  const size_t n = circ->hc.proof_len();
  if (proof_len) *proof_len = n;
  if (cap < n) return fail(SISU_ERR_BUFFER, "proof buffer of %zu bytes, need %zu", cap, n);
  if (!ev->ws) {
    int rc = workspace_alloc(ev);
    if (rc) return rc;
  }
  return SISU_OK;
}

extern "C" int sisu_gkr_prove_into(const sisu_circuit* circ, sisu_eval* ev, const sisu_transcript* tr, void* stream,
                                   uint8_t* proof, size_t cap, size_t* proof_len) {
  int rc = prepare_proof(circ, ev, proof, cap, proof_len);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  rc = launch_proof(circ, ev, tr, st);
  if (rc) return rc;
  CK(cudaStreamSynchronize(st), "prove");
  return finish_proof(circ, ev, proof);
}

// ---------------------------------------------------------------------------
// batched proving: independent instances on concurrent streams

namespace {
std::mutex g_batch_mu;
std::vector<cudaStream_t> g_batch_streams[256];
std::vector<cudaEvent_t> g_batch_events[256];
}  // namespace

extern "C" int sisu_gkr_prove_batch(const sisu_circuit* const* circs, sisu_eval* const* evals, uint32_t n,
                                    const sisu_transcript* tr, void* stream, uint32_t concurrency,
                                    uint8_t* const* proofs, const size_t* caps, size_t* lens) {
  if (n == 0) return SISU_OK;
  if (!circs || !evals || !proofs || !caps) return fail(SISU_ERR_INVALID_ARG, "NULL array");
  for (uint32_t i = 0; i < n; ++i)
    for (uint32_t j = 0; j < i; ++j)
      if (evals[i] == evals[j]) return fail(SISU_ERR_INVALID_ARG, "eval handle %u appears twice in the batch", i);
  for (uint32_t i = 0; i < n; ++i) {
    int rc = prepare_proof(circs[i], evals[i], proofs[i], caps[i], lens ? &lens[i] : nullptr);
    if (rc) return rc;
  }
  const uint32_t K = std::max(1u, std::min(concurrency ? concurrency : 4u, 32u));
  int dev = 0;
  CK(cudaGetDevice(&dev), "cudaGetDevice");
  if (dev < 0 || dev >= 256) return fail(SISU_ERR_CUDA, "device ordinal %d", dev);
  std::lock_guard<std::mutex> lock(g_batch_mu);
  auto& pool = g_batch_streams[dev];
  auto& evs = g_batch_events[dev];
  while (pool.size() < K) {
    cudaStream_t s;
    CK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking), "stream create");
    pool.push_back(s);
    cudaEvent_t e;
    CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "event create");
    evs.push_back(e);
  }
  while (evs.size() < K + 1) {
    cudaEvent_t e;
    CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "event create");
    evs.push_back(e);
  }
  cudaStream_t st = (cudaStream_t)stream;
  // the pool streams start after the caller's prior work on `stream`
  CK(cudaEventRecord(evs[K], st), "event record");
  for (uint32_t k = 0; k < K; ++k) CK(cudaStreamWaitEvent(pool[k], evs[K], 0), "stream wait");
  for (uint32_t i = 0; i < n; ++i) {
    int rc = launch_proof(circs[i], evals[i], tr, pool[i % K]);
    if (rc) return rc;
  }
  // the caller's stream continues after every instance
  for (uint32_t k = 0; k < K; ++k) {
    CK(cudaEventRecord(evs[k], pool[k]), "event record");
    CK(cudaStreamWaitEvent(st, evs[k], 0), "stream wait");
  }
  CK(cudaStreamSynchronize(st), "prove batch");
  for (uint32_t i = 0; i < n; ++i) {
    int rc = finish_proof(circs[i], evals[i], proofs[i]);
    if (rc) return rc;
  }
  return SISU_OK;
}

extern "C" int sisu_gkr_prove(const sisu_circuit* circ, sisu_eval* ev, const sisu_transcript* tr, void* stream,
                              uint8_t** proof, size_t* proof_len) {
  if (!proof || !circ) return fail(SISU_ERR_INVALID_ARG, "NULL proof pointer or circuit");
  *proof = nullptr;
  const size_t n = circ->hc.proof_len();
  uint8_t* buf = (uint8_t*)malloc(n);
  if (!buf) return fail(SISU_ERR_OOM, "host allocation of %zu bytes", n);
  int rc = sisu_gkr_prove_into(circ, ev, tr, stream, buf, n, proof_len);
  if (rc) {
    free(buf);
    return rc;
  }
  *proof = buf;
  return SISU_OK;
}

extern "C" int sisu_gkr_verify(const sisu_circuit* circ, const uint8_t* inputs, const uint8_t* outputs,
                               const uint8_t* proof, size_t proof_len, const uint8_t* domain, size_t dlen) {
  if (!circ || !inputs || !outputs || !proof) return fail(SISU_ERR_INVALID_ARG, "NULL argument");
  if (dlen > kMaxDomain) return fail(SISU_ERR_INVALID_ARG, "domain longer than %u bytes", kMaxDomain);
  const uint8_t* dom = domain;
  size_t dl = dlen;
  if (!domain || dlen == 0) {
    dom = (const uint8_t*)kDefaultDomain;
    dl = strlen(kDefaultDomain);
  }
  int rc = host_verify(circ->hc, inputs, outputs, proof, proof_len, dom, dl);
  if (rc == SISU_ERR_REJECT) return fail(rc, "proof rejected");
  if (rc == SISU_ERR_NOT_CANONICAL) return fail(rc, "an input or output element is not below r");
  return rc;
}

// ---------------------------------------------------------------------------
// field core, digests, microbenchmarks

extern "C" int sisu_fr_batch(int op, const uint8_t* a, const uint8_t* b, uint8_t* out, size_t n, void* stream) {
  if (op < 0 || op > 8) return fail(SISU_ERR_INVALID_ARG, "op %d", op);
  if (!a || !out || (op != 3 && op != 7 && op != 8 && !b)) return fail(SISU_ERR_INVALID_ARG, "NULL operand");
  if (n == 0) return SISU_OK;
  if ((((uintptr_t)a | (uintptr_t)out | (uintptr_t)(b ? b : a)) & 15) != 0)
    return fail(SISU_ERR_INVALID_ARG, "device arrays must be 16-byte aligned");
  if (int rc = require_device(a, "a")) return rc;
  if (b && op != 3 && op != 7 && op != 8)
    if (int rc = require_device(b, "b")) return rc;
  if (int rc = require_device(out, "out")) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  uint32_t *flag = nullptr, host_flag = 0;
  CK(cudaMallocAsync(&flag, 4, st), "cudaMallocAsync");
  CK(cudaMemsetAsync(flag, 0, 4, st), "memset");
  int rc = launch_fr_batch(op, (const uint32_t*)a, (const uint32_t*)(b ? b : a), (uint32_t*)out, n, flag, st);
  if (rc == 0) rc = cudaMemcpyAsync(&host_flag, flag, 4, cudaMemcpyDeviceToHost, st);
  cudaFreeAsync(flag, st);
  cudaError_t e = cudaStreamSynchronize(st);
  if (rc) return cuda_fail((cudaError_t)rc, "field op");
  if (e) return cuda_fail(e, "field op");
  if (host_flag & 1u) return fail(SISU_ERR_NOT_CANONICAL, "an operand is not below r");
  if (host_flag & 2u) return fail(SISU_ERR_ZERO_INVERSE, "inverse of zero");
  return SISU_OK;
}

extern "C" int sisu_statement_digest(const uint8_t* data, size_t len, uint8_t* out, void* stream) {
  if (!out || (len && !data)) return fail(SISU_ERR_INVALID_ARG, "NULL argument");
  if (len)
    if (int rc = require_device(data, "data")) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t words = digest_scratch_words(len) + 8;
  uint32_t* scratch = nullptr;
  CK(cudaMallocAsync(&scratch, words * 4, st), "cudaMallocAsync");
  uint32_t h[8];
  int rc = launch_digest_bytes(data, len, scratch, scratch + words - 8, st);
  if (rc == 0) rc = cudaMemcpyAsync(h, scratch + words - 8, 32, cudaMemcpyDeviceToHost, st);
  cudaFreeAsync(scratch, st);
  cudaError_t e = cudaStreamSynchronize(st);
  if (rc) return cuda_fail((cudaError_t)rc, "digest");
  if (e) return cuda_fail(e, "digest");
  for (int i = 0; i < 8; ++i) {
    out[4 * i] = (uint8_t)(h[i] >> 24); out[4 * i + 1] = (uint8_t)(h[i] >> 16);
    out[4 * i + 2] = (uint8_t)(h[i] >> 8); out[4 * i + 3] = (uint8_t)h[i];
  }
  return SISU_OK;
}

extern "C" int sisu_microbench(int kind, uint32_t blocks, uint32_t threads, uint32_t iters, void* stream, double* ms,
                               double* ops) {
  if (kind < 0 || kind > 16 || !blocks || !threads || threads > 1024 || !ms || !ops)
    return fail(SISU_ERR_INVALID_ARG, "bad microbenchmark arguments");
  int rc = run_microbench(kind, blocks, threads, iters, stream, ms, ops);
  if (rc) return cuda_fail((cudaError_t)rc, "microbenchmark");
  return SISU_OK;
}

extern "C" int sisu_tune_copy_round(uint32_t log_width, uint32_t log_pairs, uint32_t cta_threads, uint32_t form,
                                    uint32_t min_items) {
  if (set_copy_tune(log_width, log_pairs, cta_threads, form, min_items))
    return fail(SISU_ERR_INVALID_ARG, "copy-round tuning entry out of range");
  return SISU_OK;
}

extern "C" uint64_t sisu_kernel_launches(void) { return launches_add(0); }
extern "C" void sisu_free(void* p) { free(p); }
extern "C" const char* sisu_last_error(void) { return g_err; }
extern "C" const char* sisu_version(void) { return "sisu-b300 0.1 (sm_103a)"; }
