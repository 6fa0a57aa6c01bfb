// api.cu -- the C ABI (include/gbpir.h): parameter checks, resident-DB registry,
// admission by free device memory, and the answer pipeline
//   queries --NTT--> NTT form --transpose--> slot-major --modular GEMM--> slot-major
//   results --transpose--> responses (NTT form) --INTT--> responses
// (Sec. 3.2 poly-HE folding; Sec. 4.2 transposes around the parallel GEMMs;
// Sec. 4.4 per-stream fixed buffers -> the K-chunked variant here).
#include <atomic>
#include <map>
#include <mutex>
#include <set>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "common.cuh"

namespace {
// An NVTX range around one call of a public entry point, so that a profiler can
// select or group the launches of one answer (free when no tool is attached).
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};
}  // namespace

namespace gbpir {

namespace {
thread_local std::string t_last_cuda;
}

void set_cuda_error(cudaError_t e) { t_last_cuda = cudaGetErrorString(e); }
const char *last_cuda_error_cstr() { return t_last_cuda.c_str(); }

std::atomic<uint64_t> g_launches{0};

namespace {
std::mutex g_err_mu;
uint32_t *g_err_word[64] = {};
}  // namespace

cudaError_t device_error_word(uint32_t **word) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_err_mu);
  if (!g_err_word[dev]) {
    uint32_t *w = nullptr;
    if ((e = cudaMalloc(&w, sizeof(uint32_t))) != cudaSuccess) return e;
    if ((e = cudaMemset(w, 0, sizeof(uint32_t))) != cudaSuccess) return e;
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) return e;
    g_err_word[dev] = w;
  }
  *word = g_err_word[dev];
  return cudaSuccess;
}
void count_launches(uint64_t k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

pir_status_t cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return PIR_OK;
  set_cuda_error(e);
  if (e == cudaErrorMemoryAllocation) return PIR_ERR_OOM;
  return PIR_ERR_CUDA;
}

}  // namespace gbpir

using namespace gbpir;

struct pir_db {
  uint64_t magic;
  pir_params_t p;
  int layout;
  int device;
  const ParamCtx *ctx;
  void *resident;
  size_t bytes;
  std::mutex tune_mu;
  std::map<uint32_t, pir_answer_opts_t> tuned;  // batch size -> fastest options
};

// A streamed answer (pir_answer_begin): device scratch for one piece of at most
// kc_max ciphertexts per query, the slot-major result that the pieces accumulate
// into, and two staging buffers for pieces given in host memory.
struct pir_session {
  uint64_t magic;
  pir_db *db;
  cudaStream_t s;
  uint32_t B, kc_max, next, pieces;
  pir_answer_opts_t o;
  pir_status_t failed;
  void *mem;        // qhat | qs | out
  void *stage_mem;  // two host-piece staging buffers, allocated with the first host piece
  size_t qhat_bytes, qs_bytes, stage_bytes;
  cudaEvent_t arrived[2], consumed[2];
};

struct pir_graph {
  uint64_t magic;
  pir_db *db;
  cudaGraph_t graph;
  cudaGraphExec_t exec;
  uint64_t kernels;             // kernel launches per replay
  pir_expander_t expander;      // the expansion keys a packed-query graph reads, or null
  int device;                   // where its scratch memory lives
};

namespace {

constexpr uint64_t kMagic = 0x4742504952444231ull;       // "GBPIRDB1"
constexpr uint64_t kGraphMagic = 0x4742504952475231ull;  // "GBPIRGR1"
std::mutex g_reg_mu;
std::set<pir_db *> g_live;
std::set<pir_graph *> g_graphs;
std::set<pir_session *> g_sessions;
constexpr uint64_t kSessionMagic = 0x4742504952535331ull;  // "GBPIRSS1"

bool session_live(pir_session *ses) {
  std::lock_guard<std::mutex> lock(g_reg_mu);
  return ses && g_sessions.count(ses) && ses->magic == kSessionMagic;
}
// removes the session from the registry; false if it was not live
bool session_take(pir_session *ses) {
  std::lock_guard<std::mutex> lock(g_reg_mu);
  if (!ses || !g_sessions.count(ses)) return false;
  g_sessions.erase(ses);
  return true;
}

bool live(pir_db *db) {
  std::lock_guard<std::mutex> lock(g_reg_mu);
  return db && g_live.count(db) && db->magic == kMagic;
}

bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

#define CK(expr)                                   \
  do {                                             \
    cudaError_t e_ = (expr);                       \
    if (e_ != cudaSuccess) return cuda_status(e_); \
  } while (0)

// Gives the device memory back that the library keeps cached but unused: freed
// scratch in the stream-ordered pool (whose release threshold keeps it) and the
// graph memory pool's.  Called before an allocation or a graph launch is refused.
void release_cached_memory() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) cudaMemPoolTrimTo(pool, 0);
  cudaDeviceGraphMemTrim(dev);
}

thread_local bool t_capturing = false;  // launches inside a graph capture are not launches yet

// cudaMallocAsync, retried once after the cached memory has been given back.
cudaError_t malloc_async_retry(void **ptr, size_t bytes, cudaStream_t s) {
  cudaError_t e = cudaMallocAsync(ptr, bytes, s);
  if (e == cudaErrorMemoryAllocation && !t_capturing) {
    cudaGetLastError();
    release_cached_memory();
    e = cudaMallocAsync(ptr, bytes, s);
  }
  return e;
}

// Device scratch drawn from the stream-ordered allocator; freed (stream-ordered)
// when the guard goes out of scope.
struct Scratch {
  void *ptr = nullptr;
  cudaStream_t s;
  explicit Scratch(cudaStream_t st) : s(st) {}
  cudaError_t alloc(size_t bytes) { return malloc_async_retry(&ptr, bytes, s); }
  ~Scratch() {
    if (ptr) cudaFreeAsync(ptr, s);
  }
};

size_t resident_bytes(const pir_params_t &p, int layout) {
  return (size_t)(layout == PIR_LAYOUT_TENSOR ? 8 : 4) * p.L * p.n * p.D1 * p.D2;
}
size_t raw_bytes_of(const pir_params_t &p) { return (size_t)p.D1 * p.D2 * p.n * p.log2p / 8; }

uint32_t round4(uint32_t x) { return (x + 3u) & ~3u; }

// Per-layout rules of the GEMM paths.  Padded query rows: plain 4 (128-bit loads),
// limb 16 (m16 tensor tiles), tensor 8 (8-row core matrices).
uint32_t layout_rows(int layout, uint32_t M) {
  return layout == PIR_LAYOUT_LIMB ? (M + 15u) & ~15u : layout == PIR_LAYOUT_TENSOR ? tc_rows(M) : round4(M);
}
// The K-chunk a layout takes: limb 32-row blocks up to 8192 (byte-limb class sums stay
// below 2^31), tensor 64-row blocks up to 1024 (f32 sums of digit products stay exact).
uint32_t layout_chunk(int layout, uint32_t Kc) {
  if (layout == PIR_LAYOUT_LIMB) {
    if (Kc > 8192) Kc = 8192;
    Kc &= ~31u;
    return Kc ? Kc : 32;
  }
  if (layout == PIR_LAYOUT_TENSOR) {
    if (Kc > 1024) Kc = 1024;
    Kc &= ~63u;
    return Kc ? Kc : 64;
  }
  return Kc ? Kc : 1;
}
// bytes of the chunk's GEMM-layout query copy: u32 slots, four u8 limb planes, or
// four bf16 digits
size_t layout_qs_bytes(int layout, uint64_t nslots, uint32_t Kc, uint32_t Mp) {
  return (size_t)nslots * Kc * Mp * (layout == PIR_LAYOUT_TENSOR ? 8 : 4);
}
uint32_t layout_tiles(int layout) {
  return layout == PIR_LAYOUT_PLAIN ? gemm_plain_tiles() : layout == PIR_LAYOUT_LIMB ? gemm_limb_tiles()
                                                                                   : gemm_tc_tiles();
}
bool layout_tile_ok(int layout, uint32_t tile, uint32_t M, uint32_t Mp, uint32_t D2) {
  if (layout == PIR_LAYOUT_PLAIN) return gemm_plain_tile_ok(tile, M, D2);
  if (layout == PIR_LAYOUT_LIMB) return gemm_limb_tile_ok(tile, Mp);
  return gemm_tc_tile_ok(tile, Mp, D2);
}

// Keep the pool's memory once freed: repeated answers then reuse it instead of
// returning it to the driver every call.
void keep_pool_memory(int dev) {
  static std::once_flag once;
  std::call_once(once, [dev]() {
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
      uint64_t thr = ~0ull;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
  });
}

// Device memory an allocation can draw on: free memory plus what the stream-ordered
// pool holds reserved but unused (its release threshold keeps freed scratch).
size_t available_device_bytes(int dev) {
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return 0;
  cudaMemPool_t pool;
  uint64_t reserved = 0, used = 0;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess &&
      cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &reserved) == cudaSuccess &&
      cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used) == cudaSuccess && reserved > used)
    free_b += (size_t)(reserved - used);
  return free_b;
}

// Optional per-stage timing: a pair of events around every stage invocation.
struct StageMark {
  int stage;
  uint64_t launches;
  cudaEvent_t a, b;
};
thread_local std::vector<StageMark> t_marks;
thread_local std::vector<cudaEvent_t> t_free_events;

cudaEvent_t take_event() {
  if (!t_free_events.empty()) {
    cudaEvent_t e = t_free_events.back();
    t_free_events.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}


// Arrival of the query upload in pieces of kc ciphertexts (host-buffer answers): ev[k]
// is recorded on the copy stream after piece k's copies; a forward NTT over
// ciphertexts [i0, i0 + cnt) waits on every piece it touches.
constexpr uint32_t kMaxFeedChunks = 16;
struct ChunkFeed {
  uint32_t n = 0, kc = 0;
  cudaEvent_t ev[kMaxFeedChunks] = {};
  cudaError_t wait(cudaStream_t s, uint32_t i0, uint32_t cnt) const {
    if (n == 0 || cnt == 0) return cudaSuccess;
    const uint32_t last = (i0 + cnt - 1) / kc;
    for (uint32_t k = i0 / kc; k <= last && k < n; ++k) {
      cudaError_t e = cudaStreamWaitEvent(s, ev[k], 0);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
};
thread_local cudaStream_t t_copy_stream = nullptr;
cudaError_t copy_stream(cudaStream_t *out) {
  if (!t_copy_stream) {
    cudaError_t e = cudaStreamCreateWithFlags(&t_copy_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return e;
  }
  *out = t_copy_stream;
  return cudaSuccess;
}
// the device-to-host direction, so that downloads overlap the uploads
thread_local cudaStream_t t_d2h_stream = nullptr;
cudaError_t d2h_stream(cudaStream_t *out) {
  if (!t_d2h_stream) {
    cudaError_t e = cudaStreamCreateWithFlags(&t_d2h_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return e;
  }
  *out = t_d2h_stream;
  return cudaSuccess;
}

struct StageTimer {
  bool on;
  cudaStream_t s;
  cudaEvent_t a = nullptr;
  StageTimer(bool enable, cudaStream_t st) : on(enable), s(st) {}
  void begin() {
    if (on && (a = take_event())) cudaEventRecord(a, s);
  }
  void end(int stage, uint64_t launches) {
    if (!t_capturing) count_launches(launches);
    if (!on || !a) return;
    cudaEvent_t b = take_event();
    if (!b) return;
    cudaEventRecord(b, s);
    t_marks.push_back({stage, launches, a, b});
    a = nullptr;
  }
};

// One K-chunk on the DB's GEMM path: the NTT-form chunk qhat [B][kc][2][L][n] to
// the layout's query copy qs, then the GEMM accumulated into out [L*n][M][D2].
pir_status_t chunk_gemm(const pir_db *db, const uint32_t *qhat, uint32_t B, uint32_t Mp, uint32_t i0, uint32_t kc,
                        void *qs, uint32_t *out, uint32_t tile, int stall, StageTimer &tm, cudaStream_t s) {
  const ParamCtx &c = *db->ctx;
  const uint32_t D1 = db->p.D1, D2 = db->p.D2, M = 2 * B;
  tm.begin();
  if (db->layout == PIR_LAYOUT_PLAIN)
    CK(launch_query_to_slots(c, qhat, B, kc, Mp, static_cast<uint32_t *>(qs), s));
  else if (db->layout == PIR_LAYOUT_LIMB)
    CK(launch_query_to_limbs(c, qhat, B, kc, Mp, static_cast<uint8_t *>(qs), s));
  else
    CK(launch_query_to_tensor(c, qhat, B, kc, Mp, static_cast<uint16_t *>(qs), s));
  tm.end(1, 1);
  tm.begin();
  if (db->layout == PIR_LAYOUT_PLAIN)
    CK(launch_gemm_plain(c, static_cast<const uint32_t *>(db->resident), D1, D2, static_cast<const uint32_t *>(qs), M,
                         Mp, i0, kc, out, i0 > 0, tile, stall, s));
  else if (db->layout == PIR_LAYOUT_LIMB)
    CK(launch_gemm_limb(c, static_cast<const uint8_t *>(db->resident), D1, D2, static_cast<const uint8_t *>(qs), M, Mp,
                        i0, kc, out, i0 > 0, tile, s));
  else
    CK(launch_gemm_tc(c, static_cast<const uint16_t *>(db->resident), D1, D2, static_cast<const uint16_t *>(qs), M,
                      Mp, i0, kc, out, i0 > 0, tile, s));
  tm.end(2, 1);
  return PIR_OK;
}

// The device-buffer answer (stream ordered).
// qhat_ready: when set, the queries are already in NTT form for the whole of D1
// ([B][D1][2][L][n], e.g. from query expansion): no forward NTT, no K-chunking.
// ntt_out: leave the responses in NTT form (no inverse NTT, no modulus switching),
// for the folding of the remaining dimensions.
constexpr uint32_t kMinAutoChunk = 512;  // rows: shorter automatic K-chunks starve the GEMMs

pir_status_t answer_device(pir_db *db, const uint32_t *queries, uint32_t B, uint32_t *responses, cudaStream_t s,
                           const pir_answer_opts_t &o, const uint32_t *qhat_ready = nullptr, bool ntt_out = false,
                           const ChunkFeed *feed = nullptr) {
  const ParamCtx &c = *db->ctx;
  const pir_params_t &p = db->p;
  const uint32_t n = p.n, L = p.L, D1 = p.D1, D2 = p.D2;
  const bool plain = db->layout == PIR_LAYOUT_PLAIN;
  const uint32_t M = 2 * B;
  const uint32_t Mp = layout_rows(db->layout, M);
  uint32_t Kc = (o.k_chunk == 0 || o.k_chunk >= D1 || qhat_ready) ? D1 : o.k_chunk;
  if (o.k_chunk == 0 && !qhat_ready) {
    // Stream-wise buffering (Sec. 4.4): when the scratch for all of D1 would not fit
    // half of the available device memory (free, plus what the stream-ordered pool
    // keeps cached), fold D1 in as many equal chunks as needed; never in chunks
    // shorter than kMinAutoChunk rows, below which the GEMM launches stop filling the
    // GPU (a scratch allocation that then does not fit is refused with PIR_ERR_OOM,
    // after the cached memory has been given back).
    const size_t avail = available_device_bytes(db->device);
    if (avail > 0) {
      const size_t per_row = (size_t)B * 2 * L * n * 4 + layout_qs_bytes(db->layout, (uint64_t)L * n, 1, Mp);
      const size_t budget = avail / 2;
      if ((size_t)D1 * per_row > budget && per_row > 0) {
        const size_t rows = budget / per_row;
        const uint32_t chunks = (uint32_t)((D1 + (rows ? rows : 1) - 1) / (rows ? rows : 1));
        Kc = (D1 + chunks - 1) / chunks;
        const uint32_t floor = D1 < kMinAutoChunk ? D1 : kMinAutoChunk;
        if (Kc < floor) Kc = floor;
      }
    }
  }
  if (!plain) {
    Kc = layout_chunk(db->layout, Kc);
    if (qhat_ready && Kc < D1) return PIR_ERR_UNSUPPORTED;
  }
  const uint64_t nslots = (uint64_t)L * n;
  if (o.tile > layout_tiles(db->layout) ||
      (o.flags & ~(PIR_ANSWER_STAGE_TIMES | PIR_ANSWER_TEST_STALL | PIR_ANSWER_MODSWITCH |
                   PIR_ANSWER_CHECK_INPUTS)) != 0)
    return PIR_ERR_ARG;
  if (!layout_tile_ok(db->layout, o.tile, M, Mp, D2)) return PIR_ERR_ARG;
  if ((o.flags & PIR_ANSWER_CHECK_INPUTS) && !qhat_ready) {
    // every query residue canonical (below its prime) before anything is computed
    Scratch chk(s);
    CK(chk.alloc(sizeof(uint32_t)));
    CK(cudaMemsetAsync(chk.ptr, 0, sizeof(uint32_t), s));
    CK(launch_check_residues(c, queries, (uint64_t)B * D1 * 2 * L, static_cast<uint32_t *>(chk.ptr), s));
    uint32_t bad = 0;
    CK(cudaMemcpyAsync(&bad, chk.ptr, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    count_launches(1);
    if (bad) return PIR_ERR_ARG;
  }
  // With modulus switching the inverse NTT reads the full-modulus responses from
  // scratch and writes [B][D2][2][n] over q_0 to `responses`.
  const bool msw = (o.flags & PIR_ANSWER_MODSWITCH) != 0 && !ntt_out;
  const int stall = (o.flags & PIR_ANSWER_TEST_STALL) != 0;
  if (stall && (db->layout != PIR_LAYOUT_PLAIN || !scan_tma_supports(2 * B, D2) || (o.tile != 0 && o.tile != 7)))
    return PIR_ERR_ARG;

  // scratch: NTT'd query chunk | slot-major query chunk | slot-major results
  const size_t qhat_bytes = qhat_ready ? 0 : (size_t)B * Kc * 2 * L * n * 4;
  const size_t qs_bytes = layout_qs_bytes(db->layout, nslots, Kc, Mp);
  const size_t out_bytes = nslots * M * D2 * 4;
  auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
  // Batch 1 on the TMA scan: the forward NTT writes the slot layout itself (pairs of
  // a/b residues, Mp = 2) and the scan writes the response layout itself, so neither
  // transpose runs.
  // (every chunk, the last included, must hold an even number of ciphertexts)
  const bool fused = !qhat_ready && plain && B == 1 && (o.tile == 0 || o.tile == 7) && scan_tma_supports(M, D2) &&
                     Kc % 2 == 0 && D1 % 2 == 0;
  // full-modulus responses before switching: the unused result area on the fused
  // path (the same size at B = 1), an area of their own otherwise
  StageTimer tm((o.flags & PIR_ANSWER_STAGE_TIMES) != 0, s);
  const size_t full_bytes = (msw && !fused) ? (size_t)B * D2 * 2 * L * n * 4 : 0;
  // K-chunked fused path: the chunks before the last accumulate slot-major here
  const size_t slot_bytes = (fused && Kc < D1) ? out_bytes : 0;
  Scratch scratch(s);
  CK(scratch.alloc(up(qhat_bytes) + up(qs_bytes) + up(out_bytes) + up(full_bytes) + up(slot_bytes)));
  char *base = static_cast<char *>(scratch.ptr);
  const uint32_t *qhat = qhat_ready ? qhat_ready : reinterpret_cast<uint32_t *>(base);
  void *qs = base + up(qhat_bytes);
  uint32_t *out = reinterpret_cast<uint32_t *>(base + up(qhat_bytes) + up(qs_bytes));
  uint32_t *slotbuf = reinterpret_cast<uint32_t *>(base + up(qhat_bytes) + up(qs_bytes) + up(out_bytes) +
                                                   up(full_bytes));
  uint32_t *full = !msw ? responses
                        : fused ? out : reinterpret_cast<uint32_t *>(base + up(qhat_bytes) + up(qs_bytes) + up(out_bytes));
  auto finish = [&]() -> pir_status_t {  // inverse NTT (with the switch when asked)
    if (ntt_out) return PIR_OK;
    tm.begin();
    if (msw)
      CK(launch_ntt_inv_switch(c, full, responses, (uint64_t)B * D2 * 2, s));
    else
      CK(launch_ntt_inv(c, responses, responses, (uint64_t)B * D2 * 2 * L, s));
    tm.end(4, 1);
    return PIR_OK;
  };

  if (fused) {
    uint32_t *qs2 = reinterpret_cast<uint32_t *>(base);  // [L*n][Kc][2] fits the qhat area
    for (uint32_t i0 = 0; i0 < D1; i0 += Kc) {
      const uint32_t kc = D1 - i0 < Kc ? D1 - i0 : Kc;
      tm.begin();
      uint64_t nl = 1;
      if (feed && feed->n > 1 && Kc == D1) {
        // one scan pass; the forward NTT follows the upload piece by piece
        nl = 0;
        for (uint32_t p0 = 0; p0 < D1; p0 += feed->kc, ++nl) {
          const uint32_t pc = D1 - p0 < feed->kc ? D1 - p0 : feed->kc;
          CK(feed->wait(s, p0, pc));
          CK(launch_ntt_fwd_pair_slots(c, queries, p0, pc, D1, p0, qs2, s));
        }
      } else {
        if (feed) CK(feed->wait(s, i0, kc));
        CK(launch_ntt_fwd_pair_slots(c, queries, i0, kc, kc, 0, qs2, s));
      }
      tm.end(0, nl);
      tm.begin();
      // single pass: straight to the response layout; several K-chunks: slot-major
      // accumulation, and the last chunk adds it in while writing the response layout
      const bool last = i0 + kc >= D1;
      CK(launch_scan_tma(c, static_cast<const uint32_t *>(db->resident), D1, D2, qs2, M, 2, i0, kc,
                         last ? full : slotbuf, !last && i0 > 0, stall, last ? 1 : 0, (last && i0 > 0) ? slotbuf : nullptr,
                         s));
      tm.end(2, 1);
    }
    return finish();
  }
  for (uint32_t i0 = 0; i0 < D1; i0 += Kc) {
    const uint32_t kc = D1 - i0 < Kc ? D1 - i0 : Kc;
    if (feed) CK(feed->wait(s, i0, kc));
    // forward NTT of ciphertexts i0 .. i0+kc-1 of every query: per query b the rows
    // (b*D1 + i0)*2L .. +kc*2L are contiguous.
    const uint64_t G = (uint64_t)kc * 2 * L, S = (uint64_t)D1 * 2 * L;
    if (!qhat_ready) {
      tm.begin();
      CK(launch_ntt_fwd_rows(c, queries, (uint64_t)i0 * 2 * L, G, S, const_cast<uint32_t *>(qhat), (uint64_t)B * G,
                             s));
      tm.end(0, 1);
    }
    const pir_status_t st = chunk_gemm(db, qhat, B, Mp, i0, kc, qs, out, o.tile, stall, tm, s);
    if (st != PIR_OK) return st;
  }
  tm.begin();
  CK(launch_slots_to_responses(c, out, B, D2, full, s));
  tm.end(3, 1);
  return finish();
}

}  // namespace

namespace gbpir {
bool db_view(pir_db_t db, DbView *out) {
  if (!live(db) || !out) return false;
  out->p = db->p;
  out->layout = db->layout;
  out->ctx = db->ctx;
  out->resident = db->resident;
  return true;
}
}  // namespace gbpir

namespace {

// Ciphertexts i0 .. i0+kc-1 of every query, query b's at src + b * stride (words):
// forward NTT, transpose to the GEMM layout, modular GEMM accumulated into the
// session's slot-major result.  Host pieces go through a staging buffer on the copy
// stream; the call returns once that copy has completed.
pir_status_t session_piece(pir_session *ses, const uint32_t *src, uint64_t stride, uint32_t i0, uint32_t kc,
                           bool on_device) {
  pir_db *db = ses->db;
  const ParamCtx &c = *db->ctx;
  const pir_params_t &p = db->p;
  const cudaStream_t s = ses->s;
  const uint32_t B = ses->B, L = p.L, n = p.n, M = 2 * B;
  const uint32_t Mp = layout_rows(db->layout, M);
  const uint64_t ct = 2ull * L * n, G = (uint64_t)kc * 2 * L;
  auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
  char *base = static_cast<char *>(ses->mem);
  uint32_t *qhat = reinterpret_cast<uint32_t *>(base);
  void *qs = base + up(ses->qhat_bytes);
  uint32_t *out = reinterpret_cast<uint32_t *>(base + up(ses->qhat_bytes) + up(ses->qs_bytes));
  const uint32_t slot = ses->pieces & 1;
  uint64_t row_stride = stride / n;  // rows of n words
  if (!on_device) {
    if (!ses->stage_mem) {
      CK(malloc_async_retry(&ses->stage_mem, 2 * ses->stage_bytes, s));
      // the copy stream touches the staging memory only after its allocation
      CK(cudaEventRecord(ses->consumed[0], s));
      CK(cudaEventRecord(ses->consumed[1], s));
    }
    cudaStream_t cs = nullptr;
    CK(copy_stream(&cs));
    uint32_t *stage = reinterpret_cast<uint32_t *>(static_cast<char *>(ses->stage_mem) + slot * ses->stage_bytes);
    CK(cudaStreamWaitEvent(cs, ses->consumed[slot], 0));  // the piece before last has been read
    if (stride == kc * ct) {
      CK(cudaMemcpyAsync(stage, src, (size_t)B * kc * ct * 4, cudaMemcpyHostToDevice, cs));
    } else {
      for (uint32_t b = 0; b < B; ++b)
        CK(cudaMemcpyAsync(stage + b * kc * ct, src + b * stride, kc * ct * 4, cudaMemcpyHostToDevice, cs));
    }
    CK(cudaEventRecord(ses->arrived[slot], cs));
    CK(cudaStreamWaitEvent(s, ses->arrived[slot], 0));
    src = stage;
    row_stride = G;
  }
  StageTimer tm((ses->o.flags & PIR_ANSWER_STAGE_TIMES) != 0, s);
  tm.begin();
  CK(launch_ntt_fwd_rows(c, src, 0, G, row_stride, qhat, (uint64_t)B * G, s));
  tm.end(0, 1);
  if (!on_device) CK(cudaEventRecord(ses->consumed[slot], s));
  const pir_status_t st = chunk_gemm(db, qhat, B, Mp, i0, kc, qs, out, ses->o.tile, 0, tm, s);
  if (st != PIR_OK) return st;
  if (!on_device) CK(cudaEventSynchronize(ses->arrived[slot]));  // the caller's buffer is free again
  return PIR_OK;
}

// The slot-major result to responses: transpose, inverse NTT (with the switch to
// q_0 when asked), and for host responses the copy out.  Synchronous for host.
pir_status_t session_finish(pir_session *ses, uint32_t *responses, bool on_device) {
  pir_db *db = ses->db;
  const ParamCtx &c = *db->ctx;
  const pir_params_t &p = db->p;
  const cudaStream_t s = ses->s;
  const uint32_t B = ses->B, L = p.L, n = p.n, D2 = p.D2;
  const bool msw = (ses->o.flags & PIR_ANSWER_MODSWITCH) != 0;
  auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const uint32_t *out = reinterpret_cast<const uint32_t *>(static_cast<char *>(ses->mem) + up(ses->qhat_bytes) +
                                                           up(ses->qs_bytes));
  const size_t full_bytes = (size_t)B * D2 * 2 * L * n * 4, rbytes = (size_t)B * D2 * 2 * (msw ? 1 : L) * n * 4;
  // full-modulus responses: in `responses` itself unless switched or on the host;
  // the final responses: device staging for host buffers
  Scratch scr(s);
  CK(scr.alloc((msw ? up(full_bytes) : 0) + (on_device ? 0 : up(rbytes))));
  char *sb = static_cast<char *>(scr.ptr);
  uint32_t *dst = on_device ? responses : reinterpret_cast<uint32_t *>(sb + (msw ? up(full_bytes) : 0));
  uint32_t *full = msw ? reinterpret_cast<uint32_t *>(sb) : dst;
  StageTimer tm((ses->o.flags & PIR_ANSWER_STAGE_TIMES) != 0, s);
  tm.begin();
  CK(launch_slots_to_responses(c, out, B, D2, full, s));
  tm.end(3, 1);
  tm.begin();
  if (msw)
    CK(launch_ntt_inv_switch(c, full, dst, (uint64_t)B * D2 * 2, s));
  else
    CK(launch_ntt_inv(c, dst, dst, (uint64_t)B * D2 * 2 * L, s));
  tm.end(4, 1);
  if (!on_device) {
    CK(cudaMemcpyAsync(responses, dst, rbytes, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
  }
  return PIR_OK;
}

void session_release(pir_session *ses) {
  if (ses->mem) cudaFreeAsync(ses->mem, ses->s);
  if (ses->stage_mem) cudaFreeAsync(ses->stage_mem, ses->s);  // every copy was waited for on s
  for (int k = 0; k < 2; ++k) {
    if (ses->arrived[k]) cudaEventDestroy(ses->arrived[k]);
    if (ses->consumed[k]) cudaEventDestroy(ses->consumed[k]);
  }
  ses->magic = 0;
  delete ses;
}

pir_status_t session_open(pir_db *db, uint32_t B, uint32_t kc_max, cudaStream_t s, const pir_answer_opts_t &o,
                          pir_session **out) {
  const pir_params_t &p = db->p;
  if (o.k_chunk != 0 || (o.flags & ~(PIR_ANSWER_STAGE_TIMES | PIR_ANSWER_MODSWITCH)) != 0) return PIR_ERR_ARG;
  const uint32_t M = 2 * B, Mp = layout_rows(db->layout, M);
  if (o.tile > layout_tiles(db->layout) || !layout_tile_ok(db->layout, o.tile, M, Mp, p.D2)) return PIR_ERR_ARG;
  if (kc_max > p.D1) kc_max = p.D1;
  if (db->layout != PIR_LAYOUT_PLAIN) kc_max = layout_chunk(db->layout, kc_max);  // whole blocks, bounded pieces
  const uint64_t nslots = (uint64_t)p.L * p.n, ct = 2ull * p.L * p.n;
  auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
  pir_session *ses = new pir_session{};
  ses->magic = kSessionMagic;
  ses->db = db;
  ses->s = s;
  ses->B = B;
  ses->kc_max = kc_max;
  ses->o = o;
  ses->failed = PIR_OK;
  ses->qhat_bytes = (size_t)B * kc_max * ct * 4;
  ses->qs_bytes = layout_qs_bytes(db->layout, nslots, kc_max, Mp);
  ses->stage_bytes = up(ses->qhat_bytes);
  const size_t out_bytes = nslots * M * p.D2 * 4;
  void *mem = nullptr;
  cudaError_t e = malloc_async_retry(&mem, up(ses->qhat_bytes) + up(ses->qs_bytes) + up(out_bytes), s);
  if (e == cudaSuccess) ses->mem = mem;
  for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
    if ((e = cudaEventCreateWithFlags(&ses->arrived[k], cudaEventDisableTiming)) == cudaSuccess)
      e = cudaEventCreateWithFlags(&ses->consumed[k], cudaEventDisableTiming);
  }
  if (e != cudaSuccess) {
    session_release(ses);  // whatever was made
    return cuda_status(e);
  }
  {
    std::lock_guard<std::mutex> lock(g_reg_mu);
    g_sessions.insert(ses);
  }
  *out = ses;
  return PIR_OK;
}

// One piece, checked: in order, within kc_max and D1, whole 32-row blocks on the limb
// layout and whole 64-row blocks on the tensor layout.
pir_status_t session_chunk(pir_session *ses, const uint32_t *src, uint64_t stride, uint32_t i0, uint32_t kc,
                           bool on_device) {
  if (ses->failed != PIR_OK) return ses->failed;
  const pir_params_t &p = ses->db->p;
  if (!src || kc == 0 || kc > ses->kc_max || i0 != ses->next || (uint64_t)i0 + kc > p.D1) return PIR_ERR_ARG;
  if (ses->db->layout != PIR_LAYOUT_PLAIN && layout_chunk(ses->db->layout, kc) != kc) return PIR_ERR_ARG;
  if (on_device && !aligned16(src)) return PIR_ERR_ARG;
  const pir_status_t st = session_piece(ses, src, stride, i0, kc, on_device);
  if (st != PIR_OK) {
    ses->failed = st;
    return st;
  }
  ses->next += kc;
  ses->pieces += 1;
  return PIR_OK;
}

}  // namespace

namespace {
// Captures body(stream) on a private stream into an instantiated graph bound to db
// (and to the expander, for packed queries).
template <typename Body>
pir_status_t capture_graph(pir_db *db, pir_expander_t expander, Body body, pir_graph_t *out) {
  *out = nullptr;
  uint32_t *w = nullptr;
  CK(device_error_word(&w));  // lazily allocated state must exist before the capture
  cudaStream_t cs;
  CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed);
  if (e != cudaSuccess) {
    cudaStreamDestroy(cs);
    return cuda_status(e);
  }
  t_capturing = true;
  pir_status_t st = body(cs);
  t_capturing = false;
  cudaGraph_t graph = nullptr;
  e = cudaStreamEndCapture(cs, &graph);
  cudaStreamDestroy(cs);
  if (st != PIR_OK || e != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return st != PIR_OK ? st : cuda_status(e);
  }
  size_t nn = 0;
  e = cudaGraphGetNodes(graph, nullptr, &nn);
  std::vector<cudaGraphNode_t> nodes(nn);
  if (e == cudaSuccess && nn) e = cudaGraphGetNodes(graph, nodes.data(), &nn);
  uint64_t kernels = 0;
  for (size_t i = 0; e == cudaSuccess && i < nn; ++i) {
    cudaGraphNodeType t;
    if ((e = cudaGraphNodeGetType(nodes[i], &t)) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++kernels;
  }
  cudaGraphExec_t exec = nullptr;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(graph);
    return cuda_status(e);
  }
  pir_graph *g = new pir_graph{kGraphMagic, db, graph, exec, kernels, expander, db->device};
  {
    std::lock_guard<std::mutex> lock(g_reg_mu);
    g_graphs.insert(g);
  }
  *out = g;
  return PIR_OK;
}
}  // namespace

extern "C" {

const char *pir_status_str(pir_status_t st) {
  switch (st) {
    case PIR_OK: return "ok";
    case PIR_ERR_ARG: return "invalid argument";
    case PIR_ERR_OOM: return "out of memory";
    case PIR_ERR_ADMISSION: return "database does not fit the free device memory";
    case PIR_ERR_CUDA: return "CUDA error";
    case PIR_ERR_TIMEOUT: return "timed out";
    case PIR_ERR_HANDLE: return "unknown or freed database handle";
    case PIR_ERR_UNSUPPORTED: return "unsupported";
  }
  return "unknown status";
}

const char *pir_last_cuda_error(void) { return gbpir::last_cuda_error_cstr(); }

pir_status_t pir_stage_times(double *ms, uint64_t *launches) {
  cudaError_t first = cudaSuccess;
  for (const StageMark &m : t_marks) {
    float t = 0.f;
    cudaError_t e = cudaEventSynchronize(m.b);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, m.a, m.b);
    if (e != cudaSuccess && first == cudaSuccess) first = e;
    if (ms) ms[m.stage] += t;
    if (launches) launches[m.stage] += m.launches;
    t_free_events.push_back(m.a);
    t_free_events.push_back(m.b);
  }
  t_marks.clear();
  return cuda_status(first);
}

uint64_t pir_kernel_launches(void) { return g_launches.load(); }

pir_status_t pir_release_memory(void) {
  release_cached_memory();
  return cuda_status(cudaGetLastError());
}

pir_status_t pir_check_device(void *stream) {
  uint32_t *w = nullptr;
  CK(device_error_word(&w));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  uint32_t v = 0;
  CK(cudaStreamSynchronize(s));
  CK(cudaMemcpy(&v, w, sizeof(v), cudaMemcpyDeviceToHost));
  if (v) CK(cudaMemset(w, 0, sizeof(uint32_t)));
  CK(cudaDeviceSynchronize());
  return v ? PIR_ERR_TIMEOUT : PIR_OK;
}

pir_status_t pir_device_status(void) {
  uint32_t *w = nullptr;
  CK(device_error_word(&w));
  int dev = 0;
  CK(cudaGetDevice(&dev));
  static std::mutex mu;
  static cudaStream_t streams[64] = {};
  cudaStream_t s = nullptr;
  {
    std::lock_guard<std::mutex> lock(mu);
    if (!streams[dev]) CK(cudaStreamCreateWithFlags(&streams[dev], cudaStreamNonBlocking));
    s = streams[dev];
  }
  // a stream of its own that nothing else uses: the read waits for no other work
  uint32_t v = 0;
  CK(cudaMemcpyAsync(&v, w, sizeof(v), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (v) {
    CK(cudaMemsetAsync(w, 0, sizeof(uint32_t), s));
    CK(cudaStreamSynchronize(s));
  }
  return v ? PIR_ERR_TIMEOUT : PIR_OK;
}

uint32_t pir_gemm_tiles(int layout) {
  if (layout == PIR_LAYOUT_PLAIN) return gemm_plain_tiles();
  if (layout == PIR_LAYOUT_LIMB) return gemm_limb_tiles();
  if (layout == PIR_LAYOUT_TENSOR) return gemm_tc_tiles();
  return 0;
}

pir_status_t pir_setup_db(const pir_params_t *params, const void *raw_db, size_t raw_bytes, int raw_on_device,
                          int layout, void *stream, pir_db_t *out_handle) {
  NvtxRange range("pir_setup_db");
  if (!params || !raw_db || !out_handle) return PIR_ERR_ARG;
  if (layout != PIR_LAYOUT_PLAIN && layout != PIR_LAYOUT_LIMB && layout != PIR_LAYOUT_TENSOR) return PIR_ERR_ARG;
  pir_status_t st = validate_params(params);
  if (st != PIR_OK) return st;
  const pir_params_t p = *params;
  if (raw_bytes != raw_bytes_of(p)) return PIR_ERR_ARG;
  if ((p.D2 % 4) != 0) return PIR_ERR_UNSUPPORTED;  // 128-bit / paired column accesses
  if (layout == PIR_LAYOUT_LIMB && (p.D1 % 32) != 0) return PIR_ERR_UNSUPPORTED;  // k32 tensor steps
  if (layout == PIR_LAYOUT_TENSOR && !gemm_tc_shape_ok(p.D1, p.D2)) return PIR_ERR_UNSUPPORTED;  // 64-row stages, 32-column tiles
  *out_handle = nullptr;
  const ParamCtx *ctx = nullptr;
  st = get_param_ctx(&p, &ctx);
  if (st != PIR_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int dev = 0;
  CK(cudaGetDevice(&dev));
  keep_pool_memory(dev);

  // Admission: resident DB (+ the raw bytes if they must be staged) + the NTT
  // staging chunk, against the free memory less a reserve.
  const size_t bytes = resident_bytes(p, layout);
  const uint64_t polys = (uint64_t)p.D1 * p.D2;
  const uint64_t chunk_polys_target = (uint64_t)(256u << 20) / ((uint64_t)4 * p.L * p.n);
  uint64_t chunk = chunk_polys_target < polys ? chunk_polys_target : polys;
  if (layout == PIR_LAYOUT_LIMB) {  // whole columns per chunk
    uint64_t cols = chunk / p.D1;
    if (cols == 0) cols = 1;
    chunk = cols * p.D1;
  }
  const size_t staging = (size_t)chunk * p.L * p.n * 4;
  size_t free_b = 0, total_b = 0;
  CK(cudaMemGetInfo(&free_b, &total_b));
  size_t reserve = total_b / 32;
  if (reserve > ((size_t)2 << 30)) reserve = (size_t)2 << 30;
  // host bytes of the row-major layouts go up chunk by chunk, so only one chunk of
  // raw bytes is ever on the device beside the resident DB; the limb layout's
  // column-major chunks take the whole raw DB up first
  const size_t bpp = (size_t)p.n * p.log2p / 8;  // raw bytes per polynomial (whole bytes)
  const bool chunked_upload = !raw_on_device && layout != PIR_LAYOUT_LIMB;
  const size_t raw_dev_bytes = raw_on_device ? 0 : chunked_upload ? (size_t)chunk * bpp : raw_bytes;
  const size_t need = bytes + staging + raw_dev_bytes;
  if (need + reserve > free_b) {
    // answers' scratch stays cached in the stream-ordered pool, and destroyed graphs'
    // scratch in the graph pool: give back what is unused before judging the DB
    release_cached_memory();
    CK(cudaMemGetInfo(&free_b, &total_b));
  }
  if (need + reserve > free_b) return PIR_ERR_ADMISSION;

  pir_db *db = new pir_db();
  db->magic = kMagic;
  db->p = p;
  db->layout = layout;
  db->device = dev;
  db->ctx = ctx;
  db->bytes = bytes;
  cudaError_t e = cudaMalloc(&db->resident, bytes);
  if (e != cudaSuccess) {
    delete db;
    return cuda_status(e);
  }
  void *raw_dev = nullptr, *stage = nullptr;
  auto fail = [&](cudaError_t err) {
    cudaStreamSynchronize(s);
    if (raw_dev) cudaFree(raw_dev);
    if (stage) cudaFree(stage);
    cudaFree(db->resident);
    delete db;
    return cuda_status(err);
  };
  const uint8_t *raw = static_cast<const uint8_t *>(raw_db);
  if (!raw_on_device) {
    if ((e = cudaMalloc(&raw_dev, raw_dev_bytes)) != cudaSuccess) return fail(e);
    if (!chunked_upload) {
      if ((e = cudaMemcpyAsync(raw_dev, raw_db, raw_bytes, cudaMemcpyHostToDevice, s)) != cudaSuccess) return fail(e);
      raw = static_cast<const uint8_t *>(raw_dev);
    }
  }
  if ((e = cudaMalloc(&stage, staging)) != cudaSuccess) return fail(e);
  uint32_t *stg = static_cast<uint32_t *>(stage);
  if (layout != PIR_LAYOUT_LIMB) {  // row-major chunks of polynomials
    for (uint64_t first = 0; first < polys; first += chunk) {
      const uint64_t np = polys - first < chunk ? polys - first : chunk;
      if (chunked_upload) {  // this chunk's bytes only, read as polynomials 0 .. np-1
        if ((e = cudaMemcpyAsync(raw_dev, static_cast<const uint8_t *>(raw_db) + first * bpp, np * bpp,
                                 cudaMemcpyHostToDevice, s)) != cudaSuccess)
          return fail(e);
        e = launch_ntt_fwd_raw(*ctx, static_cast<const uint8_t *>(raw_dev), 0, p.D1, p.D2, 0, np, stg, s);
      } else {
        e = launch_ntt_fwd_raw(*ctx, raw, 0, p.D1, p.D2, first, np, stg, s);
      }
      if (e != cudaSuccess) return fail(e);
      e = layout == PIR_LAYOUT_PLAIN
              ? launch_db_scatter(*ctx, layout, p.D1, p.D2, stg, first, np, db->resident, s)
              : launch_db_scatter_tensor(*ctx, p.D1, p.D2, stg, first, np, static_cast<uint16_t *>(db->resident), s);
      if (e != cudaSuccess) return fail(e);
      count_launches(2);
    }
  } else {
    const uint64_t ccols = chunk / p.D1;
    for (uint64_t c0 = 0; c0 < p.D2; c0 += ccols) {
      const uint64_t nc = p.D2 - c0 < ccols ? p.D2 - c0 : ccols;
      const uint64_t np = nc * p.D1;
      if ((e = launch_ntt_fwd_raw(*ctx, raw, 1, p.D1, p.D2, c0, np, stg, s)) != cudaSuccess) return fail(e);
      if ((e = launch_db_scatter(*ctx, layout, p.D1, p.D2, stg, c0, np, db->resident, s)) != cudaSuccess)
        return fail(e);
      count_launches(2);
    }
  }
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return fail(e);
  if (layout == PIR_LAYOUT_TENSOR) {  // the tensor GEMM's error word: made here, so that
    uint32_t *w = nullptr;            // graph capture and pir_answer_noalloc never allocate
    if ((e = device_error_word(&w)) != cudaSuccess) return fail(e);
  }
  if (raw_dev) cudaFree(raw_dev);
  cudaFree(stage);
  {
    std::lock_guard<std::mutex> lock(g_reg_mu);
    g_live.insert(db);
  }
  *out_handle = db;
  return PIR_OK;
}

pir_status_t pir_answer_ex(pir_db_t db, const uint32_t *queries, uint32_t B, uint32_t *responses, int on_device,
                           void *stream, const pir_answer_opts_t *opts) {
  NvtxRange range("pir_answer");
  if (!live(db)) return PIR_ERR_HANDLE;
  if (B == 0 || !queries || !responses) return PIR_ERR_ARG;
  pir_answer_opts_t o = {};
  if (opts) o = *opts;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const pir_params_t &p = db->p;
  const size_t qbytes = (size_t)B * p.D1 * 2 * p.L * p.n * 4;
  const size_t rbytes = (size_t)B * p.D2 * 2 * ((o.flags & PIR_ANSWER_MODSWITCH) ? 1 : p.L) * p.n * 4;
  if (on_device) {
    if (!aligned16(queries) || !aligned16(responses)) return PIR_ERR_ARG;
    return answer_device(db, queries, B, responses, s, o);
  }
  // host batches above 4 GiB: a streamed answer in pieces of at most 1 GiB
  const uint64_t ct_bytes = 2ull * p.L * p.n * 4;
  if (o.k_chunk == 0 && qbytes > (4ull << 30) && (o.flags & PIR_ANSWER_TEST_STALL) == 0) {
    uint64_t kc = (1ull << 30) / ((uint64_t)B * ct_bytes);
    if (db->layout == PIR_LAYOUT_TENSOR) {
      // the tensor GEMM fills its stage ring only over long K-chunks: pieces as long
      // as the free memory holds beside the result (staging x 2, NTT-form copy, digit
      // tiles; 1 GiB kept back), up to the 1024-row exactness bound
      const size_t free_b = available_device_bytes(db->device);
      {
        const uint32_t M = 2 * B, Mp = layout_rows(db->layout, M);
        const size_t out_b = (size_t)p.L * p.n * M * p.D2 * 4 + (size_t)B * p.D2 * ct_bytes;
        const size_t per_row = 3 * (size_t)B * ct_bytes + layout_qs_bytes(db->layout, (uint64_t)p.L * p.n, 1, Mp);
        if (free_b > out_b + (1ull << 30)) {
          const uint64_t fit = (free_b - out_b - (1ull << 30)) / per_row;
          if (fit > kc) kc = fit;
        }
      }
      if (kc > 1024) kc = 1024;
    }
    if (kc == 0) kc = 1;
    if (kc > p.D1) kc = p.D1;
    if (db->layout != PIR_LAYOUT_PLAIN) kc = layout_chunk(db->layout, (uint32_t)kc);
    pir_session *ses = nullptr;
    pir_status_t st = session_open(db, B, (uint32_t)kc, s, o, &ses);
    if (st != PIR_OK) return st;
    // the first pieces ramp up (1/16, then 1/4 of a piece): the scan starts after a
    // short upload, and each upload still ends before the scan of the piece before
    // it (uploading a piece takes a quarter of the time its scan does, or less)
    uint32_t piece = layout_chunk(db->layout, (uint32_t)(kc / 16 ? kc / 16 : 1));
    for (uint32_t i0 = 0; i0 < p.D1 && st == PIR_OK;) {
      uint32_t k = piece < kc ? piece : (uint32_t)kc;
      if (k > p.D1 - i0) k = p.D1 - i0;
      st = session_chunk(ses, queries + (size_t)i0 * (ct_bytes / 4), (uint64_t)p.D1 * (ct_bytes / 4), i0, k, false);
      i0 += k;
      piece = layout_chunk(db->layout, piece * 4 < kc ? piece * 4 : (uint32_t)kc);
    }
    if (st == PIR_OK) st = session_finish(ses, responses, false);
    session_take(ses);
    session_release(ses);
    cudaStreamSynchronize(s);
    return st;
  }
  // host buffers: stage through device memory; synchronous
  Scratch dq(s), dr(s);
  CK(dq.alloc(qbytes));
  CK(dr.alloc(rbytes));
  // Batches of 16 and more (queries of 8 MiB and more, chunking left to the library)
  // run as sub-batches of at least 8 queries: sub-batch k+1 uploads on the copy
  // stream while k is answered on `stream` and k-1 downloads on a third stream, so
  // both directions of the host link stay busy and every sub-batch runs the whole
  // of D1 at once.
  if (o.k_chunk == 0 && B >= 16 && qbytes >= (8ull << 20) && (o.flags & PIR_ANSWER_TEST_STALL) == 0) {
    cudaStream_t up = nullptr, down = nullptr;
    CK(copy_stream(&up));
    CK(d2h_stream(&down));
    uint32_t nsub = B / 8;
    if (nsub > kMaxFeedChunks) nsub = kMaxFeedChunks;
    if (nsub > 4) nsub = 4;
    const uint32_t Bs = (B + nsub - 1) / nsub;
    const size_t qper = qbytes / B, rper = rbytes / B;  // bytes per query
    cudaEvent_t ready = take_event(), arrived[kMaxFeedChunks] = {}, answered[kMaxFeedChunks] = {};
    if (!ready) return PIR_ERR_CUDA;
    pir_status_t st = PIR_OK;
    auto ck = [&](cudaError_t e) {
      if (e != cudaSuccess && st == PIR_OK) st = cuda_status(e);
      return st == PIR_OK;
    };
    ck(cudaEventRecord(ready, s));  // the staging buffers are allocated in s's order
    ck(cudaStreamWaitEvent(up, ready, 0));
    uint32_t k = 0;
    for (uint32_t b0 = 0; b0 < B && st == PIR_OK; b0 += Bs, ++k) {
      const uint32_t nb = B - b0 < Bs ? B - b0 : Bs;
      if (!(arrived[k] = take_event()) || !(answered[k] = take_event())) {
        st = PIR_ERR_CUDA;
        break;
      }
      if (!ck(cudaMemcpyAsync(static_cast<char *>(dq.ptr) + b0 * qper, reinterpret_cast<const char *>(queries) + b0 * qper,
                              nb * qper, cudaMemcpyHostToDevice, up)) ||
          !ck(cudaEventRecord(arrived[k], up)) || !ck(cudaStreamWaitEvent(s, arrived[k], 0)))
        break;
      st = answer_device(db, reinterpret_cast<const uint32_t *>(static_cast<char *>(dq.ptr) + b0 * qper), nb,
                         reinterpret_cast<uint32_t *>(static_cast<char *>(dr.ptr) + b0 * rper), s, o);
      if (st != PIR_OK || !ck(cudaEventRecord(answered[k], s)) || !ck(cudaStreamWaitEvent(down, answered[k], 0)) ||
          !ck(cudaMemcpyAsync(reinterpret_cast<char *>(responses) + b0 * rper, static_cast<char *>(dr.ptr) + b0 * rper,
                              nb * rper, cudaMemcpyDeviceToHost, down)))
        break;
    }
    // the staging buffers are freed in s's order: after the last download
    cudaEvent_t fin = take_event();
    if (fin && cudaEventRecord(fin, down) == cudaSuccess) cudaStreamWaitEvent(s, fin, 0);
    cudaStreamSynchronize(up);
    cudaStreamSynchronize(down);
    cudaStreamSynchronize(s);
    t_free_events.push_back(ready);
    if (fin) t_free_events.push_back(fin);
    for (uint32_t i = 0; i < k + 1 && i < kMaxFeedChunks; ++i) {
      if (arrived[i]) t_free_events.push_back(arrived[i]);
      if (answered[i]) t_free_events.push_back(answered[i]);
    }
    return st;
  }
  // A large upload goes in K-chunk pieces on a copy stream; each chunk's forward NTT
  // waits only for its own piece, so later pieces arrive while earlier chunks are
  // being scanned.  Only when the caller leaves the chunking to the library.
  pir_answer_opts_t o2 = o;
  ChunkFeed feed;
  const bool plain = db->layout == PIR_LAYOUT_PLAIN;
  uint32_t Kc = p.D1;
  if (o.k_chunk == 0 && qbytes >= (8ull << 20) && qbytes <= (4ull << 30) && p.D1 >= 8) {
    uint32_t kc = (p.D1 + 3) / 4;
    kc = plain ? (kc + 1) & ~1u : layout_chunk(db->layout, kc);  // even pieces, or whole blocks of the layout
    if (kc < p.D1) Kc = kc;
  }
  cudaStream_t cs = nullptr;
  if (Kc < p.D1 && copy_stream(&cs) == cudaSuccess) {
    // batch 1 on the plain layout keeps one scan pass (a K-chunked scan costs more
    // than the upload it hides) and pipelines only the forward NTT behind the pieces
    if (B > 1 || !plain) o2.k_chunk = Kc;
    feed.kc = Kc;
    feed.n = (p.D1 + Kc - 1) / Kc;
    cudaEvent_t ready = take_event();  // the scratch is allocated in s's order
    if (!ready) return PIR_ERR_CUDA;
    CK(cudaEventRecord(ready, s));
    CK(cudaStreamWaitEvent(cs, ready, 0));
    t_free_events.push_back(ready);
    const size_t ct = (size_t)2 * p.L * p.n;  // words per ciphertext
    for (uint32_t k = 0; k < feed.n; ++k) {
      const uint32_t i0 = k * Kc, kc = p.D1 - i0 < Kc ? p.D1 - i0 : Kc;
      for (uint32_t b = 0; b < B; ++b) {
        const size_t off = ((size_t)b * p.D1 + i0) * ct;
        CK(cudaMemcpyAsync(static_cast<uint32_t *>(dq.ptr) + off, queries + off, (size_t)kc * ct * 4,
                           cudaMemcpyHostToDevice, cs));
      }
      if (!(feed.ev[k] = take_event())) return PIR_ERR_CUDA;
      CK(cudaEventRecord(feed.ev[k], cs));
    }
  } else {
    CK(cudaMemcpyAsync(dq.ptr, queries, qbytes, cudaMemcpyHostToDevice, s));
  }
  pir_status_t st = answer_device(db, static_cast<const uint32_t *>(dq.ptr), B, static_cast<uint32_t *>(dr.ptr), s,
                                  o2, nullptr, false, feed.n ? &feed : nullptr);
  if (st == PIR_OK) {
    cudaError_t e = cudaMemcpyAsync(responses, dr.ptr, rbytes, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) st = cuda_status(e);
  }
  cudaStreamSynchronize(s);
  if (cs) cudaStreamSynchronize(cs);  // the pieces are all consumed; their events can be reused
  for (uint32_t k = 0; k < feed.n; ++k)
    if (feed.ev[k]) t_free_events.push_back(feed.ev[k]);
  return st;
}

pir_status_t pir_answer_begin(pir_db_t db, uint32_t B, uint32_t kc_max, void *stream, const pir_answer_opts_t *opts,
                              pir_session_t *out) {
  if (!live(db)) return PIR_ERR_HANDLE;
  if (!out || B == 0 || kc_max == 0) return PIR_ERR_ARG;
  pir_answer_opts_t o = {};
  if (opts) o = *opts;
  return session_open(db, B, kc_max, static_cast<cudaStream_t>(stream), o, out);
}

pir_status_t pir_answer_chunk(pir_session_t session, const uint32_t *queries, uint32_t i0, uint32_t kc,
                              int on_device) {
  NvtxRange range("pir_answer_chunk");
  if (!session_live(session) || !live(session->db)) return PIR_ERR_HANDLE;
  const pir_params_t &p = session->db->p;
  return session_chunk(session, queries, (uint64_t)kc * 2 * p.L * p.n, i0, kc, on_device != 0);
}

pir_status_t pir_answer_end(pir_session_t session, uint32_t *responses, int on_device) {
  NvtxRange range("pir_answer_end");
  if (!session_take(session)) return PIR_ERR_HANDLE;
  pir_status_t st = session->failed;
  if (st == PIR_OK) {
    if (!live(session->db))
      st = PIR_ERR_HANDLE;
    else if (!responses || session->next != session->db->p.D1 || (on_device && !aligned16(responses)))
      st = PIR_ERR_ARG;
    else
      st = session_finish(session, responses, on_device != 0);
  }
  session_release(session);
  return st;
}

pir_status_t pir_answer_abort(pir_session_t session) {
  if (!session_take(session)) return PIR_ERR_HANDLE;
  session_release(session);
  return PIR_OK;
}

namespace {
// Packed queries pk [B][2][L][n] on the device: expansion into the D1 NTT-form
// ciphertexts of every query (scratch), then the answer (stream ordered).
pir_status_t answer_packed_device(pir_db *db, const pir_expander_impl *ex, const uint32_t *pk, uint32_t B,
                                  uint32_t *resp, cudaStream_t s, const pir_answer_opts_t &o) {
  const pir_params_t &p = db->p;
  Scratch qh(s);
  CK(qh.alloc((size_t)B * p.D1 * 2 * p.L * p.n * 4));
  StageTimer tm((o.flags & PIR_ANSWER_STAGE_TIMES) != 0, s);
  tm.begin();
  uint64_t launches = 0;
  pir_status_t st = expand_device(ex, pk, B, p.D1, static_cast<uint32_t *>(qh.ptr), s, &launches);
  tm.end(0, launches);
  if (st == PIR_OK) st = answer_device(db, nullptr, B, resp, s, o, static_cast<const uint32_t *>(qh.ptr));
  return st;
}
}  // namespace

pir_status_t pir_answer_packed(pir_db_t db, pir_expander_t expander, const uint32_t *packed, uint32_t B,
                               uint32_t *responses, int on_device, void *stream, const pir_answer_opts_t *opts) {
  NvtxRange range("pir_answer_packed");
  if (!live(db)) return PIR_ERR_HANDLE;
  const pir_expander_impl *ex = nullptr;
  if (!expander_view(expander, &ex)) return PIR_ERR_HANDLE;
  if (B == 0 || !packed || !responses) return PIR_ERR_ARG;
  pir_answer_opts_t o = {};
  if (opts) o = *opts;
  const pir_params_t &p = db->p;
  if (!expander_fits(ex, p)) return PIR_ERR_ARG;
  if ((o.k_chunk != 0 && o.k_chunk < p.D1) || (o.flags & PIR_ANSWER_TEST_STALL)) return PIR_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t pbytes = (size_t)B * 2 * p.L * p.n * 4;
  const size_t rbytes = (size_t)B * p.D2 * 2 * ((o.flags & PIR_ANSWER_MODSWITCH) ? 1 : p.L) * p.n * 4;
  Scratch dp(s), dr(s);
  const uint32_t *pk = packed;
  uint32_t *resp = responses;
  if (on_device) {
    if (!aligned16(packed) || !aligned16(responses)) return PIR_ERR_ARG;
  } else {
    CK(dp.alloc(pbytes));
    CK(dr.alloc(rbytes));
    CK(cudaMemcpyAsync(dp.ptr, packed, pbytes, cudaMemcpyHostToDevice, s));
    pk = static_cast<const uint32_t *>(dp.ptr);
    resp = static_cast<uint32_t *>(dr.ptr);
  }
  pir_status_t st = answer_packed_device(db, ex, pk, B, resp, s, o);
  if (st != PIR_OK) {
    if (!on_device) cudaStreamSynchronize(s);
    return st;
  }
  if (!on_device) {
    CK(cudaMemcpyAsync(responses, dr.ptr, rbytes, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
  }
  return PIR_OK;
}

pir_status_t pir_answer_folded(pir_db_t db, const uint32_t *queries, uint32_t B, uint32_t ell, const uint32_t *rgsw,
                               uint32_t *responses, int on_device, void *stream, const pir_answer_opts_t *opts) {
  NvtxRange range("pir_answer_folded");
  if (!live(db)) return PIR_ERR_HANDLE;
  if (B == 0 || !queries || !rgsw || !responses || ell == 0 || ell > 16) return PIR_ERR_ARG;
  pir_answer_opts_t o = {};
  if (opts) o = *opts;
  if (o.flags & PIR_ANSWER_TEST_STALL) return PIR_ERR_ARG;
  const pir_params_t &p = db->p;
  const ParamCtx &c = *db->ctx;
  if ((p.D2 & (p.D2 - 1)) != 0 || gadget_bits(p, ell) > 30) return PIR_ERR_ARG;
  uint32_t levels = 0;
  while ((1u << levels) < p.D2) ++levels;
  const bool msw = (o.flags & PIR_ANSWER_MODSWITCH) != 0;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const uint64_t ctw = 2ull * p.L * p.n;
  const size_t qbytes = (size_t)B * p.D1 * ctw * 4, gbytes = (size_t)B * levels * 2 * ell * ctw * 4;
  const size_t rbytes = (size_t)B * 2 * (msw ? 1 : p.L) * p.n * 4;
  Scratch hq(s), hg(s), hr(s), work(s);
  const uint32_t *q = queries, *g = rgsw;
  uint32_t *resp = responses;
  if (on_device) {
    if (!aligned16(queries) || !aligned16(rgsw) || !aligned16(responses)) return PIR_ERR_ARG;
  } else {
    CK(hq.alloc(qbytes));
    CK(hg.alloc(gbytes));
    CK(hr.alloc(rbytes));
    CK(cudaMemcpyAsync(hq.ptr, queries, qbytes, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(hg.ptr, rgsw, gbytes, cudaMemcpyHostToDevice, s));
    q = static_cast<const uint32_t *>(hq.ptr);
    g = static_cast<const uint32_t *>(hg.ptr);
    resp = static_cast<uint32_t *>(hr.ptr);
  }
  // NTT-form first-dimension responses | NTT-form RGSW rows | folded ciphertexts
  const size_t rn = (size_t)B * p.D2 * ctw, gn = (size_t)B * levels * 2 * ell * ctw, fn = (size_t)B * ctw;
  CK(work.alloc((rn + gn + fn) * 4));
  uint32_t *R = static_cast<uint32_t *>(work.ptr), *G = R + rn, *F = G + gn;
  pir_answer_opts_t o1 = o;
  o1.flags &= ~PIR_ANSWER_MODSWITCH;
  pir_status_t st = answer_device(db, q, B, R, s, o1, nullptr, true);
  if (st == PIR_OK) {
    StageTimer tm((o.flags & PIR_ANSWER_STAGE_TIMES) != 0, s);
    tm.begin();
    uint64_t launches = 0;
    cudaError_t e = launch_ntt_fwd(c, g, G, gn / p.n, s);
    if (e != cudaSuccess) st = cuda_status(e);
    if (st == PIR_OK) st = fold_device(c, R, B, levels, ell, G, F, s, &launches);
    if (st == PIR_OK) {
      e = msw ? launch_ntt_inv_switch(c, F, resp, (uint64_t)B * 2, s) : launch_ntt_inv(c, F, resp, (uint64_t)B * 2 * p.L, s);
      if (e != cudaSuccess) st = cuda_status(e);
    }
    tm.end(4, launches + 2);
  }
  if (st != PIR_OK) {
    cudaStreamSynchronize(s);
    return st;
  }
  if (!on_device) {
    CK(cudaMemcpyAsync(responses, hr.ptr, rbytes, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
  }
  return PIR_OK;
}

pir_status_t pir_answer(pir_db_t db, const uint32_t *queries, uint32_t B, uint32_t *responses, int on_device,
                        void *stream) {
  return pir_answer_ex(db, queries, B, responses, on_device, stream, nullptr);
}

static pir_status_t ntt_common(const pir_params_t *params, uint32_t *polys, size_t count, void *stream, bool fwd) {
  NvtxRange range(fwd ? "ntt_fwd" : "ntt_inv");
  if (!params || (!polys && count)) return PIR_ERR_ARG;
  if (count == 0) return validate_params(params);
  if (!aligned16(polys)) return PIR_ERR_ARG;
  const ParamCtx *ctx = nullptr;
  pir_status_t st = get_param_ctx(params, &ctx);
  if (st != PIR_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const uint64_t rows = (uint64_t)count * params->L;
  CK(fwd ? launch_ntt_fwd(*ctx, polys, polys, rows, s) : launch_ntt_inv(*ctx, polys, polys, rows, s));
  count_launches(1);
  return PIR_OK;
}

pir_status_t ntt_inv_modswitch(const pir_params_t *params, const uint32_t *in, size_t count, uint32_t *out,
                               void *stream) {
  if (!params || (count && (!in || !out))) return PIR_ERR_ARG;
  if (count == 0) return validate_params(params);
  if (!aligned16(in) || !aligned16(out)) return PIR_ERR_ARG;
  const uintptr_t ib = (uintptr_t)in, ob = (uintptr_t)out;
  const uint64_t in_bytes = (uint64_t)count * params->L * params->n * 4, out_bytes = (uint64_t)count * params->n * 4;
  if (ib < ob + out_bytes && ob < ib + in_bytes) return PIR_ERR_ARG;  // the kernel reads rows after others are written
  const ParamCtx *ctx = nullptr;
  pir_status_t st = get_param_ctx(params, &ctx);
  if (st != PIR_OK) return st;
  CK(launch_ntt_inv_switch(*ctx, in, out, count, static_cast<cudaStream_t>(stream)));
  count_launches(1);
  return PIR_OK;
}

pir_status_t ntt_fwd(const pir_params_t *params, uint32_t *polys, size_t count, void *stream) {
  return ntt_common(params, polys, count, stream, true);
}

pir_status_t ntt_inv(const pir_params_t *params, uint32_t *polys, size_t count, void *stream) {
  return ntt_common(params, polys, count, stream, false);
}


pir_status_t pir_graph_create(pir_db_t db, const uint32_t *queries, uint32_t B, uint32_t *responses,
                              const pir_answer_opts_t *opts, pir_graph_t *out) {
  if (!live(db)) return PIR_ERR_HANDLE;
  if (!out || !queries || !responses || B == 0 || !aligned16(queries) || !aligned16(responses)) return PIR_ERR_ARG;
  pir_answer_opts_t o = {};
  if (opts) o = *opts;
  if ((o.flags & ~PIR_ANSWER_MODSWITCH) != 0) return PIR_ERR_ARG;
  return capture_graph(
      db, nullptr, [&](cudaStream_t cs) { return answer_device(db, queries, B, responses, cs, o); }, out);
}

pir_status_t pir_graph_create_packed(pir_db_t db, pir_expander_t expander, const uint32_t *packed, uint32_t B,
                                     uint32_t *responses, const pir_answer_opts_t *opts, pir_graph_t *out) {
  if (!live(db)) return PIR_ERR_HANDLE;
  const pir_expander_impl *ex = nullptr;
  if (!expander_view(expander, &ex)) return PIR_ERR_HANDLE;
  if (!out || !packed || !responses || B == 0 || !aligned16(packed) || !aligned16(responses)) return PIR_ERR_ARG;
  pir_answer_opts_t o = {};
  if (opts) o = *opts;
  if ((o.flags & ~PIR_ANSWER_MODSWITCH) != 0 || (o.k_chunk != 0 && o.k_chunk < db->p.D1)) return PIR_ERR_ARG;
  if (!expander_fits(ex, db->p)) return PIR_ERR_ARG;
  return capture_graph(
      db, expander, [&](cudaStream_t cs) { return answer_packed_device(db, ex, packed, B, responses, cs, o); }, out);
}

static bool graph_live(pir_graph *g) {
  {
    std::lock_guard<std::mutex> lock(g_reg_mu);
    if (!(g && g_graphs.count(g) && g->magic == kGraphMagic && g_live.count(g->db))) return false;
  }
  const pir_expander_impl *ex = nullptr;  // a packed-query graph reads its expander's keys
  return !g->expander || expander_view(g->expander, &ex);
}

pir_status_t pir_graph_launch(pir_graph_t graph, void *stream) {
  NvtxRange range("pir_graph_launch");
  if (!graph_live(graph)) return PIR_ERR_HANDLE;
  cudaError_t e = cudaGraphLaunch(graph->exec, static_cast<cudaStream_t>(stream));
  if (e == cudaErrorMemoryAllocation) {  // its scratch is mapped at launch: make room and retry once
    cudaGetLastError();
    release_cached_memory();
    e = cudaGraphLaunch(graph->exec, static_cast<cudaStream_t>(stream));
  }
  CK(e);
  count_launches(graph->kernels);
  return PIR_OK;
}

pir_status_t pir_graph_destroy(pir_graph_t graph) {
  {
    std::lock_guard<std::mutex> lock(g_reg_mu);
    if (!graph || !g_graphs.count(graph)) return PIR_ERR_HANDLE;
    g_graphs.erase(graph);
  }
  cudaError_t e = cudaGraphExecDestroy(graph->exec);
  cudaError_t e2 = cudaGraphDestroy(graph->graph);
  // the scratch the capture allocated stays cached for graphs until trimmed: give it
  // back, so that later allocations and the admission checks see it
  cudaError_t e3 = cudaDeviceGraphMemTrim(graph->device);
  graph->magic = 0;
  delete graph;
  return cuda_status(e != cudaSuccess ? e : e2 != cudaSuccess ? e2 : e3);
}

pir_status_t pir_autotune(pir_db_t db, uint32_t B, void *stream, uint32_t reps, pir_answer_opts_t *best) {
  if (!live(db)) return PIR_ERR_HANDLE;
  if (!best || B == 0) return PIR_ERR_ARG;
  {
    std::lock_guard<std::mutex> lock(db->tune_mu);
    auto it = db->tuned.find(B);
    if (it != db->tuned.end()) {
      *best = it->second;
      return PIR_OK;
    }
  }
  if (reps == 0) reps = 1;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const pir_params_t &p = db->p;
  const uint32_t M = 2 * B, Mp16 = (M + 15u) & ~15u;
  const bool limb = db->layout == PIR_LAYOUT_LIMB;
  std::vector<uint32_t> tiles;
  if (db->layout == PIR_LAYOUT_TENSOR) {
    tiles.push_back(1);
    for (uint32_t t = 2; t <= gemm_tc_tiles(); ++t)
      if (gemm_tc_tile_ok(t, layout_rows(db->layout, M), p.D2)) tiles.push_back(t);
  } else if (!limb) {
    if (M <= 2) tiles.push_back(1);
    if (M <= 4) tiles.push_back(2);
    if (M <= 8) tiles.push_back(3);
    for (uint32_t t = 4; t <= 6; ++t) tiles.push_back(t);
    if (scan_tma_supports(M, p.D2)) tiles.push_back(7);
  } else {
    tiles.push_back(1);
    if (Mp16 % 32 == 0) tiles.push_back(2);
    if (Mp16 % 64 == 0) tiles.push_back(3);
  }
  std::vector<uint32_t> chunks = {0};
  for (uint32_t d : {2u, 4u}) {
    uint32_t kc = p.D1 / d;
    if (limb) kc &= ~31u;
    if (db->layout == PIR_LAYOUT_TENSOR) kc &= ~63u;
    if (kc >= 32 && kc < p.D1) chunks.push_back(kc);
  }
  const size_t qb = (size_t)B * p.D1 * 2 * p.L * p.n * 4, rb = (size_t)B * p.D2 * 2 * p.L * p.n * 4;
  Scratch dq(s), dr(s);
  CK(dq.alloc(qb));
  CK(dr.alloc(rb));
  CK(cudaMemsetAsync(dq.ptr, 0, qb, s));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  float best_ms = -1.f;
  pir_answer_opts_t win = {};
  for (uint32_t t : tiles)
    for (uint32_t kc : chunks) {
      pir_answer_opts_t o = {kc, t, 0};
      const uint32_t *qd = static_cast<const uint32_t *>(dq.ptr);
      uint32_t *rd = static_cast<uint32_t *>(dr.ptr);
      if (answer_device(db, qd, B, rd, s, o) != PIR_OK) continue;  // shape this tile does not hold
      cudaEventRecord(e0, s);
      bool ok = true;
      for (uint32_t r = 0; r < reps && ok; ++r) ok = answer_device(db, qd, B, rd, s, o) == PIR_OK;
      cudaEventRecord(e1, s);
      float ms = 0.f;
      if (!ok || cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
        continue;
      ms /= reps;
      // a later candidate (a narrower tile or more K-chunks: more launches, more
      // partial-result traffic) wins only if it is at least 1% faster, so that timing
      // noise does not flip the choice between equals
      if (best_ms < 0.f || ms < 0.99f * best_ms) best_ms = ms, win = o;
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaGetLastError();  // a refused candidate may leave a launch-configuration error behind
  if (best_ms < 0.f) return PIR_ERR_UNSUPPORTED;
  {
    std::lock_guard<std::mutex> lock(db->tune_mu);
    db->tuned[B] = win;
  }
  *best = win;
  return PIR_OK;
}

pir_status_t pir_free_db(pir_db_t db) {
  {
    std::lock_guard<std::mutex> lock(g_reg_mu);
    if (!db || !g_live.count(db)) return PIR_ERR_HANDLE;
    g_live.erase(db);
  }
  cudaDeviceSynchronize();
  cudaError_t e = cudaFree(db->resident);
  db->magic = 0;
  delete db;
  return cuda_status(e);
}

pir_status_t pir_db_bytes(pir_db_t db, size_t *bytes) {
  if (!live(db)) return PIR_ERR_HANDLE;
  if (!bytes) return PIR_ERR_ARG;
  *bytes = db->bytes;
  return PIR_OK;
}

pir_status_t pir_db_info(pir_db_t db, pir_params_t *params, int *layout) {
  if (!live(db)) return PIR_ERR_HANDLE;
  if (params) *params = db->p;
  if (layout) *layout = db->layout;
  return PIR_OK;
}

pir_status_t pir_db_read_poly(pir_db_t db, uint64_t poly_index, uint32_t *out) {
  if (!live(db)) return PIR_ERR_HANDLE;
  if (!out || poly_index >= (uint64_t)db->p.D1 * db->p.D2) return PIR_ERR_ARG;
  const size_t bytes = (size_t)db->p.L * db->p.n * 4;
  uint32_t *tmp = nullptr;
  CK(cudaMalloc(&tmp, bytes));
  cudaError_t e = db->layout == PIR_LAYOUT_TENSOR
                      ? launch_db_read_poly_tensor(*db->ctx, db->p.D1, db->p.D2,
                                                   static_cast<const uint16_t *>(db->resident), poly_index, tmp, 0)
                      : launch_db_read_poly(*db->ctx, db->layout, db->p.D1, db->p.D2, db->resident, poly_index, tmp, 0);
  if (e == cudaSuccess) e = cudaMemcpy(out, tmp, bytes, cudaMemcpyDeviceToHost);
  cudaFree(tmp);
  return cuda_status(e);
}

}  // extern "C"
