// noalloc.cu -- pir_answer_noalloc: the answer for callers that must not allocate
// device memory while they serve requests.
//
// Who needs it: a process that reserves its whole device-memory budget up front
// (for example a server that hands all free HBM to resident databases, or a host
// application whose own allocator owns the device) cannot let a library grab
// scratch memory per request; neither can a latency-critical path that cannot
// afford an allocator call and the synchronization it may bring.  This entry point
// takes its scratch from one fixed array in device memory instead.
//
// The scratch is the file-scope array below, PIR_NOALLOC_SCRATCH_BYTES (64 MiB).
// Every GPU that loads this library holds it until the process exits.  The host
// only sees a stand-in for it, so the first call on each device looks up its
// device address (cudaGetSymbolAddress, with that device current) and caches it;
// make that first call before any stream capture.  All calls on a device share
// the one array: calls that overlap on the GPU (different streams, or host
// threads) race on it and must be serialized by the caller.  Nothing in the array
// needs to start at zero: every stage writes what a later stage reads.
//
// The work is the same pipeline as pir_answer (forward NTT, slot-major layout,
// modular GEMM with its reduction, result transpose, inverse NTT), folded over D1
// in chunks small enough that one chunk of query scratch plus the result fit the
// array; requests whose result alone does not fit are refused with PIR_ERR_ARG.
// It calls no cudaMalloc, cudaFree or other allocating routine.
#include <mutex>

#include "common.cuh"

namespace gbpir {
namespace {

static __device__ __align__(256) uint8_t g_noalloc_scratch[PIR_NOALLOC_SCRATCH_BYTES];

std::mutex g_mu;
void *g_scratch_addr[64] = {};

// Device address of the scratch array on the current device (looked up once).
cudaError_t scratch_address(void **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[dev]) {
    void *ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = ptr;
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace
}  // namespace gbpir

using namespace gbpir;

extern "C" pir_status_t pir_answer_noalloc(pir_db_t db, const uint32_t *queries, uint32_t B, uint32_t *responses,
                                           void *stream) {
  DbView v;
  if (!db_view(db, &v)) return PIR_ERR_HANDLE;
  if (B == 0 || !queries || !responses) return PIR_ERR_ARG;
  if (((uintptr_t)queries & 15u) || ((uintptr_t)responses & 15u)) return PIR_ERR_ARG;
  const ParamCtx &c = *v.ctx;
  const uint32_t n = v.p.n, L = v.p.L, D1 = v.p.D1, D2 = v.p.D2;
  const bool limb = v.layout == PIR_LAYOUT_LIMB, tensor = v.layout == PIR_LAYOUT_TENSOR;
  const uint32_t M = 2 * B;
  const uint32_t Mp = limb ? (M + 15u) & ~15u : tensor ? tc_rows(M) : (M + 3u) & ~3u;
  const uint64_t nslots = (uint64_t)L * n;
  const size_t cap = PIR_NOALLOC_SCRATCH_BYTES;

  // result buffer first, then the largest K chunk whose query scratch still fits
  const size_t out_bytes = up256((size_t)nslots * M * D2 * 4);
  if (out_bytes >= cap) return PIR_ERR_ARG;
  // per folded row i: its NTT-form ciphertexts (qhat) + its GEMM-layout copy (u32 words,
  // four u8 limb planes: the same bytes; or four bf16 digits: twice that)
  const size_t per_row = (size_t)B * 2 * L * n * 4 + (size_t)nslots * Mp * (tensor ? 8 : 4);
  uint64_t kc_fit = (cap - out_bytes - 512) / per_row;
  uint32_t Kc = kc_fit >= D1 ? D1 : (uint32_t)kc_fit;
  if (limb) {
    if (Kc > 8192) Kc = 8192;
    Kc &= ~31u;
  }
  if (tensor) {  // 64-row blocks, at most 1024 rows (exact f32 digit sums)
    if (Kc > 1024) Kc = 1024;
    Kc &= ~63u;
  }
  if (Kc == 0) return PIR_ERR_ARG;

  void *base = nullptr;
  cudaError_t e = scratch_address(&base);
  if (e != cudaSuccess) return cuda_status(e);
  char *b8 = static_cast<char *>(base);
  uint32_t *out = reinterpret_cast<uint32_t *>(b8);
  uint32_t *qhat = reinterpret_cast<uint32_t *>(b8 + out_bytes);
  void *qs = b8 + out_bytes + up256((size_t)B * Kc * 2 * L * n * 4);

  // GEMM tile without the TMA scan (its error word is allocated on first use)
  const uint32_t tile = limb ? 0 : (M <= 2 ? 1 : M <= 4 ? 2 : M <= 8 ? 3 : 0);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  uint64_t launches = 0;
  for (uint32_t i0 = 0; i0 < D1; i0 += Kc) {
    const uint32_t kc = D1 - i0 < Kc ? D1 - i0 : Kc;
    const uint64_t G = (uint64_t)kc * 2 * L, S = (uint64_t)D1 * 2 * L;
    if ((e = launch_ntt_fwd_rows(c, queries, (uint64_t)i0 * 2 * L, G, S, qhat, (uint64_t)B * G, s)) != cudaSuccess)
      return cuda_status(e);
    if (tensor) {
      if ((e = launch_query_to_tensor(c, qhat, B, kc, Mp, static_cast<uint16_t *>(qs), s)) != cudaSuccess)
        return cuda_status(e);
      e = launch_gemm_tc(c, static_cast<const uint16_t *>(v.resident), D1, D2, static_cast<const uint16_t *>(qs), M,
                         Mp, i0, kc, out, i0 > 0, 0, s);
    } else if (!limb) {
      if ((e = launch_query_to_slots(c, qhat, B, kc, Mp, static_cast<uint32_t *>(qs), s)) != cudaSuccess)
        return cuda_status(e);
      e = launch_gemm_plain(c, static_cast<const uint32_t *>(v.resident), D1, D2, static_cast<const uint32_t *>(qs),
                            M, Mp, i0, kc, out, i0 > 0, tile, 0, s);
    } else {
      if ((e = launch_query_to_limbs(c, qhat, B, kc, Mp, static_cast<uint8_t *>(qs), s)) != cudaSuccess)
        return cuda_status(e);
      e = launch_gemm_limb(c, static_cast<const uint8_t *>(v.resident), D1, D2, static_cast<const uint8_t *>(qs), M,
                           Mp, i0, kc, out, i0 > 0, tile, s);
    }
    if (e != cudaSuccess) return cuda_status(e);
    launches += 3;
  }
  if ((e = launch_slots_to_responses(c, out, B, D2, responses, s)) != cudaSuccess) return cuda_status(e);
  if ((e = launch_ntt_inv(c, responses, responses, (uint64_t)B * D2 * 2 * L, s)) != cudaSuccess)
    return cuda_status(e);
  count_launches(launches + 2);
  return PIR_OK;
}
