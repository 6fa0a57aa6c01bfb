// fold.cu -- the remaining dimensions of poly-HE folding: RGSW-RLWE external
// products (Sec. 3.2 and 3.6, OnionPIR's construction; gadget of App. D.3).
//
// After the first-dimension scan every query has 2^levels response ciphertexts.
// Level l pairs them, (c_2j, c_2j+1) -> c_2j + RGSW_l (x) (c_2j+1 - c_2j), where RGSW_l
// encrypts bit l of the wanted column, until one ciphertext is left.  The external
// product writes the difference in the gadget (ell digits of the CRT lift of every
// coefficient of both components) and sums digit x RGSW row products.
//
// GPU design: ciphertexts stay in NTT form between levels (the first-dimension result
// is handed over before its inverse NTT).  A level is five launches over all pairs of
// all queries: the NTT-form difference, its inverse NTT, the gadget digits, their
// forward NTT under every prime, and one multiply-accumulate kernel adding
// sum_r NTT(d_r) RGSW[r] to c_2j.
#include "common.cuh"

namespace gbpir {
namespace {

template <typename T>
__device__ __forceinline__ T pickL(const T (&a)[PIR_MAX_L], uint32_t j) {
  T r = a[0];
#pragma unroll
  for (uint32_t i = 1; i < PIR_MAX_L; ++i) r = j == i ? a[i] : r;
  return r;
}

unsigned grid_cap(uint64_t threads) {
  const uint64_t g = (threads + 255) / 256, cap = 152ull * 32;
  return (unsigned)(g < 1 ? 1 : (g > cap ? cap : g));
}

// diff[pr] = cur[2 pr + 1] - cur[2 pr] for every residue (pairs are adjacent).
__global__ void k_fold_diff(const uint32_t *__restrict__ cur, uint64_t pairs, uint64_t ctw, uint32_t logn,
                            uint32_t L, ModConst mc, uint32_t *__restrict__ diff) {
  const uint64_t total = pairs * ctw;
  for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < total; e += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t pr = e / ctw, o = e % ctw;
    const uint32_t q = pickL(mc.q, (uint32_t)((o >> logn) % L));
    const uint32_t a = cur[(2 * pr) * ctw + o], b = cur[(2 * pr + 1) * ctw + o];
    diff[e] = b >= a ? b - a : b + q - a;
  }
}

// out[pr] = cur[2 pr] + sum_{r < 2 ell} dhat[pr][r] * G[r]  (NTT form, every residue), with
// G the RGSW ciphertext of query pr / P at this level: rgsw + ((b * levels + lev) * 2 ell) * ctw.
template <uint32_t L>
__global__ void k_fold_mac(const uint32_t *__restrict__ cur, const uint32_t *__restrict__ dhat,
                           const uint32_t *__restrict__ rgsw, uint64_t pairs, uint32_t plog, uint32_t levels,
                           uint32_t lev, uint32_t logn, uint32_t ell, ModConst mc, uint32_t *__restrict__ out) {
  const uint32_t n = 1u << logn;
  const uint64_t ctw = 2ull * L * n, total = pairs * ctw;
  for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < total; e += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t pr = e / ctw;
    const uint32_t o = (uint32_t)(e % ctw);  // (comp * L + i) * n + s
    const uint32_t s = o & (n - 1), row = o >> logn, i = row % L;
    const uint32_t q = pickL(mc.q, i);
    const uint64_t mu = pickL(mc.mu, i), k63 = pickL(mc.k63, i);
    const uint64_t b = pr >> plog;
    const uint32_t *g = rgsw + ((b * levels + lev) * 2 * ell) * ctw + o;
    const uint32_t *dh = dhat + (pr * 2 * ell * L + i) * (uint64_t)n + s;
    uint64_t acc = cur[(2 * pr) * ctw + o];
    for (uint32_t r = 0; r < 2 * ell; ++r) {
      mac_wide(acc, dh[(uint64_t)r * L * n], __ldg(g + r * ctw));
      if ((r & 7) == 7) acc = fold63(acc, k63);
    }
    out[pr * ctw + o] = reduce64(acc, q, mu);
  }
}

}  // namespace

// Fold B queries' 2^levels ciphertexts (NTT form, cur [B][2^levels][2][L][n]) with
// their RGSW ciphertexts (NTT form, rgsw [B][levels][2 ell][2][L][n]) into out
// [B][2][L][n] (NTT form).  cur is overwritten.  Scratch from the stream-ordered allocator.
pir_status_t fold_device(const ParamCtx &c, uint32_t *cur, uint32_t B, uint32_t levels, uint32_t ell,
                         const uint32_t *rgsw, uint32_t *out, cudaStream_t s, uint64_t *launch_count) {
  const uint32_t n = c.p.n, L = c.p.L, logn = c.logn;
  const uint64_t ctw = 2ull * L * n;
  *launch_count = 0;
  if (levels == 0) {
    cudaError_t e = cudaMemcpyAsync(out, cur, (uint64_t)B * ctw * 4, cudaMemcpyDeviceToDevice, s);
    return e == cudaSuccess ? PIR_OK : cuda_status(e);
  }
  const uint64_t pairs0 = (uint64_t)B << (levels - 1);
  // scratch: next level | difference | its digits | their NTT
  const uint64_t words = pairs0 * ctw + pairs0 * ctw + pairs0 * 2 * ell * n + pairs0 * 2 * ell * L * n;
  void *scratch = nullptr;
  cudaError_t e = cudaMallocAsync(&scratch, words * 4, s);
  if (e != cudaSuccess) return cuda_status(e);
  uint32_t *nxt = static_cast<uint32_t *>(scratch);
  uint32_t *diff = nxt + pairs0 * ctw;
  uint32_t *dig = diff + pairs0 * ctw;
  uint32_t *dhat = dig + pairs0 * 2 * ell * n;
  pir_status_t st = PIR_OK;
  auto ck = [&](cudaError_t err) {
    if (err != cudaSuccess && st == PIR_OK) st = cuda_status(err);
    return err == cudaSuccess;
  };
  for (uint32_t lev = 0; lev < levels; ++lev) {
    const uint32_t plog = levels - 1 - lev;  // pairs per query = 2^plog
    const uint64_t pairs = (uint64_t)B << plog;
    uint32_t *dst = lev + 1 == levels ? out : nxt;
    k_fold_diff<<<grid_cap(pairs * ctw), 256, 0, s>>>(cur, pairs, ctw, logn, L, c.mod, diff);
    if (!ck(cudaGetLastError())) break;
    // coefficient form of both components: rows [pairs][2][L]
    if (!ck(launch_ntt_inv(c, diff, diff, pairs * 2 * L, s))) break;
    if (!ck(launch_gadget_digits(c, diff, pairs * 2, ell, dig, s))) break;  // [pairs][2][ell][n] = [pairs][2 ell][n]
    if (!ck(launch_ntt_fwd_rows_t(c, dig, 0, L, 1, 0, dhat, pairs * 2 * ell * L, s))) break;
    const unsigned gm = grid_cap(pairs * ctw);
    switch (L) {
      case 1: k_fold_mac<1><<<gm, 256, 0, s>>>(cur, dhat, rgsw, pairs, plog, levels, lev, logn, ell, c.mod, dst); break;
      case 2: k_fold_mac<2><<<gm, 256, 0, s>>>(cur, dhat, rgsw, pairs, plog, levels, lev, logn, ell, c.mod, dst); break;
      case 3: k_fold_mac<3><<<gm, 256, 0, s>>>(cur, dhat, rgsw, pairs, plog, levels, lev, logn, ell, c.mod, dst); break;
      default: k_fold_mac<4><<<gm, 256, 0, s>>>(cur, dhat, rgsw, pairs, plog, levels, lev, logn, ell, c.mod, dst); break;
    }
    if (!ck(cudaGetLastError())) break;
    *launch_count += 5;
    // the level's output becomes the next input; the old input area takes the next output
    uint32_t *t = cur;
    cur = nxt;
    nxt = t;
  }
  cudaFreeAsync(scratch, s);
  return st;
}

}  // namespace gbpir

using namespace gbpir;

extern "C" pir_status_t pir_fold(const pir_params_t *params, const uint32_t *cts, uint32_t B, uint32_t levels,
                                 uint32_t ell, const uint32_t *rgsw, uint32_t *out, void *stream) {
  if (!params || !cts || !rgsw || !out || B == 0 || levels > 20 || ell == 0 || ell > 16) return PIR_ERR_ARG;
  if (((uintptr_t)cts & 15u) || ((uintptr_t)rgsw & 15u) || ((uintptr_t)out & 15u)) return PIR_ERR_ARG;
  const ParamCtx *ctx = nullptr;
  pir_status_t st = get_param_ctx(params, &ctx);
  if (st != PIR_OK) return st;
  if (gadget_bits(ctx->p, ell) > 30) return PIR_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const uint32_t L = params->L, n = params->n;
  const uint64_t ctw = 2ull * L * n, count = 1ull << levels;
  const uint64_t cur_words = (uint64_t)B * count * ctw, g_words = (uint64_t)B * levels * 2 * ell * ctw;
  void *scratch = nullptr;
  cudaError_t e = cudaMallocAsync(&scratch, (cur_words + g_words) * 4, s);
  if (e != cudaSuccess) return cuda_status(e);
  uint32_t *cur = static_cast<uint32_t *>(scratch), *g = cur + cur_words;
  // NTT form of the inputs and of the RGSW rows (rows [..][L][n], row r under prime r % L)
  if ((e = launch_ntt_fwd(*ctx, cts, cur, cur_words / n, s)) == cudaSuccess &&
      (e = launch_ntt_fwd(*ctx, rgsw, g, g_words / n, s)) == cudaSuccess) {
    uint64_t launches = 0;
    st = fold_device(*ctx, cur, B, levels, ell, g, out, s, &launches);
    count_launches(2 + launches);
    if (st == PIR_OK && (e = launch_ntt_inv(*ctx, out, out, (uint64_t)B * 2 * L, s)) != cudaSuccess)
      st = cuda_status(e);
    if (st == PIR_OK) count_launches(1);
  } else {
    st = cuda_status(e);
  }
  cudaFreeAsync(scratch, s);
  return st;
}
