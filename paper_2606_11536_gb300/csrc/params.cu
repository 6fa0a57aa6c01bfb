// params.cu -- host-side parameter generation and device constant tables.
//
// RNS primes (App. A.4): q_j = 1 mod 2n (negacyclic NTT exists) and q_j = 1 mod p
// (so Delta * p + 1 = q); both moduli are powers of two, so q_j = 1 mod max(2n, p).
// This library takes the L largest such primes in (2^29, 2^30), decreasing, and
// psi_j = h^((q_j - 1) / 2n) for the smallest h >= 2 with psi_j^n = -1.
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "common.cuh"

namespace gbpir {
namespace {

uint64_t mul_mod32(uint64_t a, uint64_t b, uint64_t m) { return (a * b) % m; }  // a, b < 2^32

uint64_t pow_mod32(uint64_t b, uint64_t e, uint64_t m) {
  uint64_t r = 1;
  b %= m;
  for (; e; e >>= 1) {
    if (e & 1) r = mul_mod32(r, b, m);
    b = mul_mod32(b, b, m);
  }
  return r;
}

// Miller-Rabin with bases {2, 7, 61}: deterministic for all n < 4,759,123,141,
// which covers every candidate below 2^30.
bool prime32(uint32_t n) {
  if (n < 2) return false;
  for (uint32_t sp : {2u, 3u, 5u, 7u, 11u, 13u, 61u})
    if (n % sp == 0) return n == sp;
  uint32_t d = n - 1, r = 0;
  while (!(d & 1)) d >>= 1, ++r;
  for (uint32_t a : {2u, 7u, 61u}) {
    uint64_t x = pow_mod32(a, d, n);
    if (x == 1 || x == n - 1) continue;
    bool witness = true;
    for (uint32_t i = 1; i < r && witness; ++i) {
      x = mul_mod32(x, x, n);
      if (x == n - 1) witness = false;
    }
    if (witness) return false;
  }
  return true;
}

uint32_t log2_exact(uint32_t n) {
  uint32_t l = 0;
  while ((1u << l) < n) ++l;
  return (1u << l) == n ? l : 0xFFFFFFFFu;
}

uint32_t brv(uint32_t x, uint32_t bits) {
  uint32_t r = 0;
  for (uint32_t i = 0; i < bits; ++i, x >>= 1) r = (r << 1) | (x & 1);
  return r;
}

uint32_t shoup(uint32_t w, uint32_t q) { return (uint32_t)(((uint64_t)w << 32) / q); }

}  // namespace

pir_status_t validate_params(const pir_params_t *p) {
  if (!p) return PIR_ERR_ARG;
  uint32_t lg = log2_exact(p->n);
  if (lg < 11 || lg > 13) return PIR_ERR_ARG;
  if (p->L < 1 || p->L > PIR_MAX_L || p->log2p < 1 || p->log2p > 28 || p->D1 == 0 || p->D2 == 0)
    return PIR_ERR_ARG;
  if (((uint64_t)p->n * p->log2p) % 8) return PIR_ERR_ARG;  // whole bytes per polynomial
  const uint64_t plain = 1ull << p->log2p;
  for (uint32_t j = 0; j < p->L; ++j) {
    uint32_t q = p->q[j];
    if (q <= (1u << 29) || q >= (1u << 30)) return PIR_ERR_ARG;
    if ((q - 1) % (2ull * p->n) != 0 || (q - 1) % plain != 0) return PIR_ERR_ARG;
    if (!prime32(q)) return PIR_ERR_ARG;
    if (pow_mod32(p->psi[j], p->n, q) != q - 1) return PIR_ERR_ARG;
    for (uint32_t i = 0; i < j; ++i)
      if (p->q[i] == q) return PIR_ERR_ARG;
  }
  return PIR_OK;
}

extern "C" pir_status_t pir_make_params(uint32_t n, uint32_t log2p, uint32_t D1, uint32_t D2, uint32_t L,
                                        pir_params_t *out) {
  if (!out) return PIR_ERR_ARG;
  uint32_t lg = log2_exact(n);
  if (lg < 11 || lg > 13 || L < 1 || L > PIR_MAX_L || log2p < 1 || log2p > 28 || D1 == 0 || D2 == 0)
    return PIR_ERR_ARG;
  pir_params_t p = {};
  p.n = n;
  p.L = L;
  p.log2p = log2p;
  p.D1 = D1;
  p.D2 = D2;
  uint64_t step = 2ull * n;
  if ((1ull << log2p) > step) step = 1ull << log2p;
  uint64_t cand = ((1ull << 30) - 2) / step * step + 1;
  uint32_t found = 0;
  for (; found < L && cand > (1ull << 29); cand -= step)
    if (prime32((uint32_t)cand)) p.q[found++] = (uint32_t)cand;
  if (found < L) return PIR_ERR_UNSUPPORTED;
  for (uint32_t j = 0; j < L; ++j) {
    const uint32_t q = p.q[j];
    const uint64_t e = (q - 1) / (2ull * n);
    for (uint64_t h = 2;; ++h) {
      uint64_t psi = pow_mod32(h, e, q);
      if (pow_mod32(psi, n, q) == q - 1) {
        p.psi[j] = (uint32_t)psi;
        break;
      }
    }
  }
  *out = p;
  return validate_params(&p);
}

// ---------------------------------------------------------------------------
// Device tables, built once per (device, parameter set) and kept until exit.
// ---------------------------------------------------------------------------
namespace {
struct Key {
  int dev;
  uint32_t n, L, log2p;
  uint32_t q[PIR_MAX_L], psi[PIR_MAX_L];
  bool operator<(const Key &o) const {
    return std::tie(dev, n, L, log2p, q[0], q[1], q[2], q[3], psi[0], psi[1], psi[2], psi[3]) <
           std::tie(o.dev, o.n, o.L, o.log2p, o.q[0], o.q[1], o.q[2], o.q[3], o.psi[0], o.psi[1], o.psi[2],
                    o.psi[3]);
  }
};
std::mutex g_mu;
std::map<Key, ParamCtx *> g_cache;
}  // namespace

pir_status_t get_param_ctx(const pir_params_t *p, const ParamCtx **out) {
  pir_status_t st = validate_params(p);
  if (st != PIR_OK) return st;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_status(e);
  Key k = {};
  k.dev = dev;
  k.n = p->n;
  k.L = p->L;
  k.log2p = p->log2p;
  for (uint32_t j = 0; j < p->L; ++j) k.q[j] = p->q[j], k.psi[j] = p->psi[j];
  std::lock_guard<std::mutex> lock(g_mu);
  auto it = g_cache.find(k);
  if (it != g_cache.end()) {
    *out = it->second;
    return PIR_OK;
  }
  const uint32_t n = p->n, lg = log2_exact(n);
  // per prime and direction: the n twiddle pairs, then their lane-major copy for the
  // first two stages of a radix-16 pass on the lowest index bits (kNttLaneMajorWords)
  const size_t dir_words = 2 * (size_t)n + ntt_lane_major_words(n), prime_words = 2 * dir_words;
  std::vector<uint32_t> host(prime_words * p->L);
  ParamCtx *ctx = new ParamCtx();
  ctx->p = *p;
  ctx->p.D1 = ctx->p.D2 = 0;  // the context describes the ring only; shapes travel per call
  ctx->logn = lg;
  for (uint32_t j = 0; j < p->L; ++j) {
    const uint32_t q = p->q[j];
    const uint32_t psi = p->psi[j];
    const uint32_t psi_inv = (uint32_t)pow_mod32(psi, q - 2, q);
    // per prime: forward pairs [n][2] and their lane-major copy, then the same inverse
    uint32_t *f = &host[j * prime_words], *iv = &host[j * prime_words + dir_words];
    for (uint32_t i = 0; i < n; ++i) {
      f[2 * i] = (uint32_t)pow_mod32(psi, brv(i, lg), q);
      f[2 * i + 1] = shoup(f[2 * i], q);
      iv[2 * i] = (uint32_t)pow_mod32(psi_inv, brv(i, lg), q);
      iv[2 * i + 1] = shoup(iv[2 * i], q);
    }
    ntt_lane_major_fill(f, n);
    ntt_lane_major_fill(iv, n);
    ctx->ntt.q[j] = q;
    ctx->ntt.ninv[j] = (uint32_t)pow_mod32(n, q - 2, q);
    ctx->ntt.ninv_sh[j] = shoup(ctx->ntt.ninv[j], q);
    ctx->mod.q[j] = q;
    ctx->mod.mu[j] = (uint64_t)(~0ull / q);  // floor((2^64 - 1) / q) = floor(2^64 / q) for q not a power of 2
    ctx->mod.k63[j] = ((1ull << 63) / q) * q;
  }
  {  // modulus switching to q_0
    SwitchConst &sw = ctx->sw;
    const uint32_t q0 = p->q[0];
    for (uint32_t k = 1; k < p->L; ++k)
      for (uint32_t i = 1; i < k; ++i) {
        const uint32_t qk = p->q[k];
        sw.c[k][i] = (uint32_t)pow_mod32(p->q[i] % qk, qk - 2, qk);
        sw.c_sh[k][i] = shoup(sw.c[k][i], qk);
      }
    uint64_t wk = 1;                // q_1 ... q_{k-1} mod q_0
    unsigned __int128 Qd = 1;       // Q' = q_1 ... q_{L-1} (< 2^90)
    for (uint32_t k = 1; k < p->L; ++k) {
      sw.w[k] = (uint32_t)wk;
      sw.w_sh[k] = shoup(sw.w[k], q0);
      wk = wk * p->q[k] % q0;
      Qd *= p->q[k];
    }
    sw.qinv = (uint32_t)pow_mod32(wk, q0 - 2, q0);  // wk = Q' mod q_0 (nonzero: distinct primes)
    sw.qinv_sh = shoup(sw.qinv, q0);
    unsigned __int128 H = (Qd - 1) / 2;
    for (uint32_t k = 1; k < p->L; ++k) {
      sw.h[k] = (uint32_t)(H % p->q[k]);
      H /= p->q[k];
    }
  }
  uint32_t *dtab = nullptr;
  e = cudaMalloc(&dtab, host.size() * sizeof(uint32_t));
  if (e != cudaSuccess) {
    delete ctx;
    return cuda_status(e);
  }
  e = cudaMemcpy(dtab, host.data(), host.size() * sizeof(uint32_t), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(dtab);
    delete ctx;
    return cuda_status(e);
  }
  for (uint32_t j = 0; j < p->L; ++j) {
    ctx->ntt.fwd[j] = reinterpret_cast<const uint2 *>(dtab + j * prime_words);
    ctx->ntt.inv[j] = reinterpret_cast<const uint2 *>(dtab + j * prime_words + dir_words);
  }
  g_cache[k] = ctx;
  *out = ctx;
  return PIR_OK;
}

}  // namespace gbpir
