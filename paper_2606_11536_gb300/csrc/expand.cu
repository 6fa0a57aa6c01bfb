// expand.cu -- server-side query expansion (Sec. 3.5 "ExpPack" expansion; App. C.2:
// SealPIR's recursive expansion after pre-scaling by 2^-levels; App. D.3: expansion
// keys with a gadget of ell digits in base t = 2^ceil(log2 q / ell)).
//
// A client sends one ciphertext encrypting m = sum_i m_i X^i instead of D1
// ciphertexts; the server expands it into the D1 ciphertexts Enc(m_i).  Level j of
// the recursion turns each of its 2^j ciphertexts c (index k) into
//     c + Subs(c, g_j)                               at index k,
//     c X^-2^j + Subs(c X^-2^j, g_j)                 at index k + 2^j,
// with g_j = n / 2^j + 1 and Subs = substitution X -> X^g followed by key switching
// back to the secret s with level j's key.
//
// GPU design: ciphertexts stay in NTT form between levels.  In that form the
// substitution is a permutation of slots (NTT(tau_g a)[k] = NTT(a)[perm(k)], no
// arithmetic) and X^-2^j is a pointwise factor.  The gadget digits are those of the
// level's input a-part, moved by the same shift and substitution as the ciphertext
// (signed digits in (-t, t); sum_k t^k tau_g(d_k X^-C) = tau_g(a X^-C)).  Moved
// digits are permuted and scaled copies of NTT(d_k), so both branches share one
// key-switching sum S[s] = sum_k NTT(d_k)[perm(s)] K_k[s]; branch 1 multiplies it by
// NTT(X^-C)[perm(s)].  Each level is four launches over all its ciphertexts:
//   1. inverse NTT of the a-parts;
//   2. decomposition: CRT lift of every coefficient (Garner, 128-bit) into ell
//      digits of w bits;
//   3. forward NTT of every digit row under every prime;
//   4. the shared sums and both branches' outputs, reduced once per residue.
#include <cstring>
#include <mutex>
#include <set>
#include <vector>

#include "common.cuh"

namespace gbpir {
namespace {

constexpr uint64_t kExpanderMagic = 0x4558504e44455231ull;  // "EXPNDER1"
constexpr uint32_t kMaxEll = 16;

// Decomposition constants: Garner inverses gc[k][i] = q_i^-1 mod q_k (i < k).
struct ExpConst {
  uint32_t q[PIR_MAX_L];
  uint64_t mu[PIR_MAX_L];
  uint32_t gc[PIR_MAX_L][PIR_MAX_L], gc_sh[PIR_MAX_L][PIR_MAX_L];
  uint32_t inv2l[PIR_MAX_L], inv2l_sh[PIR_MAX_L];  // 2^-levels mod q_i
};

template <typename T>
__device__ __forceinline__ T pick4(const T (&a)[PIR_MAX_L], uint32_t j) {
  T r = a[0];
#pragma unroll
  for (uint32_t i = 1; i < PIR_MAX_L; ++i) r = j == i ? a[i] : r;
  return r;
}

__device__ __forceinline__ uint32_t csub(uint32_t x, uint32_t m) { return min(x, x - m); }

// x * 2^-levels for every residue of rows [rows][n] (row r under prime r % L).
__global__ void k_expand_scale(uint32_t *__restrict__ x, uint64_t words, uint32_t logn, uint32_t L, ExpConst E) {
  for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < words; e += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t i = (uint32_t)((e >> logn) % L);
    const uint32_t q = pick4(E.q, i);
    x[e] = csub(shoup_mul(x[e], pick4(E.inv2l, i), pick4(E.inv2l_sh, i), q), q);
  }
}

// Gadget digits of the a-parts.  acoef [cts][L][n] (coefficient form, canonical);
// dig [cts][ell][n].  Thread = (ciphertext, coefficient u).
__global__ void k_expand_decompose(const uint32_t *__restrict__ acoef, uint64_t cts, uint32_t logn, uint32_t L,
                                   uint32_t ell, uint32_t w, ExpConst E, uint32_t *__restrict__ dig) {
  const uint32_t n = 1u << logn;
  const uint64_t total = cts << logn;
  for (uint64_t idx = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t ct = idx >> logn;
    const uint32_t u = (uint32_t)(idx & (n - 1));
    const uint32_t *a = acoef + ct * L * n + u;
    uint32_t x[PIR_MAX_L];
#pragma unroll
    for (uint32_t i = 0; i < PIR_MAX_L; ++i) x[i] = i < L ? a[(uint64_t)i * n] : 0;
    // Garner: x = a_0 + q_0 (a_1 + q_1 (a_2 + q_2 a_3)), a_k in [0, q_k)
#pragma unroll
    for (uint32_t k = 1; k < PIR_MAX_L; ++k) {
      if (k < L) {
        const uint32_t qk = E.q[k];
        uint32_t v = x[k];
#pragma unroll
        for (uint32_t i = 0; i < k; ++i) {
          const uint32_t ai = csub(x[i], qk);
          v = csub(shoup_mul(v + qk - ai, E.gc[k][i], E.gc_sh[k][i], qk), qk);
        }
        x[k] = v;
      }
    }
    unsigned __int128 X = 0;
#pragma unroll
    for (int k = PIR_MAX_L - 1; k >= 0; --k)
      if ((uint32_t)k < L) X = X * E.q[k] + x[k];
    const uint32_t mask = (1u << w) - 1;
    uint32_t *d = dig + ct * ell * n + u;
    for (uint32_t k = 0; k < ell; ++k) d[(uint64_t)k * n] = (uint32_t)(X >> (w * k)) & mask;
  }
}

// Key-switching sums and outputs of one level.  cur [cts][2][L][n] (NTT form, the
// level's inputs, C per query), dhat [cts][ell][L][n], key [ell][2][L][n], mon [L][n]
// (NTT of X^-C) with Shoup companions, perm [n].  Thread = (ciphertext, prime, slot s):
//   S_a = sum_k dhat_k[perm(s)] K_k.a[s],  S_b likewise,
//   branch 0 -> (a + S_a, b + b[p] + S_b),
//   branch 1 -> (a m[s] + S_a m[p], b m[s] + (b[p] + S_b) m[p]),   p = perm(s), m = mon.
// Output ciphertext (query b, index k) goes to out + (b * ostride + k) * 2 L n when
// k < olimit.
template <uint32_t L>
__global__ void k_expand_mac(const uint32_t *__restrict__ cur, const uint32_t *__restrict__ dhat,
                             const uint32_t *__restrict__ key, const uint32_t *__restrict__ mon,
                             const uint32_t *__restrict__ mon_sh, const uint32_t *__restrict__ perm, uint64_t cts,
                             uint32_t lev, uint32_t logn, uint32_t ell, uint32_t ostride, uint32_t olimit, ExpConst E,
                             uint32_t *__restrict__ out) {
  const uint32_t n = 1u << logn, C = 1u << lev;
  const uint64_t total = cts * L * (uint64_t)n;
  for (uint64_t idx = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t s = (uint32_t)(idx & (n - 1));
    const uint64_t row = idx >> logn;  // ciphertext * L + prime
    const uint32_t i = (uint32_t)(row % L);
    const uint64_t ct = row / L;
    const uint64_t b = ct >> lev;
    const uint32_t k0 = (uint32_t)(ct & (C - 1)), k1 = k0 + C;
    if (k0 >= olimit) continue;
    const uint32_t q = pick4(E.q, i);
    const uint64_t mu = pick4(E.mu, i);
    const uint32_t p = __ldg(perm + s);
    const uint32_t *dh = dhat + (ct * ell * L + i) * (uint64_t)n + p;
    const uint32_t *ka = key + (uint64_t)i * n + s;  // key[d][comp][i][s]
    const uint64_t kstride = 2ull * L * n, dstride = (uint64_t)L * n;
    const uint64_t k63 = (((uint64_t)1 << 63) / q) * q;
    uint64_t acc_a = 0, acc_b = 0;
    for (uint32_t d = 0; d < ell; ++d) {
      const uint32_t dv = dh[d * dstride];
      mac_wide(acc_a, dv, __ldg(ka + d * kstride));
      mac_wide(acc_b, dv, __ldg(ka + d * kstride + dstride));
      if ((d & 7) == 7) acc_a = fold63(acc_a, k63), acc_b = fold63(acc_b, k63);
    }
    const uint32_t sa = reduce64(acc_a, q, mu), sb = reduce64(acc_b, q, mu);
    const uint32_t *ca = cur + ((ct * 2 + 0) * L + i) * n;
    const uint32_t *cb = cur + ((ct * 2 + 1) * L + i) * n;
    const uint32_t a = ca[s], bs = cb[s], bp = cb[p];
    const uint32_t tb = csub(bp + sb, q);  // b[p] + S_b
    uint32_t *o0 = out + ((b * ostride + k0) * 2 * L + i) * (uint64_t)n + s;
    o0[0] = csub(a + sa, q);
    o0[dstride] = csub(bs + tb, q);
    if (k1 < olimit) {
      const uint32_t *m = mon + (uint64_t)i * n, *msh = mon_sh + (uint64_t)i * n;
      const uint32_t ms = __ldg(m + s), mss = __ldg(msh + s), mp = __ldg(m + p), mps = __ldg(msh + p);
      const uint32_t a1 = csub(csub(shoup_mul(a, ms, mss, q), q) + csub(shoup_mul(sa, mp, mps, q), q), q);
      const uint32_t b1 = csub(csub(shoup_mul(bs, ms, mss, q), q) + csub(shoup_mul(tb, mp, mps, q), q), q);
      uint32_t *o1 = out + ((b * ostride + k1) * 2 * L + i) * (uint64_t)n + s;
      o1[0] = a1;
      o1[dstride] = b1;
    }
  }
}

uint64_t mul_mod64(uint64_t a, uint64_t b, uint64_t m) { return (uint64_t)((unsigned __int128)a * b % m); }
uint64_t pow_mod64(uint64_t b, uint64_t e, uint64_t m);
uint32_t shoup32(uint32_t w, uint32_t q);

// Reduction and Garner constants of a ring (2^-levels too, for the expansion's pre-scaling).
ExpConst make_exp_const(const pir_params_t &p, uint32_t levels) {
  ExpConst E;
  std::memset(&E, 0, sizeof(E));
  for (uint32_t k = 0; k < p.L; ++k) {
    const uint32_t qk = p.q[k];
    E.q[k] = qk;
    E.mu[k] = ~0ull / qk;
    const uint32_t inv = (uint32_t)pow_mod64(pow_mod64(2, levels, qk), qk - 2, qk);
    E.inv2l[k] = inv;
    E.inv2l_sh[k] = shoup32(inv, qk);
    for (uint32_t i = 0; i < k; ++i) {
      E.gc[k][i] = (uint32_t)pow_mod64(p.q[i] % qk, qk - 2, qk);
      E.gc_sh[k][i] = shoup32(E.gc[k][i], qk);
    }
  }
  return E;
}
uint64_t pow_mod64(uint64_t b, uint64_t e, uint64_t m) {
  uint64_t r = 1 % m;
  b %= m;
  for (; e; e >>= 1) {
    if (e & 1) r = mul_mod64(r, b, m);
    b = mul_mod64(b, b, m);
  }
  return r;
}
uint32_t shoup32(uint32_t w, uint32_t q) { return (uint32_t)(((uint64_t)w << 32) / q); }
uint32_t brv32(uint32_t x, uint32_t bits) {
  uint32_t r = 0;
  for (uint32_t b = 0; b < bits; ++b) r |= ((x >> b) & 1u) << (bits - 1 - b);
  return r;
}

unsigned grid_for(uint64_t threads, unsigned block) {
  uint64_t g = (threads + block - 1) / block;
  const uint64_t cap = 152ull * 32;  // grid-stride loops cover the rest
  return (unsigned)(g < 1 ? 1 : (g > cap ? cap : g));
}

}  // namespace

struct pir_expander_impl {
  uint64_t magic;
  pir_params_t p;
  const ParamCtx *ctx;
  int device;
  uint32_t levels, ell, w;
  uint32_t *tables;  // one allocation: keys | mon | mon_sh | perm
  const uint32_t *keys, *mon, *mon_sh, *perm;
  ExpConst E;
};

namespace {
std::mutex g_ex_mu;
std::set<const void *> g_ex_live;

bool ex_live(const void *e) {
  std::lock_guard<std::mutex> lock(g_ex_mu);
  return e && g_ex_live.count(e) && static_cast<const pir_expander_impl *>(e)->magic == kExpanderMagic;
}

// ceil(log2 q) for q = prod q_j
uint32_t modulus_bits(const pir_params_t &p) {
  unsigned __int128 q = 1;
  for (uint32_t j = 0; j < p.L; ++j) q *= p.q[j];
  uint32_t bits = 0;
  while (bits < 128 && ((unsigned __int128)1 << bits) < q) ++bits;
  return bits;
}
}  // namespace

// Expansion of B packed ciphertexts (device, coefficient form [B][2][L][n]) into
// out [B][count][2][L][n] in NTT form.  Scratch from the stream-ordered allocator.
pir_status_t expand_device(const pir_expander_impl *ex, const uint32_t *packed, uint32_t B, uint32_t count,
                           uint32_t *out, cudaStream_t s, uint64_t *launch_count) {
  const ParamCtx &c = *ex->ctx;
  const uint32_t n = ex->p.n, L = ex->p.L, logn = c.logn, levels = ex->levels, ell = ex->ell;
  const uint64_t ctw = 2ull * L * n;             // words per ciphertext
  const uint64_t full = 1ull << levels;           // ciphertexts per query after the last level
  const uint64_t half = full >> 1 ? full >> 1 : 1;
  // per query: two ciphertext buffers of `full`, a-coefficients, digits and their NTT
  const uint64_t per_q = (2 * full * ctw + half * L * n + half * ell * n + half * ell * L * n) * 4;
  size_t free_b = 0, total_b = 0;
  uint64_t budget = 1ull << 30;
  if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess && free_b / 4 > budget) budget = free_b / 4;
  uint32_t Bc = (uint32_t)(budget / per_q);
  if (Bc < 1) Bc = 1;
  if (Bc > B) Bc = B;
  void *scratch = nullptr;
  cudaError_t e = cudaMallocAsync(&scratch, per_q * Bc, s);
  if (e != cudaSuccess) return cuda_status(e);
  uint32_t *cur = static_cast<uint32_t *>(scratch);
  uint32_t *nxt = cur + Bc * full * ctw;
  uint32_t *acoef = nxt + Bc * full * ctw;
  uint32_t *dig = acoef + Bc * half * L * n;
  uint32_t *dhat = dig + Bc * half * ell * n;
  pir_status_t st = PIR_OK;
  auto ck = [&](cudaError_t err) {
    if (err != cudaSuccess && st == PIR_OK) st = cuda_status(err);
    return err == cudaSuccess;
  };
  uint64_t launches = 0;
  for (uint32_t b0 = 0; b0 < B && st == PIR_OK; b0 += Bc) {
    const uint32_t nb = B - b0 < Bc ? B - b0 : Bc;
    // level-0 input: NTT of the packed ciphertexts, times 2^-levels
    if (!ck(launch_ntt_fwd(c, packed + (uint64_t)b0 * ctw, cur, (uint64_t)nb * 2 * L, s))) break;
    k_expand_scale<<<grid_for((uint64_t)nb * ctw, 256), 256, 0, s>>>(cur, (uint64_t)nb * ctw, logn, L, ex->E);
    if (!ck(cudaGetLastError())) break;
    launches += 2;
    for (uint32_t lev = 0; lev < levels; ++lev) {
      const uint32_t C = 1u << lev;
      const uint64_t cts = (uint64_t)nb * C;
      const bool last = lev + 1 == levels;
      // 1. a-parts to coefficient form: local row r reads ciphertext r / L, prime r % L
      if (!ck(launch_ntt_inv_rows(c, cur, 0, L, 2ull * L, 1, acoef, cts * L, s))) break;
      // 2. gadget digits of the a-parts
      k_expand_decompose<<<grid_for(cts * n, 256), 256, 0, s>>>(acoef, cts, logn, L, ell, ex->w, ex->E, dig);
      if (!ck(cudaGetLastError())) break;
      // 3. every digit row under every prime: local row r reads digit row r / L
      if (!ck(launch_ntt_fwd_rows_t(c, dig, 0, L, 1, 0, dhat, cts * ell * L, s))) break;
      // 4. key products and sums
      const uint32_t *key = ex->keys + (uint64_t)lev * ell * ctw;
      const uint32_t *mon = ex->mon + (uint64_t)lev * L * n, *msh = ex->mon_sh + (uint64_t)lev * L * n;
      const uint32_t *perm = ex->perm + (uint64_t)lev * n;
      uint32_t *dst = last ? out + (uint64_t)b0 * count * ctw : nxt;
      const uint32_t ostride = last ? count : 2 * C, olimit = last ? count : 2 * C;
      const unsigned gmac = grid_for(cts * L * n, 256);
      switch (L) {
        case 1: k_expand_mac<1><<<gmac, 256, 0, s>>>(cur, dhat, key, mon, msh, perm, cts, lev, logn, ell, ostride, olimit, ex->E, dst); break;
        case 2: k_expand_mac<2><<<gmac, 256, 0, s>>>(cur, dhat, key, mon, msh, perm, cts, lev, logn, ell, ostride, olimit, ex->E, dst); break;
        case 3: k_expand_mac<3><<<gmac, 256, 0, s>>>(cur, dhat, key, mon, msh, perm, cts, lev, logn, ell, ostride, olimit, ex->E, dst); break;
        default: k_expand_mac<4><<<gmac, 256, 0, s>>>(cur, dhat, key, mon, msh, perm, cts, lev, logn, ell, ostride, olimit, ex->E, dst); break;
      }
      if (!ck(cudaGetLastError())) break;
      launches += 4;
      uint32_t *t = cur;
      cur = nxt;
      nxt = t;
    }
    if (levels == 0 && st == PIR_OK) {  // one ciphertext: the scaled input itself
      ck(cudaMemcpyAsync(out + (uint64_t)b0 * count * ctw, cur, (uint64_t)nb * ctw * 4, cudaMemcpyDeviceToDevice, s));
    }
  }
  cudaFreeAsync(scratch, s);
  *launch_count = launches;
  return st;
}

uint32_t gadget_bits(const pir_params_t &p, uint32_t ell) { return (modulus_bits(p) + ell - 1) / ell; }

cudaError_t launch_gadget_digits(const ParamCtx &c, const uint32_t *coef, uint64_t polys, uint32_t ell,
                                 uint32_t *dig, cudaStream_t s) {
  if (polys == 0) return cudaSuccess;
  const ExpConst E = make_exp_const(c.p, 0);
  const uint32_t n = c.p.n;
  k_expand_decompose<<<grid_for(polys * n, 256), 256, 0, s>>>(coef, polys, c.logn, c.p.L, ell, gadget_bits(c.p, ell), E,
                                                              dig);
  return cudaGetLastError();
}

bool expander_view(pir_expander_t h, const pir_expander_impl **out) {
  if (!ex_live(h)) return false;
  *out = reinterpret_cast<const pir_expander_impl *>(h);
  return true;
}

bool expander_fits(const pir_expander_impl *ex, const pir_params_t &p) {
  if (ex->p.n != p.n || ex->p.L != p.L) return false;
  for (uint32_t j = 0; j < p.L; ++j)
    if (ex->p.q[j] != p.q[j] || ex->p.psi[j] != p.psi[j]) return false;
  return (1ull << ex->levels) >= p.D1;
}

}  // namespace gbpir

using namespace gbpir;

extern "C" {

pir_status_t pir_expander_create(const pir_params_t *params, uint32_t levels, uint32_t ell, const uint32_t *keys,
                                 int keys_on_device, void *stream, pir_expander_t *out) {
  if (!params || !keys || !out) return PIR_ERR_ARG;
  *out = nullptr;
  pir_status_t st = validate_params(params);
  if (st != PIR_OK) return st;
  const uint32_t n = params->n, L = params->L;
  if ((1u << levels) > n || levels > 31 || ell == 0 || ell > kMaxEll) return PIR_ERR_ARG;
  const uint32_t bits = modulus_bits(*params);
  const uint32_t w = (bits + ell - 1) / ell;
  if (w > 30 || w * (ell - 1) >= 128) return PIR_ERR_ARG;  // digits must stay below every prime's 2^30
  const ParamCtx *ctx = nullptr;
  if ((st = get_param_ctx(params, &ctx)) != PIR_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const uint32_t logn = ctx->logn;
  const uint64_t key_words = (uint64_t)levels * ell * 2 * L * n;
  const uint64_t mon_words = (uint64_t)levels * L * n;
  const uint64_t words = key_words + 2 * mon_words + (uint64_t)levels * n;

  auto *ex = new pir_expander_impl();
  ex->magic = kExpanderMagic;
  ex->p = *params;
  ex->p.D1 = ex->p.D2 = 0;
  ex->ctx = ctx;
  cudaGetDevice(&ex->device);
  ex->levels = levels;
  ex->ell = ell;
  ex->w = w;
  // host tables: NTT(X^-2^j) per prime (squares of NTT(X^-1)), slot permutations
  std::vector<uint32_t> host(2 * mon_words + (uint64_t)levels * n);
  uint32_t *hmon = host.data(), *hsh = hmon + mon_words, *hperm = hsh + mon_words;
  for (uint32_t i = 0; i < L; ++i) {
    const uint64_t q = params->q[i];
    const uint64_t psi_inv = pow_mod64(params->psi[i], q - 2, q);
    std::vector<uint64_t> v(n);
    for (uint32_t k = 0; k < n; ++k) v[k] = pow_mod64(psi_inv, 2ull * brv32(k, logn) + 1, q);  // X^-1 at slot k
    for (uint32_t j = 0; j < levels; ++j) {
      for (uint32_t k = 0; k < n; ++k) {
        const uint64_t o = ((uint64_t)j * L + i) * n + k;
        hmon[o] = (uint32_t)v[k];
        hsh[o] = shoup32((uint32_t)v[k], (uint32_t)q);
        v[k] = mul_mod64(v[k], v[k], q);  // X^-2^(j+1)
      }
    }
  }
  for (uint32_t j = 0; j < levels; ++j) {
    const uint64_t g = (n >> j) + 1, two_n = 2ull * n;
    for (uint32_t k = 0; k < n; ++k) {
      const uint64_t e = (2ull * brv32(k, logn) + 1) * g % two_n;
      hperm[(uint64_t)j * n + k] = brv32((uint32_t)((e - 1) / 2), logn);
    }
  }
  ex->E = make_exp_const(*params, levels);
  cudaError_t e = cudaMalloc(&ex->tables, words * 4);
  if (e != cudaSuccess) {
    delete ex;
    return cuda_status(e);
  }
  ex->keys = ex->tables;
  ex->mon = ex->tables + key_words;
  ex->mon_sh = ex->mon + mon_words;
  ex->perm = ex->mon_sh + mon_words;
  auto fail = [&](cudaError_t err) {
    cudaFree(ex->tables);
    delete ex;
    return cuda_status(err);
  };
  if ((e = cudaMemcpyAsync(ex->tables, keys, key_words * 4,
                           keys_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s)) != cudaSuccess)
    return fail(e);
  if ((e = cudaMemcpyAsync(ex->tables + key_words, host.data(), host.size() * 4, cudaMemcpyHostToDevice, s)) !=
      cudaSuccess)
    return fail(e);
  // keys to NTT form: rows [levels][ell][2][L] with row r under prime r % L
  if ((e = launch_ntt_fwd(*ctx, ex->tables, ex->tables, key_words / n, s)) != cudaSuccess) return fail(e);
  count_launches(1);
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return fail(e);
  {
    std::lock_guard<std::mutex> lock(g_ex_mu);
    g_ex_live.insert(ex);
  }
  *out = reinterpret_cast<pir_expander_t>(ex);
  return PIR_OK;
}

pir_status_t pir_expander_free(pir_expander_t h) {
  if (!ex_live(h)) return PIR_ERR_HANDLE;
  auto *ex = reinterpret_cast<pir_expander_impl *>(h);
  {
    std::lock_guard<std::mutex> lock(g_ex_mu);
    g_ex_live.erase(ex);
  }
  cudaDeviceSynchronize();
  cudaFree(ex->tables);
  ex->magic = 0;
  delete ex;
  return PIR_OK;
}

pir_status_t pir_expand(pir_expander_t h, const uint32_t *packed, uint32_t B, uint32_t count, uint32_t *out,
                        void *stream) {
  const pir_expander_impl *ex = nullptr;
  if (!expander_view(h, &ex)) return PIR_ERR_HANDLE;
  if (!packed || !out || B == 0 || count == 0 || count > (1u << ex->levels)) return PIR_ERR_ARG;
  if (((uintptr_t)packed & 15u) || ((uintptr_t)out & 15u)) return PIR_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  uint64_t launches = 0;
  pir_status_t st = expand_device(ex, packed, B, count, out, s, &launches);
  count_launches(launches);
  if (st != PIR_OK) return st;
  // the public result is in coefficient form, like the queries pir_answer takes
  cudaError_t e = launch_ntt_inv(*ex->ctx, out, out, (uint64_t)B * count * 2 * ex->p.L, s);
  if (e != cudaSuccess) return cuda_status(e);
  count_launches(1);
  return PIR_OK;
}

}  // extern "C"
