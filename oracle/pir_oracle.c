/*
 * pir_oracle.c -- plain, slow, CPU-only oracle for the RLWE-PIR first-dimension
 * scan of VIPIR (arXiv 2606.11536).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or call
 * this file: only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark use it.  It shares no code, header, table or constant generator with
 * the CUDA library; it computes every parameter (primes, roots of unity, powers)
 * from scratch, in uint64 / unsigned __int128, with one modular reduction per
 * operation and no lazy or Montgomery forms.
 *
 * What it computes, and where the paper defines it:
 *   - RNS prime selection: q_j = 1 (mod 2n) and q_j = 1 (mod p)      (App. A.4)
 *   - polynomial ring R_q = Z_q[X]/(X^n + 1), RNS rows per prime      (Sec. 2.3, App. A.2)
 *   - negacyclic NTT / inverse NTT, one row per prime                 (Sec. 2.3)
 *   - RLWE encryption / decryption with Delta = floor(q/p)            (App. A.2)
 *   - modulus switching q -> q_0: round(x q_0 / q) mod q_0, and decryption over
 *     the single prime q_0 afterwards                                 (App. D.5, Sec. 4.3)
 *   - scalar-HE (LWE) DB GEMM: out = DB Q^T mod 2^32 with an INT8 DB         (Sec. 2.5, 4.1, App. A.1)
 *   - RGSW encryption, RGSW-RLWE external product and the folding of the
 *     remaining dimensions c_2j + RGSW (x) (c_2j+1 - c_2j)         (Sec. 3.2, 3.6, App. D.3)
 *   - query expansion: substitutions tau_g, key switching with the base-t gadget
 *     (t = 2^ceil(log2 q / ell)), SealPIR's recursive expansion with the
 *     2^-levels pre-scaling                                         (Sec. 3.5, App. C.2, D.3)
 *   - first-dimension folding: out_c = sum_i DB[i][c] * ct_i in R_q^2 (Sec. 3.2, Sec. 4 "INT32
 *     modular GEMM", Sec. 4.2): in the NTT domain, for every prime q_j and slot k,
 *     out[b][c][k] = sum_i DB[i][c][k] * Q[b][i][k]  (mod q_j).
 *
 * Readings where the paper is silent:
 *   - primes are the L largest primes in (2^29, 2^30) with q = 1 mod max(2n, p);
 *   - psi_j = h^((q_j-1)/(2n)) for the smallest h >= 2 with psi_j^n = -1;
 *   - NTT(a)[k] = sum_t a_t psi^((2 brv(k) + 1) t)  (bit-reversed evaluation order);
 *   - a raw DB is a little-endian bit stream of log2(p)-bit coefficients, poly after
 *     poly, poly (i, c) at position i*D2 + c;
 *   - each query ciphertext contributes its a- and b-polynomial as two GEMM rows;
 *   - modulus switching keeps q_0, the largest prime (#RNS = 1, about 2^30), and
 *     rounds to nearest;
 *   - expansion level j substitutes with g = n/2^j + 1 and keeps the SealPIR index
 *     order (c + Subs(c) at k, c X^-2^j + Subs(.) at k + 2^j); the gadget digits are
 *     those of the CRT lift in [0, q) of each coefficient of the level's input
 *     a-part, moved (with their signs) by the same shift and substitution as the
 *     ciphertext, so a moved digit lies in (-t, t).  The textbook order (digits of
 *     the substituted a-part, in [0, t)) is kept beside it (orc_subs_textbook,
 *     orc_expand_textbook); with error-free keys the two give the same phase.
 *
 * Parity: pinned.  The tests check this file against primality by an independent
 * library, the defining congruences, the NTT evaluated by its definition, schoolbook
 * negacyclic multiplication, the convolution theorem, and the BFV decryption
 * invariant (decrypting the answer returns exactly the requested record); modulus
 * switching against values built as t Q' + r, the rounding-error bound of App. D.5
 * and decryption after the switch; substitution against polynomial evaluation at
 * the primitive 2n-th roots and the ring-automorphism laws, key switching and
 * expansion against decryption (every coefficient, with the exact aliasing above
 * 2^levels) and worst-case noise bounds, and an expanded query that answers and
 * decrypts.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef uint8_t u8;
typedef uint32_t u32;
typedef uint64_t u64;
typedef unsigned __int128 u128;
typedef __int128 i128;
typedef int64_t i64;

#define ORC_MAX_L 4

/* Parameters of one PIR instance, as the oracle sees them.  Own layout, not the
 * CUDA library's. */
typedef struct {
  u32 n;        /* ring degree (a power of two)                       */
  u32 L;        /* number of RNS primes                                */
  u32 log2p;    /* plaintext modulus p = 2^log2p                       */
  u32 D1, D2;   /* first-dimension size (summed index i), columns (c) */
  u64 q[ORC_MAX_L];
  u64 psi[ORC_MAX_L];
} orc_params;

/* ------------------------------------------------------------------------- */
/* Modular arithmetic, one reduction per operation.                          */
/* ------------------------------------------------------------------------- */

static u64 mulmod(u64 a, u64 b, u64 m) {
  if (a <= 0xFFFFFFFFull && b <= 0xFFFFFFFFull) return (a * b) % m; /* product fits u64 */
  return (u64)(((u128)a * b) % m);
}
static u64 addmod(u64 a, u64 b, u64 m) { return (a + b) % m; }
static u64 submod(u64 a, u64 b, u64 m) { return (a + m - b) % m; }

u64 orc_powmod(u64 base, u64 e, u64 m) {
  u64 r = 1 % m;
  base %= m;
  while (e) {
    if (e & 1) r = mulmod(r, base, m);
    base = mulmod(base, base, m);
    e >>= 1;
  }
  return r;
}

/* Inverse modulo a prime by Fermat's little theorem. */
static u64 invmod_prime(u64 a, u64 q) { return orc_powmod(a, q - 2, q); }

/* Deterministic Miller-Rabin for 64-bit inputs with the first twelve primes as
 * bases (these bases are known to decide primality for every n < 3.3e24). */
int orc_is_prime(u64 x) {
  static const u64 bases[12] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
  if (x < 2) return 0;
  for (int i = 0; i < 12; i++) {
    if (x == bases[i]) return 1;
    if (x % bases[i] == 0) return 0;
  }
  u64 d = x - 1;
  int s = 0;
  while ((d & 1) == 0) {
    d >>= 1;
    s++;
  }
  for (int i = 0; i < 12; i++) {
    u64 y = orc_powmod(bases[i], d, x);
    if (y == 1 || y == x - 1) continue;
    int composite = 1;
    for (int r = 1; r < s; r++) {
      y = mulmod(y, y, x);
      if (y == x - 1) {
        composite = 0;
        break;
      }
    }
    if (composite) return 0;
  }
  return 1;
}

/* App. A.4: q_j = 1 mod 2n enables the negacyclic NTT; q_j = 1 mod p makes
 * Delta*p + 1 = q.  Both moduli are powers of two, so the joint condition is
 * q_j = 1 mod max(2n, p).  We take the L largest such primes in (2^29, 2^30),
 * in decreasing order.  Returns 0 on success, -1 if fewer than L exist. */
int orc_select_primes(u32 n, u32 log2p, u32 L, u64 *q_out) {
  if (L == 0 || L > ORC_MAX_L || n < 2 || (n & (n - 1)) || log2p == 0 || log2p > 28) return -1;
  u64 M = 2ull * n;
  u64 p = 1ull << log2p;
  if (p > M) M = p;
  const u64 lo = 1ull << 29, hi = 1ull << 30;
  u64 c = ((hi - 2) / M) * M + 1; /* largest value = 1 mod M below 2^30 */
  u32 found = 0;
  while (found < L && c > lo) {
    if (orc_is_prime(c)) q_out[found++] = c;
    c -= M;
  }
  return found == L ? 0 : -1;
}

/* psi = h^((q-1)/(2n)) for the smallest h >= 2 with psi^n = -1 (mod q); such a
 * psi is a primitive 2n-th root of unity. */
u64 orc_find_psi(u64 q, u32 n) {
  u64 e = (q - 1) / (2ull * n);
  for (u64 h = 2; h < q; h++) {
    u64 psi = orc_powmod(h, e, q);
    if (orc_powmod(psi, n, q) == q - 1) return psi;
  }
  return 0;
}

int orc_make_params(u32 n, u32 log2p, u32 D1, u32 D2, u32 L, orc_params *P) {
  memset(P, 0, sizeof(*P));
  P->n = n;
  P->L = L;
  P->log2p = log2p;
  P->D1 = D1;
  P->D2 = D2;
  if (orc_select_primes(n, log2p, L, P->q) != 0) return -1;
  for (u32 j = 0; j < L; j++) {
    P->psi[j] = orc_find_psi(P->q[j], n);
    if (P->psi[j] == 0) return -1;
  }
  return 0;
}

/* ------------------------------------------------------------------------- */
/* NTT                                                                       */
/* ------------------------------------------------------------------------- */

static u32 ilog2(u32 n) {
  u32 l = 0;
  while ((1u << l) < n) l++;
  return l;
}

static u32 bitrev(u32 x, u32 bits) {
  u32 r = 0;
  for (u32 b = 0; b < bits; b++) r |= ((x >> b) & 1u) << (bits - 1 - b);
  return r;
}

/* Definition (O(n^2)): out[k] = sum_t a_t * psi^((2 brv(k) + 1) t) mod q, i.e. the
 * polynomial evaluated at the odd powers of psi (the roots of X^n + 1), listed in
 * bit-reversed order. */
void orc_ntt_definition(const u32 *a, u32 *out, u32 n, u64 q, u64 psi) {
  u32 lg = ilog2(n);
  for (u32 k = 0; k < n; k++) {
    u64 root = orc_powmod(psi, 2ull * bitrev(k, lg) + 1, q);
    u64 acc = 0, x = 1;
    for (u32 t = 0; t < n; t++) {
      acc = addmod(acc, mulmod(a[t] % q, x, q), q);
      x = mulmod(x, root, q);
    }
    out[k] = (u32)acc;
  }
}

/* Inverse of the definition (O(n^2)): a_t = n^-1 * sum_k A[k] * root_k^-t. */
void orc_intt_definition(const u32 *A, u32 *out, u32 n, u64 q, u64 psi) {
  u32 lg = ilog2(n);
  u64 ninv = invmod_prime(n, q);
  for (u32 t = 0; t < n; t++) out[t] = 0;
  for (u32 k = 0; k < n; k++) {
    u64 root = orc_powmod(psi, 2ull * bitrev(k, lg) + 1, q);
    u64 rinv = invmod_prime(root, q);
    u64 x = 1;
    for (u32 t = 0; t < n; t++) {
      out[t] = (u32)addmod(out[t], mulmod(A[k] % q, x, q), q);
      x = mulmod(x, rinv, q);
    }
  }
  for (u32 t = 0; t < n; t++) out[t] = (u32)mulmod(out[t], ninv, q);
}

/* Powers psi^brv(i) for i < n, the twiddles of the radix-2 transform below. */
static void psi_powers_brv(u64 *tab, u32 n, u64 q, u64 psi) {
  u32 lg = ilog2(n);
  for (u32 i = 0; i < n; i++) tab[i] = orc_powmod(psi, bitrev(i, lg), q);
}

/* Fast forward negacyclic NTT, in place, radix-2 decimation in time with the
 * psi powers folded into the butterflies.  Stage with half-width t: the block g
 * of 2t elements uses w = psi^brv(m + g) with m = n / (2t).  The result equals
 * orc_ntt_definition (pinned by the tests). */
void orc_ntt_fwd(u32 *a, u32 n, u64 q, u64 psi) {
  u64 *w = (u64 *)malloc(sizeof(u64) * n);
  psi_powers_brv(w, n, q, psi);
  for (u32 i = 0; i < n; i++) a[i] = (u32)(a[i] % q);
  u32 t = n;
  for (u32 m = 1; m < n; m <<= 1) {
    t >>= 1;
    for (u32 g = 0; g < m; g++) {
      u64 wg = w[m + g];
      for (u32 x = 2 * g * t; x < 2 * g * t + t; x++) {
        u64 u = a[x], v = mulmod(a[x + t], wg, q);
        a[x] = (u32)addmod(u, v, q);
        a[x + t] = (u32)submod(u, v, q);
      }
    }
  }
  free(w);
}

/* Fast inverse: the butterflies of orc_ntt_fwd undone in reverse order
 * (decimation in frequency with psi^-brv(m + g)), then a scale by n^-1. */
void orc_ntt_inv(u32 *a, u32 n, u64 q, u64 psi) {
  u64 *w = (u64 *)malloc(sizeof(u64) * n);
  psi_powers_brv(w, n, q, invmod_prime(psi, q));
  u64 ninv = invmod_prime(n, q);
  for (u32 i = 0; i < n; i++) a[i] = (u32)(a[i] % q);
  u32 t = 1;
  for (u32 m = n >> 1; m >= 1; m >>= 1) {
    for (u32 g = 0; g < m; g++) {
      u64 wg = w[m + g];
      for (u32 x = 2 * g * t; x < 2 * g * t + t; x++) {
        u64 u = a[x], v = a[x + t];
        a[x] = (u32)addmod(u, v, q);
        a[x + t] = (u32)mulmod(submod(u, v, q), wg, q);
      }
    }
    t <<= 1;
  }
  for (u32 i = 0; i < n; i++) a[i] = (u32)mulmod(a[i], ninv, q);
  free(w);
}

/* Apply the fast NTT / INTT to `count` RNS polynomials laid out [count][L][n]. */
void orc_ntt_fwd_rns(const orc_params *P, u32 *polys, u64 count) {
  for (u64 c = 0; c < count; c++)
    for (u32 j = 0; j < P->L; j++) orc_ntt_fwd(polys + (c * P->L + j) * P->n, P->n, P->q[j], P->psi[j]);
}
void orc_ntt_inv_rns(const orc_params *P, u32 *polys, u64 count) {
  for (u64 c = 0; c < count; c++)
    for (u32 j = 0; j < P->L; j++) orc_ntt_inv(polys + (c * P->L + j) * P->n, P->n, P->q[j], P->psi[j]);
}

/* Schoolbook product in Z_q[X]/(X^n + 1): X^n = -1, so the term a_s*b_t with
 * s + t >= n lands at s + t - n with a minus sign. */
void orc_negacyclic_schoolbook(const u32 *a, const u32 *b, u32 *out, u32 n, u64 q) {
  for (u32 k = 0; k < n; k++) out[k] = 0;
  for (u32 s = 0; s < n; s++) {
    for (u32 t = 0; t < n; t++) {
      u64 pr = mulmod(a[s] % q, b[t] % q, q);
      u32 k = s + t;
      if (k < n)
        out[k] = (u32)addmod(out[k], pr, q);
      else
        out[k - n] = (u32)submod(out[k - n], pr, q);
    }
  }
}

/* ------------------------------------------------------------------------- */
/* Database encoding                                                         */
/* ------------------------------------------------------------------------- */

/* Coefficient t of plaintext polynomial `poly`: bits [(poly*n + t)*log2p, +log2p)
 * of the raw byte stream, little-endian bit order (bit b is bit b%8 of byte b/8). */
static u32 raw_coeff(const u8 *raw, u32 log2p, u32 n, u64 poly, u32 t) {
  const u64 bit0 = ((u64)poly * n + t) * log2p, bit_end = bit0 + log2p; /* [bit0, bit_end) */
  const u64 byte0 = bit0 >> 3;
  u64 w = 0;
  for (u64 by = byte0; by * 8 < bit_end; by++) w |= (u64)raw[by] << (8 * (by - byte0));
  return (u32)((w >> (bit0 & 7)) & ((1ull << log2p) - 1));
}

void orc_unpack_poly(const u8 *raw, u32 log2p, u32 n, u64 poly, u32 *coef) {
  for (u32 t = 0; t < n; t++) coef[t] = raw_coeff(raw, log2p, n, poly, t);
}

/* ------------------------------------------------------------------------- */
/* Threads: a plain static partition of [0, count) over worker threads.      */
/* ------------------------------------------------------------------------- */

typedef void (*orc_task_fn)(void *ctx, u64 item, void *scratch);
typedef struct {
  orc_task_fn fn;
  void *ctx;
  u64 begin, end;
  size_t scratch_bytes;
} orc_worker;

static void *orc_worker_main(void *arg) {
  orc_worker *w = (orc_worker *)arg;
  void *scratch = w->scratch_bytes ? malloc(w->scratch_bytes) : NULL;
  for (u64 it = w->begin; it < w->end; it++) w->fn(w->ctx, it, scratch);
  free(scratch);
  return NULL;
}

static void orc_parallel_for(u64 count, int nthreads, orc_task_fn fn, void *ctx, size_t scratch_bytes) {
  if (nthreads < 1) nthreads = 1;
  if ((u64)nthreads > count) nthreads = (int)(count ? count : 1);
  pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * nthreads);
  orc_worker *ws = (orc_worker *)malloc(sizeof(orc_worker) * nthreads);
  for (int t = 0; t < nthreads; t++) {
    ws[t].fn = fn;
    ws[t].ctx = ctx;
    ws[t].begin = count * t / nthreads;
    ws[t].end = count * (t + 1) / nthreads;
    ws[t].scratch_bytes = scratch_bytes;
  }
  for (int t = 1; t < nthreads; t++) pthread_create(&th[t], NULL, orc_worker_main, &ws[t]);
  orc_worker_main(&ws[0]);
  for (int t = 1; t < nthreads; t++) pthread_join(th[t], NULL);
  free(th);
  free(ws);
}

/* ------------------------------------------------------------------------- */
/* The answer: first-dimension folding                                       */
/* ------------------------------------------------------------------------- */


/* NTT-form of plaintext DB polynomials.  poly_ids[t] = i*D2 + c; out is
 * [count][L][n].  Lifting a coefficient < p < q_j to residue j is the identity. */
typedef struct {
  const orc_params *P;
  const u8 *raw;
  const u64 *ids;
  u32 *out;
} encode_ctx;

static void encode_one(void *vctx, u64 t, void *scratch) {
  (void)scratch;
  encode_ctx *x = (encode_ctx *)vctx;
  const orc_params *P = x->P;
  for (u32 j = 0; j < P->L; j++) {
    u32 *dst = x->out + (t * P->L + j) * P->n;
    orc_unpack_poly(x->raw, P->log2p, P->n, x->ids[t], dst);
    orc_ntt_fwd(dst, P->n, P->q[j], P->psi[j]);
  }
}

void orc_encode_polys(const orc_params *P, const u8 *raw, const u64 *poly_ids, u64 count, u32 *out, int nthreads) {
  encode_ctx x = {P, raw, poly_ids, out};
  orc_parallel_for(count, nthreads, encode_one, &x, 0);
}

/* Forward NTT of every query polynomial: queries [B][D1][2][L][n] -> same layout. */
typedef struct {
  const orc_params *P;
  u32 *polys;
} ntt_ctx;

static void ntt_one(void *vctx, u64 r, void *scratch) {
  (void)scratch;
  ntt_ctx *x = (ntt_ctx *)vctx;
  u32 j = (u32)(r % x->P->L);
  orc_ntt_fwd(x->polys + r * x->P->n, x->P->n, x->P->q[j], x->P->psi[j]);
}
static void intt_one(void *vctx, u64 r, void *scratch) {
  (void)scratch;
  ntt_ctx *x = (ntt_ctx *)vctx;
  u32 j = (u32)(r % x->P->L);
  orc_ntt_inv(x->polys + r * x->P->n, x->P->n, x->P->q[j], x->P->psi[j]);
}

void orc_ntt_fwd_rns_mt(const orc_params *P, u32 *polys, u64 count, int nthreads) {
  ntt_ctx x = {P, polys};
  orc_parallel_for(count * P->L, nthreads, ntt_one, &x, 0);
}
void orc_ntt_inv_rns_mt(const orc_params *P, u32 *polys, u64 count, int nthreads) {
  ntt_ctx x = {P, polys};
  orc_parallel_for(count * P->L, nthreads, intt_one, &x, 0);
}

/* The answer for a set of columns, given their NTT-form DB polynomials.
 *   dbhat     [ncols][D1][L][n]   NTT form of DB[i][cols[t]]
 *   qhat      [B][D1][2][L][n]    NTT form of the query ciphertexts
 *   responses [B][ncols][2][L][n] coefficient form
 * For every prime j and slot k: acc[b][comp][j][k] = sum_i dbhat[i][j][k] * qhat[b][i][comp][j][k]
 * mod q_j (Sec. 4 / Sec. 4.2), then the inverse NTT of acc. */
typedef struct {
  const orc_params *P;
  const u32 *dbhat;
  const u32 *qhat;
  u32 B, ncols;
  u32 *resp;
} fold_ctx;

static void fold_column(void *vctx, u64 t, void *scratch) {
  fold_ctx *x = (fold_ctx *)vctx;
  const orc_params *P = x->P;
  const u32 n = P->n, L = P->L, D1 = P->D1, B = x->B;
  u32 *acc = (u32 *)scratch; /* [B][2][L][n] */
  memset(acc, 0, sizeof(u32) * (size_t)B * 2 * L * n);
  for (u32 i = 0; i < D1; i++)
    for (u32 j = 0; j < L; j++) {
      const u32 *d = x->dbhat + ((t * D1 + i) * L + j) * n;
      for (u32 b = 0; b < B; b++)
        for (u32 comp = 0; comp < 2; comp++) {
          const u32 *qv = x->qhat + ((((u64)b * D1 + i) * 2 + comp) * L + j) * n;
          u32 *av = acc + (((u64)b * 2 + comp) * L + j) * n;
          for (u32 k = 0; k < n; k++) av[k] = (u32)addmod(av[k], mulmod(d[k], qv[k], P->q[j]), P->q[j]);
        }
    }
  for (u32 b = 0; b < B; b++)
    for (u32 comp = 0; comp < 2; comp++)
      for (u32 j = 0; j < L; j++) {
        u32 *av = acc + (((u64)b * 2 + comp) * L + j) * n;
        orc_ntt_inv(av, n, P->q[j], P->psi[j]);
        memcpy(x->resp + (((((u64)b * x->ncols + t) * 2 + comp) * L + j) * n), av, sizeof(u32) * n);
      }
}

void orc_answer_encoded(const orc_params *P, const u32 *dbhat, u32 ncols, const u32 *qhat, u32 B, u32 *responses,
                        int nthreads) {
  fold_ctx x = {P, dbhat, qhat, B, ncols, responses};
  orc_parallel_for(ncols, nthreads, fold_column, &x, sizeof(u32) * (size_t)B * 2 * P->L * P->n);
}

/* Whole answer for the requested columns from the raw DB and coefficient-form
 * queries: encode the needed DB polynomials, NTT the queries, fold, INTT.
 * Returns 0, or -1 if memory runs out. */
int orc_answer(const orc_params *P, const u8 *raw, const u32 *queries, u32 B, const u32 *cols, u32 ncols,
               u32 *responses, int nthreads) {
  const u64 qwords = (u64)B * P->D1 * 2 * P->L * P->n;
  u32 *qhat = (u32 *)malloc(sizeof(u32) * qwords);
  u64 *ids = (u64 *)malloc(sizeof(u64) * (u64)ncols * P->D1);
  u32 *dbhat = (u32 *)malloc(sizeof(u32) * (u64)ncols * P->D1 * P->L * P->n);
  if (!qhat || !ids || !dbhat) {
    free(qhat);
    free(ids);
    free(dbhat);
    return -1;
  }
  memcpy(qhat, queries, sizeof(u32) * qwords);
  orc_ntt_fwd_rns_mt(P, qhat, (u64)B * P->D1 * 2, nthreads);
  for (u32 t = 0; t < ncols; t++)
    for (u32 i = 0; i < P->D1; i++) ids[(u64)t * P->D1 + i] = (u64)i * P->D2 + cols[t];
  orc_encode_polys(P, raw, ids, (u64)ncols * P->D1, dbhat, nthreads);
  orc_answer_encoded(P, dbhat, ncols, qhat, B, responses, nthreads);
  free(qhat);
  free(ids);
  free(dbhat);
  return 0;
}

/* The same answer straight from the definition of folding (Sec. 3.2): every
 * response polynomial is sum_i DB[i][c](X) * ct_i(X) in Z_{q_j}[X]/(X^n + 1) by
 * schoolbook products, no NTT anywhere.  O(D1 n^2) per output; tiny rings only. */
void orc_answer_schoolbook(const orc_params *P, const u8 *raw, const u32 *queries, u32 B, u32 *responses) {
  const u32 n = P->n, L = P->L, D1 = P->D1, D2 = P->D2;
  u32 *d = (u32 *)malloc(sizeof(u32) * n);
  u32 *prod = (u32 *)malloc(sizeof(u32) * n);
  for (u32 b = 0; b < B; b++)
    for (u32 c = 0; c < D2; c++)
      for (u32 comp = 0; comp < 2; comp++)
        for (u32 j = 0; j < L; j++) {
          u32 *out = responses + ((((u64)b * D2 + c) * 2 + comp) * L + j) * n;
          memset(out, 0, sizeof(u32) * n);
          for (u32 i = 0; i < D1; i++) {
            orc_unpack_poly(raw, P->log2p, n, (u64)i * D2 + c, d);
            const u32 *ct = queries + ((((u64)b * D1 + i) * 2 + comp) * L + j) * n;
            orc_negacyclic_schoolbook(d, ct, prod, n, P->q[j]);
            for (u32 k = 0; k < n; k++) out[k] = (u32)addmod(out[k], prod[k], P->q[j]);
          }
        }
  free(d);
  free(prod);
}

/* ------------------------------------------------------------------------- */
/* Toy RLWE (BFV-style) client, App. A.2                                     */
/* ------------------------------------------------------------------------- */

/* Product in Z_q[X]/(X^n+1) through the (pinned) fast NTT. */
static void ring_mul(const u32 *a, const u32 *b, u32 *out, u32 n, u64 q, u64 psi) {
  u32 *fb = (u32 *)malloc(sizeof(u32) * n);
  memcpy(out, a, sizeof(u32) * n);
  memcpy(fb, b, sizeof(u32) * n);
  orc_ntt_fwd(out, n, q, psi);
  orc_ntt_fwd(fb, n, q, psi);
  for (u32 k = 0; k < n; k++) out[k] = (u32)mulmod(out[k], fb[k], q);
  orc_ntt_inv(out, n, q, psi);
  free(fb);
}

/* q = prod_j q_j (< 2^120 for L <= 4) and Delta = floor(q / p). */
static u128 full_modulus(const orc_params *P) {
  u128 q = 1;
  for (u32 j = 0; j < P->L; j++) q *= P->q[j];
  return q;
}

/* Writes q (as two u64 halves, low first) and Delta; lets the tests check
 * Delta*p + 1 = q (App. A.4). */
void orc_modulus_info(const orc_params *P, u64 *q_lo_hi, u64 *delta_lo_hi) {
  u128 q = full_modulus(P);
  u128 delta = q >> P->log2p; /* floor(q / p), p = 2^log2p */
  q_lo_hi[0] = (u64)q;
  q_lo_hi[1] = (u64)(q >> 64);
  delta_lo_hi[0] = (u64)delta;
  delta_lo_hi[1] = (u64)(delta >> 64);
}

/* Encrypt(m) -> (a, b) with a*s + b = Delta*m + e (mod q).
 *   s [n] ternary in {-1,0,1};  a [L][n] residues (uniform mod q by CRT);
 *   e [n] small signed error;   m [n] plaintext coefficients in [0, p).
 *   ct [2][L][n]: component 0 = a, 1 = b. */
void orc_bfv_encrypt(const orc_params *P, const int8_t *s, const u32 *a, const int8_t *e, const u32 *m, u32 *ct) {
  const u32 n = P->n, L = P->L;
  u128 delta = full_modulus(P) >> P->log2p;
  u32 *sj = (u32 *)malloc(sizeof(u32) * n);
  u32 *as = (u32 *)malloc(sizeof(u32) * n);
  for (u32 j = 0; j < L; j++) {
    const u64 q = P->q[j];
    const u64 dj = (u64)(delta % q);
    for (u32 t = 0; t < n; t++) sj[t] = (u32)((s[t] + (i128)q) % q);
    ring_mul(a + (u64)j * n, sj, as, n, q, P->psi[j]);
    for (u32 t = 0; t < n; t++) {
      u64 et = (u64)((e[t] + (i128)q) % q);
      u64 bt = addmod(mulmod(dj, m[t] % q, q), et, q);
      ct[(u64)j * n + t] = a[(u64)j * n + t];
      ct[((u64)L + j) * n + t] = (u32)submod(bt, as[t], q);
    }
  }
  free(sj);
  free(as);
}

/* Phase phi = a*s + b (mod q), recombined from the residues by CRT (Garner). */
static void phase(const orc_params *P, const int8_t *s, const u32 *ct, u128 *phi) {
  const u32 n = P->n, L = P->L;
  u32 *sj = (u32 *)malloc(sizeof(u32) * n);
  u32 *res = (u32 *)malloc(sizeof(u32) * (size_t)L * n);
  for (u32 j = 0; j < L; j++) {
    const u64 q = P->q[j];
    for (u32 t = 0; t < n; t++) sj[t] = (u32)((s[t] + (i128)q) % q);
    ring_mul(ct + (u64)j * n, sj, res + (u64)j * n, n, q, P->psi[j]);
    for (u32 t = 0; t < n; t++) res[(u64)j * n + t] = (u32)addmod(res[(u64)j * n + t], ct[((u64)L + j) * n + t], q);
  }
  for (u32 t = 0; t < n; t++) {
    u128 x = res[t], M = P->q[0];
    for (u32 j = 1; j < L; j++) {
      const u64 q = P->q[j];
      u64 xm = (u64)(x % q);
      u64 inv = invmod_prime((u64)(M % q), q);
      u64 h = mulmod(submod(res[(u64)j * n + t], xm, q), inv, q);
      x += (u128)h * M;
      M *= q;
    }
    phi[t] = x;
  }
  free(sj);
  free(res);
}

/* Decrypt: centre the phase in (-q/2, q/2], m = round(phi / Delta) mod p. */
void orc_bfv_decrypt(const orc_params *P, const int8_t *s, const u32 *ct, u32 *m_out) {
  const u32 n = P->n;
  const u128 q = full_modulus(P);
  const i128 delta = (i128)(q >> P->log2p);
  const u64 pmask = (1ull << P->log2p) - 1;
  u128 *phi = (u128 *)malloc(sizeof(u128) * n);
  phase(P, s, ct, phi);
  for (u32 t = 0; t < n; t++) {
    i128 v = (phi[t] > q / 2) ? (i128)phi[t] - (i128)q : (i128)phi[t];
    /* round(v / delta) = floor((2v + delta) / (2 delta)), floor for negatives too */
    i128 num = 2 * v + delta, den = 2 * delta;
    i128 qt = num / den;
    if ((num % den != 0) && (num < 0)) qt -= 1;
    m_out[t] = (u32)((u64)qt & pmask);
  }
  free(phi);
}

/* Noise of a ciphertext that should encrypt m: the centred phase minus Delta*m,
 * per coefficient, as a signed 64-bit value (saturated).  Used to report the
 * decryption margin against Delta/2 (App. A.2). */
void orc_bfv_noise(const orc_params *P, const int8_t *s, const u32 *ct, const u32 *m, int64_t *noise) {
  const u32 n = P->n;
  const u128 q = full_modulus(P);
  const u128 delta = q >> P->log2p;
  u128 *phi = (u128 *)malloc(sizeof(u128) * n);
  phase(P, s, ct, phi);
  for (u32 t = 0; t < n; t++) {
    u128 dm = (delta * m[t]) % q;
    u128 diff = (phi[t] + q - dm) % q;
    i128 v = (diff > q / 2) ? (i128)diff - (i128)q : (i128)diff;
    if (v > (i128)INT64_MAX) v = INT64_MAX;
    if (v < (i128)INT64_MIN) v = INT64_MIN;
    noise[t] = (int64_t)v;
  }
  free(phi);
}

/* ------------------------------------------------------------------------- */
/* Freivalds check of a full response tensor                                 */
/* ------------------------------------------------------------------------- */

/* With r[j][c] random residues, folding is linear in the DB, so
 *   sum_c r_c * R[b][c]  ==  INTT( sum_i NTT(y_i) . NTT(ct_{b,i}) ),  y_i = sum_c r_c * DB[i][c]
 * holds for a correct R; a wrong coefficient survives with probability <= 1/q_j.
 * The check never forms the NTT-form DB.  Returns the number of mismatching
 * coefficients over [B][2][L][n], or -1 if memory runs out. */
typedef struct {
  const orc_params *P;
  const u8 *raw;
  const u32 *r;
  u32 *yhat; /* [D1][L][n] */
} fr_ctx;

static void fr_row(void *vctx, u64 i, void *scratch) {
  fr_ctx *x = (fr_ctx *)vctx;
  const orc_params *P = x->P;
  const u32 n = P->n, L = P->L, D2 = P->D2;
  u32 *d = (u32 *)scratch;
  u32 *y = x->yhat + i * L * n;
  memset(y, 0, sizeof(u32) * L * n);
  for (u32 c = 0; c < D2; c++) {
    orc_unpack_poly(x->raw, P->log2p, n, i * D2 + c, d);
    for (u32 j = 0; j < L; j++) {
      const u64 q = P->q[j], rc = x->r[(u64)j * D2 + c];
      u32 *yj = y + (u64)j * n;
      for (u32 t = 0; t < n; t++) yj[t] = (u32)addmod(yj[t], mulmod(d[t], rc, q), q);
    }
  }
  for (u32 j = 0; j < L; j++) orc_ntt_fwd(y + (u64)j * n, n, P->q[j], P->psi[j]);
}

long long orc_freivalds(const orc_params *P, const u8 *raw, const u32 *queries, u32 B, const u32 *responses,
                        const u32 *r, int nthreads) {
  const u32 n = P->n, L = P->L, D1 = P->D1, D2 = P->D2;
  u32 *yhat = (u32 *)malloc(sizeof(u32) * (u64)D1 * L * n);
  u32 *qhat = (u32 *)malloc(sizeof(u32) * (u64)B * D1 * 2 * L * n);
  u32 *acc = (u32 *)malloc(sizeof(u32) * n);
  if (!yhat || !qhat || !acc) {
    free(yhat);
    free(qhat);
    free(acc);
    return -1;
  }
  fr_ctx x = {P, raw, r, yhat};
  orc_parallel_for(D1, nthreads, fr_row, &x, sizeof(u32) * n);
  memcpy(qhat, queries, sizeof(u32) * (u64)B * D1 * 2 * L * n);
  orc_ntt_fwd_rns_mt(P, qhat, (u64)B * D1 * 2, nthreads);
  long long bad = 0;
  for (u32 b = 0; b < B; b++)
    for (u32 comp = 0; comp < 2; comp++)
      for (u32 j = 0; j < L; j++) {
        const u64 q = P->q[j];
        memset(acc, 0, sizeof(u32) * n);
        for (u32 i = 0; i < D1; i++) {
          const u32 *yv = yhat + ((u64)i * L + j) * n;
          const u32 *qv = qhat + ((((u64)b * D1 + i) * 2 + comp) * L + j) * n;
          for (u32 k = 0; k < n; k++) acc[k] = (u32)addmod(acc[k], mulmod(yv[k], qv[k], q), q);
        }
        orc_ntt_inv(acc, n, q, P->psi[j]);
        for (u32 k = 0; k < n; k++) {
          u64 rhs = 0;
          for (u32 c = 0; c < D2; c++)
            rhs = addmod(rhs, mulmod(r[(u64)j * D2 + c], responses[((((u64)b * D2 + c) * 2 + comp) * L + j) * n + k], q), q);
          if (rhs != acc[k]) bad++;
        }
      }
  free(yhat);
  free(qhat);
  free(acc);
  return bad;
}

/* The phase a*s + b (mod q) of a ciphertext, each coefficient as two u64 halves
 * (low first), in [0, q).  Lets the tests check App. A.2 / A.4 identities exactly. */
void orc_bfv_phase(const orc_params *P, const int8_t *s, const u32 *ct, u64 *phi_lo_hi) {
  u128 *phi = (u128 *)malloc(sizeof(u128) * P->n);
  phase(P, s, ct, phi);
  for (u32 t = 0; t < P->n; t++) {
    phi_lo_hi[2 * t] = (u64)phi[t];
    phi_lo_hi[2 * t + 1] = (u64)(phi[t] >> 64);
  }
  free(phi);
}

/* ------------------------------------------------------------------------- */
/* Modulus switching down to the single prime q_0                            */
/* ------------------------------------------------------------------------- */

/* The integer x in [0, q) with x = res[j * stride] (mod q_j) for every j: Chinese
 * remaindering, built up one prime at a time (x stays below q_0 ... q_j). */
static u128 crt_lift(const orc_params *P, const u32 *res, u64 stride) {
  u128 x = res[0], M = P->q[0];
  for (u32 j = 1; j < P->L; j++) {
    const u64 q = P->q[j];
    const u64 h = mulmod(submod(res[(u64)j * stride], (u64)(x % q), q), invmod_prime((u64)(M % q), q), q);
    x += (u128)h * M;
    M *= q;
  }
  return x;
}

/* Modulus switching of RLWE ciphertext polynomials (App. D.5, "Error analysis of
 * RLWE modulus switching"; Sec. 4.3 fuses it with the inverse NTT): every
 * coefficient x in [0, q) goes to
 *     y = round(x * q_0 / q) mod q_0,
 * so the ciphertext modulus drops from q = q_0 q_1 ... q_{L-1} to the single prime
 * q_0 (#RNS = 1).  With Q' = q / q_0 = q_1 ... q_{L-1}, x q_0 / q = x / Q', and
 * round(x / Q') = floor((2x + Q') / (2Q')): Q' is odd, so no value sits exactly
 * half way.  polys [count][L][n] in coefficient form; out [count][n]. */
void orc_modswitch(const orc_params *P, const u32 *polys, u64 count, u32 *out) {
  const u32 n = P->n, L = P->L;
  u128 Qd = 1;
  for (u32 j = 1; j < L; j++) Qd *= P->q[j];
  for (u64 c = 0; c < count; c++)
    for (u32 t = 0; t < n; t++) {
      const u128 x = crt_lift(P, polys + c * L * n + t, n);
      const u128 r = (2 * x + Qd) / (2 * Qd);
      out[c * n + t] = (u32)(r % P->q[0]);
    }
}

/* Phase phi = a*s + b (mod q_0) of a ciphertext [2][n] over the single prime q_0
 * (what modulus switching leaves), each coefficient in [0, q_0). */
void orc_bfv_phase_q0(const orc_params *P, const int8_t *s, const u32 *ct, u64 *phi) {
  const u32 n = P->n;
  const u64 q = P->q[0];
  u32 *sj = (u32 *)calloc(n, sizeof(u32));
  u32 *as = (u32 *)malloc(sizeof(u32) * n);
  for (u32 t = 0; t < n; t++) sj[t] = (u32)((s[t] + (i128)q) % q);
  ring_mul(ct, sj, as, n, q, P->psi[0]);
  for (u32 t = 0; t < n; t++) phi[t] = addmod(as[t], ct[n + t], q);
  free(sj);
  free(as);
}

/* Decrypt a ciphertext [2][n] over q_0: m = round(p * phi / q_0) mod p (App. A.2,
 * the scale after switching being about q_0 / p). */
void orc_bfv_decrypt_q0(const orc_params *P, const int8_t *s, const u32 *ct, u32 *m_out) {
  const u32 n = P->n;
  const u64 q = P->q[0], pmask = (1ull << P->log2p) - 1;
  u64 *phi = (u64 *)malloc(sizeof(u64) * n);
  orc_bfv_phase_q0(P, s, ct, phi);
  for (u32 t = 0; t < n; t++) {
    const u128 num = ((u128)phi[t] << (P->log2p + 1)) + q; /* 2 p phi + q_0 */
    m_out[t] = (u32)((u64)(num / (2 * (u128)q)) & pmask);
  }
  free(phi);
}

/* ------------------------------------------------------------------------- */
/* Server-side query expansion (Sec. 3.5; App. C.2; decomposition of App. D.3) */
/* ------------------------------------------------------------------------- */

/* tau_g: a(X) -> a(X^g) in Z_q[X]/(X^n + 1), g odd.  Coefficient t moves to
 * e = t g mod 2n, negated when e >= n (X^n = -1). */
void orc_automorphism(const u32 *a, u32 *out, u32 n, u64 q, u32 g) {
  for (u32 t = 0; t < n; t++) {
    const u64 e = (u64)t * g % (2ull * n);
    if (e < n)
      out[e] = a[t];
    else
      out[e - n] = (u32)((q - a[t]) % q);
  }
}

/* out = a X^-k in Z_q[X]/(X^n + 1), 0 <= k < n: coefficient t goes to t - k, or to
 * t - k + n negated (X^(t-k) = -X^(t-k+n)). */
static void monomial_div(const u32 *a, u32 *out, u32 n, u64 q, u32 k) {
  for (u32 t = 0; t < n; t++) {
    if (t >= k)
      out[t - k] = a[t];
    else
      out[t + n - k] = (u32)((q - a[t]) % q);
  }
}

/* Gadget of the expansion keys (App. D.3): base t = 2^w with w = ceil(log2 q / ell),
 * ell digits; x in [0, q) is sum_k d_k t^k with d_k = (x >> (w k)) mod t. */
u32 orc_gadget_bits(const orc_params *P, u32 ell) {
  const u128 q = full_modulus(P);
  u32 bits = 0;
  while (bits < 128 && ((u128)1 << bits) < q) bits++; /* ceil(log2 q) */
  return (bits + ell - 1) / ell;
}

/* Key-switching key from s' = tau_g(s) to s: for k < ell, ksk[k] = (a_k, b_k) with
 * a_k s + b_k = t^k s' + e_k (mod q), i.e. b_k = t^k s' + e_k - a_k s.  a [ell][L][n]
 * (uniform residues) and e [ell][n] are the caller's draws; ksk [ell][2][L][n],
 * coefficient form. */
void orc_ksk_gen(const orc_params *P, const int8_t *s, u32 g, u32 ell, const u32 *a, const int8_t *e, u32 *ksk) {
  const u32 n = P->n, L = P->L, w = orc_gadget_bits(P, ell);
  u32 *sj = (u32 *)calloc(n, sizeof(u32));
  u32 *sg = (u32 *)calloc(n, sizeof(u32));
  u32 *as = (u32 *)calloc(n, sizeof(u32));
  for (u32 k = 0; k < ell; k++)
    for (u32 j = 0; j < L; j++) {
      const u64 q = P->q[j];
      const u64 tk = (u64)(((u128)1 << (w * k)) % q); /* t^k mod q_j (w k < 128) */
      for (u32 t = 0; t < n; t++) sj[t] = (u32)((s[t] + (i128)q) % q);
      orc_automorphism(sj, sg, n, q, g);
      const u32 *ak = a + ((u64)k * L + j) * n;
      ring_mul(ak, sj, as, n, q, P->psi[j]);
      u32 *ka = ksk + (((u64)k * 2 + 0) * L + j) * n;
      u32 *kb = ksk + (((u64)k * 2 + 1) * L + j) * n;
      for (u32 t = 0; t < n; t++) {
        const u64 et = (u64)((e[(u64)k * n + t] + (i128)q) % q);
        ka[t] = ak[t];
        kb[t] = (u32)submod(addmod(mulmod(tk, sg[t], q), et, q), as[t], q);
      }
    }
  free(sj);
  free(sg);
  free(as);
}

/* Gadget digits of a polynomial a [L][n] (coefficient form): d [ell][n] with
 * d_k[t] = (x_t >> (w k)) mod 2^w for the CRT lift x_t in [0, q) of coefficient t,
 * so that sum_k d_k t^k = a (App. D.3's decomposition). */
static void gadget_digits(const orc_params *P, const u32 *a, u32 ell, u32 *d) {
  const u32 n = P->n, w = orc_gadget_bits(P, ell);
  const u128 mask = ((u128)1 << w) - 1;
  for (u32 t = 0; t < n; t++) {
    const u128 x = crt_lift(P, a + t, n);
    for (u32 k = 0; k < ell; k++) d[(u64)k * n + t] = (u32)((x >> (w * k)) & mask);
  }
}

/* The key-switching sums (sum_k e_k K_k.a, b + sum_k e_k K_k.b) for digit
 * polynomials e_k given as residues [ell][L][n]; b [L][n]; out [2][L][n]. */
static void key_switch_sum(const orc_params *P, const u32 *e, const u32 *b, const u32 *ksk, u32 ell, u32 *out) {
  const u32 n = P->n, L = P->L;
  u32 *prod = (u32 *)calloc(n, sizeof(u32));
  for (u32 j = 0; j < L; j++) {
    const u64 q = P->q[j];
    u32 *oa = out + (u64)j * n, *ob = out + ((u64)L + j) * n;
    for (u32 t = 0; t < n; t++) {
      oa[t] = 0;
      ob[t] = b[(u64)j * n + t];
    }
    for (u32 k = 0; k < ell; k++) {
      const u32 *ek = e + ((u64)k * L + j) * n;
      ring_mul(ek, ksk + (((u64)k * 2 + 0) * L + j) * n, prod, n, q, P->psi[j]);
      for (u32 t = 0; t < n; t++) oa[t] = (u32)addmod(oa[t], prod[t], q);
      ring_mul(ek, ksk + (((u64)k * 2 + 1) * L + j) * n, prod, n, q, P->psi[j]);
      for (u32 t = 0; t < n; t++) ob[t] = (u32)addmod(ob[t], prod[t], q);
    }
  }
  free(prod);
}

/* Subs of (a X^-shift, b X^-shift) by g, with the decomposition taken of a itself:
 * the digit polynomials of a are moved by the same signed permutations as the
 * ciphertext (X^-shift, then tau_g), which keeps sum_k t^k tau_g(d_k X^-shift) =
 * tau_g(a X^-shift) since both maps fix the constants t^k; the digits of the moved
 * ciphertext are thus in (-t, t).  Then the key-switching sums.  ct, out [2][L][n]. */
static void subs_shifted(const orc_params *P, const u32 *ct, u32 shift, u32 g, const u32 *ksk, u32 ell, u32 *out) {
  const u32 n = P->n, L = P->L;
  u32 *d = (u32 *)calloc((size_t)ell * n, sizeof(u32));
  u32 *e = (u32 *)calloc((size_t)ell * L * n, sizeof(u32));
  u32 *bs = (u32 *)calloc((size_t)L * n, sizeof(u32));
  u32 *tmp = (u32 *)calloc(n, sizeof(u32));
  gadget_digits(P, ct, ell, d);
  for (u32 j = 0; j < L; j++) {
    const u64 q = P->q[j];
    for (u32 k = 0; k < ell; k++) {
      for (u32 t = 0; t < n; t++) tmp[t] = (u32)(d[(u64)k * n + t] % q);
      u32 *ek = e + ((u64)k * L + j) * n;
      monomial_div(tmp, ek, n, q, shift);
      memcpy(tmp, ek, sizeof(u32) * n);
      orc_automorphism(tmp, ek, n, q, g);
    }
    monomial_div(ct + ((u64)L + j) * n, tmp, n, q, shift);
    orc_automorphism(tmp, bs + (u64)j * n, n, q, g);
  }
  key_switch_sum(P, e, bs, ksk, ell, out);
  free(d);
  free(e);
  free(bs);
  free(tmp);
}

/* Subs of (a X^-shift, b X^-shift) by g in the textbook order: the ciphertext is
 * shifted and substituted first, and the gadget digits are those of the CRT lift in
 * [0, q) of the substituted a-part tau_g(a X^-shift), so every digit lies in [0, t).
 * Then the same key-switching sums.  Kept beside subs_shifted as the second reading
 * of App. D.3's key switch; both equal tau_g(a X^-shift) as sum_k t^k e_k, so with
 * error-free keys both give the same phase.  ct, out [2][L][n]. */
static void subs_textbook(const orc_params *P, const u32 *ct, u32 shift, u32 g, const u32 *ksk, u32 ell, u32 *out) {
  const u32 n = P->n, L = P->L;
  u32 *sub = (u32 *)calloc((size_t)2 * L * n, sizeof(u32));
  u32 *d = (u32 *)calloc((size_t)ell * n, sizeof(u32));
  u32 *e = (u32 *)calloc((size_t)ell * L * n, sizeof(u32));
  u32 *tmp = (u32 *)calloc(n, sizeof(u32));
  for (u32 c = 0; c < 2; c++)
    for (u32 j = 0; j < L; j++) {
      monomial_div(ct + ((u64)c * L + j) * n, tmp, n, P->q[j], shift);
      orc_automorphism(tmp, sub + ((u64)c * L + j) * n, n, P->q[j], g);
    }
  gadget_digits(P, sub, ell, d);
  for (u32 k = 0; k < ell; k++)
    for (u32 j = 0; j < L; j++)
      for (u32 t = 0; t < n; t++) e[((u64)k * L + j) * n + t] = (u32)(d[(u64)k * n + t] % P->q[j]);
  key_switch_sum(P, e, sub + (u64)L * n, ksk, ell, out);
  free(sub);
  free(d);
  free(e);
  free(tmp);
}

/* Subs(ct, g): the substitution X -> X^g (the result decrypts under tau_g(s)) with
 * key switching back to s by that substitution's key; the gadget digits are those
 * of ct's a-part, substituted along with it.  ct, out [2][L][n]. */
void orc_subs(const orc_params *P, const u32 *ct, u32 g, const u32 *ksk, u32 ell, u32 *out) {
  subs_shifted(P, ct, 0, g, ksk, ell, out);
}

/* Subs(ct X^-shift, g) in the textbook order (digits of the substituted a-part). */
void orc_subs_textbook(const orc_params *P, const u32 *ct, u32 shift, u32 g, const u32 *ksk, u32 ell, u32 *out) {
  subs_textbook(P, ct, shift, g, ksk, ell, out);
}

/* Subs(ct X^-shift, g) with the digits of ct's a-part moved along (the order
 * orc_expand uses). */
void orc_subs_moved(const orc_params *P, const u32 *ct, u32 shift, u32 g, const u32 *ksk, u32 ell, u32 *out) {
  subs_shifted(P, ct, shift, g, ksk, ell, out);
}

typedef void (*subs_fn)(const orc_params *, const u32 *, u32, u32, const u32 *, u32, u32 *);

/* Query expansion, SealPIR's recursion as App. C.2 applies it.  ct [2][L][n]
 * encrypts sum_i m_i X^i (i < 2^levels <= n).  It is first multiplied by
 * 2^-levels mod q.  Level j = 0 .. levels-1 maps each of the 2^j ciphertexts c_k to
 *     c_k + Subs(c_k, n/2^j + 1)                at index k,
 *     c'  + Subs(c',  n/2^j + 1), c' = c_k X^-2^j   at index k + 2^j,
 * so that ciphertext i finally encrypts m_i as a constant polynomial.  ksk
 * [levels][ell][2][L][n] holds level j's key (g = n/2^j + 1) at index j.  out
 * [count][2][L][n] receives ciphertexts 0 .. count-1 (count <= 2^levels). */
static void expand_with(const orc_params *P, const u32 *ct, u32 levels, u32 ell, const u32 *ksk, u32 count, u32 *out,
                        subs_fn subs_c) {
  const u32 n = P->n, L = P->L;
  const u64 csz = (u64)2 * L * n;
  const u64 total = 1ull << levels;
  u32 *cur = (u32 *)calloc(total * csz, sizeof(u32));
  u32 *nxt = (u32 *)calloc(total * csz, sizeof(u32));
  u32 *c1 = (u32 *)calloc(csz, sizeof(u32));
  u32 *sb = (u32 *)calloc(csz, sizeof(u32));
  for (u32 j = 0; j < L; j++) {
    const u64 q = P->q[j];
    const u64 inv = invmod_prime(orc_powmod(2, levels, q), q);
    for (u32 c = 0; c < 2; c++)
      for (u32 t = 0; t < n; t++) {
        const u64 i = ((u64)c * L + j) * n + t;
        cur[i] = (u32)mulmod(ct[i], inv, q);
      }
  }
  for (u32 lev = 0; lev < levels; lev++) {
    const u64 C = 1ull << lev;
    const u32 g = (n >> lev) + 1;
    const u32 *key = ksk + (u64)lev * ell * csz;
    for (u64 k = 0; k < C; k++) {
      const u32 *c0 = cur + k * csz;
      for (u32 c = 0; c < 2; c++)
        for (u32 j = 0; j < L; j++)
          monomial_div(c0 + ((u64)c * L + j) * n, c1 + ((u64)c * L + j) * n, n, P->q[j], (u32)C);
      for (u32 br = 0; br < 2; br++) {
        const u32 *src = br ? c1 : c0;
        u32 *dst = nxt + (k + br * C) * csz;
        /* Subs(c X^-C): subs_shifted moves the digits of c's a-part along,
         * subs_textbook takes the digits of the substituted a-part */
        subs_c(P, c0, br ? (u32)C : 0, g, key, ell, sb);
        for (u32 c = 0; c < 2; c++)
          for (u32 j = 0; j < L; j++) {
            const u64 q = P->q[j], o = ((u64)c * L + j) * n;
            for (u32 t = 0; t < n; t++) dst[o + t] = (u32)addmod(src[o + t], sb[o + t], q);
          }
      }
    }
    u32 *sw = cur;
    cur = nxt;
    nxt = sw;
  }
  memcpy(out, cur, sizeof(u32) * count * csz);
  free(cur);
  free(nxt);
  free(c1);
  free(sb);
}

void orc_expand(const orc_params *P, const u32 *ct, u32 levels, u32 ell, const u32 *ksk, u32 count, u32 *out) {
  expand_with(P, ct, levels, ell, ksk, count, out, subs_shifted);
}

/* The same recursion with every key switch in the textbook order. */
void orc_expand_textbook(const orc_params *P, const u32 *ct, u32 levels, u32 ell, const u32 *ksk, u32 count,
                         u32 *out) {
  expand_with(P, ct, levels, ell, ksk, count, out, subs_textbook);
}

/* ------------------------------------------------------------------------- */
/* Scalar-HE (LWE) DB GEMM of the online SimplePIR step (Sec. 2.5, Sec. 4.1)  */
/* ------------------------------------------------------------------------- */

/* out[b][i] = sum_j A[i][j] * Q[b][j]  (mod 2^32): A [D1][D0] INT8 plaintexts (signed),
 * Q [B][D0] the query ciphertexts' Z_{2^32} entries, out [B][D1].  Every product and
 * sum is taken exactly in 64-bit arithmetic (D0 <= 2^24) and reduced mod 2^32 once
 * per output. */
void orc_lwe_gemm(const int8_t *A, u32 D1, u32 D0, const u32 *Q, u32 B, u32 *out) {
  for (u32 b = 0; b < B; b++)
    for (u32 i = 0; i < D1; i++) {
      i64 acc = 0;
      const int8_t *a = A + (u64)i * D0;
      const u32 *q = Q + (u64)b * D0;
      for (u32 j = 0; j < D0; j++) acc += (i64)a[j] * (i64)q[j]; /* |acc| < 2^7 2^32 2^24 */
      out[(u64)b * D1 + i] = (u32)((u64)acc & 0xFFFFFFFFull);
    }
}

/* ------------------------------------------------------------------------- */
/* RGSW-RLWE external products for the remaining dimensions (Sec. 3.2, 3.6)   */
/* ------------------------------------------------------------------------- */

/* RGSW encryption of mu (a polynomial with small non-negative coefficients, e.g. a
 * selection bit) with the ell-digit base-t gadget of App. D.3: 2 ell rows, each an
 * RLWE encryption of zero (a s + b = e) plus mu t^k in the a-part (row k < ell) or in
 * the b-part (row ell + k).  a [2 ell][L][n] uniform residues, e [2 ell][n] errors;
 * out [2 ell][2][L][n], coefficient form. */
void orc_rgsw_encrypt(const orc_params *P, const int8_t *s, const u32 *mu, u32 ell, const u32 *a, const int8_t *e,
                      u32 *out) {
  const u32 n = P->n, L = P->L, w = orc_gadget_bits(P, ell);
  u32 *sj = (u32 *)calloc(n, sizeof(u32));
  u32 *as = (u32 *)calloc(n, sizeof(u32));
  for (u32 r = 0; r < 2 * ell; r++) {
    const u32 k = r % ell, in_b = r >= ell;
    for (u32 j = 0; j < L; j++) {
      const u64 q = P->q[j];
      const u64 tk = (u64)(((u128)1 << (w * k)) % q);
      for (u32 t = 0; t < n; t++) sj[t] = (u32)((s[t] + (i128)q) % q);
      const u32 *ar = a + ((u64)r * L + j) * n;
      ring_mul(ar, sj, as, n, q, P->psi[j]);
      u32 *oa = out + (((u64)r * 2 + 0) * L + j) * n, *ob = out + (((u64)r * 2 + 1) * L + j) * n;
      for (u32 t = 0; t < n; t++) {
        const u64 et = (u64)((e[(u64)r * n + t] + (i128)q) % q);
        const u64 mt = mulmod(tk, mu[t] % q, q);
        const u64 b0 = submod(et, as[t], q); /* a s + b = e */
        oa[t] = (u32)(in_b ? ar[t] : addmod(ar[t], mt, q));
        ob[t] = (u32)(in_b ? addmod(b0, mt, q) : b0);
      }
    }
  }
  free(sj);
  free(as);
}

/* External product RGSW(mu) (x) ct: with a = sum_k t^k d_k(a) and b = sum_k t^k d_k(b)
 * (digits of the CRT lifts of the coefficients), out = sum_k d_k(a) row_k +
 * sum_k d_k(b) row_(ell+k); its phase is mu (a s + b) plus the rows' errors weighted
 * by the digits.  rgsw [2 ell][2][L][n], ct and out [2][L][n], coefficient form. */
void orc_external_product(const orc_params *P, const u32 *rgsw, u32 ell, const u32 *ct, u32 *out) {
  const u32 n = P->n, L = P->L;
  u32 *d = (u32 *)calloc((size_t)2 * ell * n, sizeof(u32));
  u32 *dk = (u32 *)calloc(n, sizeof(u32));
  u32 *prod = (u32 *)calloc(n, sizeof(u32));
  gadget_digits(P, ct, ell, d);                              /* digits of a */
  gadget_digits(P, ct + (u64)L * n, ell, d + (u64)ell * n);  /* digits of b */
  memset(out, 0, sizeof(u32) * 2 * L * n);
  for (u32 r = 0; r < 2 * ell; r++)
    for (u32 c = 0; c < 2; c++)
      for (u32 j = 0; j < L; j++) {
        const u64 q = P->q[j];
        for (u32 t = 0; t < n; t++) dk[t] = (u32)(d[(u64)r * n + t] % q);
        ring_mul(dk, rgsw + (((u64)r * 2 + c) * L + j) * n, prod, n, q, P->psi[j]);
        u32 *o = out + ((u64)c * L + j) * n;
        for (u32 t = 0; t < n; t++) o[t] = (u32)addmod(o[t], prod[t], q);
      }
  free(d);
  free(dk);
  free(prod);
}

/* Folding of 2^levels ciphertexts [2^levels][2][L][n] into one (OnionPIR's remaining
 * dimensions, Sec. 3.2 / 3.6): level l pairs ciphertexts (2j, 2j + 1) and keeps
 * c_2j + RGSW_l (x) (c_2j+1 - c_2j), which is c_2j+1 when RGSW_l encrypts 1 and c_2j
 * when it encrypts 0.  rgsw [levels][2 ell][2][L][n]; out [2][L][n]. */
void orc_fold(const orc_params *P, const u32 *cts, u32 levels, const u32 *rgsw, u32 ell, u32 *out) {
  const u32 n = P->n, L = P->L;
  const u64 csz = (u64)2 * L * n;
  u64 count = 1ull << levels;
  u32 *cur = (u32 *)calloc(count * csz, sizeof(u32));
  u32 *diff = (u32 *)calloc(csz, sizeof(u32));
  u32 *ep = (u32 *)calloc(csz, sizeof(u32));
  memcpy(cur, cts, sizeof(u32) * count * csz);
  for (u32 l = 0; l < levels; l++) {
    const u32 *g = rgsw + (u64)l * 2 * ell * csz;
    for (u64 j = 0; j < count / 2; j++) {
      const u32 *c0 = cur + (2 * j) * csz, *c1 = cur + (2 * j + 1) * csz;
      for (u32 c = 0; c < 2; c++)
        for (u32 i = 0; i < L; i++) {
          const u64 q = P->q[i], o = ((u64)c * L + i) * n;
          for (u32 t = 0; t < n; t++) diff[o + t] = (u32)submod(c1[o + t], c0[o + t], q);
        }
      orc_external_product(P, g, ell, diff, ep);
      u32 *dst = cur + j * csz; /* j <= 2j: c0 was read above */
      for (u32 c = 0; c < 2; c++)
        for (u32 i = 0; i < L; i++) {
          const u64 q = P->q[i], o = ((u64)c * L + i) * n;
          for (u32 t = 0; t < n; t++) dst[o + t] = (u32)addmod(c0[o + t], ep[o + t], q);
        }
    }
    count /= 2;
  }
  memcpy(out, cur, sizeof(u32) * csz);
  free(cur);
  free(diff);
  free(ep);
}
