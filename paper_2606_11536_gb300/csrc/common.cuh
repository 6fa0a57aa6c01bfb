// common.cuh -- internal declarations of the GB300 PIR scan library.
//
// Shared by the .cu files of this library only (never by the CPU oracle).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gbpir.h"

namespace gbpir {

// ---------------------------------------------------------------------------
// Per-prime NTT constants handed to kernels by value.
// ---------------------------------------------------------------------------
// Lane-major twiddles.  In a radix-16 pass over the lowest index bits (units of 16
// consecutive elements, unit hi = thread), stage 0 takes pairs n/2 + 8 hi .. +7 and
// stage 1 pairs n/4 + 4 hi .. +3 of the table: each thread its own 64 (32) bytes,
// which a warp reads with 16 (8) L1 wavefronts per 16-byte load.  The same pairs
// are kept after the table in lane-major order, [stage 0: 4][n/16] then
// [stage 1: 2][n/16] 16-byte pairs of pairs, so that a warp's load is one
// contiguous 512-byte run.
inline size_t ntt_lane_major_words(uint32_t n) { return (size_t)6 * (n / 16) * 4; }
inline void ntt_lane_major_fill(uint32_t *tab, uint32_t n) {  // tab: n pairs, then the copy
  uint32_t *lm = tab + 2 * (size_t)n;
  const uint32_t units = n / 16;
  for (uint32_t hi = 0; hi < units; ++hi) {
    for (uint32_t k = 0; k < 4; ++k)  // stage 0: pairs n/2 + 8 hi + 2k, +1
      for (uint32_t w = 0; w < 4; ++w) lm[((size_t)k * units + hi) * 4 + w] = tab[2 * (n / 2 + 8 * hi + 2 * k) + w];
    for (uint32_t k = 0; k < 2; ++k)  // stage 1: pairs n/4 + 4 hi + 2k, +1
      for (uint32_t w = 0; w < 4; ++w)
        lm[((size_t)(4 + k) * units + hi) * 4 + w] = tab[2 * (n / 4 + 4 * hi + 2 * k) + w];
  }
}

struct NttConst {
  uint32_t q[PIR_MAX_L];
  uint32_t ninv[PIR_MAX_L];        // n^-1 mod q
  uint32_t ninv_sh[PIR_MAX_L];     // Shoup companion of n^-1
  const uint2 *fwd[PIR_MAX_L];     // [n] {psi^brv(i), floor(psi^brv(i) * 2^32 / q)}: twiddle, Shoup companion;
                                   // the lane-major copy follows at fwd + n
  const uint2 *inv[PIR_MAX_L];     // [n] {psi^-brv(i), its Shoup companion}; lane-major copy at inv + n
};

// Reduction constants of the modular GEMM epilogues.
struct ModConst {
  uint32_t q[PIR_MAX_L];
  uint64_t mu[PIR_MAX_L];   // floor(2^64 / q)
  uint64_t k63[PIR_MAX_L];  // q * floor(2^63 / q): the largest multiple of q <= 2^63
};

// Modulus switching from q = q_0 q_1 ... q_{L-1} down to q_0 (App. D.5; fused into
// the inverse NTT as in Sec. 4.3): y = round(x / Q') mod q_0, Q' = q_1 ... q_{L-1}.
// x mod Q' is formed in mixed radix over q_1 .. q_{L-1} (Garner):
// x mod Q' = a_1 + a_2 q_1 + a_3 q_1 q_2, digits a_k in [0, q_k).
struct SwitchConst {
  uint32_t c[PIR_MAX_L][PIR_MAX_L];     // c[k][i] = q_i^-1 mod q_k, 1 <= i < k < L
  uint32_t c_sh[PIR_MAX_L][PIR_MAX_L];  // Shoup companions (mod q_k)
  uint32_t w[PIR_MAX_L], w_sh[PIR_MAX_L];  // w[k] = q_1 ... q_{k-1} mod q_0 (w[1] = 1)
  uint32_t h[PIR_MAX_L];                   // mixed-radix digits of (Q' - 1) / 2
  uint32_t qinv, qinv_sh;                  // Q'^-1 mod q_0
};

// Host-side: the ring (n, L, primes, roots) plus device tables, cached per device
// and ring.  p.D1 / p.D2 are zero here: database shapes are passed per call.
struct ParamCtx {
  pir_params_t p;
  uint32_t logn;
  NttConst ntt;
  ModConst mod;
  SwitchConst sw;
};

// params.cu
pir_status_t validate_params(const pir_params_t *p);
pir_status_t get_param_ctx(const pir_params_t *p, const ParamCtx **out);  // cached, device-resident tables

// expand.cu: query expansion.  expand_device writes B x count expanded ciphertexts
// [B][count][2][L][n] in NTT form from packed [B][2][L][n] (coefficient form) and
// reports its kernel launches; expander_fits checks ring and depth against a DB.
struct pir_expander_impl;
// Gadget digits (App. D.3): for every polynomial [L][n] (coefficient form, canonical)
// of coef [polys][L][n], dig [polys][ell][n] holds the w-bit digits of the CRT lift of
// each coefficient, w = gadget_bits(p, ell) = ceil(ceil(log2 q) / ell).
uint32_t gadget_bits(const pir_params_t &p, uint32_t ell);
cudaError_t launch_gadget_digits(const ParamCtx &c, const uint32_t *coef, uint64_t polys, uint32_t ell,
                                 uint32_t *dig, cudaStream_t s);
bool expander_view(pir_expander_t h, const pir_expander_impl **out);
bool expander_fits(const pir_expander_impl *ex, const pir_params_t &p);
pir_status_t expand_device(const pir_expander_impl *ex, const uint32_t *packed, uint32_t B, uint32_t count,
                           uint32_t *out, cudaStream_t s, uint64_t *launch_count);

// fold.cu: folding of the remaining dimensions with RGSW external products; cur
// [B][2^levels][2][L][n] and rgsw [B][levels][2 ell][2][L][n] in NTT form, out
// [B][2][L][n] in NTT form; cur is overwritten.
pir_status_t fold_device(const ParamCtx &c, uint32_t *cur, uint32_t B, uint32_t levels, uint32_t ell,
                         const uint32_t *rgsw, uint32_t *out, cudaStream_t s, uint64_t *launch_count);

// Read-only view of a live DB handle (api.cu); false for unknown or freed handles.
struct DbView {
  pir_params_t p;
  int layout;
  const ParamCtx *ctx;
  const void *resident;
};
bool db_view(pir_db_t db, DbView *out);
void count_launches(uint64_t k);

// Error bookkeeping (api.cu)
// Per-device error word that kernels with bounded waits set on a timeout.
cudaError_t device_error_word(uint32_t **word);
pir_status_t cuda_status(cudaError_t e);
void set_cuda_error(cudaError_t e);
const char *last_cuda_error_cstr();

// ntt.cu.  Rows are polynomials of n residues; row r uses prime r % L.
cudaError_t launch_ntt_fwd(const ParamCtx &c, const uint32_t *src, uint32_t *dst, uint64_t rows, cudaStream_t s);
// Forward NTT of `rows` rows where local row r reads source row off + (r / G) * S + r % G.
cudaError_t launch_ntt_fwd_rows(const ParamCtx &c, const uint32_t *src, uint64_t off, uint64_t G, uint64_t S,
                                uint32_t *dst, uint64_t rows, cudaStream_t s);
cudaError_t launch_ntt_inv(const ParamCtx &c, const uint32_t *src, uint32_t *dst, uint64_t rows, cudaStream_t s);
// Row-mapped variants: local row r (prime r % L) reads source row
// off + (r / G) * S + (r % G) * T.
cudaError_t launch_ntt_inv_rows(const ParamCtx &c, const uint32_t *src, uint64_t off, uint64_t G, uint64_t S,
                                uint64_t T, uint32_t *dst, uint64_t rows, cudaStream_t s);
cudaError_t launch_ntt_fwd_rows_t(const ParamCtx &c, const uint32_t *src, uint64_t off, uint64_t G, uint64_t S,
                                  uint64_t T, uint32_t *dst, uint64_t rows, cudaStream_t s);
// Inverse NTT of `count` RNS polynomials src [count][L][n] with modulus switching to
// q_0 fused in: dst [count][n] over q_0.  src and dst must not overlap.
cudaError_t launch_ntt_inv_switch(const ParamCtx &c, const uint32_t *src, uint32_t *dst, uint64_t count,
                                  cudaStream_t s);
// Batch-1 queries [1][D1][2][L][n]: forward NTT of ciphertexts i0 .. i0+kc-1 written
// directly into the plain slot layout [L*n][stride][2] (Mp = 2), columns col0 .. col0+kc-1.
cudaError_t launch_ntt_fwd_pair_slots(const ParamCtx &c, const uint32_t *queries, uint32_t i0, uint32_t kc,
                                      uint32_t stride, uint32_t col0, uint32_t *slots, cudaStream_t s);
// Forward NTT of DB plaintexts read from the raw bit stream (RNS lift fused: a
// coefficient < p < q_j is its own residue).  Row-major: polys first .. first+np-1;
// column-major: local poly p is (i, c) = (p % D1, first + p / D1).  dst is [np][L][n].
cudaError_t launch_ntt_fwd_raw(const ParamCtx &c, const uint8_t *raw, int col_major, uint32_t D1, uint32_t D2,
                               uint64_t first, uint64_t npolys, uint32_t *dst, cudaStream_t s);

// layout.cu (layouts are described at the top of layout.cu)
// Sets *bad (device word) when a residue of rows [nrows][n] is not below its prime
// (row r over q_{r % L}).
cudaError_t launch_check_residues(const ParamCtx &c, const uint32_t *rows, uint64_t nrows, uint32_t *bad,
                                  cudaStream_t s);
cudaError_t launch_query_to_slots(const ParamCtx &c, const uint32_t *qhat, uint32_t B, uint32_t Kc, uint32_t Mp,
                                  uint32_t *qs, cudaStream_t s);
cudaError_t launch_query_to_limbs(const ParamCtx &c, const uint32_t *qhat, uint32_t B, uint32_t Kc, uint32_t Mp,
                                  uint8_t *ql, cudaStream_t s);
cudaError_t launch_slots_to_responses(const ParamCtx &c, const uint32_t *out, uint32_t B, uint32_t D2,
                                      uint32_t *resp, cudaStream_t s);
// first = first poly id (plain, row-major chunk) or first column (limb, column-major chunk)
cudaError_t launch_db_scatter(const ParamCtx &c, int layout, uint32_t D1, uint32_t D2, const uint32_t *polys,
                              uint64_t first, uint64_t np, void *resident, cudaStream_t s);
cudaError_t launch_db_read_poly(const ParamCtx &c, int layout, uint32_t D1, uint32_t D2, const void *resident,
                                uint64_t poly, uint32_t *out, cudaStream_t s);

// gemm_plain.cu: for every slot s, out[s][m][c] = (acc ? out[s][m][c] : 0) + sum over the
// Kc rows i0.. of qs[s][i - i0][m] * db[s][i][c], reduced mod q_j, for m < M, c < D2.
cudaError_t launch_gemm_plain(const ParamCtx &c, const uint32_t *db, uint32_t D1, uint32_t D2, const uint32_t *qs,
                              uint32_t M, uint32_t Mp, uint32_t i0, uint32_t Kc, uint32_t *out, int acc,
                              uint32_t tile, int stall_test, cudaStream_t s);
uint32_t gemm_plain_tiles();

// scan_tma.cu: the same contract for M <= 8 rows and D2 <= 512 (D2 % 4 == 0), as a
// TMA-staged stream; stall_test makes its consumers wait on a barrier that never
// completes (exercises the bounded-wait error path).
bool scan_tma_supports(uint32_t M, uint32_t D2);
// out_poly = 1 writes the response layout [B][D2][2][L][n] (NTT domain) directly.
// acc_src, when set, is a slot-major partial result [L*n][M][D2] added in before the
// write (the K-chunks before the last accumulate there with coalesced accesses).
cudaError_t launch_scan_tma(const ParamCtx &c, const uint32_t *db, uint32_t D1, uint32_t D2, const uint32_t *qs,
                            uint32_t M, uint32_t Mp, uint32_t i0, uint32_t Kc, uint32_t *out, int acc, int stall_test,
                            int out_poly, const uint32_t *acc_src, cudaStream_t s);

// gemm_limb.cu: the same contract on the limb layouts (db [s][4][D2][D1] u8,
// ql [s][4][Mp][Kc] u8), exact through u8 x u8 -> s32 tensor-pipe products.
// The bf16 tensor-core path (PIR_LAYOUT_TENSOR): signed base-256 digits of every
// residue in tensor-core operand tiles.  Query rows pad to tc_rows(M) (a multiple
// of 8); K-chunks are multiples of 64 rows, at most 1024.
bool gemm_tc_shape_ok(uint32_t D1, uint32_t D2);
uint32_t tc_rows(uint32_t M);
cudaError_t launch_query_to_tensor(const ParamCtx &c, const uint32_t *qhat, uint32_t B, uint32_t Kc, uint32_t Mp,
                                   uint16_t *qt, cudaStream_t s);
cudaError_t launch_db_scatter_tensor(const ParamCtx &c, uint32_t D1, uint32_t D2, const uint32_t *polys,
                                     uint64_t first, uint64_t np, uint16_t *resident, cudaStream_t s);
cudaError_t launch_db_read_poly_tensor(const ParamCtx &c, uint32_t D1, uint32_t D2, const uint16_t *resident,
                                       uint64_t poly, uint32_t *out, cudaStream_t s);
cudaError_t launch_gemm_tc(const ParamCtx &c, const uint16_t *db, uint32_t D1, uint32_t D2, const uint16_t *qt,
                           uint32_t M, uint32_t Mp, uint32_t i0, uint32_t Kc, uint32_t *out, int acc, uint32_t tile,
                           cudaStream_t s);
uint32_t gemm_tc_tiles();
bool gemm_tc_tile_ok(uint32_t tile, uint32_t Mp, uint32_t D2);
cudaError_t launch_gemm_limb(const ParamCtx &c, const uint8_t *db, uint32_t D1, uint32_t D2, const uint8_t *ql,
                             uint32_t M, uint32_t Mp, uint32_t i0, uint32_t Kc, uint32_t *out, int acc,
                             uint32_t tile, cudaStream_t s);
uint32_t gemm_limb_tiles();
// Whether a tile id holds a shape (the plain tiles 1-3 and 7 bound the query rows;
// the limb tiles need the padded rows to fill whole warp tiles).
bool gemm_plain_tile_ok(uint32_t tile, uint32_t M, uint32_t D2);
bool gemm_limb_tile_ok(uint32_t tile, uint32_t Mp);

// ---------------------------------------------------------------------------
// Device helpers
// ---------------------------------------------------------------------------

// Shoup multiplication by a constant w < q with wsh = floor(w * 2^32 / q):
// returns x * w mod q in [0, 2q) for any x < 2^32 (needs q < 2^31).
__device__ __forceinline__ uint32_t shoup_mul(uint32_t x, uint32_t w, uint32_t wsh, uint32_t q) {
  uint32_t hi = __umulhi(x, wsh);
  return x * w - hi * q;
}

// Lazy reduction of a 64-bit accumulator without a multiply (compare + predicated
// 64-bit subtract: integer ALU pipe, leaving the multiply-add pipe to the products):
// if acc >= 2^63, subtract k63 = q * floor(2^63 / q) > 2^63 - q.  The result is
// congruent mod q and below 2^63 + q, so with q < 2^30 it takes 8 more products
// (q-1)^2 < 2^60 before it could reach 2^64 (2^63 + q + 8 (q-1)^2 < 2^64).
constexpr int kFoldProducts = 8;
__device__ __forceinline__ uint64_t fold63(uint64_t acc, uint64_t k63) {
  // sign test on the high word, then a predicated 64-bit subtract
  asm("{\n .reg .pred p;\n .reg .u32 lo, hi;\n mov.b64 {lo, hi}, %0;\n setp.lt.s32 p, hi, 0;\n"
      " @p sub.u64 %0, %0, %1;\n}"
      : "+l"(acc)
      : "l"(k63));
  return acc;
}

// acc += a * b with a, b < 2^32: one 32 x 32 -> 64-bit multiply-add.  Written as
// PTX mad.wide.u32 because the C++ form `acc += (uint64_t)a * b` does not always
// reach the single-instruction form inside the streaming loops (measured: ~10
// instructions per product in the TMA scan, one with this helper).
__device__ __forceinline__ void mac_wide(uint64_t &acc, uint32_t a, uint32_t b) {
  asm("mad.wide.u32 %0, %1, %2, %0;" : "+l"(acc) : "r"(a), "r"(b));
}

// Full reduction of a 64-bit value mod q (q < 2^30): Barrett with mu = floor(2^64/q).
__device__ __forceinline__ uint32_t reduce64(uint64_t x, uint32_t q, uint64_t mu) {
  uint64_t qt = __umul64hi(x, mu);
  uint64_t r = x - qt * q;  // in [0, 2q) (Barrett's error is at most one q here)
  if (r >= q) r -= q;
  if (r >= q) r -= q;
  return (uint32_t)r;
}

}  // namespace gbpir
