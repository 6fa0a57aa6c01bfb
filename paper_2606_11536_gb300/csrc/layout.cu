// layout.cu -- transposes between the polynomial-major layout the NTT wants and
// the slot-major ("tile-major") layout the per-slot modular GEMMs want (Sec. 4.2:
// the paper inserts such transpositions around its (#RNS*N)-parallel GEMMs).
//
//   queries, NTT form   [B][Kc][2][L][n]       (one chunk of ciphertexts i0..i0+Kc-1)
//   plain slot layout   qs [L*n][Kc][Mp]        m = 2b + comp, Mp = M rounded up to 4, zero padded
//   limb slot layout    ql [L*n][4][Mp][Kc] u8  byte `limb` of each residue, i fastest
//   GEMM result         out [L*n][M][D2]
//   responses           [B][D2][2][L][n]
//   resident DB, plain  [L*n][D1][D2] u32
//   resident DB, limb   [L*n][4][D2][D1] u8
// Slot s = j*n + k (prime j, NTT slot k).
#include "common.cuh"

namespace gbpir {
namespace {

constexpr int TK = 32;  // slots per tile
constexpr int TF = 64;  // flattened (row, column) entries per tile

// qhat chunk [B][Kc][2][L][n] -> qs[s][i][mp] for f = i*Mp + mp in one tile of TF.
__global__ void __launch_bounds__(256) k_query_to_slots(const uint32_t *__restrict__ qhat, uint32_t B, uint32_t Kc,
                                                        uint32_t L, uint32_t logn, uint32_t Mp,
                                                        uint32_t *__restrict__ qs) {
  __shared__ uint32_t tile[TF][TK + 1];
  const uint32_t n = 1u << logn;
  const uint64_t F = (uint64_t)Kc * Mp;
  const uint64_t f0 = (uint64_t)blockIdx.x * TF;
  const uint32_t s0 = blockIdx.y * TK;  // slots s0 .. s0+31, all of one prime since n >= 32
  const uint32_t j = s0 >> logn, k0 = s0 & (n - 1);
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (uint32_t r = warp; r < TF; r += 8) {
    const uint64_t f = f0 + r;
    uint32_t v = 0;
    if (f < F) {
      const uint32_t i = (uint32_t)(f / Mp), m = (uint32_t)(f % Mp);
      if (m < 2 * B) {
        const uint32_t b = m >> 1, comp = m & 1;
        const uint64_t row = (((uint64_t)b * Kc + i) * 2 + comp) * L + j;
        v = qhat[row * n + k0 + lane];
      }
    }
    tile[r][lane] = v;
  }
  __syncthreads();
  for (uint32_t kk = warp; kk < TK; kk += 8) {
    const uint64_t base = (uint64_t)(s0 + kk) * F;
    for (uint32_t r = lane; r < TF; r += 32) {
      const uint64_t f = f0 + r;
      if (f < F) qs[base + f] = tile[r][kk];
    }
  }
}

// qhat chunk -> ql[s][limb][mp][i]: a tile is 32 slots x 32 ciphertexts i of one row m.
__global__ void __launch_bounds__(256) k_query_to_limbs(const uint32_t *__restrict__ qhat, uint32_t B, uint32_t Kc,
                                                        uint32_t L, uint32_t logn, uint32_t Mp,
                                                        uint8_t *__restrict__ ql) {
  __shared__ uint32_t tile[32][TK + 1];
  const uint32_t n = 1u << logn;
  const uint32_t i0 = blockIdx.x * 32;
  const uint32_t m = blockIdx.z;
  const uint32_t s0 = blockIdx.y * TK;
  const uint32_t j = s0 >> logn, k0 = s0 & (n - 1);
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (uint32_t r = warp; r < 32; r += 8) {
    const uint32_t i = i0 + r;
    uint32_t v = 0;
    if (i < Kc && m < 2 * B) {
      const uint64_t row = (((uint64_t)(m >> 1) * Kc + i) * 2 + (m & 1)) * L + j;
      v = qhat[row * n + k0 + lane];
    }
    tile[r][lane] = v;
  }
  __syncthreads();
  // each warp writes 4 slots x 4 limbs x 32 i (one byte per lane)
  for (uint32_t kk = warp; kk < TK; kk += 8) {
    const uint32_t i = i0 + lane;
    if (i >= Kc) continue;
    const uint32_t v = tile[lane][kk];
    const uint64_t s = s0 + kk;
#pragma unroll
    for (uint32_t limb = 0; limb < 4; ++limb)
      ql[((s * 4 + limb) * Mp + m) * Kc + i] = (uint8_t)(v >> (8 * limb));
  }
}

// out[s][m][c] -> resp[b][c][comp][j][k] for f = m*D2 + c.
__global__ void __launch_bounds__(256) k_slots_to_responses(const uint32_t *__restrict__ out, uint32_t M, uint32_t D2,
                                                            uint32_t L, uint32_t logn, uint32_t *__restrict__ resp) {
  __shared__ uint32_t tile[TK][TF + 1];
  const uint32_t n = 1u << logn;
  const uint64_t F = (uint64_t)M * D2;
  const uint64_t f0 = (uint64_t)blockIdx.x * TF;
  const uint32_t s0 = blockIdx.y * TK;
  const uint32_t j = s0 >> logn, k0 = s0 & (n - 1);
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (uint32_t kk = warp; kk < TK; kk += 8) {
    const uint64_t base = (uint64_t)(s0 + kk) * F;
    for (uint32_t r = lane; r < TF; r += 32) {
      const uint64_t f = f0 + r;
      tile[kk][r] = f < F ? out[base + f] : 0u;
    }
  }
  __syncthreads();
  for (uint32_t r = warp; r < TF; r += 8) {
    const uint64_t f = f0 + r;
    if (f >= F) continue;
    const uint32_t m = (uint32_t)(f / D2), c = (uint32_t)(f % D2);
    const uint64_t row = (((uint64_t)(m >> 1) * D2 + c) * 2 + (m & 1)) * L + j;
    resp[row * n + k0 + lane] = tile[lane][r];
  }
}

// 64 x 64 tiles with 16-byte global accesses on both sides (the batched path's
// transposes).  Shared tile rows are padded to 65 words.
constexpr int VT = 64;

// qhat chunk -> qs[s][f], f = i*Mp + m, m = 2b + comp; needs Kc*Mp % 4 == 0.
__global__ void __launch_bounds__(256) k_query_to_slots_v(const uint32_t *__restrict__ qhat, uint32_t B, uint32_t Kc,
                                                          uint32_t L, uint32_t logn, uint32_t Mp,
                                                          uint32_t *__restrict__ qs) {
  __shared__ uint32_t tile[VT][VT + 1];  // [f][k]
  const uint32_t n = 1u << logn;
  const uint64_t F = (uint64_t)Kc * Mp;
  const uint64_t f0 = (uint64_t)blockIdx.x * VT;
  const uint32_t s0 = blockIdx.y * VT;
  const uint32_t j = s0 >> logn, k0 = s0 & (n - 1);
  const uint32_t t = threadIdx.x, lane16 = t & 15, row = t >> 4;  // 16 rows of 16 lanes
  // read: row f, columns k0 + 4*lane16 .. +3
  for (uint32_t r = row; r < VT; r += 16) {
    const uint64_t f = f0 + r;
    uint4 v = make_uint4(0, 0, 0, 0);
    if (f < F) {
      const uint32_t i = (uint32_t)(f / Mp), m = (uint32_t)(f % Mp);
      if (m < 2 * B) {
        const uint64_t src = ((((uint64_t)(m >> 1) * Kc + i) * 2 + (m & 1)) * L + j) * n + k0 + 4 * lane16;
        v = *reinterpret_cast<const uint4 *>(qhat + src);
      }
    }
    tile[r][4 * lane16] = v.x, tile[r][4 * lane16 + 1] = v.y, tile[r][4 * lane16 + 2] = v.z,
    tile[r][4 * lane16 + 3] = v.w;
  }
  __syncthreads();
  // write: slot s0 + kk, f0 + 4*lane16 .. +3
  for (uint32_t kk = row; kk < VT; kk += 16) {
    const uint64_t f = f0 + 4 * lane16;
    if (f >= F) continue;
    const uint4 v = make_uint4(tile[4 * lane16][kk], tile[4 * lane16 + 1][kk], tile[4 * lane16 + 2][kk],
                               tile[4 * lane16 + 3][kk]);
    *reinterpret_cast<uint4 *>(qs + (uint64_t)(s0 + kk) * F + f) = v;
  }
}

// out[s][f], f = m*D2 + c -> resp[b][c][comp][j][k]; needs M*D2 % 4 == 0.
__global__ void __launch_bounds__(256) k_slots_to_responses_v(const uint32_t *__restrict__ out, uint32_t M,
                                                              uint32_t D2, uint32_t L, uint32_t logn,
                                                              uint32_t *__restrict__ resp) {
  __shared__ uint32_t tile[VT][VT + 1];  // [k][f]
  const uint32_t n = 1u << logn;
  const uint64_t F = (uint64_t)M * D2;
  const uint64_t f0 = (uint64_t)blockIdx.x * VT;
  const uint32_t s0 = blockIdx.y * VT;
  const uint32_t j = s0 >> logn, k0 = s0 & (n - 1);
  const uint32_t t = threadIdx.x, lane16 = t & 15, row = t >> 4;
  for (uint32_t kk = row; kk < VT; kk += 16) {
    const uint64_t f = f0 + 4 * lane16;
    uint4 v = make_uint4(0, 0, 0, 0);
    if (f < F) v = *reinterpret_cast<const uint4 *>(out + (uint64_t)(s0 + kk) * F + f);
    tile[kk][4 * lane16] = v.x, tile[kk][4 * lane16 + 1] = v.y, tile[kk][4 * lane16 + 2] = v.z,
    tile[kk][4 * lane16 + 3] = v.w;
  }
  __syncthreads();
  for (uint32_t r = row; r < VT; r += 16) {
    const uint64_t f = f0 + r;
    if (f >= F) continue;
    const uint32_t m = (uint32_t)(f / D2), c = (uint32_t)(f % D2);
    const uint64_t dst = ((((uint64_t)(m >> 1) * D2 + c) * 2 + (m & 1)) * L + j) * n + k0 + 4 * lane16;
    *reinterpret_cast<uint4 *>(resp + dst) = make_uint4(tile[4 * lane16][r], tile[4 * lane16 + 1][r],
                                                        tile[4 * lane16 + 2][r], tile[4 * lane16 + 3][r]);
  }
}

// NTT-form DB polys [np][L][n] -> resident layout.  Plain: polys are row-major ids
// poly0 + p = i*D2 + c.  Tile = 32 polys x 32 slots of one prime.
__global__ void __launch_bounds__(256) k_db_scatter_plain(const uint32_t *__restrict__ polys, uint64_t poly0,
                                                          uint64_t np, uint32_t D1, uint32_t D2, uint32_t L,
                                                          uint32_t logn, uint32_t *__restrict__ res) {
  __shared__ uint32_t tile[32][TK + 1];
  const uint32_t n = 1u << logn;
  const uint64_t p0 = (uint64_t)blockIdx.x * 32;
  const uint32_t s0 = blockIdx.y * TK;
  const uint32_t j = s0 >> logn, k0 = s0 & (n - 1);
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (uint32_t r = warp; r < 32; r += 8) {
    const uint64_t p = p0 + r;
    tile[r][lane] = p < np ? polys[(p * L + j) * n + k0 + lane] : 0u;
  }
  __syncthreads();
  for (uint32_t kk = warp; kk < TK; kk += 8) {
    const uint64_t p = p0 + lane;
    if (p >= np) continue;
    const uint64_t P = poly0 + p;
    const uint64_t i = P / D2, c = P % D2;
    res[((uint64_t)(s0 + kk) * D1 + i) * D2 + c] = tile[lane][kk];
  }
}

// Limb layout: polys are column-major ids, p -> (c = c0 + p / D1, i = p % D1).
__global__ void __launch_bounds__(256) k_db_scatter_limb(const uint32_t *__restrict__ polys, uint64_t c0,
                                                         uint64_t np, uint32_t D1, uint32_t D2, uint32_t L,
                                                         uint32_t logn, uint8_t *__restrict__ res) {
  __shared__ uint32_t tile[32][TK + 1];
  const uint32_t n = 1u << logn;
  const uint64_t p0 = (uint64_t)blockIdx.x * 32;
  const uint32_t s0 = blockIdx.y * TK;
  const uint32_t j = s0 >> logn, k0 = s0 & (n - 1);
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (uint32_t r = warp; r < 32; r += 8) {
    const uint64_t p = p0 + r;
    tile[r][lane] = p < np ? polys[(p * L + j) * n + k0 + lane] : 0u;
  }
  __syncthreads();
  for (uint32_t kk = warp; kk < TK; kk += 8) {
    const uint64_t p = p0 + lane;
    if (p >= np) continue;
    const uint64_t c = c0 + p / D1, i = p % D1;
    const uint32_t v = tile[lane][kk];
    const uint64_t s = s0 + kk;
#pragma unroll
    for (uint32_t limb = 0; limb < 4; ++limb) res[((s * 4 + limb) * D2 + c) * D1 + i] = (uint8_t)(v >> (8 * limb));
  }
}

// Gather the residues of one DB polynomial back out of the resident layout.
__global__ void k_db_read_poly(const void *__restrict__ res, int layout, uint64_t poly, uint32_t D1, uint32_t D2,
                               uint32_t L, uint32_t logn, uint32_t *__restrict__ out) {
  const uint32_t n = 1u << logn;
  const uint64_t i = poly / D2, c = poly % D2;
  for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < (uint64_t)L * n;
       t += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t s = t;  // t = j*n + k is the slot index
    uint32_t v;
    if (layout == PIR_LAYOUT_PLAIN) {
      v = static_cast<const uint32_t *>(res)[(s * D1 + i) * D2 + c];
    } else {
      const uint8_t *r8 = static_cast<const uint8_t *>(res);
      v = 0;
      for (uint32_t limb = 0; limb < 4; ++limb) v |= (uint32_t)r8[((s * 4 + limb) * D2 + c) * D1 + i] << (8 * limb);
    }
    out[t] = v;
  }
}

}  // namespace

cudaError_t launch_query_to_slots(const ParamCtx &c, const uint32_t *qhat, uint32_t B, uint32_t Kc, uint32_t Mp,
                                  uint32_t *qs, cudaStream_t s) {
  const uint64_t F = (uint64_t)Kc * Mp;
  if (F % 4 == 0) {
    dim3 grid((unsigned)((F + VT - 1) / VT), (c.p.L << c.logn) / VT);
    k_query_to_slots_v<<<grid, 256, 0, s>>>(qhat, B, Kc, c.p.L, c.logn, Mp, qs);
    return cudaGetLastError();
  }
  dim3 grid((unsigned)((F + TF - 1) / TF), (c.p.L << c.logn) / TK);
  k_query_to_slots<<<grid, 256, 0, s>>>(qhat, B, Kc, c.p.L, c.logn, Mp, qs);
  return cudaGetLastError();
}

cudaError_t launch_query_to_limbs(const ParamCtx &c, const uint32_t *qhat, uint32_t B, uint32_t Kc, uint32_t Mp,
                                  uint8_t *ql, cudaStream_t s) {
  dim3 grid((Kc + 31) / 32, (c.p.L << c.logn) / TK, Mp);
  k_query_to_limbs<<<grid, 256, 0, s>>>(qhat, B, Kc, c.p.L, c.logn, Mp, ql);
  return cudaGetLastError();
}

cudaError_t launch_slots_to_responses(const ParamCtx &c, const uint32_t *out, uint32_t B, uint32_t D2,
                                      uint32_t *resp, cudaStream_t s) {
  const uint64_t F = (uint64_t)2 * B * D2;
  if (F % 4 == 0) {
    dim3 grid((unsigned)((F + VT - 1) / VT), (c.p.L << c.logn) / VT);
    k_slots_to_responses_v<<<grid, 256, 0, s>>>(out, 2 * B, D2, c.p.L, c.logn, resp);
    return cudaGetLastError();
  }
  dim3 grid((unsigned)((F + TF - 1) / TF), (c.p.L << c.logn) / TK);
  k_slots_to_responses<<<grid, 256, 0, s>>>(out, 2 * B, D2, c.p.L, c.logn, resp);
  return cudaGetLastError();
}

cudaError_t launch_db_scatter(const ParamCtx &c, int layout, uint32_t D1, uint32_t D2, const uint32_t *polys,
                              uint64_t first, uint64_t np, void *resident, cudaStream_t s) {
  if (np == 0) return cudaSuccess;
  dim3 grid((unsigned)((np + 31) / 32), (c.p.L << c.logn) / TK);
  if (layout == PIR_LAYOUT_PLAIN)
    k_db_scatter_plain<<<grid, 256, 0, s>>>(polys, first, np, D1, D2, c.p.L, c.logn, static_cast<uint32_t *>(resident));
  else
    k_db_scatter_limb<<<grid, 256, 0, s>>>(polys, first, np, D1, D2, c.p.L, c.logn, static_cast<uint8_t *>(resident));
  return cudaGetLastError();
}

cudaError_t launch_db_read_poly(const ParamCtx &c, int layout, uint32_t D1, uint32_t D2, const void *resident,
                                uint64_t poly, uint32_t *out, cudaStream_t s) {
  k_db_read_poly<<<(c.p.L << c.logn) / 256, 256, 0, s>>>(resident, layout, poly, D1, D2, c.p.L, c.logn, out);
  return cudaGetLastError();
}

// Range check of residue rows: rows [rows][n], row r over prime q_{r % L}; sets *bad
// when any word is not below its prime (input validation, not on the answer path).
__global__ void k_check_residues(const uint4 *__restrict__ rows, uint64_t nrows, uint32_t n4, uint32_t L,
                                 NttConst C, uint32_t *__restrict__ bad) {
  const uint64_t total = nrows * n4;
  uint32_t found = 0;
  for (uint64_t w = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; w < total; w += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t j = (uint32_t)((w / n4) % L);
    uint32_t q = C.q[0];
#pragma unroll
    for (uint32_t i = 1; i < PIR_MAX_L; ++i) q = j == i ? C.q[i] : q;
    const uint4 v = __ldg(rows + w);
    found |= (v.x >= q) | (v.y >= q) | (v.z >= q) | (v.w >= q);
  }
  if (__any_sync(0xffffffffu, found) && (threadIdx.x & 31) == 0) atomicOr(bad, 1u);
}

cudaError_t launch_check_residues(const ParamCtx &c, const uint32_t *rows, uint64_t nrows, uint32_t *bad,
                                  cudaStream_t s) {
  if (nrows == 0) return cudaSuccess;
  const uint32_t n4 = (1u << c.logn) / 4;
  const uint64_t words = nrows * n4;
  uint64_t blocks = (words + 255) / 256;
  if (blocks > 152ull * 16) blocks = 152ull * 16;
  k_check_residues<<<(unsigned)blocks, 256, 0, s>>>(reinterpret_cast<const uint4 *>(rows), nrows, n4, c.p.L, c.ntt,
                                                    bad);
  return cudaGetLastError();
}

}  // namespace gbpir
