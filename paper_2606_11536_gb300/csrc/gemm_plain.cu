// gemm_plain.cu -- the first-dimension modular GEMM on CUDA cores (Sec. 4 "INT32
// modular GEMM", Sec. 4.2; the paper also keeps a CUDA-core kernel for batch 1,
// Sec. 5).
//
// For every slot s = j*n + k (prime q_j, NTT slot k):
//   out[s][m][c] = sum_{i < Kc} qs[s][i][m] * db[s][i0 + i][c]   (mod q_j)
// with m = 2b + comp the query rows (a- and b-polynomial of each ciphertext).
//
// Products of two residues are below 2^60 and go into u64 accumulators with one
// u32 x u32 + u64 multiply-add each (Sec. 4.2's lazy reduction, re-derived for
// 30-bit primes: fold63 after at most 8 products keeps every accumulator below
// 2^64; the paper's 32-MAC bound is for primes below 2^29).
//
// Two kernels:
//   k_gemv  -- few query rows (M <= 8): a stream over the resident DB, one slot per
//              CTA, 128-bit loads along c, query rows broadcast from shared memory.
//              Bound by HBM bandwidth.
//   k_gemm  -- M >= 16: a tiled SIMT GEMM per slot, operands staged through shared
//              memory with cp.async double buffering; thread tile RM rows x 8 columns,
//              the columns in two groups of 4 half a tile apart so that a warp's
//              128-bit shared loads cover contiguous 256-byte spans (no bank conflicts).
//              Bound by the INT32 multiply-add pipe.
#include "common.cuh"

namespace gbpir {
namespace {

// ---------------------------------------------------------------------------
// GEMV-shaped kernel (M <= MB, MB in {2, 4, 8})
// ---------------------------------------------------------------------------
constexpr int kGemvThreads = 256;
constexpr int kGemvSmemWords = 8192;  // 32 KiB: query chunk, later the phase partials
constexpr int kGemvUnroll = 8;        // products per accumulator between folds

template <int MB>
__global__ void __launch_bounds__(kGemvThreads) k_gemv(const uint32_t *__restrict__ db, const uint32_t *__restrict__ qs,
                                                       uint32_t M, uint32_t Mp, uint32_t D1, uint32_t D2, uint32_t i0,
                                                       uint32_t Kc, uint32_t *__restrict__ out, ModConst mc,
                                                       uint32_t logn, uint32_t nslots, int acc_in) {
  __shared__ __align__(16) uint32_t sm[kGemvSmemWords];
  const uint32_t nq = D2 >> 2;                        // column quads
  const uint32_t QT = nq < kGemvThreads ? nq : kGemvThreads;
  const uint32_t P = kGemvThreads / QT;               // i-phases
  const uint32_t tid = threadIdx.x;
  const uint32_t p = tid / QT, cq0 = tid % QT;
  const bool phase_ok = p < P;                        // 256 % QT threads idle when QT does not divide 256
  const uint32_t IC = kGemvSmemWords / MB;            // ciphertexts per query chunk in smem

  for (uint32_t s = blockIdx.x; s < nslots; s += gridDim.x) {
    const uint32_t j = s >> logn;
    const uint32_t q = mc.q[j];
    const uint64_t mu = mc.mu[j], k63 = mc.k63[j];
    const uint32_t *dbs = db + ((uint64_t)s * D1 + i0) * D2;
    const uint32_t *qss = qs + (uint64_t)s * Kc * Mp;
    for (uint32_t cqb = 0; cqb < nq; cqb += QT) {  // uniform trip count: the body synchronizes
      const uint32_t cq = cqb + cq0;
      const bool active = phase_ok && cq < nq;
      uint64_t acc[MB][4];
#pragma unroll
      for (int m = 0; m < MB; ++m)
#pragma unroll
        for (int e = 0; e < 4; ++e) acc[m][e] = 0;
      for (uint32_t ic = 0; ic < Kc; ic += IC) {
        const uint32_t icn = Kc - ic < IC ? Kc - ic : IC;
        __syncthreads();
        // query chunk -> sm[i][MB], zero padded for m >= M
        for (uint32_t t = tid; t < icn * MB; t += kGemvThreads) {
          const uint32_t i = t / MB, m = t % MB;
          sm[t] = m < M ? qss[(uint64_t)(ic + i) * Mp + m] : 0u;
        }
        __syncthreads();
        const uint32_t *rowp = dbs + (uint64_t)ic * D2 + 4 * cq;
        uint32_t i = active ? p : icn;
        for (; i + (kGemvUnroll - 1) * P < icn; i += kGemvUnroll * P) {
          uint4 d[kGemvUnroll];
#pragma unroll
          for (int u = 0; u < kGemvUnroll; ++u)
            d[u] = __ldcs(reinterpret_cast<const uint4 *>(rowp + (uint64_t)(i + u * P) * D2));
#pragma unroll
          for (int u = 0; u < kGemvUnroll; ++u) {
            const uint32_t *qv = sm + (i + u * P) * MB;
#pragma unroll
            for (int m = 0; m < MB; ++m) {
              const uint32_t a = qv[m];
              mac_wide(acc[m][0], a, d[u].x);
              mac_wide(acc[m][1], a, d[u].y);
              mac_wide(acc[m][2], a, d[u].z);
              mac_wide(acc[m][3], a, d[u].w);
            }
          }
#pragma unroll
          for (int m = 0; m < MB; ++m)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[m][e] = fold63(acc[m][e], k63);
        }
        for (; i < icn; i += P) {
          const uint4 d = __ldcs(reinterpret_cast<const uint4 *>(rowp + (uint64_t)i * D2));
          const uint32_t *qv = sm + i * MB;
#pragma unroll
          for (int m = 0; m < MB; ++m) {
            const uint32_t a = qv[m];
            mac_wide(acc[m][0], a, d.x);
            mac_wide(acc[m][1], a, d.y);
            mac_wide(acc[m][2], a, d.z);
            mac_wide(acc[m][3], a, d.w);
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[m][e] = fold63(acc[m][e], k63);
          }
        }
      }
      // combine the P phases: partials -> smem [p][m][4 * cq_local + e] -> phase 0 sums
      __syncthreads();
      const uint32_t stride = MB * 4 * QT;  // words per phase
      if (phase_ok) {
#pragma unroll
        for (int m = 0; m < MB; ++m)
#pragma unroll
          for (int e = 0; e < 4; ++e) sm[p * stride + (m * QT + cq0) * 4 + e] = reduce64(acc[m][e], q, mu);
      }
      __syncthreads();
      if (p == 0 && cq < nq) {
#pragma unroll
        for (int m = 0; m < MB; ++m) {
          if ((uint32_t)m >= M) break;
          uint32_t r[4];
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            uint64_t sum = 0;
            for (uint32_t pp = 0; pp < P; ++pp) sum += sm[pp * stride + (m * QT + cq0) * 4 + e];
            r[e] = reduce64(sum, q, mu);
          }
          uint4 *o = reinterpret_cast<uint4 *>(out + ((uint64_t)s * M + m) * D2 + 4 * cq);
          if (acc_in) {
            const uint4 prev = *o;
            r[0] = reduce64((uint64_t)r[0] + prev.x, q, mu);
            r[1] = reduce64((uint64_t)r[1] + prev.y, q, mu);
            r[2] = reduce64((uint64_t)r[2] + prev.z, q, mu);
            r[3] = reduce64((uint64_t)r[3] + prev.w, q, mu);
          }
          *o = make_uint4(r[0], r[1], r[2], r[3]);
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Tiled GEMM (M >= 16): CTA tile TM rows x TC columns, K stages of KS rows, NT
// threads, thread tile RM x 8; MINB CTAs per SM asked of the register allocator
// (0: no request).
// ---------------------------------------------------------------------------
constexpr int kKS = 16;

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem, bool pred) {
  const uint32_t sa = (uint32_t)__cvta_generic_to_shared(smem);
  const int sz = pred ? 16 : 0;  // zero-fill when out of range
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(gmem), "r"(sz));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;\n" ::); }

// KS: K rows per stage (a multiple of the 8 products between folds); the narrow tiles
// for small batches take fewer rows so that their wide column tile fits static
// shared memory.
template <int TM, int TC, int RM, int KS = kKS, int NT = 256, int MINB = 0>
__global__ void __launch_bounds__(NT, MINB) k_gemm(const uint32_t *__restrict__ db, const uint32_t *__restrict__ qs,
                                              uint32_t M, uint32_t Mp, uint32_t D1, uint32_t D2, uint32_t i0,
                                              uint32_t Kc, uint32_t *__restrict__ out, ModConst mc, uint32_t logn,
                                              int acc_in) {
  static_assert((TM / RM) * (TC / 8) == NT, "thread tile RM x 8 over NT threads");
  static_assert(kFoldProducts == 8, "one of the thread tile's 8 columns is folded per K row");
  static_assert(KS % kFoldProducts == 0, "every stage ends with each column folded once per 8 rows");
  __shared__ __align__(16) uint32_t As[2][KS][TM];
  __shared__ __align__(16) uint32_t Bs[2][KS][TC];
  const uint32_t nct = (D2 + TC - 1) / TC, nmt = (Mp + TM - 1) / TM;
  const uint64_t bid = blockIdx.x;
  const uint32_t ct = (uint32_t)(bid % nct);
  const uint32_t mt = (uint32_t)((bid / nct) % nmt);
  const uint32_t s = (uint32_t)(bid / ((uint64_t)nct * nmt));
  const uint32_t j = s >> logn;
  const uint32_t q = mc.q[j];
  const uint64_t mu = mc.mu[j], k63 = mc.k63[j];
  const uint32_t m0 = mt * TM, c0 = ct * TC;
  const uint32_t *dbs = db + ((uint64_t)s * D1 + i0) * D2;
  const uint32_t *qss = qs + (uint64_t)s * Kc * Mp;
  const uint32_t tid = threadIdx.x;
  const uint32_t tc = tid % (TC / 8), tm = tid / (TC / 8);

  // loader mapping: A tile = kKS x TM words = kKS*TM/4 uint4; B tile = kKS*TC/4 uint4
  auto load_tiles = [&](int buf, uint32_t k0) {
    for (uint32_t t = tid; t < KS * TM / 4; t += NT) {
      const uint32_t r = t / (TM / 4), c4 = (t % (TM / 4)) * 4;
      const bool ok = (k0 + r < Kc) && (m0 + c4 < Mp);
      const uint32_t *g = ok ? qss + (uint64_t)(k0 + r) * Mp + m0 + c4 : qss;
      cp_async16(&As[buf][r][c4], g, ok);
    }
    for (uint32_t t = tid; t < KS * TC / 4; t += NT) {
      const uint32_t r = t / (TC / 4), c4 = (t % (TC / 4)) * 4;
      const bool ok = (k0 + r < Kc) && (c0 + c4 < D2);
      const uint32_t *g = ok ? dbs + (uint64_t)(k0 + r) * D2 + c0 + c4 : dbs;
      cp_async16(&Bs[buf][r][c4], g, ok);
    }
    cp_async_commit();
  };

  uint64_t acc[RM][8];
#pragma unroll
  for (int a = 0; a < RM; ++a)
#pragma unroll
    for (int b = 0; b < 8; ++b) acc[a][b] = 0;

  const uint32_t nk = (Kc + KS - 1) / KS;
  load_tiles(0, 0);
  for (uint32_t kt = 0; kt < nk; ++kt) {
    const int buf = kt & 1;
    cp_async_wait0();
    __syncthreads();
    if (kt + 1 < nk) load_tiles(buf ^ 1, (kt + 1) * KS);
#pragma unroll
    for (int kk = 0; kk < KS; ++kk) {
      uint32_t av[RM];
      if constexpr (RM == 8) {
        const uint4 a0 = *reinterpret_cast<const uint4 *>(&As[buf][kk][tm * 8]);
        const uint4 a1 = *reinterpret_cast<const uint4 *>(&As[buf][kk][tm * 8 + 4]);
        av[0] = a0.x, av[1] = a0.y, av[2] = a0.z, av[3] = a0.w;
        av[4] = a1.x, av[5] = a1.y, av[6] = a1.z, av[7] = a1.w;
      } else if constexpr (RM == 4) {
        const uint4 a = *reinterpret_cast<const uint4 *>(&As[buf][kk][tm * 4]);
        av[0] = a.x, av[1] = a.y, av[2] = a.z, av[3] = a.w;
      } else if constexpr (RM == 2) {
        const uint2 a = *reinterpret_cast<const uint2 *>(&As[buf][kk][tm * 2]);
        av[0] = a.x, av[1] = a.y;
      } else {
        av[0] = As[buf][kk][tm];  // one row per thread: a broadcast within the warp
      }
      const uint4 b0 = *reinterpret_cast<const uint4 *>(&Bs[buf][kk][tc * 4]);
      const uint4 b1 = *reinterpret_cast<const uint4 *>(&Bs[buf][kk][TC / 2 + tc * 4]);
      const uint32_t bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int x = 0; x < RM; ++x)
#pragma unroll
        // the plain C++ form: here (operands from 128-bit shared loads, 32 independent
        // accumulators) the compiler emits one 32x32+64 multiply-add per product and
        // schedules them better than the opaque PTX helper (measured 7.1 vs 6.5 T/s)
        for (int y = 0; y < 8; ++y) acc[x][y] += (uint64_t)av[x] * bv[y];
      // staggered lazy reduction: after K row kk, column kk % 8 of the thread tile has
      // taken 8 products since its last fold.  Folding one column per row (instead of
      // all 32 accumulators every 8 rows) keeps the folds, on the integer ALU, beside
      // the multiply-adds instead of in bursts that leave the multiply-add pipe idle
      // while a CTA's warps, aligned by its barriers, all fold at once (measured 4%
      // faster at 2B = 64 and 2B = 16).
#pragma unroll
      for (int x = 0; x < RM; ++x) acc[x][kk & 7] = fold63(acc[x][kk & 7], k63);
    }
    __syncthreads();
  }

#pragma unroll
  for (int x = 0; x < RM; ++x) {
    const uint32_t m = m0 + tm * RM + x;
    if (m >= M) continue;
    uint32_t *orow = out + ((uint64_t)s * M + m) * D2;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const uint32_t c = c0 + h * (TC / 2) + tc * 4;
      if (c >= D2) continue;
      uint32_t r[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) r[e] = reduce64(acc[x][h * 4 + e], q, mu);
      uint4 *o = reinterpret_cast<uint4 *>(orow + c);
      if (acc_in) {
        const uint4 prev = *o;
        r[0] = reduce64((uint64_t)r[0] + prev.x, q, mu);
        r[1] = reduce64((uint64_t)r[1] + prev.y, q, mu);
        r[2] = reduce64((uint64_t)r[2] + prev.z, q, mu);
        r[3] = reduce64((uint64_t)r[3] + prev.w, q, mu);
      }
      *o = make_uint4(r[0], r[1], r[2], r[3]);
    }
  }
}

template <int MB>
cudaError_t gemv_launch(const ParamCtx &c, const uint32_t *db, uint32_t D1, uint32_t D2, const uint32_t *qs,
                        uint32_t M, uint32_t Mp, uint32_t i0, uint32_t Kc, uint32_t *out, int acc, cudaStream_t s) {
  const uint32_t nslots = c.p.L << c.logn;
  k_gemv<MB><<<nslots, kGemvThreads, 0, s>>>(db, qs, M, Mp, D1, D2, i0, Kc, out, c.mod, c.logn, nslots, acc);
  return cudaGetLastError();
}

template <int TM, int TC, int RM, int KS = kKS, int NT = 256, int MINB = 0>
cudaError_t gemm_launch(const ParamCtx &c, const uint32_t *db, uint32_t D1, uint32_t D2, const uint32_t *qs,
                        uint32_t M, uint32_t Mp, uint32_t i0, uint32_t Kc, uint32_t *out, int acc, cudaStream_t s) {
  const uint64_t nslots = (uint64_t)c.p.L << c.logn;
  const uint64_t blocks = nslots * ((D2 + TC - 1) / TC) * ((Mp + TM - 1) / TM);
  if (blocks > 0x7FFFFFFFull) return cudaErrorInvalidConfiguration;
  k_gemm<TM, TC, RM, KS, NT, MINB><<<(unsigned)blocks, NT, 0, s>>>(db, qs, M, Mp, D1, D2, i0, Kc, out, c.mod, c.logn, acc);
  return cudaGetLastError();
}

}  // namespace

// Tile ids: 1 = GEMV MB=2, 2 = GEMV MB=4, 3 = GEMV MB=8, 4 = GEMM 16x256, 5 = GEMM 32x256,
// 6 = GEMM 64x128, 7 = TMA-staged scan (M <= 8, D2 <= 512; scan_tma.cu), 8 = GEMM 8x256
// (one query row per thread, for a few queries).  0 picks the TMA scan up to 4 rows,
// the 8-row GEMM up to 8, else a GEMM tile by M.
uint32_t gemm_plain_tiles() { return 8; }

bool gemm_plain_tile_ok(uint32_t tile, uint32_t M, uint32_t D2) {
  switch (tile) {
    case 0: case 4: case 5: case 6: case 8: return true;
    case 1: return M <= 2;
    case 2: return M <= 4;
    case 3: return M <= 8;
    case 7: return scan_tma_supports(M, D2);
  }
  return false;
}

cudaError_t launch_gemm_plain(const ParamCtx &c, const uint32_t *db, uint32_t D1, uint32_t D2, const uint32_t *qs,
                              uint32_t M, uint32_t Mp, uint32_t i0, uint32_t Kc, uint32_t *out, int acc,
                              uint32_t tile, int stall_test, cudaStream_t s) {
  if (tile == 0) {
    // measured on GB300: the TMA scan wins up to 4 query rows; with 6-8 rows its
    // accumulators cap it at one or two CTAs per SM and the GEMV-shaped kernel wins
    // (5-8 rows: the 8-row GEMM tile measured 15-17% ahead of the GEMV)
    if (M <= 4 && scan_tma_supports(M, D2)) tile = 7;
    else if (M <= 2) tile = 1;
    else if (M <= 4) tile = 2;
    else if (M <= 8) tile = 8;
    else if (M <= 16) tile = 4;
    else if (M <= 32) tile = 5;
    else tile = 6;
  }
  if (stall_test && tile != 7) return cudaErrorInvalidValue;
  switch (tile) {
    case 7: return launch_scan_tma(c, db, D1, D2, qs, M, Mp, i0, Kc, out, acc, stall_test, 0, nullptr, s);
    case 1: return M <= 2 ? gemv_launch<2>(c, db, D1, D2, qs, M, Mp, i0, Kc, out, acc, s) : cudaErrorInvalidValue;
    case 2: return M <= 4 ? gemv_launch<4>(c, db, D1, D2, qs, M, Mp, i0, Kc, out, acc, s) : cudaErrorInvalidValue;
    case 3: return M <= 8 ? gemv_launch<8>(c, db, D1, D2, qs, M, Mp, i0, Kc, out, acc, s) : cudaErrorInvalidValue;
    case 4: return gemm_launch<16, 256, 2>(c, db, D1, D2, qs, M, Mp, i0, Kc, out, acc, s);
    // the same 8 x 8 tiles (4.7% faster at 2B = 32); at 2B = 16 a 16 x 512 tile of them
    // measured 4% slower than tile 4's 2 x 8 tiles over 256 threads
    case 5: return gemm_launch<32, 256, 8, 16, 128, 3>(c, db, D1, D2, qs, M, Mp, i0, Kc, out, acc, s);
    // 8 x 8 thread tiles over 128 threads, three CTAs per SM (168 registers): half the
    // shared-memory loads per multiply-add of 4 x 8 tiles over 256 threads, measured
    // 3.4% faster at 2B = 64; 32-row stages
    case 6: return gemm_launch<64, 128, 8, 32, 128, 3>(c, db, D1, D2, qs, M, Mp, i0, Kc, out, acc, s);
    case 8: return gemm_launch<8, 256, 1>(c, db, D1, D2, qs, M, Mp, i0, Kc, out, acc, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace gbpir
