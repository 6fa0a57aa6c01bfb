// lwe.cu -- the scalar-HE (LWE) DB GEMM of SimplePIR's online step (Sec. 2.5) on the
// INT8 tensor pipe, as Sec. 4.1 builds it:
//     out[b][i] = sum_j A[i][j] * Q[b][j]   (mod 2^32)
// with A the raw DB (D1 x D0 signed INT8 plaintexts, no NTT encoding, no bloating)
// and Q the B query vectors of Z_{2^32} entries.  Every query word splits into four
// byte planes Q_p (Q = sum_p 2^(8p) Q_p); each A Q_p is an s8 x u8 product with s32
// accumulation, and out = sum_p (A Q_p) << 8p.  Wrapping 32-bit arithmetic is exactly
// arithmetic mod 2^32, so the accumulators need no K chunking.
//
// Tensor path: mma.sync m16n8k32 s8.u8 -> s32 (this toolkit has no tcgen05 INT8 for
// sm_103a).  A warp owns 64 rows x 8 queries; its four n8 tiles are the four byte
// planes of the same 8 queries, so one thread holds all planes of its outputs and
// combines them with shifts.  The byte planes come straight from the staged query
// words: for 4 consecutive words of one query, eight prmt (a 4 x 4 byte transpose)
// give the four plane registers the B fragment wants.  A and Q tiles are staged by
// cp.async into double-buffered shared memory (A swizzled for ldmatrix).
//
// CUDA-core path (small batches, where the n8 query tile would be mostly padding):
// dp4a s8 x u8 over the same byte planes, one DB row per thread, the query planes
// transposed once per stage in shared memory and read as broadcasts.
#include "common.cuh"

namespace gbpir {
namespace {

constexpr int KS = 128;  // DB bytes of K per stage

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void cp16z(uint32_t saddr, const void *g, bool ok) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(saddr), "l"(g), "r"(ok ? 16 : 0));
}

__device__ __forceinline__ uint32_t prmt(uint32_t a, uint32_t b, uint32_t sel) {
  uint32_t d;
  asm("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(sel));
  return d;
}

// Byte planes of four words w0..w3: plane p = {w0.p, w1.p, w2.p, w3.p} (a 4 x 4 byte
// transpose in eight prmt).
__device__ __forceinline__ void byte_planes(uint32_t w0, uint32_t w1, uint32_t w2, uint32_t w3, uint32_t (&p)[4]) {
  const uint32_t t0 = prmt(w0, w1, 0x5140), t1 = prmt(w0, w1, 0x7362);  // {w0.0 w1.0 w0.1 w1.1}, {.2 .2 .3 .3}
  const uint32_t t2 = prmt(w2, w3, 0x5140), t3 = prmt(w2, w3, 0x7362);
  p[0] = prmt(t0, t2, 0x5410);
  p[1] = prmt(t0, t2, 0x7632);
  p[2] = prmt(t1, t3, 0x5410);
  p[3] = prmt(t1, t3, 0x7632);
}

// A tile: rows of KS bytes, 16-byte chunks XOR-swizzled by row (ldmatrix without
// bank conflicts).
__device__ __forceinline__ uint32_t swz_a(uint32_t r, uint32_t ch) { return r * KS + ((ch ^ (r & 7)) << 4); }
// Q tile: rows of KS words (512 B); chunk c of query n at c ^ (4 (n & 1)), so the
// fragment reads of a quarter warp (two queries x four chunks) hit distinct banks.
__device__ __forceinline__ uint32_t swz_q(uint32_t n, uint32_t c) { return n * KS * 4 + ((c ^ ((n & 1) << 2)) << 4); }

__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t (&r)[4]) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(addr));
}

__device__ __forceinline__ void mma_s8u8(int (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k32.row.col.s32.s8.u8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
      : "+r"(d[0]), "+r"(d[1]), "+r"(d[2]), "+r"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// CTA = 4 warps: WR along rows x WQ along queries; warp tile 64 rows x 8 queries.
template <int WQ>
__global__ void __launch_bounds__(128) k_lwe_mma(const int8_t *__restrict__ A, uint32_t D1, uint32_t D0,
                                                 const uint32_t *__restrict__ Q, uint32_t B, uint32_t *__restrict__ out) {
  constexpr int WR = 4 / WQ, TM = 64 * WR, TQ = 8 * WQ;
  constexpr int A_BYTES = TM * KS, Q_BYTES = TQ * KS * 4, STAGE = A_BYTES + Q_BYTES;
  extern __shared__ __align__(128) uint8_t smem[];
  const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t wr = warp % WR, wq = warp / WR;
  const uint64_t m0 = (uint64_t)blockIdx.x * TM;
  const uint32_t q0 = blockIdx.y * TQ;

  auto load_stage = [&](int buf, uint32_t k0) {
    const uint32_t sbase = smem_addr(smem + buf * STAGE);
    for (uint32_t t = tid; t < TM * (KS / 16); t += 128) {  // A: TM rows x 8 chunks
      const uint32_t ch = t & 7, r = t >> 3;
      const bool ok = (m0 + r < D1) && (k0 + ch * 16 < D0);
      const int8_t *g = A + (m0 + r) * D0 + k0 + ch * 16;
      cp16z(sbase + swz_a(r, ch), ok ? g : A, ok);
    }
    for (uint32_t t = tid; t < TQ * (KS / 4); t += 128) {  // Q: TQ queries x 32 chunks of 4 words
      const uint32_t c = t & 31, n = t >> 5;
      const bool ok = (q0 + n < B) && (k0 + c * 4 < D0);
      const uint32_t *g = Q + (uint64_t)(q0 + n) * D0 + k0 + c * 4;
      cp16z(sbase + A_BYTES + swz_q(n, c), ok ? g : Q, ok);
    }
    asm volatile("cp.async.commit_group;\n" ::);
  };

  int acc[4][4][4];  // [m16 tile][byte plane][fragment]
#pragma unroll
  for (int mt = 0; mt < 4; ++mt)
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
      for (int f = 0; f < 4; ++f) acc[mt][p][f] = 0;

  const uint32_t nk = (D0 + KS - 1) / KS;
  const uint32_t n_loc = wq * 8 + (lane >> 2), tg = lane & 3;
  load_stage(0, 0);
  for (uint32_t kt = 0; kt < nk; ++kt) {
    const int buf = kt & 1;
    asm volatile("cp.async.wait_group 0;\n" ::);
    __syncthreads();
    if (kt + 1 < nk) load_stage(buf ^ 1, (kt + 1) * KS);
    const uint32_t sA = smem_addr(smem + buf * STAGE), sQ = sA + A_BYTES;
#pragma unroll
    for (int kk = 0; kk < KS / 32; ++kk) {
      // B fragments of the four byte planes: words k = 32 kk + 4 tg + (0..3) and +16
      uint32_t b0[4], b1[4];
      {
        uint4 lo, hi;
        asm volatile("ld.shared.v4.u32 {%0,%1,%2,%3}, [%4];\n"
                     : "=r"(lo.x), "=r"(lo.y), "=r"(lo.z), "=r"(lo.w)
                     : "r"(sQ + swz_q(n_loc, kk * 8 + tg)));
        asm volatile("ld.shared.v4.u32 {%0,%1,%2,%3}, [%4];\n"
                     : "=r"(hi.x), "=r"(hi.y), "=r"(hi.z), "=r"(hi.w)
                     : "r"(sQ + swz_q(n_loc, kk * 8 + 4 + tg)));
        byte_planes(lo.x, lo.y, lo.z, lo.w, b0);
        byte_planes(hi.x, hi.y, hi.z, hi.w, b1);
      }
#pragma unroll
      for (int mt = 0; mt < 4; ++mt) {
        uint32_t a[4];
        const uint32_t ar = wr * 64 + mt * 16 + (lane & 15), ach = 2 * kk + (lane >> 4);
        ldsm_x4(sA + swz_a(ar, ach), a);
#pragma unroll
        for (int p = 0; p < 4; ++p) mma_s8u8(acc[mt][p], a, b0[p], b1[p]);
      }
    }
  }

  // epilogue: out = sum_p acc_p << 8p (mod 2^32); fragment f: row g + 8 (f >> 1), query 2 tg + (f & 1)
  const uint32_t g = lane >> 2;
#pragma unroll
  for (int mt = 0; mt < 4; ++mt)
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      const uint64_t i = m0 + wr * 64 + mt * 16 + g + 8 * (f >> 1);
      const uint32_t b = q0 + wq * 8 + 2 * tg + (f & 1);
      if (i >= D1 || b >= B) continue;
      uint32_t v = 0;
#pragma unroll
      for (int p = 0; p < 4; ++p) v += (uint32_t)acc[mt][p][f] << (8 * p);
      out[(uint64_t)b * D1 + i] = v;
    }
}

// CUDA-core path: 256 rows per CTA (one per thread) x QB queries.  Per stage the raw
// query words are staged, then transposed once into planes [QB][KS/4][4] that every
// thread reads as broadcasts.  blockIdx.z takes K stages [z * kper, (z + 1) * kper):
// with more than one split the partial sums are added into the zeroed output with
// wrapping atomics, exact in any order because the result is taken mod 2^32.
template <int QB>
__global__ void __launch_bounds__(256) k_lwe_dp4a(const int8_t *__restrict__ A, uint32_t D1, uint32_t D0,
                                                  const uint32_t *__restrict__ Q, uint32_t B, uint32_t kper,
                                                  uint32_t *__restrict__ out) {
  constexpr int A_BYTES = 256 * KS, QR_BYTES = QB * KS * 4, STAGE = A_BYTES + QR_BYTES;
  extern __shared__ __align__(128) uint8_t smem[];
  uint4 *planes = reinterpret_cast<uint4 *>(smem + 2 * STAGE);  // [QB][KS/4] of {p0, p1, p2, p3}
  const uint32_t tid = threadIdx.x;
  const uint64_t m0 = (uint64_t)blockIdx.x * 256;
  const uint32_t q0 = blockIdx.y * QB;

  auto load_stage = [&](int buf, uint32_t k0) {
    const uint32_t sbase = smem_addr(smem + buf * STAGE);
    for (uint32_t t = tid; t < 256 * (KS / 16); t += 256) {  // 8 threads per 128-byte row segment
      const uint32_t ch = t & 7, r = t >> 3;
      const bool ok = (m0 + r < D1) && (k0 + ch * 16 < D0);
      const int8_t *g = A + (m0 + r) * D0 + k0 + ch * 16;
      cp16z(sbase + swz_a(r, ch), ok ? g : A, ok);
    }
    for (uint32_t t = tid; t < QB * (KS / 4); t += 256) {
      const uint32_t c = t % (KS / 4), n = t / (KS / 4);
      const bool ok = (q0 + n < B) && (k0 + c * 4 < D0);
      const uint32_t *g = Q + (uint64_t)(q0 + n) * D0 + k0 + c * 4;
      cp16z(sbase + A_BYTES + (n * (KS / 4) + c) * 16, ok ? g : Q, ok);
    }
    asm volatile("cp.async.commit_group;\n" ::);
  };

  int acc[QB][4];
#pragma unroll
  for (int b = 0; b < QB; ++b)
#pragma unroll
    for (int p = 0; p < 4; ++p) acc[b][p] = 0;

  const uint32_t nk_all = (D0 + KS - 1) / KS, kbeg = blockIdx.z * kper;
  const uint32_t nk = kbeg >= nk_all ? 0 : (nk_all - kbeg < kper ? nk_all - kbeg : kper);
  if (nk > 0) load_stage(0, kbeg * KS);
  for (uint32_t kt = 0; kt < nk; ++kt) {
    const int buf = kt & 1;
    asm volatile("cp.async.wait_group 0;\n" ::);
    __syncthreads();  // this stage landed; the previous stage's planes are no longer read
    const uint8_t *st = smem + buf * STAGE;
    for (uint32_t t = tid; t < QB * (KS / 4); t += 256) {
      const uint4 w = reinterpret_cast<const uint4 *>(st + A_BYTES)[t];
      uint32_t p[4];
      byte_planes(w.x, w.y, w.z, w.w, p);
      planes[t] = make_uint4(p[0], p[1], p[2], p[3]);
    }
    if (kt + 1 < nk) load_stage(buf ^ 1, (kbeg + kt + 1) * KS);
    __syncthreads();
#pragma unroll 2
    for (uint32_t ch = 0; ch < KS / 16; ++ch) {
      const uint4 a = *reinterpret_cast<const uint4 *>(st + swz_a(tid, ch));
      const uint32_t aw[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
      for (int b = 0; b < QB; ++b)
#pragma unroll
        for (int w = 0; w < 4; ++w) {
          const uint4 pl = planes[b * (KS / 4) + ch * 4 + w];  // the same address in every thread
          asm("dp4a.s32.u32 %0, %1, %2, %0;" : "+r"(acc[b][0]) : "r"(aw[w]), "r"(pl.x));
          asm("dp4a.s32.u32 %0, %1, %2, %0;" : "+r"(acc[b][1]) : "r"(aw[w]), "r"(pl.y));
          asm("dp4a.s32.u32 %0, %1, %2, %0;" : "+r"(acc[b][2]) : "r"(aw[w]), "r"(pl.z));
          asm("dp4a.s32.u32 %0, %1, %2, %0;" : "+r"(acc[b][3]) : "r"(aw[w]), "r"(pl.w));
        }
    }
  }
  const uint64_t i = m0 + tid;
  if (i >= D1) return;
#pragma unroll
  for (int b = 0; b < QB; ++b) {
    if (q0 + b >= B) break;
    uint32_t v = 0;
#pragma unroll
    for (int p = 0; p < 4; ++p) v += (uint32_t)acc[b][p] << (8 * p);
    if (gridDim.z > 1)
      atomicAdd(out + (uint64_t)(q0 + b) * D1 + i, v);
    else
      out[(uint64_t)(q0 + b) * D1 + i] = v;
  }
}

template <int WQ>
cudaError_t mma_launch(const int8_t *A, uint32_t D1, uint32_t D0, const uint32_t *Q, uint32_t B, uint32_t *out,
                       cudaStream_t s) {
  constexpr int TM = 64 * (4 / WQ), TQ = 8 * WQ;
  constexpr int smem = 2 * (TM * KS + TQ * KS * 4);
  cudaError_t e = cudaFuncSetAttribute(k_lwe_mma<WQ>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  const uint64_t gx = (D1 + TM - 1) / TM, gy = (B + TQ - 1) / TQ;
  if (gx > 0x7FFFFFFFull || gy > 65535) return cudaErrorInvalidConfiguration;
  k_lwe_mma<WQ><<<dim3((unsigned)gx, (unsigned)gy), 128, smem, s>>>(A, D1, D0, Q, B, out);
  return cudaGetLastError();
}

template <int QB>
cudaError_t dp4a_launch(const int8_t *A, uint32_t D1, uint32_t D0, const uint32_t *Q, uint32_t B, uint32_t *out,
                        cudaStream_t s, uint32_t *launches) {
  constexpr int smem = 2 * (256 * KS + QB * KS * 4) + QB * KS * 4;
  cudaError_t e = cudaFuncSetAttribute(k_lwe_dp4a<QB>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  const uint64_t gx = (D1 + 255) / 256, gy = (B + QB - 1) / QB;
  if (gx > 0x7FFFFFFFull || gy > 65535) return cudaErrorInvalidConfiguration;
  // split K until the grid fills about four waves of resident CTAs
  int dev = 0, sms = 0, per_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_lwe_dp4a<QB>, 256, smem)) != cudaSuccess) return e;
  const uint32_t nk = (D0 + KS - 1) / KS;
  const uint64_t target = 4ull * sms * (per_sm > 0 ? per_sm : 1);
  uint64_t splits = (target + gx * gy - 1) / (gx * gy);
  const uint64_t max_splits = nk / 8 > 0 ? nk / 8 : 1;  // at least 8 stages per split
  if (splits > max_splits) splits = max_splits;
  if (splits > 64) splits = 64;
  if (splits < 1) splits = 1;
  const uint32_t kper = (uint32_t)((nk + splits - 1) / splits);
  splits = (nk + kper - 1) / kper;
  if (splits > 1) {
    if ((e = cudaMemsetAsync(out, 0, (size_t)B * D1 * sizeof(uint32_t), s)) != cudaSuccess) return e;
  }
  k_lwe_dp4a<QB><<<dim3((unsigned)gx, (unsigned)gy, (unsigned)splits), 256, smem, s>>>(A, D1, D0, Q, B, kper, out);
  *launches = 1;
  return cudaGetLastError();
}

}  // namespace

// path: PIR_LWE_AUTO picks the tensor path from 8 queries up.
cudaError_t launch_lwe_gemm(const int8_t *A, uint32_t D1, uint32_t D0, const uint32_t *Q, uint32_t B, uint32_t *out,
                            uint32_t path, cudaStream_t s) {
  if (path == PIR_LWE_AUTO) path = B >= 8 ? PIR_LWE_TENSOR : PIR_LWE_SIMT;
  if (path == PIR_LWE_TENSOR) return B >= 16 ? mma_launch<2>(A, D1, D0, Q, B, out, s) : mma_launch<1>(A, D1, D0, Q, B, out, s);
  if (path == PIR_LWE_SIMT) {
    uint32_t launches = 0;
    if (B >= 4) return dp4a_launch<4>(A, D1, D0, Q, B, out, s, &launches);
    if (B == 3) return dp4a_launch<3>(A, D1, D0, Q, B, out, s, &launches);
    if (B == 2) return dp4a_launch<2>(A, D1, D0, Q, B, out, s, &launches);
    return dp4a_launch<1>(A, D1, D0, Q, B, out, s, &launches);
  }
  return cudaErrorInvalidValue;
}

}  // namespace gbpir

extern "C" pir_status_t pir_lwe_answer(const int8_t *db, uint32_t D1, uint32_t D0, const uint32_t *queries,
                                       uint32_t B, uint32_t *out, uint32_t path, void *stream) {
  using namespace gbpir;
  if (!db || !queries || !out || D1 == 0 || D0 == 0 || B == 0 || path > PIR_LWE_SIMT) return PIR_ERR_ARG;
  if (D0 % 16 != 0 || D0 > (1u << 24)) return PIR_ERR_ARG;
  if (((uintptr_t)db & 15u) || ((uintptr_t)queries & 15u) || ((uintptr_t)out & 15u)) return PIR_ERR_ARG;
  cudaError_t e = launch_lwe_gemm(db, D1, D0, queries, B, out, path, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_status(e);
  count_launches(1);
  return PIR_OK;
}
