// scan_tma.cu -- the batch-1..4 first-dimension scan as a TMA-staged stream over
// the resident NTT-form DB (the memory-bound GEMV of Sec. 5 / the (#RNS*N)-parallel
// modular GEMMs of Sec. 4.2 with 2B <= 8 query rows).
//
//   out[s][m][c] = sum_{i < Kc} qs[s][i][m] * db[s][i0 + i][c]   (mod q_j),  s = j*n + k
//
// Persistent CTAs, as many per SM as registers and shared memory allow (three for
// batch 1): warp 8 is the producer, warps 0..7 consume.  The producer walks this
// CTA's slots (s = blockIdx.x, + gridDim.x, ...) in chunks of R DB rows and, per
// chunk, issues two 1-D bulk copies (cp.async.bulk, the TMA engine) into a ring of 4
// shared-memory stages: R*D2*4 bytes of DB rows (L2 evict-first: the DB is read
// once) and the matching R*Mp*4 bytes of slot-major query rows.  Each stage has a
// "full" mbarrier (expect-tx bytes) and an "empty" mbarrier (one arrival per
// consumer warp).  The rings keep up to 12 chunks (~192 KiB) in flight per SM across
// slot boundaries, so the stream never drains between slots.
//
// Consumers own whole columns: lane = (phase ph, quad ql) with QW quads x PH row
// phases per warp; warp w covers quads w*QW + ql + 8*QW*t.  Each lane accumulates
// u32 x u32 -> u64 products (fold63 every <= 8 products keeps them below 2^64); at
// a slot's end the PH phases combine with warp shuffles, so no block barrier is
// ever needed after set-up.
//
// Every barrier wait is bounded (about one second of %globaltimer).  A wait that runs
// out sets the per-device error word; the producer then stops issuing, waits (again
// bounded) for the copies it has in flight, and the CTA returns.
#include "async.cuh"
#include "common.cuh"

namespace gbpir {
namespace {

constexpr int kConsumerWarps = 8;
constexpr int kThreads = (kConsumerWarps + 1) * 32;
constexpr int kStages = 4;
constexpr uint32_t kChunkTarget = 16384;       // DB bytes per stage
using async::bulk_g2s;
using async::mbar_arrive;
using async::mbar_expect_tx;
using async::mbar_init;
using async::saddr;
using async::wait_bounded;

struct ScanArgs {
  const uint32_t *db;  // plain resident layout [L*n][D1][D2]
  const uint32_t *qs;  // [L*n][Kc][Mp]
  uint32_t *out;       // [L*n][M][D2]
  uint32_t *err;       // per-device error word
  uint32_t M, Mp, D1, D2, i0, Kc;
  uint32_t R;          // DB rows per stage
  uint32_t stage_bytes;
  uint32_t nslots, logn;
  int acc_in;
  int stall_test;      // consumers wait on a barrier nobody arrives on (tests the timeout path)
  int out_poly;        // 1: out is the response layout [B][D2][2][L*n] (NTT domain), else [L*n][M][D2]
  const uint32_t *acc_src;  // optional slot-major partial [L*n][M][D2] added before the write
};

// Rows per unrolled group and CTAs per SM, by accumulator count (MB rows x T quads):
// the batch-1 shape keeps three CTAs (27 warps) per SM, two rows of loads per group.
template <int MB, int T>
struct ScanShape {
  static constexpr int U = (MB * T <= 4) ? 2 : 1;
  static constexpr int kMinBlocks = (MB * T <= 2) ? 3 : (MB * T <= 4) ? 2 : 1;
};

template <int MB, int T>
__global__ void __launch_bounds__(kThreads, ScanShape<MB, T>::kMinBlocks) k_scan_tma(ScanArgs a, ModConst mc) {
  constexpr int U = ScanShape<MB, T>::U;
  extern __shared__ __align__(128) uint8_t smem[];
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + kStages * a.stage_bytes);
  const uint32_t full0 = saddr(bars), empty0 = saddr(bars + kStages), stall = saddr(bars + 2 * kStages);
  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int st = 0; st < kStages; ++st) {
      mbar_init(full0 + 8 * st, 1);
      mbar_init(empty0 + 8 * st, kConsumerWarps);
    }
    mbar_init(stall, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  const uint32_t db_bytes_full = a.R * a.D2 * 4;

  if (warp == kConsumerWarps) {
    // ---------------- producer ----------------
    if (lane != 0) return;
    uint64_t pol_stream, pol_keep;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol_stream));
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol_keep));
    uint32_t it = 0;
    bool ok = true;
    for (uint32_t s = blockIdx.x; ok && s < a.nslots; s += gridDim.x) {
      for (uint32_t r0 = 0; r0 < a.Kc; r0 += a.R) {
        const uint32_t rows = a.Kc - r0 < a.R ? a.Kc - r0 : a.R;
        const uint32_t st = it % kStages, ph = (it / kStages) & 1;
        if (!wait_bounded(empty0 + 8 * st, ph ^ 1)) {
          atomicExch(a.err, 1u);
          ok = false;
          break;
        }
        const uint32_t dbb = rows * a.D2 * 4, qb = rows * a.Mp * 4;
        const uint32_t dst = saddr(smem + st * a.stage_bytes);
        mbar_expect_tx(full0 + 8 * st, dbb + qb);
        bulk_g2s(dst, a.db + ((uint64_t)s * a.D1 + a.i0 + r0) * a.D2, dbb, full0 + 8 * st, pol_stream);
        bulk_g2s(dst + db_bytes_full, a.qs + ((uint64_t)s * a.Kc + r0) * a.Mp, qb, full0 + 8 * st, pol_keep);
        ++it;
      }
    }
    // drain: never leave with copies in flight
    const uint32_t first = it > (uint32_t)kStages ? it - kStages : 0;
    for (uint32_t k = first; k < it; ++k)
      if (!wait_bounded(full0 + 8 * (k % kStages), (k / kStages) & 1)) atomicExch(a.err, 1u);
    return;
  }

  // ---------------- consumers ----------------
  if (a.stall_test) {
    // nothing ever arrives on this barrier: the bounded wait runs out
    if (!__all_sync(0xffffffffu, wait_bounded(stall, 0)) && lane == 0) atomicExch(a.err, 1u);
    return;
  }
  const uint32_t nq = a.D2 >> 2;
  uint32_t QW = 8;
  while (QW > nq) QW >>= 1;
  const uint32_t PH = 32 / QW;
  const uint32_t ql = lane % QW, phs = lane / QW;
  uint32_t quad[T];
  bool qv[T];
#pragma unroll
  for (int t = 0; t < T; ++t) {
    quad[t] = warp * QW + ql + kConsumerWarps * QW * t;
    qv[t] = quad[t] < nq;
  }

  uint32_t it = 0;
  for (uint32_t s = blockIdx.x; s < a.nslots; s += gridDim.x) {
    const uint32_t j = s >> a.logn;
    const uint32_t q = mc.q[j];
    const uint64_t mu = mc.mu[j], k63 = mc.k63[j];
    uint32_t pend = 0;  // products per accumulator since the last fold
    uint64_t acc[T][MB][4];
#pragma unroll
    for (int t = 0; t < T; ++t)
#pragma unroll
      for (int m = 0; m < MB; ++m)
#pragma unroll
        for (int e = 0; e < 4; ++e) acc[t][m][e] = 0;

    for (uint32_t r0 = 0; r0 < a.Kc; r0 += a.R) {
      const uint32_t rows = a.Kc - r0 < a.R ? a.Kc - r0 : a.R;
      const uint32_t st = it % kStages, ph = (it / kStages) & 1;
      // every lane observes the barrier (acquire); the vote keeps the warp uniform
      if (!__all_sync(0xffffffffu, wait_bounded(full0 + 8 * st, ph))) {
        if (lane == 0) atomicExch(a.err, 1u);
        return;
      }
      const uint32_t *dbs = reinterpret_cast<const uint32_t *>(smem + st * a.stage_bytes);
      const uint32_t *qsm = reinterpret_cast<const uint32_t *>(smem + st * a.stage_bytes + db_bytes_full);
      // rows phs, phs + PH, ... of this chunk, U at a time: all shared loads of a
      // group issue before its multiply-adds; a fold before any group that would
      // take an accumulator past kFoldProducts products.
      for (uint32_t r0l = phs; r0l < rows; r0l += U * PH) {
        if (pend + U > kFoldProducts) {
#pragma unroll
          for (int t = 0; t < T; ++t)
#pragma unroll
            for (int m = 0; m < MB; ++m)
#pragma unroll
              for (int e = 0; e < 4; ++e) acc[t][m][e] = fold63(acc[t][m][e], k63);
          pend = 0;
        }
        pend += U;
        uint32_t qrow[U][MB];
        uint4 d[U][T];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const uint32_t r = r0l + u * PH;
          const bool rv = r < rows;
          if constexpr (MB == 2) {
            const uint2 v = rv ? *reinterpret_cast<const uint2 *>(qsm + r * a.Mp) : make_uint2(0, 0);
            qrow[u][0] = v.x, qrow[u][1] = v.y;
          } else {
#pragma unroll
            for (int m4 = 0; m4 < MB; m4 += 4) {
              const uint4 v = rv ? *reinterpret_cast<const uint4 *>(qsm + r * a.Mp + m4) : make_uint4(0, 0, 0, 0);
              qrow[u][m4] = v.x, qrow[u][m4 + 1] = v.y, qrow[u][m4 + 2] = v.z, qrow[u][m4 + 3] = v.w;
            }
          }
#pragma unroll
          for (int t = 0; t < T; ++t)
            d[u][t] = (rv && qv[t]) ? *reinterpret_cast<const uint4 *>(dbs + r * a.D2 + 4 * quad[t])
                                    : make_uint4(0, 0, 0, 0);
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
          for (int t = 0; t < T; ++t)
#pragma unroll
            for (int m = 0; m < MB; ++m) {
              mac_wide(acc[t][m][0], qrow[u][m], d[u][t].x);
              mac_wide(acc[t][m][1], qrow[u][m], d[u][t].y);
              mac_wide(acc[t][m][2], qrow[u][m], d[u][t].z);
              mac_wide(acc[t][m][3], qrow[u][m], d[u][t].w);
            }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(empty0 + 8 * st);
      ++it;
    }

    // combine the PH row phases of each quad (lanes ql, ql + QW, ...) and write
#pragma unroll
    for (int t = 0; t < T; ++t) {
#pragma unroll
      for (int m = 0; m < MB; ++m) {
        uint32_t r[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          uint32_t v = (phs < PH) ? reduce64(acc[t][m][e], q, mu) : 0u;
          for (uint32_t off = QW; off < 32; off <<= 1) {
            const uint32_t o = __shfl_xor_sync(0xffffffffu, v, off);
            v += o;
            v = v >= q ? v - q : v;
          }
          r[e] = v;
        }
        if (phs == 0 && qv[t] && (uint32_t)m < a.M) {
          if (a.acc_src) {  // earlier K-chunks, slot-major: one coalesced 16-byte read
            const uint4 prev = *reinterpret_cast<const uint4 *>(a.acc_src + ((uint64_t)s * a.M + m) * a.D2 + 4 * quad[t]);
            r[0] = reduce64((uint64_t)r[0] + prev.x, q, mu);
            r[1] = reduce64((uint64_t)r[1] + prev.y, q, mu);
            r[2] = reduce64((uint64_t)r[2] + prev.z, q, mu);
            r[3] = reduce64((uint64_t)r[3] + prev.w, q, mu);
          }
          if (a.out_poly) {
            // response layout: element (b, c, comp, j, k) at ((b*D2 + c)*2 + comp)*L*n + s.
            // Consecutive slots go to consecutive CTAs at about the same time, so the
            // 4-byte stores of neighbouring k meet in L2 before reaching DRAM.
            const uint32_t b = (uint32_t)m >> 1, comp = (uint32_t)m & 1;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              uint32_t *o = a.out + (((uint64_t)b * a.D2 + 4 * quad[t] + e) * 2 + comp) * a.nslots + s;
              *o = a.acc_in ? reduce64((uint64_t)r[e] + *o, q, mu) : r[e];
            }
          } else {
            uint4 *o = reinterpret_cast<uint4 *>(a.out + ((uint64_t)s * a.M + m) * a.D2 + 4 * quad[t]);
            if (a.acc_in) {
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
}

template <int MB, int T>
cudaError_t scan_launch(const ParamCtx &c, const ScanArgs &a0, cudaStream_t s) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  ScanArgs a = a0;
  const size_t smem = (size_t)kStages * a.stage_bytes + (2 * kStages + 1) * sizeof(uint64_t);
  e = cudaFuncSetAttribute(k_scan_tma<MB, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_scan_tma<MB, T>, kThreads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const uint64_t want = (uint64_t)sms * per_sm;
  const uint32_t grid = a.nslots < want ? a.nslots : (uint32_t)want;
  k_scan_tma<MB, T><<<grid, kThreads, smem, s>>>(a, c.mod);
  return cudaGetLastError();
}

}  // namespace

// The TMA scan holds M <= 8 rows and D2 <= 8 * 8 * 4 * 2 = 512 columns per lane
// budget (T <= 2 quads per lane).
bool scan_tma_supports(uint32_t M, uint32_t D2) { return M <= 8 && D2 % 4 == 0 && D2 <= 512; }

cudaError_t launch_scan_tma(const ParamCtx &c, const uint32_t *db, uint32_t D1, uint32_t D2, const uint32_t *qs,
                            uint32_t M, uint32_t Mp, uint32_t i0, uint32_t Kc, uint32_t *out, int acc, int stall_test,
                            int out_poly, const uint32_t *acc_src, cudaStream_t s) {
  // query rows are bulk-copied: Mp = 2 needs an even Kc (16-byte chunk starts)
  if (!scan_tma_supports(M, D2) || Kc == 0 || !(Mp % 4 == 0 || (Mp == 2 && M <= 2 && Kc % 2 == 0)))
    return cudaErrorInvalidValue;
  uint32_t *err = nullptr;
  cudaError_t e = device_error_word(&err);
  if (e != cudaSuccess) return e;
  ScanArgs a = {};
  a.db = db;
  a.qs = qs;
  a.out = out;
  a.err = err;
  a.M = M;
  a.Mp = Mp;
  a.D1 = D1;
  a.D2 = D2;
  a.i0 = i0;
  a.Kc = Kc;
  a.R = kChunkTarget / (D2 * 4);
  if (a.R == 0) a.R = 1;
  if (a.R > Kc) a.R = Kc;
  if (Mp == 2 && (a.R & 1)) a.R = a.R > 1 ? a.R - 1 : 2;  // even row counts keep bulk copies 16-byte sized
  a.stage_bytes = (a.R * D2 * 4 + a.R * Mp * 4 + 127) & ~127u;
  a.nslots = c.p.L << c.logn;
  a.logn = c.logn;
  a.acc_in = acc;
  a.stall_test = stall_test;
  a.out_poly = out_poly;
  a.acc_src = acc_src;
  const uint32_t nq = D2 / 4;
  const int T = nq > 64 ? 2 : 1;  // 8 warps x 8 quads per pass
  const int MB = M <= 2 ? 2 : M <= 4 ? 4 : 8;
  if (MB == 2) return T == 1 ? scan_launch<2, 1>(c, a, s) : scan_launch<2, 2>(c, a, s);
  if (MB == 4) return T == 1 ? scan_launch<4, 1>(c, a, s) : scan_launch<4, 2>(c, a, s);
  return T == 1 ? scan_launch<8, 1>(c, a, s) : scan_launch<8, 2>(c, a, s);
}

}  // namespace gbpir
