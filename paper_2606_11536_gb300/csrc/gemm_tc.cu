// gemm_tc.cu -- the batched first-dimension modular GEMM on the bf16 tensor cores:
// tcgen05.mma with its accumulators in tensor memory.  This is the paper's limb
// decomposition of an INT32 GEMM into narrow tensor-core products (Sec. 4.1),
// re-targeted to the tensor format GB300 runs at full rate (its INT8 tensor rate
// is a small fraction of the bf16 one) and to modular arithmetic.
//
// Digits.  A residue x in [0, q), q < 2^30, is x = sum_{l<4} 256^l d_l with signed
// digits d_0..d_2 in [-128, 127] and d_3 in [0, 64]; such integers are exact in
// bf16.  For slot s the modular GEMM splits into 16 digit GEMMs
//     P_ab[c][m] = sum_{i < Kc} DB_b[i][c] * Q_a[i][m],    |P_ab| <= Kc * 2^14,
// so for Kc <= 1024 every partial sum is an integer of at most 2^24 in magnitude
// that the f32 accumulator holds exactly, in any summation order.
//
// One MMA (M = 128, N = 4 * query rows, K = 16) forms all 16 digit products at once.
//   A rows are (DB column, DB digit) pairs: r = 4 * c_local + b, 32 columns per tile.
//   B rows are (query row, query digit) pairs: n = 4 * m + a.
// The epilogue reads P back with tcgen05.ld, converts to integers, weights digit
// pair (a, b) by 2^(8(a+b)) mod q and sums: in int64 over a within a thread, then over
// b across the 4 lanes that hold one column.  Then it reduces mod q and writes
// out[s][m][c] (or adds it to the earlier K-chunks' partial).
//
// Layouts.  Both operands are bf16, in the K-major no-swizzle canonical layout of
// the tensor-core shared-memory descriptors.  Core matrices are 8 rows x 16 bytes;
// element (row r, k < 16) of a [rows][16] block is at
//     (r / 8) * 128 + (k / 8) * 64 + (r % 8) * 8 + k % 8        (elements)
// so a block is contiguous, and a run of 8-row groups is a contiguous sub-range.
//   resident DB   dbt[s][u][4 * D2 rows][16]   u = i / 16
//   query digits  qt[s][u][4 * Mp rows][16]    u over one K-chunk
// Descriptors: LBO (K direction) = 128 bytes, SBO (8-row groups) = 256 bytes.
//
// Work unit = (slot, T tiles of 32 DB columns, one tile of <= 64 query rows); its
// accumulators take T * N <= 256 tensor-memory columns.  One persistent CTA per SM
// runs its units through two accumulator buffers.  In the cluster forms (C = 2 or 4
// CTAs, one per SM) the C CTAs of a cluster take units of one slot side by side, and
// each one loads 1/C of every stage's query digits and multicasts it to all C: the
// query digits cross from L2 to the SMs once per C units instead of once per unit.
//   warp 8   streams the units' K stages (KS16 x 16 rows) back to back into a
//            ring of S shared-memory stages with 1-D bulk copies;
//   warp 9   allocates the tensor memory and issues the MMAs from one thread;
//   warps 0..7  run the epilogue of the previous unit meanwhile.
// Every barrier wait is bounded; a wait that runs out sets the device error word.
#include <cuda.h>  // CUtensorMap and its enums only: the encoder is reached through the runtime
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "async.cuh"
#include "common.cuh"

namespace gbpir {
namespace {

using async::bulk_g2s;
using async::mbar_expect_tx;
using async::mbar_init;
using async::saddr;
using async::wait_bounded;

constexpr int kEpiWarps = 8;  // two sets of the four tensor-memory lane quarters
constexpr int kProducerWarp = kEpiWarps, kMmaWarp = kEpiWarps + 1;
constexpr int kThreads = (kEpiWarps + 2) * 32;
constexpr int kMaxStages = 4;
// One persistent CTA per SM with two tensor-memory accumulator buffers of
// kTmemBudget columns each (the MMAs of one unit overlap the epilogue of the one
// before).  Every CTA takes more than half of an SM's shared memory, so a second
// never lands on the same SM (its tensor-memory allocation would wait for the first).
constexpr uint32_t kTmemCols = 512;                   // the whole tensor memory of the SM
constexpr uint32_t kTmemBudget = kTmemCols / 2;        // one of two accumulator buffers
constexpr uint32_t kSmemBudget = 200u << 10, kSmemFloor = 116u << 10;
constexpr uint32_t kBlockBytes = 128 * 16 * 2;  // one 128-row x K16 bf16 block
// The 2-SM form: stage budget, and a spare run after the barriers so that no operand
// read of the last stage can leave the CTA's shared memory.
constexpr uint32_t kSmemBudget2 = 200u << 10, kSpareBytes2 = 8u << 10;

// Signed base-256 digits of x < 2^30.
__device__ __forceinline__ void digits4(uint32_t x, int (&d)[4]) {
  int v = (int)x;
#pragma unroll
  for (int l = 0; l < 3; ++l) {
    d[l] = (int)(int8_t)(v & 0xFF);
    v = (v - d[l]) >> 8;  // exact: v - d[l] is a multiple of 256
  }
  d[3] = v;
}

__device__ __forceinline__ uint16_t bf16_bits(int d) { return __bfloat16_as_ushort(__float2bfloat16_rn((float)d)); }

// Element offset of (row r, k) inside one [rows][16] core-matrix block.
__host__ __device__ __forceinline__ uint32_t cm_off(uint32_t r, uint32_t k) {
  return (r >> 3) * 128 + (k >> 3) * 64 + (r & 7) * 8 + (k & 7);
}

// Shared-memory matrix descriptor: K-major, no swizzle, LBO 128 B, SBO 256 B.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(256 >> 4) << 32) |
         (1ull << 46);
}

// Instruction descriptor, kind::f16: D f32, A and B bf16, both K-major, M x N.
__device__ __forceinline__ uint32_t instr_desc(uint32_t M, uint32_t N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((N >> 3) << 17) | ((M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

// Arrive on `bar` in every CTA of the cluster set in cta_mask once this thread's MMAs
// issued so far complete.
__device__ __forceinline__ void mma_commit_multicast(uint32_t bar, uint16_t cta_mask) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(bar),
      "h"(cta_mask)
      : "memory");
}

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\nbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Arrive on the mbarrier at local offset `bar` in CTA `rank` of the cluster.
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t bar, uint32_t rank) {
  uint32_t remote;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(bar), "r"(rank));
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(remote) : "memory");
}

// 32 consecutive accumulator columns of this warp's 32 lanes
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// 32 x 32 -> 64-bit signed multiply-add
__device__ __forceinline__ int64_t mad_wide(int32_t x, int32_t y, int64_t acc) {
  int64_t d;
  asm("mad.wide.s32 %0, %1, %2, %3;" : "=l"(d) : "r"(x), "r"(y), "l"(acc));
  return d;
}

struct TcArgs {
  const uint16_t *db;  // resident DB digits
  const uint16_t *qt;  // query digits of this K-chunk
  uint32_t *out;       // [L*n][M][D2]
  uint32_t *err;       // per-device error word
  uint32_t M, Mp, D1, D2, i0, Kc;
  uint32_t T, KS16, S, stage_bytes, ctiles, mtiles, nunits;
  uint32_t nbuf, buf_cols;  // accumulator buffers in tensor memory and their column stride
  uint32_t logn;
  int acc_in;
};

template <typename T>
__device__ __forceinline__ T pick(const T (&v)[PIR_MAX_L], uint32_t j) {
  T r = v[0];
#pragma unroll
  for (uint32_t i = 1; i < PIR_MAX_L; ++i) r = j == i ? v[i] : r;
  return r;
}

// Work unit u = (slot s, query-row tile mt, column tile ct), ct fastest: CTAs that
// run side by side take the column tiles of one slot and share its query digits in L2.
struct Unit {
  uint32_t s, mt, ct, n0, Nt;
};

__device__ __forceinline__ Unit unit_of(const TcArgs &a, uint32_t u) {
  Unit w;
  w.ct = u % a.ctiles;
  const uint32_t rest = u / a.ctiles;
  w.mt = rest % a.mtiles;
  w.s = rest / a.mtiles;
  const uint32_t Ntot = 4 * a.Mp;
  w.n0 = w.mt * 256;
  w.Nt = Ntot - w.n0 < 256 ? Ntot - w.n0 : 256;
  return w;
}

// Persistent: cluster g of G = gridDim.x / C takes unit groups g, g + G, ... and its
// CTA of rank r the unit C * group + r (C = 1: CTA b takes units b, b + gridDim.x, ...).
// The producer streams the units' K stages back to back through the ring; the MMA
// thread accumulates unit k into tensor-memory buffer k % 2 while the epilogue drains
// buffer (k - 1) % 2.  With C > 1 a stage slot is refilled only after the MMAs of all
// C CTAs have read it: each MMA thread's commit arrives on the empty barrier of every
// CTA in the cluster (C arrivals per phase), because every producer writes its part
// of the query digits into all C rings.
template <int C>
__global__ void __launch_bounds__(kThreads, 1) k_gemm_tc(TcArgs a, ModConst mc) {
  extern __shared__ __align__(1024) uint8_t smem[];
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + a.S * a.stage_bytes);
  const uint32_t full0 = saddr(bars), empty0 = saddr(bars + kMaxStages);
  const uint32_t tfull0 = saddr(bars + 2 * kMaxStages), tempty0 = saddr(bars + 2 * kMaxStages + 2);
  const uint32_t done = saddr(bars + 2 * kMaxStages + 4);
  uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + 2 * kMaxStages + 5);
  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t R = 4 * a.D2, U = a.D1 / 16, Uc = a.Kc / 16;
  const uint32_t nst = Uc / a.KS16, Ntot = 4 * a.Mp;
  const uint32_t db_stage = a.KS16 * a.T * kBlockBytes;
  const uint32_t rank = C > 1 ? cluster_rank() : 0, cl0 = blockIdx.x / C, ncl = gridDim.x / C;
  const uint32_t ngroups = a.nunits / C;
  const uint16_t all_ctas = (uint16_t)((1u << C) - 1);

  if (threadIdx.x == 0) {
    for (int st = 0; st < kMaxStages; ++st) {
      mbar_init(full0 + 8 * st, 1);
      mbar_init(empty0 + 8 * st, C);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(tfull0 + 8 * b, 1);
      mbar_init(tempty0 + 8 * b, kEpiWarps);
    }
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == kMmaWarp) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(tslot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (C > 1) cluster_sync();  // every CTA's barriers exist before any multicast copy or commit
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;

  if (warp == kProducerWarp) {
    if (lane == 0) {
      const uint64_t pol_db = async::policy_evict_first(), pol_q = async::policy_evict_last();
      const uint8_t *dbs = reinterpret_cast<const uint8_t *>(a.db);
      const uint8_t *qs = reinterpret_cast<const uint8_t *>(a.qt);
      uint32_t it = 0;
      bool ok = true;
      for (uint32_t gi = cl0; ok && gi < ngroups; gi += ncl) {
        const Unit w = unit_of(a, gi * C + rank);
        const uint32_t qbytes = a.KS16 * w.Nt * 32;  // all of the stage's query digits land here
        for (uint32_t st = 0; st < nst; ++st, ++it) {
          const uint32_t slot = it % a.S, ph = (it / a.S) & 1;
          if (!wait_bounded(empty0 + 8 * slot, ph ^ 1)) {
            atomicExch(a.err, 1u);
            ok = false;
            break;
          }
          const uint32_t dst = saddr(smem + slot * a.stage_bytes);
          mbar_expect_tx(full0 + 8 * slot, db_stage + qbytes);
          for (uint32_t v = 0; v < a.KS16; ++v) {
            const uint64_t uu = a.i0 / 16 + (uint64_t)st * a.KS16 + v;
            const uint64_t e = (((uint64_t)w.s * U + uu) * R + (uint64_t)w.ct * a.T * 128) * 16;
            bulk_g2s(dst + v * a.T * kBlockBytes, dbs + 2 * e, a.T * kBlockBytes, full0 + 8 * slot, pol_db);
          }
          // query digits: this CTA's 1/C share of each contiguous run, to all C CTAs
          if (w.Nt == Ntot) {  // the stage's query rows are one contiguous run
            const uint64_t e = ((uint64_t)w.s * Uc + (uint64_t)st * a.KS16) * Ntot * 16;
            const uint32_t part = qbytes / C, o = rank * part;
            if (C == 1)
              bulk_g2s(dst + db_stage, qs + 2 * e, qbytes, full0 + 8 * slot, pol_q);
            else
              async::bulk_g2s_multicast(dst + db_stage + o, qs + 2 * e + o, part, full0 + 8 * slot, all_ctas, pol_q);
          } else {
            const uint32_t part = w.Nt * 32 / C, o = rank * part;
            for (uint32_t v = 0; v < a.KS16; ++v) {
              const uint64_t e = (((uint64_t)w.s * Uc + (uint64_t)st * a.KS16 + v) * Ntot + w.n0) * 16;
              if (C == 1)
                bulk_g2s(dst + db_stage + v * w.Nt * 32, qs + 2 * e, w.Nt * 32, full0 + 8 * slot, pol_q);
              else
                async::bulk_g2s_multicast(dst + db_stage + v * w.Nt * 32 + o, qs + 2 * e + o, part, full0 + 8 * slot,
                                          all_ctas, pol_q);
            }
          }
        }
      }
      // drain: never leave with copies in flight
      const uint32_t first = it > a.S ? it - a.S : 0;
      for (uint32_t k = first; k < it; ++k)
        if (!wait_bounded(full0 + 8 * (k % a.S), (k / a.S) & 1)) atomicExch(a.err, 1u);
      // and, in a cluster, no commit of a peer's MMAs still on its way to this CTA's
      // empty barriers: wait for the release of the last stages by all C CTAs
      if (C > 1)
        for (uint32_t k = first; k < it; ++k)
          if (!wait_bounded(empty0 + 8 * (k % a.S), (k / a.S) & 1)) atomicExch(a.err, 1u);
    }
    __syncwarp();
  } else if (warp == kMmaWarp) {
    if (lane == 0) {
      uint32_t it = 0, k = 0;
      bool ok = true;
      for (uint32_t gi = cl0; ok && gi < ngroups; gi += ncl, ++k) {
        const Unit w = unit_of(a, gi * C + rank);
        const uint32_t buf = k % a.nbuf, use = k / a.nbuf;
        if (!wait_bounded(tempty0 + 8 * buf, (use & 1) ^ 1)) {  // the epilogue has drained this buffer
          atomicExch(a.err, 1u);
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t idesc = instr_desc(128, w.Nt), dcol = tmem + buf * a.buf_cols;
        for (uint32_t st = 0; st < nst; ++st, ++it) {
          const uint32_t slot = it % a.S;
          if (!wait_bounded(full0 + 8 * slot, (it / a.S) & 1)) {
            atomicExch(a.err, 1u);
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t base = saddr(smem + slot * a.stage_bytes);
          for (uint32_t v = 0; v < a.KS16; ++v) {
            const uint64_t bdesc = smem_desc(base + db_stage + v * w.Nt * 32);
            for (uint32_t t = 0; t < a.T; ++t) {
              const uint64_t adesc = smem_desc(base + (v * a.T + t) * kBlockBytes);
              mma_bf16(dcol + t * w.Nt, adesc, bdesc, idesc, (st | v) != 0);
            }
          }
          // the stage is free once these MMAs have read it (in every CTA that fills it)
          if (C == 1)
            mma_commit(empty0 + 8 * slot);
          else
            mma_commit_multicast(empty0 + 8 * slot, all_ctas);
        }
        mma_commit(tfull0 + 8 * buf);  // this unit's accumulators are complete
      }
      // on every path: no MMA may still be running when the tensor memory is freed
      mma_commit(done);
      if (!wait_bounded(done, 0)) atomicExch(a.err, 1u);
    }
    __syncwarp();
  } else {
    // ---------------- epilogue: warps 0..7 ----------------
    const uint32_t quarter = warp & 3, b = lane & 3;
    const uint32_t row = 32 * quarter + lane;  // accumulator lane: column c_local = row / 4, DB digit b
    const bool hi2 = (b & 2) != 0, hi1 = (b & 1) != 0;
    uint32_t k = 0;
    for (uint32_t gi = cl0; gi < ngroups; gi += ncl, ++k) {
      const Unit w = unit_of(a, gi * C + rank);
      const uint32_t buf = k % a.nbuf, use = k / a.nbuf;
      if (!__all_sync(0xffffffffu, wait_bounded(tfull0 + 8 * buf, use & 1))) {
        if (lane == 0) atomicExch(a.err, 1u);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t j = w.s >> a.logn;
      const uint32_t q = pick(mc.q, j);
      const uint64_t mu = pick(mc.mu, j);
      const int64_t off = (int64_t)q << 29;  // > 2^58 > |sum of the 16 weighted digit products|
      // digit-pair weights 2^(8(a + b)) mod q for this lane's DB digit b
      uint32_t pw[7];
      pw[0] = 1;
#pragma unroll
      for (int t = 1; t < 7; ++t) pw[t] = reduce64((uint64_t)pw[t - 1] << 8, q, mu);
      int32_t wgt[4];  // < 2^30
#pragma unroll
      for (int d = 0; d < 4; ++d)
        wgt[d] = (int32_t)(b == 0 ? pw[d] : b == 1 ? pw[d + 1] : b == 2 ? pw[d + 2] : pw[d + 3]);
      // items (column tile t, group of 8 query rows x 4 digits), shared by the sets
      const uint32_t G = w.Nt / 32;
      for (uint32_t item = warp >> 2; item < a.T * G; item += kEpiWarps / 4) {
        const uint32_t t = item / G, g = item % G;
        const uint32_t c = (w.ct * a.T + t) * 32 + (row >> 2);
        uint32_t f[32];
        tmem_ld32(tmem + buf * a.buf_cols + ((32 * quarter) << 16) + t * w.Nt + 32 * g, f);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          // this lane's DB digit b, weighted over the query digits a, for rows 8g + 4h + mm
          int64_t sum[4];
#pragma unroll
          for (int mm = 0; mm < 4; ++mm) {
            int64_t v = 0;
#pragma unroll
            for (int d = 0; d < 4; ++d)
              v = mad_wide(__float2int_rn(__uint_as_float(f[16 * h + 4 * mm + d])), wgt[d], v);
            sum[mm] = v;
          }
          // reduce-scatter over the column's 4 lanes: lane b ends with row 8g + 4h + b's total
          int64_t k0 = hi2 ? sum[2] : sum[0], k1 = hi2 ? sum[3] : sum[1];
          const int64_t o0 = hi2 ? sum[0] : sum[2], o1 = hi2 ? sum[1] : sum[3];
          k0 += __shfl_xor_sync(0xffffffffu, o0, 2);
          k1 += __shfl_xor_sync(0xffffffffu, o1, 2);
          int64_t mine = hi1 ? k1 : k0;
          mine += __shfl_xor_sync(0xffffffffu, hi1 ? k0 : k1, 1);
          const uint32_t m = w.n0 / 4 + 8 * g + 4 * h + b;
          if (m < a.M) {
            uint32_t r = reduce64((uint64_t)(mine + off), q, mu);
            uint32_t *o = a.out + ((uint64_t)w.s * a.M + m) * a.D2 + c;
            if (a.acc_in) {
              r += *o;
              if (r >= q) r -= q;
            }
            *o = r;
          }
        }
      }
      // this warp's reads of the buffer are complete: hand it back to the MMA thread
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) async::mbar_arrive(tempty0 + 8 * buf);
    }
  }

  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (C > 1) cluster_sync();  // no CTA leaves while a peer may still copy into it or arrive on it
  if (warp == kMmaWarp) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols)
                 : "memory");
  }
}

// ---------------------------------------------------------------------------
// The 2-SM form: one MMA per CTA pair (cta_group::2, M = 256).
//
// A cluster of two CTAs on two SMs takes a unit of 64 DB columns: each CTA holds
// its own 32 columns (128 A rows = (column, digit) pairs) and half of the query
// digits (N/2 B rows); the pair's MMA, issued by the even CTA, reads A from both
// CTAs' shared memory (rows 0..127 from the even CTA, 128..255 from the odd one)
// and B as the two halves, and leaves each CTA the accumulator rows of its own A
// half, [128 lanes][N columns], in its own tensor memory.  Per SM and MMA that is
// 4 KiB of DB digits plus N/2 x 32 bytes of query digits instead of N x 32 bytes:
// a third fewer operand bytes than the 1-SM form at N = 256, so the same stages
// in flight keep the tensor cores busy for longer.
//
// Barriers (mbarriers at the same shared-memory offsets in both CTAs):
//   full[st]    local: this CTA's stage `st` has arrived (expect-tx by its producer)
//   pfull[st]   even CTA only: the odd CTA's stage `st` has arrived (one remote
//               arrive by the odd CTA's relay thread, which waits on its own full)
//   empty[st]   both: the pair's MMAs have read stage `st` (multicast commit)
//   tfull[b]    both: accumulator buffer b is complete (multicast commit)
//   tempty[b]   even CTA only: both CTAs' epilogues have drained buffer b
//               (2 x kEpiWarps arrivals, the odd CTA's remote)
// Every wait is bounded; the end is a cluster barrier, after which both CTAs
// release the pair's tensor memory.

__device__ __forceinline__ void mma_bf16_pair(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc,
                                              uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}

// Arrive on `bar` in both CTAs of the pair once the pair MMAs issued so far complete.
__device__ __forceinline__ void mma_commit_pair(uint32_t bar) {
  const uint16_t both = 0x3;
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(bar),
      "h"(both)
      : "memory");
}

// The pair's work unit u = (slot s, query-row tile mt, column-tile pair cp), cp fastest.
__device__ __forceinline__ Unit unit_of_pair(const TcArgs &a, uint32_t u, uint32_t rank) {
  Unit w;
  const uint32_t pairs = a.ctiles / 2;
  const uint32_t cp = u % pairs;
  const uint32_t rest = u / pairs;
  w.ct = 2 * cp + rank;
  w.mt = rest % a.mtiles;
  w.s = rest / a.mtiles;
  const uint32_t Ntot = 4 * a.Mp;
  w.n0 = w.mt * 256;
  w.Nt = Ntot - w.n0 < 256 ? Ntot - w.n0 : 256;
  return w;
}

constexpr int kMaxStages2 = 8;

// Tensor-map load of a 3-D box into this CTA's shared memory at dst, completing its
// bytes on the barrier at shared::cluster address bar, which .cta_group::2 lets lie
// in either CTA of the pair (here: the pair's leader).  Coordinates are elements.
__device__ __forceinline__ void tma_load_3d_pair(uint32_t dst, const CUtensorMap *map, uint32_t c0, uint32_t c1,
                                                 uint32_t c2, uint32_t bar, uint64_t policy) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.cta_group::2"
      ".L2::cache_hint [%0], [%1, {%2, %3, %4}], [%5], %6;" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(bar), "l"(policy)
      : "memory");
}

// TMA = false: 1-D bulk copies into each CTA's own ring and a relay thread in the odd
// CTA; TMA = true: tensor-map loads (maps tm_db, tm_q) whose bytes complete on the
// even CTA's barrier directly, so the pair's MMAs wait on one barrier and no relay
// runs.  The TMA form needs every unit's query rows to be a full half of one tile
// (4 Mp <= 256 or a multiple of 256): a tensor map has one box size.
template <bool TMA>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kThreads, 1)
    k_gemm_tc2(TcArgs a, ModConst mc, const __grid_constant__ CUtensorMap tm_db,
               const __grid_constant__ CUtensorMap tm_q) {
  extern __shared__ __align__(1024) uint8_t smem[];
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + a.S * a.stage_bytes);
  const uint32_t full0 = saddr(bars), empty0 = saddr(bars + kMaxStages2), pfull0 = saddr(bars + 2 * kMaxStages2);
  const uint32_t tfull0 = saddr(bars + 3 * kMaxStages2), tempty0 = saddr(bars + 3 * kMaxStages2 + 2);
  const uint32_t done = saddr(bars + 3 * kMaxStages2 + 4);
  uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + 3 * kMaxStages2 + 5);
  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = cluster_rank(), cluster = blockIdx.x >> 1, nclusters = gridDim.x >> 1;
  const uint32_t R = 4 * a.D2, U = a.D1 / 16, Uc = a.Kc / 16;
  const uint32_t nst = Uc / a.KS16, Ntot = 4 * a.Mp;
  const uint32_t db_stage = a.KS16 * kBlockBytes;

  if (threadIdx.x == 0) {
    for (int st = 0; st < kMaxStages2; ++st) {
      mbar_init(full0 + 8 * st, 1);
      mbar_init(empty0 + 8 * st, 1);
      mbar_init(pfull0 + 8 * st, 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(tfull0 + 8 * b, 1);
      mbar_init(tempty0 + 8 * b, 2 * kEpiWarps);
    }
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == kMmaWarp) {
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(tslot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  cluster_sync();  // both CTAs' barriers exist before any remote arrive or multicast commit
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;

  if (warp == kProducerWarp) {
    if (lane == 0) {
      const uint64_t pol_db = async::policy_evict_first(), pol_q = async::policy_evict_last();
      const uint8_t *dbs = reinterpret_cast<const uint8_t *>(a.db);
      const uint8_t *qs = reinterpret_cast<const uint8_t *>(a.qt);
      uint32_t it = 0;
      bool ok = true;
      for (uint32_t u = cluster; ok && u < a.nunits; u += nclusters) {
        const Unit w = unit_of_pair(a, u, rank);
        const uint32_t half = w.Nt / 2, qbytes = a.KS16 * half * 32;
        for (uint32_t st = 0; st < nst; ++st, ++it) {
          const uint32_t slot = it % a.S, ph = (it / a.S) & 1;
          if (!wait_bounded(empty0 + 8 * slot, ph ^ 1)) {
            atomicExch(a.err, 1u);
            ok = false;
            break;
          }
          const uint32_t dst = saddr(smem + slot * a.stage_bytes);
          if (TMA) {
            // this CTA's 128 DB digit rows and half of the query rows, as two boxes
            // [KS16][rows / 8][128 elements]; both CTAs' bytes complete on the even
            // CTA's barrier, which it arms for the pair's two stages
            uint32_t lead;
            asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(lead) : "r"(full0 + 8 * slot), "r"(0u));
            if (rank == 0) mbar_expect_tx(full0 + 8 * slot, 2 * (db_stage + qbytes));
            tma_load_3d_pair(dst, &tm_db, 0, w.ct * 16, w.s * U + a.i0 / 16 + st * a.KS16, lead, pol_db);
            tma_load_3d_pair(dst + db_stage, &tm_q, 0, (w.n0 + rank * half) / 8, w.s * Uc + st * a.KS16, lead,
                             pol_q);
          } else {
            mbar_expect_tx(full0 + 8 * slot, db_stage + qbytes);
            for (uint32_t v = 0; v < a.KS16; ++v) {
              const uint64_t uu = a.i0 / 16 + (uint64_t)st * a.KS16 + v;
              const uint64_t e = (((uint64_t)w.s * U + uu) * R + (uint64_t)w.ct * 128) * 16;
              bulk_g2s(dst + v * kBlockBytes, dbs + 2 * e, kBlockBytes, full0 + 8 * slot, pol_db);
            }
            for (uint32_t v = 0; v < a.KS16; ++v) {  // this CTA's half of the stage's query rows
              const uint64_t e =
                  (((uint64_t)w.s * Uc + (uint64_t)st * a.KS16 + v) * Ntot + w.n0 + rank * half) * 16;
              bulk_g2s(dst + db_stage + v * half * 32, qs + 2 * e, half * 32, full0 + 8 * slot, pol_q);
            }
          }
        }
      }
      // drain: never leave with copies in flight (in the TMA form the even CTA's
      // barriers count both CTAs' bytes; the odd CTA's copies are complete once the
      // even CTA has drained, before the closing cluster barrier)
      const uint32_t first = it > a.S ? it - a.S : 0;
      if (!TMA || rank == 0)
        for (uint32_t k = first; k < it; ++k)
          if (!wait_bounded(full0 + 8 * (k % a.S), (k / a.S) & 1)) atomicExch(a.err, 1u);
    }
    __syncwarp();
  } else if (warp == kMmaWarp) {
    if (lane == 0 && rank == 1 && !TMA) {
      // relay: tell the even CTA's MMA thread when this CTA's stages have arrived
      uint32_t it = 0;
      bool ok = true;
      for (uint32_t u = cluster; ok && u < a.nunits; u += nclusters)
        for (uint32_t st = 0; st < nst; ++st, ++it) {
          if (!wait_bounded(full0 + 8 * (it % a.S), (it / a.S) & 1)) {
            atomicExch(a.err, 1u);
            ok = false;
            break;
          }
          mbar_arrive_cluster(pfull0 + 8 * (it % a.S), 0);
        }
    } else if (lane == 0 && rank == 0) {
      uint32_t it = 0, k = 0;
      bool ok = true;
      for (uint32_t u = cluster; ok && u < a.nunits; u += nclusters, ++k) {
        const Unit w = unit_of_pair(a, u, 0);
        const uint32_t buf = k % a.nbuf, use = k / a.nbuf, half = w.Nt / 2;
        if (!wait_bounded(tempty0 + 8 * buf, (use & 1) ^ 1)) {  // both epilogues have drained this buffer
          atomicExch(a.err, 1u);
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t idesc = instr_desc(256, w.Nt), dcol = tmem + buf * a.buf_cols;
        for (uint32_t st = 0; st < nst; ++st, ++it) {
          const uint32_t slot = it % a.S, ph = (it / a.S) & 1;
          if (!wait_bounded(full0 + 8 * slot, ph) || (!TMA && !wait_bounded(pfull0 + 8 * slot, ph))) {
            atomicExch(a.err, 1u);
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t base = saddr(smem + slot * a.stage_bytes);
          for (uint32_t v = 0; v < a.KS16; ++v) {
            const uint64_t adesc = smem_desc(base + v * kBlockBytes);
            const uint64_t bdesc = smem_desc(base + db_stage + v * half * 32);
            mma_bf16_pair(dcol, adesc, bdesc, idesc, (st | v) != 0);
          }
          mma_commit_pair(empty0 + 8 * slot);  // both CTAs' stage is free once these MMAs have read it
        }
        mma_commit_pair(tfull0 + 8 * buf);  // this unit's accumulators are complete in both CTAs
      }
      // on every path: no MMA may still be running when the tensor memory is freed
      asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(done)
                   : "memory");
      if (!wait_bounded(done, 0)) atomicExch(a.err, 1u);
    }
    __syncwarp();
  } else {
    // ---------------- epilogue: warps 0..7 of each CTA, on its own accumulator rows ----------------
    const uint32_t quarter = warp & 3, b = lane & 3;
    const uint32_t row = 32 * quarter + lane;  // accumulator lane: column c_local = row / 4, DB digit b
    const bool hi2 = (b & 2) != 0, hi1 = (b & 1) != 0;
    uint32_t k = 0;
    for (uint32_t u = cluster; u < a.nunits; u += nclusters, ++k) {
      const Unit w = unit_of_pair(a, u, rank);
      const uint32_t buf = k % a.nbuf, use = k / a.nbuf;
      if (!__all_sync(0xffffffffu, wait_bounded(tfull0 + 8 * buf, use & 1))) {
        if (lane == 0) atomicExch(a.err, 1u);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t j = w.s >> a.logn;
      const uint32_t q = pick(mc.q, j);
      const uint64_t mu = pick(mc.mu, j);
      const int64_t off = (int64_t)q << 29;  // > 2^58 > |sum of the 16 weighted digit products|
      uint32_t pw[7];
      pw[0] = 1;
#pragma unroll
      for (int t = 1; t < 7; ++t) pw[t] = reduce64((uint64_t)pw[t - 1] << 8, q, mu);
      int32_t wgt[4];
#pragma unroll
      for (int d = 0; d < 4; ++d)
        wgt[d] = (int32_t)(b == 0 ? pw[d] : b == 1 ? pw[d + 1] : b == 2 ? pw[d + 2] : pw[d + 3]);
      const uint32_t G = w.Nt / 32;
      const uint32_t c = w.ct * 32 + (row >> 2);
      for (uint32_t g = warp >> 2; g < G; g += kEpiWarps / 4) {
        uint32_t f[32];
        tmem_ld32(tmem + buf * a.buf_cols + ((32 * quarter) << 16) + 32 * g, f);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          int64_t sum[4];
#pragma unroll
          for (int mm = 0; mm < 4; ++mm) {
            int64_t v = 0;
#pragma unroll
            for (int d = 0; d < 4; ++d)
              v = mad_wide(__float2int_rn(__uint_as_float(f[16 * h + 4 * mm + d])), wgt[d], v);
            sum[mm] = v;
          }
          int64_t k0 = hi2 ? sum[2] : sum[0], k1 = hi2 ? sum[3] : sum[1];
          const int64_t o0 = hi2 ? sum[0] : sum[2], o1 = hi2 ? sum[1] : sum[3];
          k0 += __shfl_xor_sync(0xffffffffu, o0, 2);
          k1 += __shfl_xor_sync(0xffffffffu, o1, 2);
          int64_t mine = hi1 ? k1 : k0;
          mine += __shfl_xor_sync(0xffffffffu, hi1 ? k0 : k1, 1);
          const uint32_t m = w.n0 / 4 + 8 * g + 4 * h + b;
          if (m < a.M) {
            uint32_t r = reduce64((uint64_t)(mine + off), q, mu);
            uint32_t *o = a.out + ((uint64_t)w.s * a.M + m) * a.D2 + c;
            if (a.acc_in) {
              r += *o;
              if (r >= q) r -= q;
            }
            *o = r;
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive_cluster(tempty0 + 8 * buf, 0);
    }
  }

  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  cluster_sync();  // the pair's MMAs are complete and both epilogues are done with the tensor memory
  if (warp == kMmaWarp) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols)
                 : "memory");
  }
}

// Two digits (|d| < 2^22) as a bf16 pair, exactly: 1.5 * 2^23 + d is exact in f32
// with unit spacing, so adding d to that constant's bit pattern and subtracting the
// constant gives (float)d; a digit of at most 8 significant bits leaves the low 16
// bits of the f32 zero, so its top half is the bf16 value.
__device__ __forceinline__ uint32_t bf16x2_of(int d0, int d1) {
  const float f0 = __int_as_float(0x4B400000 + d0) - 12582912.0f;
  const float f1 = __int_as_float(0x4B400000 + d1) - 12582912.0f;
  return __byte_perm(__float_as_uint(f0), __float_as_uint(f1), 0x7632);
}

// qhat chunk [B][Kc][2][L][n] -> qt[s][u][4*Mp rows][16] bf16 digits, row n = 4m + a.
// CTA = 32 slots of one prime x 16 ciphertexts (one u) x 8 query rows m; residues
// are staged in shared memory (coalesced reads along slots).  Then a thread takes
// (slot, row m, K half): the digits of its 8 residues, once, and the four 16-byte
// digit rows n = 4m..4m+3 (64 contiguous bytes; 16 threads = 1 KiB per slot).
__global__ void __launch_bounds__(256) k_query_to_tensor(const uint32_t *__restrict__ qhat, uint32_t M, uint32_t Mp,
                                                          uint32_t Kc, uint32_t L, uint32_t logn,
                                                          uint16_t *__restrict__ qt) {
  __shared__ uint32_t vals[16][8][33];
  const uint32_t n = 1u << logn;
  const uint32_t s0 = blockIdx.x * 32, u = blockIdx.y, mb = blockIdx.z;
  const uint32_t j = s0 >> logn, k0 = s0 & (n - 1);
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // all 16 loads of a thread in flight at once, then the shared-memory stores
  uint32_t v[16];
#pragma unroll
  for (uint32_t r = 0; r < 16; ++r) {
    const uint32_t p = warp + 8 * r, il = p >> 3, ml = p & 7, m = mb * 8 + ml, i = u * 16 + il;
    v[r] = m < M ? __ldg(qhat + ((uint64_t)((m >> 1) * Kc + i) * 2 + (m & 1)) * L * n + (uint64_t)j * n + k0 + lane)
                 : 0u;
  }
#pragma unroll
  for (uint32_t r = 0; r < 16; ++r) {
    const uint32_t p = warp + 8 * r;
    vals[p >> 3][p & 7][lane] = v[r];
  }
  __syncthreads();
  const uint32_t Ntot = 4 * Mp, Uc = Kc / 16;
  for (uint32_t w = threadIdx.x; w < 32 * 16; w += 256) {
    // w = slot * 16 + ((m / 2) * 4 + h * 2 + m % 2): 64-byte pieces in memory order
    const uint32_t sl = w >> 4, t = w & 15;
    const uint32_t ml = ((t >> 2) << 1) | (t & 1), h = (t >> 1) & 1;
    int d[8][4];
#pragma unroll
    for (int e = 0; e < 8; ++e) digits4(vals[8 * h + e][ml][sl], d[e]);
    const uint64_t s = s0 + sl;
    uint16_t *dst = qt + (s * Uc + u) * Ntot * 16 + cm_off(32 * mb + 4 * ml, 8 * h);
#pragma unroll
    for (int a = 0; a < 4; ++a)  // digit rows 4m + a: consecutive 16-byte rows of one core matrix
      *reinterpret_cast<uint4 *>(dst + 8 * a) =
          make_uint4(bf16x2_of(d[0][a], d[1][a]), bf16x2_of(d[2][a], d[3][a]), bf16x2_of(d[4][a], d[5][a]),
                     bf16x2_of(d[6][a], d[7][a]));
  }
}

// NTT-form DB polys [np][L][n] (row-major ids first + p = i*D2 + c) -> dbt digits.
__global__ void __launch_bounds__(256) k_db_scatter_tensor(const uint32_t *__restrict__ polys, uint64_t first,
                                                            uint64_t np, uint32_t D1, uint32_t D2, uint32_t L,
                                                            uint32_t logn, uint16_t *__restrict__ res) {
  __shared__ uint32_t tile[32][33];
  const uint32_t n = 1u << logn;
  const uint64_t p0 = (uint64_t)blockIdx.x * 32;
  const uint32_t s0 = blockIdx.y * 32;
  const uint32_t j = s0 >> logn, k0 = s0 & (n - 1);
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (uint32_t r = warp; r < 32; r += 8) {
    const uint64_t p = p0 + r;
    tile[r][lane] = p < np ? polys[(p * L + j) * n + k0 + lane] : 0u;
  }
  __syncthreads();
  const uint64_t R = 4ull * D2, U = D1 / 16;
  for (uint32_t kk = warp; kk < 32; kk += 8) {
    const uint64_t p = p0 + lane;
    if (p >= np) continue;
    const uint64_t P = first + p, i = P / D2, c = P % D2;
    int d[4];
    digits4(tile[lane][kk], d);
    const uint64_t blk = ((s0 + kk) * U + i / 16) * R * 16;
#pragma unroll
    for (uint32_t b = 0; b < 4; ++b) res[blk + cm_off((uint32_t)(4 * c + b), (uint32_t)(i % 16))] = bf16_bits(d[b]);
  }
}

__global__ void k_db_read_poly_tensor(const uint16_t *__restrict__ res, uint64_t poly, uint32_t D1, uint32_t D2,
                                      uint32_t nslots, uint32_t *__restrict__ out) {
  const uint64_t i = poly / D2, c = poly % D2, R = 4ull * D2, U = D1 / 16;
  for (uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; s < nslots; s += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t blk = (s * U + i / 16) * R * 16;
    int64_t v = 0;
    for (int b = 3; b >= 0; --b)
      v = v * 256 + (int64_t)__bfloat162float(__ushort_as_bfloat16(res[blk + cm_off((uint32_t)(4 * c + b),
                                                                                      (uint32_t)(i % 16))]));
    out[s] = (uint32_t)v;
  }
}

}  // namespace

bool gemm_tc_shape_ok(uint32_t D1, uint32_t D2) { return D1 % 64 == 0 && D2 % 32 == 0; }

// Tensor-layout GEMM forms: 0 = automatic (5 where it applies, else 1), 1 = one SM per unit
// (k_gemm_tc), 2 = CTA pairs (k_gemm_tc2; D2 a multiple of 64), 3 and 4 = the 1-SM
// form in clusters of 2 and 4 CTAs with the query digits multicast (D2 a multiple of
// 64 and 128), 5 = CTA pairs loading by tensor maps (D2 a multiple of 64, the padded
// query rows 4 Mp at most 256 or a multiple of 256).
uint32_t gemm_tc_tiles() { return 5; }
bool gemm_tc_tile_ok(uint32_t tile, uint32_t Mp, uint32_t D2) {
  const uint32_t Ntot = 4 * Mp;
  return tile <= 1 || ((tile == 2 || tile == 3) && D2 % 64 == 0) || (tile == 4 && D2 % 128 == 0) ||
         (tile == 5 && D2 % 64 == 0 && (Ntot <= 256 || Ntot % 256 == 0));
}

uint32_t tc_rows(uint32_t M) { return (M + 7u) & ~7u; }

cudaError_t launch_query_to_tensor(const ParamCtx &c, const uint32_t *qhat, uint32_t B, uint32_t Kc, uint32_t Mp,
                                   uint16_t *qt, cudaStream_t s) {
  if (Kc % 16 != 0 || Mp % 8 != 0) return cudaErrorInvalidValue;
  dim3 grid((c.p.L << c.logn) / 32, Kc / 16, Mp / 8);
  k_query_to_tensor<<<grid, 256, 0, s>>>(qhat, 2 * B, Mp, Kc, c.p.L, c.logn, qt);
  return cudaGetLastError();
}

cudaError_t launch_db_scatter_tensor(const ParamCtx &c, uint32_t D1, uint32_t D2, const uint32_t *polys,
                                     uint64_t first, uint64_t np, uint16_t *resident, cudaStream_t s) {
  if (np == 0) return cudaSuccess;
  dim3 grid((unsigned)((np + 31) / 32), (c.p.L << c.logn) / 32);
  k_db_scatter_tensor<<<grid, 256, 0, s>>>(polys, first, np, D1, D2, c.p.L, c.logn, resident);
  return cudaGetLastError();
}

cudaError_t launch_db_read_poly_tensor(const ParamCtx &c, uint32_t D1, uint32_t D2, const uint16_t *resident,
                                       uint64_t poly, uint32_t *out, cudaStream_t s) {
  const uint32_t nslots = c.p.L << c.logn;
  k_db_read_poly_tensor<<<(nslots + 255) / 256, 256, 0, s>>>(resident, poly, D1, D2, nslots, out);
  return cudaGetLastError();
}

// cuTensorMapEncodeTiled, reached through the runtime (no link to the driver library).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, []() {
    void *f = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    else
      cudaGetLastError();
  });
  return fn;
}

// A digit array [blocks][groups][128] (bf16 bits; a group = 8 rows x 16 K values, one
// core-matrix pair) as a 3-D tensor map with boxes of box_groups groups x box_blocks
// blocks.  False if the encoder refuses it (or is missing).
bool digit_tensor_map(CUtensorMap *map, const uint16_t *base, uint64_t groups, uint64_t blocks, uint32_t box_groups,
                      uint32_t box_blocks) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return false;
  const cuuint64_t dims[3] = {128, groups, blocks};
  const cuuint64_t strides[2] = {256, groups * 256};  // bytes, of dims 1 and 2
  const cuuint32_t box[3] = {128, box_groups, box_blocks};
  const cuuint32_t estride[3] = {1, 1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT16, 3, const_cast<uint16_t *>(base), dims, strides, box, estride,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// The 2-SM form (k_gemm_tc2): clusters of two CTAs, each unit 64 DB columns; tma
// selects the tensor-map form.
cudaError_t launch_gemm_tc_pair(const ParamCtx &c, const uint16_t *db, uint32_t D1, uint32_t D2, const uint16_t *qt,
                                uint32_t M, uint32_t Mp, uint32_t i0, uint32_t Kc, uint32_t *out, int acc, bool tma,
                                cudaStream_t s) {
  uint32_t *err = nullptr;
  cudaError_t e = device_error_word(&err);
  if (e != cudaSuccess) return e;
  TcArgs a = {};
  a.db = db;
  a.qt = qt;
  a.out = out;
  a.err = err;
  a.M = M;
  a.Mp = Mp;
  a.D1 = D1;
  a.D2 = D2;
  a.i0 = i0;
  a.Kc = Kc;
  const uint32_t Ntot = 4 * Mp, Nmax = Ntot < 256 ? Ntot : 256;
  a.mtiles = (Ntot + 255) / 256;
  a.T = 1;
  a.nbuf = 2;
  a.buf_cols = kTmemBudget;
  a.ctiles = D2 / 32;
  // per CTA and K16 step: its 128 DB digit rows and half of the query digit rows
  const uint32_t per16 = kBlockBytes + (Nmax / 2) * 32;
  uint32_t ks = 4;
  while (ks > 1 && (Kc / 16) % ks) ks /= 2;
  a.KS16 = ks;
  a.stage_bytes = ks * per16;
  uint32_t S = kSmemBudget2 / a.stage_bytes;
  if (S > (uint32_t)kMaxStages2) S = kMaxStages2;
  if (S < 2) return cudaErrorInvalidValue;
  a.S = S;
  a.logn = c.logn;
  a.acc_in = acc;
  const uint64_t nunits = (uint64_t)(c.p.L << c.logn) * (a.ctiles / 2) * a.mtiles;
  if (nunits > 0x7fffffffull) return cudaErrorInvalidValue;
  a.nunits = (uint32_t)nunits;
  // the tensor maps: the whole resident DB ([L n U][D2 / 2][128], boxes of this CTA's
  // 16 groups x KS16 blocks) and this K-chunk's query digits ([L n Uc][Mp / 2][128],
  // boxes of half a query tile); coordinates stay below 2^31
  alignas(64) CUtensorMap tm_db = {}, tm_q = {};
  const uint64_t nslots = (uint64_t)c.p.L << c.logn;
  if (tma) {
    if ((Ntot > 256 && Ntot % 256 != 0) || nslots * (D1 / 16) >= (1ull << 31)) return cudaErrorInvalidValue;
    if (!digit_tensor_map(&tm_db, db, D2 / 2, nslots * (D1 / 16), 16, ks) ||
        !digit_tensor_map(&tm_q, qt, Ntot / 8, nslots * (Kc / 16), Nmax / 16, ks))
      return cudaErrorInvalidValue;
  }
  // stages | full, empty, pfull (kMaxStages2 each), two tensor-memory full/empty pairs,
  // done | tensor-memory address | a spare run past the end
  size_t smem = (size_t)S * a.stage_bytes + (3 * kMaxStages2 + 5) * 8 + 16 + kSpareBytes2;
  if (smem < kSmemFloor) smem = kSmemFloor;
  auto kernel = tma ? k_gemm_tc2<true> : k_gemm_tc2<false>;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  // clusters that fit at once (the pairs land on SM pairs); every cluster loops over its units
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(sms & ~1), 1, 1);
  cfg.blockDim = dim3(kThreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  int nclusters = 0;
  if (cudaOccupancyMaxActiveClusters(&nclusters, kernel, &cfg) != cudaSuccess || nclusters <= 0) {
    cudaGetLastError();  // clear the query's error: fall back to one cluster per SM pair
    nclusters = sms / 2;
  }
  if ((uint64_t)nclusters > nunits) nclusters = (int)nunits;
  kernel<<<2 * (unsigned)nclusters, kThreads, smem, s>>>(a, c.mod, tm_db, tm_q);
  return cudaGetLastError();
}

// The cluster forms of k_gemm_tc: as many clusters of C CTAs as fit on the GPU at
// once (one CTA per SM), each looping over its unit groups.
template <int C>
cudaError_t launch_tc_clusters(const TcArgs &a, const ModConst &mod, size_t smem, int sms, cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(k_gemm_tc<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(sms / C * C), 1, 1);
  cfg.blockDim = dim3(kThreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int nclusters = 0;
  if (cudaOccupancyMaxActiveClusters(&nclusters, k_gemm_tc<C>, &cfg) != cudaSuccess || nclusters <= 0) {
    cudaGetLastError();  // clear the query's error: fall back to one cluster per C SMs
    nclusters = sms / C;
  }
  const uint32_t groups = a.nunits / C;
  if ((uint32_t)nclusters > groups) nclusters = (int)groups;
  cfg.gridDim = dim3((unsigned)(nclusters * C), 1, 1);
  return cudaLaunchKernelEx(&cfg, k_gemm_tc<C>, a, mod);
}

// out[s][m][c] (+)= sum_{i < Kc} Q[s][i][m] * DB[s][i0 + i][c] mod q_j for the
// query digits qt of one K-chunk (Mp = tc_rows(M) rows).
cudaError_t launch_gemm_tc(const ParamCtx &c, const uint16_t *db, uint32_t D1, uint32_t D2, const uint16_t *qt,
                           uint32_t M, uint32_t Mp, uint32_t i0, uint32_t Kc, uint32_t *out, int acc, uint32_t tile,
                           cudaStream_t s) {
  if (!gemm_tc_shape_ok(D1, D2) || Kc == 0 || Kc % 64 != 0 || Kc > 1024 || i0 % 64 != 0 || i0 + Kc > D1 ||
      Mp % 8 != 0 || Mp < M || !gemm_tc_tile_ok(tile, Mp, D2))
    return cudaErrorInvalidValue;
  // the built-in choice: the tensor-map CTA pair where the shape allows it (1.25x the
  // 1-SM form's GEMM at batch 32 on the 16 GiB DB), else the 1-SM form
  if (tile == 0 && gemm_tc_tile_ok(5, Mp, D2) && tensor_map_encoder() != nullptr) tile = 5;
  if (tile == 2 || tile == 5) return launch_gemm_tc_pair(c, db, D1, D2, qt, M, Mp, i0, Kc, out, acc, tile == 5, s);
  uint32_t *err = nullptr;
  cudaError_t e = device_error_word(&err);
  if (e != cudaSuccess) return e;
  TcArgs a = {};
  a.db = db;
  a.qt = qt;
  a.out = out;
  a.err = err;
  a.M = M;
  a.Mp = Mp;
  a.D1 = D1;
  a.D2 = D2;
  a.i0 = i0;
  a.Kc = Kc;
  const uint32_t Ntot = 4 * Mp, Nmax = Ntot < 256 ? Ntot : 256;
  a.mtiles = (Ntot + 255) / 256;
  // 32-column tiles per unit: as many as half of the tensor memory and D2 allow, so
  // that two accumulator buffers alternate
  const uint32_t C = tile == 3 ? 2 : tile == 4 ? 4 : 1;  // CTAs per cluster
  uint32_t T = 1;
  while (2 * T * Nmax <= kTmemBudget && (D2 / 32) % (2 * T * C) == 0) T *= 2;
  a.T = T;
  a.nbuf = 2;
  a.buf_cols = kTmemBudget;
  a.ctiles = D2 / (32 * T);
  // K16 steps per stage: as many as leave room for three stages
  const uint32_t per16 = T * kBlockBytes + Nmax * 32;
  uint32_t ks = 4;
  while (ks > 1 && (3 * ks * per16 > kSmemBudget || (Kc / 16) % ks)) ks /= 2;
  a.KS16 = ks;
  a.stage_bytes = ks * per16;
  uint32_t S = kSmemBudget / a.stage_bytes;
  if (S > (uint32_t)kMaxStages) S = kMaxStages;
  if (S < 2) return cudaErrorInvalidValue;
  a.S = S;
  a.logn = c.logn;
  a.acc_in = acc;
  const uint64_t nunits = (uint64_t)(c.p.L << c.logn) * a.ctiles * a.mtiles;
  if (nunits > 0x7fffffffull) return cudaErrorInvalidValue;
  a.nunits = (uint32_t)nunits;
  // stages | full, empty (kMaxStages each), two tensor-memory full/empty pairs, done |
  // tensor-memory address
  size_t smem = (size_t)S * a.stage_bytes + (2 * kMaxStages + 5) * 8 + 16;
  if (smem < kSmemFloor) smem = kSmemFloor;
  int dev = 0, sms = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if (C == 1) {
    e = cudaFuncSetAttribute(k_gemm_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const uint32_t grid = a.nunits < (uint32_t)sms ? a.nunits : (uint32_t)sms;
    k_gemm_tc<1><<<grid, kThreads, smem, s>>>(a, c.mod);
    return cudaGetLastError();
  }
  return C == 2 ? launch_tc_clusters<2>(a, c.mod, smem, sms, s) : launch_tc_clusters<4>(a, c.mod, smem, sms, s);
}

}  // namespace gbpir
