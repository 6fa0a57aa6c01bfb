// gemm_limb.cu -- the first-dimension modular GEMM on the INT8 tensor pipe
// (the paper's INT32-as-four-INT8 decomposition, Sec. 4.1, re-targeted to
// modular arithmetic: both operands are 30-bit residues).
//
// Every residue x = sum_{l<4} 2^(8l) x_l with bytes x_l (the top byte is below 64).
// For a slot s the product Q[m][i] * DB[i][c] splits into 16 byte products; the
// ones of equal shift class t = a + b (t = 0..6) share one s32 accumulator:
//   C_t[m][c] = sum_i sum_{a+b=t} Q_a[m][i] * DB_b[i][c]      (u8 x u8 -> s32 MMA)
// The largest class sums at most three 255*255 products and one 255*63 pair per i,
// so C_t < 2^31 for up to 8192 rows per K chunk (every chunk here is at most 8192).
// The epilogue recombines out = sum_t (C_t * (2^(8t) mod q)) mod q in u64 (seven
// terms below 2^61 each) and reduces once.
//
// Operands (byte planes written by the setup scatter and the query transpose):
//   A = query limbs  ql[s][a][Mp][Kc]  (row-major: m rows, i contiguous)
//   B = DB limbs     db[s][b][D2][D1]  ("col" operand: column c, i contiguous)
// Tensor op: mma.sync.aligned.m16n8k32.row.col.s32.u8.u8.s32 (warp level; this
// toolkit rejects tcgen05.mma kind::i8 for sm_103a).  Tiles are staged with
// cp.async into shared memory rows of 128 bytes, 16-byte chunks XOR-swizzled by
// row so that ldmatrix reads are free of bank conflicts.
#include "common.cuh"

namespace gbpir {
namespace {

constexpr int KS = 128;  // bytes of K per stage (four m16n8k32 steps)

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void cp16(uint32_t saddr, const void *g, bool ok) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(saddr), "l"(g), "r"(ok ? 16 : 0));
}

// Byte offset of 16-byte chunk `ch` (0..7) of row `r` in a [rows][128 B] tile.
__device__ __forceinline__ uint32_t swz(uint32_t r, uint32_t ch) { return r * KS + ((ch ^ (r & 7)) << 4); }

__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(addr));
}

__device__ __forceinline__ void mma_u8(int (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k32.row.col.s32.u8.u8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
      : "+r"(d[0]), "+r"(d[1]), "+r"(d[2]), "+r"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// CTA = 4 warps laid out WM x (4 / WM); warp tile 16 rows x 32 columns (four n8 tiles).
template <int WM>
__global__ void __launch_bounds__(128) k_gemm_limb(const uint8_t *__restrict__ db, const uint8_t *__restrict__ ql,
                                                   uint32_t M, uint32_t Mp, uint32_t D1, uint32_t D2, uint32_t i0,
                                                   uint32_t Kc, uint32_t *__restrict__ out, ModConst mc,
                                                   uint32_t logn, int acc_in) {
  constexpr int WN = 4 / WM;
  constexpr int TM = 16 * WM, TN = 32 * WN;
  constexpr int A_BYTES = 4 * TM * KS, B_BYTES = 4 * TN * KS, STAGE = A_BYTES + B_BYTES;
  extern __shared__ __align__(128) uint8_t smem[];

  const uint32_t nct = (D2 + TN - 1) / TN, nmt = Mp / TM;
  const uint64_t bid = blockIdx.x;
  const uint32_t ct = (uint32_t)(bid % nct);
  const uint32_t mt = (uint32_t)((bid / nct) % nmt);
  const uint32_t s = (uint32_t)(bid / ((uint64_t)nct * nmt));
  const uint32_t j = s >> logn;
  const uint32_t m0 = mt * TM, c0 = ct * TN;
  const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t wm = warp % WM, wn = warp / WM;

  const uint8_t *qa = ql + (uint64_t)s * 4 * Mp * Kc;      // [4][Mp][Kc]
  const uint8_t *dbb = db + (uint64_t)s * 4 * D2 * D1 + i0;  // [4][D2][D1], columns from row i0

  auto load_stage = [&](int buf, uint32_t k0) {
    const uint32_t sbase = smem_u32(smem + buf * STAGE);
    // A: 4 limbs x TM rows x 8 chunks
    for (uint32_t t = tid; t < 4 * TM * 8; t += 128) {
      const uint32_t ch = t & 7, r = (t >> 3) % TM, limb = (t >> 3) / TM;
      const bool ok = k0 + ch * 16 < Kc;
      const uint8_t *g = qa + ((uint64_t)limb * Mp + m0 + r) * Kc + k0 + ch * 16;
      cp16(sbase + limb * TM * KS + swz(r, ch), ok ? g : qa, ok);
    }
    // B: 4 limbs x TN columns x 8 chunks
    for (uint32_t t = tid; t < 4 * TN * 8; t += 128) {
      const uint32_t ch = t & 7, r = (t >> 3) % TN, limb = (t >> 3) / TN;
      const bool ok = (k0 + ch * 16 < Kc) && (c0 + r < D2);
      const uint8_t *g = dbb + ((uint64_t)limb * D2 + c0 + r) * D1 + k0 + ch * 16;
      cp16(sbase + A_BYTES + limb * TN * KS + swz(r, ch), ok ? g : dbb, ok);
    }
    asm volatile("cp.async.commit_group;\n" ::);
  };

  int acc[7][4][4];  // [shift class][n8 tile][fragment]
#pragma unroll
  for (int t = 0; t < 7; ++t)
#pragma unroll
    for (int nt = 0; nt < 4; ++nt)
#pragma unroll
      for (int f = 0; f < 4; ++f) acc[t][nt][f] = 0;

  const uint32_t nk = (Kc + KS - 1) / KS;
  load_stage(0, 0);
  for (uint32_t kt = 0; kt < nk; ++kt) {
    const int buf = kt & 1;
    asm volatile("cp.async.wait_group 0;\n" ::);
    __syncthreads();
    if (kt + 1 < nk) load_stage(buf ^ 1, (kt + 1) * KS);
    const uint32_t sA = smem_u32(smem + buf * STAGE), sB = sA + A_BYTES;
#pragma unroll
    for (int kk = 0; kk < KS / 32; ++kk) {
      // A fragments, 4 limbs: rows wm*16 + (lane & 15), chunk 2*kk + (lane >> 4)
      uint32_t a[4][4];
      const uint32_t ar = wm * 16 + (lane & 15), ach = 2 * kk + (lane >> 4);
#pragma unroll
      for (int l = 0; l < 4; ++l) ldsm_x4(sA + l * TM * KS + swz(ar, ach), a[l][0], a[l][1], a[l][2], a[l][3]);
      // B fragments, 4 limbs x 4 n8 tiles: one x4 covers two n8 tiles of one limb
      uint32_t b[4][4][2];
#pragma unroll
      for (int l = 0; l < 4; ++l)
#pragma unroll
        for (int np = 0; np < 2; ++np) {
          // matrices: (tile 2np, chunk lo), (tile 2np, chunk hi), (tile 2np+1, lo), (tile 2np+1, hi)
          const uint32_t mat = lane >> 3;
          const uint32_t br = wn * 32 + (2 * np + (mat >> 1)) * 8 + (lane & 7);
          const uint32_t bch = 2 * kk + (mat & 1);
          ldsm_x4(sB + l * TN * KS + swz(br, bch), b[l][2 * np][0], b[l][2 * np][1], b[l][2 * np + 1][0],
                  b[l][2 * np + 1][1]);
        }
#pragma unroll
      for (int la = 0; la < 4; ++la)
#pragma unroll
        for (int lb = 0; lb < 4; ++lb)
#pragma unroll
          for (int nt = 0; nt < 4; ++nt) mma_u8(acc[la + lb][nt], a[la], b[lb][nt][0], b[lb][nt][1]);
    }
  }

  // epilogue: recombine the seven classes mod q_j
  const uint32_t q = mc.q[j];
  const uint64_t mu = mc.mu[j];
  uint32_t w[7];
  w[0] = 1 % q;
#pragma unroll
  for (int t = 1; t < 7; ++t) w[t] = (uint32_t)(((uint64_t)w[t - 1] << 8) % q);
  const uint32_t g = lane >> 2, tg = lane & 3;
#pragma unroll
  for (int nt = 0; nt < 4; ++nt) {
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      const uint32_t m = m0 + wm * 16 + g + 8 * half;
      const uint32_t c = c0 + wn * 32 + nt * 8 + 2 * tg;
      if (m >= M || c >= D2) continue;  // D2 % 4 == 0, so c + 1 < D2 too
      uint32_t r[2];
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        uint64_t v = 0;
#pragma unroll
        for (int t = 0; t < 7; ++t) v += (uint64_t)(uint32_t)acc[t][nt][2 * half + e] * w[t];
        r[e] = reduce64(v, q, mu);
      }
      uint2 *o = reinterpret_cast<uint2 *>(out + ((uint64_t)s * M + m) * D2 + c);
      if (acc_in) {
        const uint2 prev = *o;
        r[0] = reduce64((uint64_t)r[0] + prev.x, q, mu);
        r[1] = reduce64((uint64_t)r[1] + prev.y, q, mu);
      }
      *o = make_uint2(r[0], r[1]);
    }
  }
}

template <int WM>
cudaError_t limb_launch(const ParamCtx &c, const uint8_t *db, uint32_t D1, uint32_t D2, const uint8_t *ql,
                        uint32_t M, uint32_t Mp, uint32_t i0, uint32_t Kc, uint32_t *out, int acc, cudaStream_t s) {
  constexpr int TM = 16 * WM, TN = 32 * (4 / WM);
  constexpr int smem = 2 * (4 * TM * KS + 4 * TN * KS);
  // per device and cheap: set on every launch so every device the library runs on has it
  cudaError_t e = cudaFuncSetAttribute(k_gemm_limb<WM>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  if (Mp % TM != 0) return cudaErrorInvalidValue;
  const uint64_t nslots = (uint64_t)c.p.L << c.logn;
  const uint64_t blocks = nslots * ((D2 + TN - 1) / TN) * (Mp / TM);
  if (blocks > 0x7FFFFFFFull) return cudaErrorInvalidConfiguration;
  k_gemm_limb<WM><<<(unsigned)blocks, 128, smem, s>>>(db, ql, M, Mp, D1, D2, i0, Kc, out, c.mod, c.logn, acc);
  return cudaGetLastError();
}

}  // namespace

// Tile ids: 1 = 16 x 128 (warps along columns), 2 = 32 x 64, 3 = 64 x 32 (warps along rows).
// 0 picks by the padded row count Mp (a multiple of 16).
uint32_t gemm_limb_tiles() { return 3; }

bool gemm_limb_tile_ok(uint32_t tile, uint32_t Mp) {
  switch (tile) {
    case 0: return true;
    case 1: return Mp % 16 == 0;
    case 2: return Mp % 32 == 0;
    case 3: return Mp % 64 == 0;
  }
  return false;
}

cudaError_t launch_gemm_limb(const ParamCtx &c, const uint8_t *db, uint32_t D1, uint32_t D2, const uint8_t *ql,
                             uint32_t M, uint32_t Mp, uint32_t i0, uint32_t Kc, uint32_t *out, int acc,
                             uint32_t tile, cudaStream_t s) {
  if (Kc > 8192 || (Kc % 32) != 0 || (Mp % 16) != 0) return cudaErrorInvalidValue;
  if (tile == 0) tile = (Mp % 64 == 0) ? 3 : (Mp % 32 == 0) ? 2 : 1;
  switch (tile) {
    case 1: return limb_launch<1>(c, db, D1, D2, ql, M, Mp, i0, Kc, out, acc, s);
    case 2: return limb_launch<2>(c, db, D1, D2, ql, M, Mp, i0, Kc, out, acc, s);
    case 3: return limb_launch<4>(c, db, D1, D2, ql, M, Mp, i0, Kc, out, acc, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace gbpir
