// ntt.cu -- forward / inverse negacyclic NTT over 30-bit primes (Sec. 2.3; the
// paper's single-kernel, on-chip NTT, Sec. 4.3).
//
// One CTA transforms one polynomial row of n residues (row r uses prime r % L).
// Each thread holds 16 residues in registers and applies four butterfly stages
// to them; the rows pass through shared memory (padded one word in sixteen) between
// such radix-16 passes: n = 2^11 -> 4+4+3 bits, 2^12 -> 4+4+4, 2^13 -> 4+4+4+1.
//
// Arithmetic: twiddles are psi^brv(i) (forward) and psi^-brv(i) (inverse) with
// Shoup companions floor(w * 2^32 / q), so each twiddle product is one high and
// two low 32-bit multiplies.  Butterflies keep values lazily reduced (Harvey):
// forward values live in [0, 4q), inverse values in [0, 2q); 4q < 2^32 because
// q < 2^30.  The last pass reduces to canonical [0, q) (and, for the inverse,
// multiplies by n^-1).
//
// Output order: forward NTT(a)[k] = sum_t a_t psi^((2 brv(k) + 1) t), the natural
// result of decimation in time with psi powers in bit-reversed order.
#include "common.cuh"

namespace gbpir {
namespace {

__device__ __forceinline__ uint32_t padx(uint32_t i) { return i + (i >> 4); }

// Padded shared index of element e of a unit whose base index has bits
// [BLO, BLO + RB) clear: when BLO >= 4, or BLO == 0 (a base aligned to 2^RB, RB <= 4),
// the padding of base + e 2^BLO is that of base plus a constant, so the address is
// the unit's padded base plus a compile-time offset.
template <int BLO>
__device__ __forceinline__ uint32_t pidx(uint32_t pbase, uint32_t base, int e) {
  if constexpr (BLO >= 4)
    return pbase + (uint32_t)e * ((1u << BLO) + (1u << (BLO - 4)));
  else if constexpr (BLO == 0)
    return pbase + (uint32_t)e;
  else
    return padx(base + ((uint32_t)e << BLO));
}

// x - m if x >= m, else x (x < 2m <= 2^32): as unsigned values x - m wraps above x
// exactly when x < m, so the minimum picks the right one in two integer operations.
__device__ __forceinline__ uint32_t csub(uint32_t x, uint32_t m) { return min(x, x - m); }

// Element j < L of a per-prime parameter array, by compare and select: indexing a
// kernel parameter array with a run-time j makes the compiler copy the whole
// parameter block to local memory first.
template <typename T>
__device__ __forceinline__ T pick(const T (&a)[PIR_MAX_L], uint32_t j) {
  T r = a[0];
#pragma unroll
  for (uint32_t i = 1; i < PIR_MAX_L; ++i) r = j == i ? a[i] : r;
  return r;
}

// Source kinds of the first pass.
enum { SRC_SMEM = 0, SRC_U32 = 1, SRC_RAW = 2 };

// Destinations of a pass: shared memory (not the last pass), global memory
// (canonical), a second shared buffer (canonical; the first row of a pair), or the
// slot-major query layout as (first row, this row) pairs.
enum { DST_SMEM = 0, DST_GLOBAL = 1, DST_PAIR = 2 };

// (DST_PAIR parks a row's canonical results in its shared buffer; the pair kernel
// then writes element k of rows (i, comp 0) and (i, comp 1) of prime j to
// slots[((j*n + k) * Kc + i) * 2 + comp], the plain slot layout with Mp = 2.)
struct SlotDst {};

struct RawSrc {
  const uint8_t *raw;  // little-endian bit stream of log2p-bit coefficients
  uint64_t poly0;      // row-major order: local polynomial p is poly0 + p
  uint32_t log2p;
  uint32_t col_major;  // 1: local polynomial p is (i, c) = (p % D1, c0 + p / D1)
  uint32_t D1, D2;
  uint64_t c0;
  __device__ __forceinline__ uint64_t poly(uint64_t p) const {
    return col_major ? (p % D1) * D2 + (c0 + p / D1) : poly0 + p;
  }
};

// Source rows of a launch: local row r reads row off + (r / G) * S + r % G, so a
// chunk of ciphertexts can be taken out of every query of a batch without a copy.
struct RowMap {  // local row r reads source row off + (r / G) * S + (r % G) * T
  uint64_t off, G, S, T;
  __device__ __forceinline__ uint64_t operator()(uint64_t r) const { return off + (r / G) * S + (r % G) * T; }
};

// Coefficient `t` of plaintext polynomial `poly` from the raw bit stream.
__device__ __forceinline__ uint32_t raw_coeff(const RawSrc &rs, uint64_t poly, uint32_t t, uint32_t logn) {
  const uint64_t bit0 = ((poly << logn) + t) * rs.log2p;
  const uint64_t byte0 = bit0 >> 3;
  const uint32_t nbytes = (uint32_t)(((bit0 & 7) + rs.log2p + 7) >> 3);
  uint64_t w = 0;
  for (uint32_t b = 0; b < nbytes; ++b) w |= (uint64_t)__ldg(rs.raw + byte0 + b) << (8 * b);
  return (uint32_t)((w >> (bit0 & 7)) & ((1ull << rs.log2p) - 1));
}

// Twiddle pairs {w, Shoup companion} used by one stage of one radix-2^RB unit.
// Stage bit b pairs (x, x + 2^b); the pair belongs to block g = index >> (b+1) and
// uses twiddle m + g, m = n >> (b+1).  Within a unit the blocks of stage LB are the
// 2^(RB-1-LB) consecutive entries from m + (hi << (RB-1-LB)), a run aligned to its
// own length, so they arrive in 16-byte loads (8 bytes for a single pair).
template <int CNT>
struct Pairs {  // CNT twiddle pairs held as whole 16-byte vectors (8 bytes when CNT = 1)
  uint4 v[(CNT + 1) / 2];
  __device__ __forceinline__ void load(const uint2 *__restrict__ src) {
    if constexpr (CNT == 1) {
      const uint2 x = __ldg(src);
      v[0] = make_uint4(x.x, x.y, 0u, 0u);
    } else {
#pragma unroll
      for (int i = 0; i < CNT / 2; ++i) v[i] = __ldg(reinterpret_cast<const uint4 *>(src) + i);
    }
  }
  // CNT pairs as CNT/2 16-byte loads spaced `stride` 16-byte words apart (the
  // lane-major copy: load i of every thread is one contiguous run)
  __device__ __forceinline__ void load_lane_major(const uint4 *__restrict__ src, uint32_t stride) {
#pragma unroll
    for (int i = 0; i < CNT / 2; ++i) v[i] = __ldg(src + (size_t)i * stride);
  }
  template <int I>
  __device__ __forceinline__ uint32_t w() const { return (I & 1) ? v[I / 2].z : v[I / 2].x; }
  template <int I>
  __device__ __forceinline__ uint32_t ws() const { return (I & 1) ? v[I / 2].w : v[I / 2].y; }
};

// One forward (Cooley-Tukey) butterfly of stage LB on elements E and E + 2^LB.
template <int RB, int LB, int E, int CNT>
__device__ __forceinline__ void fwd_bfly(uint32_t (&v)[1 << RB], const Pairs<CNT> &p, uint32_t q) {
  if constexpr (E < (1 << RB)) {
    if constexpr ((E & (1 << LB)) == 0) {
      const uint32_t q2 = 2 * q;
      uint32_t x = v[E];
      const uint32_t y = v[E | (1 << LB)];
      x = csub(x, q2);                                                              // [0, 2q)
      const uint32_t t = shoup_mul(y, p.template w<(E >> (LB + 1))>(), p.template ws<(E >> (LB + 1))>(), q);  // [0, 2q)
      v[E] = x + t;                                                                 // [0, 4q)
      v[E | (1 << LB)] = x - t + q2;                                                // (0, 4q)
    }
    fwd_bfly<RB, LB, E + 1, CNT>(v, p, q);
  }
}

// One forward stage on the unit's bit BLO + LB.
template <int RB, int BLO, int LOGN, int LB>
__device__ __forceinline__ void fwd_stage(uint32_t (&v)[1 << RB], uint32_t hi, const uint2 *__restrict__ tw,
                                          uint32_t q) {
  constexpr int CNT = 1 << (RB - 1 - LB);
  constexpr uint32_t m = 1u << (LOGN - 1 - (BLO + LB));
  Pairs<CNT> p;
  if constexpr (BLO == 0 && RB == 4 && LB <= 1) {  // the lane-major copy after the table
    constexpr uint32_t units = 1u << (LOGN - 4);
    p.load_lane_major(reinterpret_cast<const uint4 *>(tw + (1u << LOGN)) + (LB == 0 ? 0u : 4 * units) + hi, units);
  } else {
    p.load(tw + m + (hi << (RB - 1 - LB)));
  }
  fwd_bfly<RB, LB, 0, CNT>(v, p, q);
}

// Forward stages on one unit: bits BLO+RB-1 down to BLO of the element index.
template <int RB, int BLO, int LOGN, int LB = RB - 1>
__device__ __forceinline__ void fwd_stages(uint32_t (&v)[1 << RB], uint32_t hi, const uint2 *__restrict__ tw,
                                           uint32_t q) {
  fwd_stage<RB, BLO, LOGN, LB>(v, hi, tw, q);
  if constexpr (LB > 0) fwd_stages<RB, BLO, LOGN, LB - 1>(v, hi, tw, q);
}

// One inverse (Gentleman-Sande) butterfly of stage LB; values in [0, 2q).
template <int RB, int LB, int E, int CNT>
__device__ __forceinline__ void inv_bfly(uint32_t (&v)[1 << RB], const Pairs<CNT> &p, uint32_t q) {
  if constexpr (E < (1 << RB)) {
    if constexpr ((E & (1 << LB)) == 0) {
      const uint32_t q2 = 2 * q;
      const uint32_t x = v[E], y = v[E | (1 << LB)];
      uint32_t s = x + y;
      s = csub(s, q2);
      v[E] = s;
      v[E | (1 << LB)] = shoup_mul(x - y + q2, p.template w<(E >> (LB + 1))>(), p.template ws<(E >> (LB + 1))>(), q);
    }
    inv_bfly<RB, LB, E + 1, CNT>(v, p, q);
  }
}

// One inverse stage on bit BLO + LB.
template <int RB, int BLO, int LOGN, int LB>
__device__ __forceinline__ void inv_stage(uint32_t (&v)[1 << RB], uint32_t hi, const uint2 *__restrict__ tw,
                                          uint32_t q) {
  constexpr int CNT = 1 << (RB - 1 - LB);
  constexpr uint32_t m = 1u << (LOGN - 1 - (BLO + LB));
  Pairs<CNT> p;
  if constexpr (BLO == 0 && RB == 4 && LB <= 1) {  // the lane-major copy after the table
    constexpr uint32_t units = 1u << (LOGN - 4);
    p.load_lane_major(reinterpret_cast<const uint4 *>(tw + (1u << LOGN)) + (LB == 0 ? 0u : 4 * units) + hi, units);
  } else {
    p.load(tw + m + (hi << (RB - 1 - LB)));
  }
  inv_bfly<RB, LB, 0, CNT>(v, p, q);
}

// Inverse stages on one unit: bits BLO up to BLO+RB-1.
template <int RB, int BLO, int LOGN, int LB = 0>
__device__ __forceinline__ void inv_stages(uint32_t (&v)[1 << RB], uint32_t hi, const uint2 *__restrict__ tw,
                                           uint32_t q) {
  inv_stage<RB, BLO, LOGN, LB>(v, hi, tw, q);
  if constexpr (LB < RB - 1) inv_stages<RB, BLO, LOGN, LB + 1>(v, hi, tw, q);
}

// One radix-2^RB pass over the whole row: unit u holds the 2^RB elements whose
// index has bits [BLO, BLO+RB) free and the rest fixed by u.
template <int LOGN, int RB, int BLO, bool FWD, int SRC, int DST>
__device__ __forceinline__ void ntt_pass(uint32_t *sm, const uint32_t *__restrict__ gin, const RawSrc &rs,
                                         uint64_t poly, uint32_t *__restrict__ gout, const uint2 *__restrict__ tw,
                                         uint32_t q, uint32_t ninv,
                                         uint32_t ninv_sh, const SlotDst *sd = nullptr,
                                         uint32_t tid = threadIdx.x) {
  constexpr int N = 1 << LOGN, T = N / 16, UNITS = N >> RB, PER = UNITS / T;
  static_assert(UNITS % T == 0, "pass plan");
#pragma unroll
  for (int r = 0; r < PER; ++r) {
    const uint32_t u = tid + r * T;
    const uint32_t lo = u & ((1u << BLO) - 1), hi = u >> BLO;
    const uint32_t base = (hi << (BLO + RB)) | lo;
    const uint32_t pbase = padx(base);
    uint32_t v[1 << RB];
    if constexpr (SRC == SRC_U32 && BLO == 0 && RB >= 2) {
#pragma unroll
      for (int e = 0; e < (1 << RB); e += 4) {
        const uint4 x = __ldg(reinterpret_cast<const uint4 *>(gin + base + e));
        v[e] = x.x, v[e + 1] = x.y, v[e + 2] = x.z, v[e + 3] = x.w;
      }
    } else {
#pragma unroll
      for (int e = 0; e < (1 << RB); ++e) {
        const uint32_t idx = base + ((uint32_t)e << BLO);
        if constexpr (SRC == SRC_SMEM)
          v[e] = sm[pidx<BLO>(pbase, base, e)];
        else if constexpr (SRC == SRC_U32)
          v[e] = __ldg(gin + idx);
        else
          v[e] = raw_coeff(rs, poly, idx, LOGN);
      }
    }
    if constexpr (FWD)
      fwd_stages<RB, BLO, LOGN>(v, hi, tw, q);
    else
      inv_stages<RB, BLO, LOGN>(v, hi, tw, q);
    if constexpr (DST != DST_SMEM) {
#pragma unroll
      for (int e = 0; e < (1 << RB); ++e) {
        uint32_t x = v[e];
        if constexpr (FWD) {
          x = csub(x, 2 * q);
          x = csub(x, q);
        } else {
          x = shoup_mul(x, ninv, ninv_sh, q);
          x = csub(x, q);
        }
        v[e] = x;
      }
      if constexpr (DST == DST_PAIR) {
#pragma unroll
        for (int e = 0; e < (1 << RB); ++e) sm[pidx<BLO>(pbase, base, e)] = v[e];
      } else if constexpr (BLO == 0 && RB >= 2) {
#pragma unroll
        for (int e = 0; e < (1 << RB); e += 4)
          *reinterpret_cast<uint4 *>(gout + base + e) = make_uint4(v[e], v[e + 1], v[e + 2], v[e + 3]);
      } else if constexpr (BLO == 0 && RB == 1) {
        *reinterpret_cast<uint2 *>(gout + base) = make_uint2(v[0], v[1]);
      } else {
#pragma unroll
        for (int e = 0; e < (1 << RB); ++e) gout[base + ((uint32_t)e << BLO)] = v[e];
      }
    } else {
#pragma unroll
      for (int e = 0; e < (1 << RB); ++e) sm[pidx<BLO>(pbase, base, e)] = v[e];
    }
  }
}

template <int LOGN, int SRC>
__global__ void __launch_bounds__((1 << LOGN) / 16, 20480 >> LOGN)  // >= 1280 threads per SM (measured fastest)
    k_ntt_fwd(const uint32_t *__restrict__ src, RowMap rm, RawSrc rs, uint32_t *__restrict__ dst, NttConst C,
              uint32_t L, uint64_t rows) {
  constexpr int N = 1 << LOGN;
  extern __shared__ uint32_t sm[];
  for (uint64_t row = blockIdx.x; row < rows; row += gridDim.x) {
    const uint32_t j = (uint32_t)(row % L);
    const uint32_t q = pick(C.q, j);
    const uint2 *tw = pick(C.fwd, j);
    const uint32_t *gin = src ? src + rm(row) * N : nullptr;
    uint32_t *gout = dst + row * N;
    const uint64_t poly = SRC == SRC_RAW ? rs.poly(row / L) : 0;
    if constexpr (LOGN == 11) {
      ntt_pass<11, 4, 7, true, SRC, DST_SMEM>(sm, gin, rs, poly, gout, tw, q, 0, 0);
      __syncthreads();
      ntt_pass<11, 4, 3, true, SRC_SMEM, DST_SMEM>(sm, gin, rs, poly, gout, tw, q, 0, 0);
      __syncthreads();
      ntt_pass<11, 3, 0, true, SRC_SMEM, DST_GLOBAL>(sm, gin, rs, poly, gout, tw, q, 0, 0);
    } else if constexpr (LOGN == 12) {
      ntt_pass<12, 4, 8, true, SRC, DST_SMEM>(sm, gin, rs, poly, gout, tw, q, 0, 0);
      __syncthreads();
      ntt_pass<12, 4, 4, true, SRC_SMEM, DST_SMEM>(sm, gin, rs, poly, gout, tw, q, 0, 0);
      __syncthreads();
      ntt_pass<12, 4, 0, true, SRC_SMEM, DST_GLOBAL>(sm, gin, rs, poly, gout, tw, q, 0, 0);
    } else {
      ntt_pass<13, 4, 9, true, SRC, DST_SMEM>(sm, gin, rs, poly, gout, tw, q, 0, 0);
      __syncthreads();
      ntt_pass<13, 4, 5, true, SRC_SMEM, DST_SMEM>(sm, gin, rs, poly, gout, tw, q, 0, 0);
      __syncthreads();
      ntt_pass<13, 4, 1, true, SRC_SMEM, DST_SMEM>(sm, gin, rs, poly, gout, tw, q, 0, 0);
      __syncthreads();
      ntt_pass<13, 1, 0, true, SRC_SMEM, DST_GLOBAL>(sm, gin, rs, poly, gout, tw, q, 0, 0);
    }
    __syncthreads();  // the next row reuses shared memory
  }
}

template <int LOGN>
__global__ void __launch_bounds__((1 << LOGN) / 16, 20480 >> LOGN)  // >= 1280 threads per SM (measured fastest)
    k_ntt_inv(const uint32_t *__restrict__ src, RowMap rm, uint32_t *__restrict__ dst, NttConst C, uint32_t L,
              uint64_t rows) {
  constexpr int N = 1 << LOGN;
  extern __shared__ uint32_t sm[];
  const RawSrc rs = {};
  for (uint64_t row = blockIdx.x; row < rows; row += gridDim.x) {
    const uint32_t j = (uint32_t)(row % L);
    const uint32_t q = pick(C.q, j), ni = pick(C.ninv, j), nis = pick(C.ninv_sh, j);
    const uint2 *tw = pick(C.inv, j);
    const uint32_t *gin = src + rm(row) * N;
    uint32_t *gout = dst + row * N;
    if constexpr (LOGN == 11) {
      ntt_pass<11, 4, 0, false, SRC_U32, DST_SMEM>(sm, gin, rs, 0, gout, tw, q, ni, nis);
      __syncthreads();
      ntt_pass<11, 4, 4, false, SRC_SMEM, DST_SMEM>(sm, gin, rs, 0, gout, tw, q, ni, nis);
      __syncthreads();
      ntt_pass<11, 3, 8, false, SRC_SMEM, DST_GLOBAL>(sm, gin, rs, 0, gout, tw, q, ni, nis);
    } else if constexpr (LOGN == 12) {
      ntt_pass<12, 4, 0, false, SRC_U32, DST_SMEM>(sm, gin, rs, 0, gout, tw, q, ni, nis);
      __syncthreads();
      ntt_pass<12, 4, 4, false, SRC_SMEM, DST_SMEM>(sm, gin, rs, 0, gout, tw, q, ni, nis);
      __syncthreads();
      ntt_pass<12, 4, 8, false, SRC_SMEM, DST_GLOBAL>(sm, gin, rs, 0, gout, tw, q, ni, nis);
    } else {
      ntt_pass<13, 4, 0, false, SRC_U32, DST_SMEM>(sm, gin, rs, 0, gout, tw, q, ni, nis);
      __syncthreads();
      ntt_pass<13, 4, 4, false, SRC_SMEM, DST_SMEM>(sm, gin, rs, 0, gout, tw, q, ni, nis);
      __syncthreads();
      ntt_pass<13, 4, 8, false, SRC_SMEM, DST_SMEM>(sm, gin, rs, 0, gout, tw, q, ni, nis);
      __syncthreads();
      ntt_pass<13, 1, 12, false, SRC_SMEM, DST_GLOBAL>(sm, gin, rs, 0, gout, tw, q, ni, nis);
    }
    __syncthreads();
  }
}

// One coefficient switched to q_0 from its L canonical residues in shared memory
// (row j at sm + j * padn, position pt): Garner digits a_k of x mod Q', that value
// mod q_0 and its comparison with (Q' - 1) / 2 (digit by digit from the top), then
// y = (x_0 - (x mod Q')) Q'^-1 + [x mod Q' > (Q' - 1) / 2]  (mod q_0),
// which is round(x / Q') mod q_0: x = Q' floor(x / Q') + (x mod Q').  Every residue
// is below 2^30 < 2 q_k, so one conditional subtraction brings it under any q_k.
__device__ __forceinline__ uint32_t switch_coeff(const uint32_t *sm, uint32_t padn, uint32_t pt, const NttConst &C,
                                                 const SwitchConst &W, uint32_t L) {
  const uint32_t q0 = C.q[0];
  uint32_t a[PIR_MAX_L];
  uint32_t xm = 0;
#pragma unroll
  for (int k = 1; k < PIR_MAX_L; ++k) {
    a[k] = 0;
    if ((uint32_t)k < L) {
      const uint32_t qk = C.q[k];
      uint32_t t = sm[k * padn + pt];
#pragma unroll
      for (int i = 1; i < k; ++i) {
        const uint32_t ai = a[i] >= qk ? a[i] - qk : a[i];
        t = shoup_mul(t + qk - ai, W.c[k][i], W.c_sh[k][i], qk);
        t = t >= qk ? t - qk : t;
      }
      a[k] = t;
      const uint32_t ak = t >= q0 ? t - q0 : t;
      uint32_t pr = shoup_mul(ak, W.w[k], W.w_sh[k], q0);
      pr = pr >= q0 ? pr - q0 : pr;
      xm += pr;
      xm = xm >= q0 ? xm - q0 : xm;
    }
  }
  bool up = false, eq = true;
#pragma unroll
  for (int k = PIR_MAX_L - 1; k >= 1; --k)
    if ((uint32_t)k < L && eq && a[k] != W.h[k]) {
      up = a[k] > W.h[k];
      eq = false;
    }
  uint32_t y = shoup_mul(sm[pt] + q0 - xm, W.qinv, W.qinv_sh, q0);
  y = y >= q0 ? y - q0 : y;
  y += up ? 1u : 0u;
  return y >= q0 ? y - q0 : y;
}

// Inverse NTT with modulus switching fused into its epilogue (Sec. 4.3 fuses the
// modulus reduction into the inverse NTT; App. D.5 defines the switch): block c
// takes the L residue rows src + (c L + j) n of one polynomial (NTT form) and
// writes dst + c n, its coefficients over the single prime q_0.  2 x n/16 threads:
// half h inverts rows h, h + 2, ... into their own shared buffers (canonical), then
// all threads switch the coefficients, four per 16-byte store.
template <int LOGN>
__global__ void __launch_bounds__((1 << LOGN) / 8, 8192 >> LOGN)  // <= 64 registers: 1024 threads per SM
    k_ntt_inv_switch(const uint32_t *__restrict__ src, uint32_t *__restrict__ dst, NttConst C, SwitchConst W,
                     uint32_t L) {
  constexpr int N = 1 << LOGN, PADN = N + N / 16, T = N / 16;
  extern __shared__ uint32_t sm[];
  const uint32_t half = threadIdx.x / T, tid = threadIdx.x % T;
  const RawSrc rs = {};
  uint32_t *gout = nullptr;
  for (uint32_t r = 0; r < (L + 1) / 2; ++r) {
    const uint32_t j = 2 * r + half;
    const bool act = j < L;  // the barriers below are reached by both halves
    const uint32_t jj = act ? j : 0;
    uint32_t *smh = sm + jj * PADN;
    const uint32_t q = pick(C.q, jj), ni = pick(C.ninv, jj), nis = pick(C.ninv_sh, jj);
    const uint2 *tw = pick(C.inv, jj);
    const uint32_t *gin = src + ((uint64_t)blockIdx.x * L + jj) * N;
    if constexpr (LOGN == 11) {
      if (act) ntt_pass<11, 4, 0, false, SRC_U32, DST_SMEM>(smh, gin, rs, 0, gout, tw, q, ni, nis, nullptr, tid);
      __syncthreads();
      if (act) ntt_pass<11, 4, 4, false, SRC_SMEM, DST_SMEM>(smh, gin, rs, 0, gout, tw, q, ni, nis, nullptr, tid);
      __syncthreads();
      if (act) ntt_pass<11, 3, 8, false, SRC_SMEM, DST_PAIR>(smh, gin, rs, 0, gout, tw, q, ni, nis, nullptr, tid);
    } else if constexpr (LOGN == 12) {
      if (act) ntt_pass<12, 4, 0, false, SRC_U32, DST_SMEM>(smh, gin, rs, 0, gout, tw, q, ni, nis, nullptr, tid);
      __syncthreads();
      if (act) ntt_pass<12, 4, 4, false, SRC_SMEM, DST_SMEM>(smh, gin, rs, 0, gout, tw, q, ni, nis, nullptr, tid);
      __syncthreads();
      if (act) ntt_pass<12, 4, 8, false, SRC_SMEM, DST_PAIR>(smh, gin, rs, 0, gout, tw, q, ni, nis, nullptr, tid);
    } else {
      if (act) ntt_pass<13, 4, 0, false, SRC_U32, DST_SMEM>(smh, gin, rs, 0, gout, tw, q, ni, nis, nullptr, tid);
      __syncthreads();
      if (act) ntt_pass<13, 4, 4, false, SRC_SMEM, DST_SMEM>(smh, gin, rs, 0, gout, tw, q, ni, nis, nullptr, tid);
      __syncthreads();
      if (act) ntt_pass<13, 4, 8, false, SRC_SMEM, DST_SMEM>(smh, gin, rs, 0, gout, tw, q, ni, nis, nullptr, tid);
      __syncthreads();
      if (act) ntt_pass<13, 1, 12, false, SRC_SMEM, DST_PAIR>(smh, gin, rs, 0, gout, tw, q, ni, nis, nullptr, tid);
    }
    __syncthreads();
  }
  uint32_t *out = dst + (uint64_t)blockIdx.x * N;
  for (uint32_t g = threadIdx.x; g < (uint32_t)N / 4; g += blockDim.x) {
    const uint32_t pt = padx(4 * g);  // four consecutive positions stay consecutive
    uint4 y;
    y.x = switch_coeff(sm, PADN, pt + 0, C, W, L);
    y.y = switch_coeff(sm, PADN, pt + 1, C, W, L);
    y.z = switch_coeff(sm, PADN, pt + 2, C, W, L);
    y.w = switch_coeff(sm, PADN, pt + 3, C, W, L);
    *reinterpret_cast<uint4 *>(out + 4 * g) = y;
  }
}

// Forward NTT of the a- and b-polynomial of one ciphertext (rows (i, comp 0) and
// (i, comp 1) of prime j of a batch-1 query chunk), written straight into the
// slot-major layout [L*n][stride][2] that the batch-1 scan reads (column col0 + i): the transpose of
// Sec. 4.2 fused into the NTT.  Block = i * L + j, 2 x n/16 threads: each half
// transforms one row in its own shared buffer, then all threads write the pairs.
template <int LOGN>
__global__ void __launch_bounds__((1 << LOGN) / 8)
    k_ntt_fwd_pair_slots(const uint32_t *__restrict__ src, uint64_t row0, NttConst C, uint32_t L, uint32_t stride,
                         uint32_t col0, uint32_t *__restrict__ slots) {
  constexpr int N = 1 << LOGN, PADN = N + N / 16, T = N / 16;
  extern __shared__ uint32_t sm[];
  const uint32_t i = blockIdx.x / L, j = blockIdx.x % L;
  const uint32_t half = threadIdx.x / T, tid = threadIdx.x % T;
  uint32_t *smh = sm + half * PADN;
  const uint32_t q = pick(C.q, j);
  const uint2 *tw = pick(C.fwd, j);
  const uint32_t *gin = src + (row0 + (uint64_t)i * 2 * L + (uint64_t)half * L + j) * N;
  const RawSrc rs = {};
  uint32_t *gout = nullptr;
  if constexpr (LOGN == 11) {
    ntt_pass<11, 4, 7, true, SRC_U32, DST_SMEM>(smh, gin, rs, 0, gout, tw, q, 0, 0, nullptr, tid);
    __syncthreads();
    ntt_pass<11, 4, 3, true, SRC_SMEM, DST_SMEM>(smh, gin, rs, 0, gout, tw, q, 0, 0, nullptr, tid);
    __syncthreads();
    ntt_pass<11, 3, 0, true, SRC_SMEM, DST_PAIR>(smh, gin, rs, 0, gout, tw, q, 0, 0, nullptr, tid);
  } else if constexpr (LOGN == 12) {
    ntt_pass<12, 4, 8, true, SRC_U32, DST_SMEM>(smh, gin, rs, 0, gout, tw, q, 0, 0, nullptr, tid);
    __syncthreads();
    ntt_pass<12, 4, 4, true, SRC_SMEM, DST_SMEM>(smh, gin, rs, 0, gout, tw, q, 0, 0, nullptr, tid);
    __syncthreads();
    ntt_pass<12, 4, 0, true, SRC_SMEM, DST_PAIR>(smh, gin, rs, 0, gout, tw, q, 0, 0, nullptr, tid);
  } else {
    ntt_pass<13, 4, 9, true, SRC_U32, DST_SMEM>(smh, gin, rs, 0, gout, tw, q, 0, 0, nullptr, tid);
    __syncthreads();
    ntt_pass<13, 4, 5, true, SRC_SMEM, DST_SMEM>(smh, gin, rs, 0, gout, tw, q, 0, 0, nullptr, tid);
    __syncthreads();
    ntt_pass<13, 4, 1, true, SRC_SMEM, DST_SMEM>(smh, gin, rs, 0, gout, tw, q, 0, 0, nullptr, tid);
    __syncthreads();
    ntt_pass<13, 1, 0, true, SRC_SMEM, DST_PAIR>(smh, gin, rs, 0, gout, tw, q, 0, 0, nullptr, tid);
  }
  __syncthreads();
  uint32_t *dst = slots + ((uint64_t)j * N * stride + col0 + i) * 2;
  for (uint32_t k = threadIdx.x; k < (uint32_t)N; k += 2 * T)
    *reinterpret_cast<uint2 *>(dst + (uint64_t)k * stride * 2) = make_uint2(sm[padx(k)], sm[PADN + padx(k)]);
}

constexpr uint64_t kMaxGrid = 1u << 30;

template <int LOGN>
cudaError_t fwd_launch(const ParamCtx &c, const uint32_t *src, const RowMap &rm, const RawSrc &rs, uint32_t *dst,
                       uint64_t rows, cudaStream_t s, bool raw) {
  const int T = (1 << LOGN) / 16;
  const size_t smem = ((1u << LOGN) + (1u << LOGN) / 16) * sizeof(uint32_t);
  const unsigned grid = (unsigned)(rows < kMaxGrid ? rows : kMaxGrid);
  if (raw)
    k_ntt_fwd<LOGN, SRC_RAW><<<grid, T, smem, s>>>(nullptr, rm, rs, dst, c.ntt, c.p.L, rows);
  else
    k_ntt_fwd<LOGN, SRC_U32><<<grid, T, smem, s>>>(src, rm, rs, dst, c.ntt, c.p.L, rows);
  return cudaGetLastError();
}

template <int LOGN>
cudaError_t inv_launch(const ParamCtx &c, const uint32_t *src, const RowMap &rm, uint32_t *dst, uint64_t rows,
                       cudaStream_t s) {
  const int T = (1 << LOGN) / 16;
  const size_t smem = ((1u << LOGN) + (1u << LOGN) / 16) * sizeof(uint32_t);
  const unsigned grid = (unsigned)(rows < kMaxGrid ? rows : kMaxGrid);
  k_ntt_inv<LOGN><<<grid, T, smem, s>>>(src, rm, dst, c.ntt, c.p.L, rows);
  return cudaGetLastError();
}

cudaError_t fwd_any(const ParamCtx &c, const uint32_t *src, const RowMap &rm, const RawSrc &rs, uint32_t *dst,
                    uint64_t rows, cudaStream_t s, bool raw) {
  if (rows == 0) return cudaSuccess;
  switch (c.logn) {
    case 11: return fwd_launch<11>(c, src, rm, rs, dst, rows, s, raw);
    case 12: return fwd_launch<12>(c, src, rm, rs, dst, rows, s, raw);
    case 13: return fwd_launch<13>(c, src, rm, rs, dst, rows, s, raw);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_ntt_fwd(const ParamCtx &c, const uint32_t *src, uint32_t *dst, uint64_t rows, cudaStream_t s) {
  const RawSrc rs = {};
  const RowMap rm = {0, rows ? rows : 1, 0, 1};
  return fwd_any(c, src, rm, rs, dst, rows, s, false);
}

cudaError_t launch_ntt_fwd_rows(const ParamCtx &c, const uint32_t *src, uint64_t off, uint64_t G, uint64_t S,
                                uint32_t *dst, uint64_t rows, cudaStream_t s) {
  const RawSrc rs = {};
  const RowMap rm = {off, G, S, 1};
  return fwd_any(c, src, rm, rs, dst, rows, s, false);
}

cudaError_t launch_ntt_fwd_raw(const ParamCtx &c, const uint8_t *raw, int col_major, uint32_t D1, uint32_t D2,
                               uint64_t first, uint64_t npolys, uint32_t *dst, cudaStream_t s) {
  RawSrc rs = {};
  rs.raw = raw;
  rs.log2p = c.p.log2p;
  rs.col_major = col_major ? 1u : 0u;
  rs.D1 = D1;
  rs.D2 = D2;
  if (col_major)
    rs.c0 = first;
  else
    rs.poly0 = first;
  const RowMap rm = {0, 1, 1, 1};
  return fwd_any(c, nullptr, rm, rs, dst, npolys * c.p.L, s, true);
}

template <int LOGN>
cudaError_t pair_launch(const ParamCtx &c, const uint32_t *src, uint64_t row0, uint32_t kc, uint32_t stride,
                        uint32_t col0, uint32_t *slots, cudaStream_t s) {
  const int T = (1 << LOGN) / 8;  // two rows in parallel
  const int smem = 2 * ((1 << LOGN) + (1 << LOGN) / 16) * (int)sizeof(uint32_t);
  cudaError_t e = cudaFuncSetAttribute(k_ntt_fwd_pair_slots<LOGN>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  k_ntt_fwd_pair_slots<LOGN><<<kc * c.p.L, T, smem, s>>>(src, row0, c.ntt, c.p.L, stride, col0, slots);
  return cudaGetLastError();
}

cudaError_t launch_ntt_fwd_pair_slots(const ParamCtx &c, const uint32_t *queries, uint32_t i0, uint32_t kc,
                                      uint32_t stride, uint32_t col0, uint32_t *slots, cudaStream_t s) {
  if (kc == 0) return cudaSuccess;
  if (col0 + (uint64_t)kc > stride) return cudaErrorInvalidValue;
  const uint64_t row0 = (uint64_t)i0 * 2 * c.p.L;  // row (b = 0, i0, comp 0, j = 0)
  switch (c.logn) {
    case 11: return pair_launch<11>(c, queries, row0, kc, stride, col0, slots, s);
    case 12: return pair_launch<12>(c, queries, row0, kc, stride, col0, slots, s);
    case 13: return pair_launch<13>(c, queries, row0, kc, stride, col0, slots, s);
  }
  return cudaErrorInvalidValue;
}

template <int LOGN>
cudaError_t switch_launch(const ParamCtx &c, const uint32_t *src, uint32_t *dst, uint64_t count, cudaStream_t s) {
  constexpr int N = 1 << LOGN, PADN = N + N / 16;
  const uint32_t L = c.p.L;
  const int smem = (int)(L * PADN * sizeof(uint32_t));
  cudaError_t e = cudaFuncSetAttribute(k_ntt_inv_switch<LOGN>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  for (uint64_t first = 0; first < count; first += kMaxGrid) {
    const uint64_t nb = count - first < kMaxGrid ? count - first : kMaxGrid;
    k_ntt_inv_switch<LOGN><<<(unsigned)nb, N / 8, smem, s>>>(src + first * L * N, dst + first * N, c.ntt, c.sw, L);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_ntt_inv_switch(const ParamCtx &c, const uint32_t *src, uint32_t *dst, uint64_t count,
                                  cudaStream_t s) {
  if (count == 0) return cudaSuccess;
  switch (c.logn) {
    case 11: return switch_launch<11>(c, src, dst, count, s);
    case 12: return switch_launch<12>(c, src, dst, count, s);
    case 13: return switch_launch<13>(c, src, dst, count, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_ntt_inv(const ParamCtx &c, const uint32_t *src, uint32_t *dst, uint64_t rows, cudaStream_t s) {
  if (rows == 0) return cudaSuccess;
  const RowMap rm = {0, rows, 0, 1};
  switch (c.logn) {
    case 11: return inv_launch<11>(c, src, rm, dst, rows, s);
    case 12: return inv_launch<12>(c, src, rm, dst, rows, s);
    case 13: return inv_launch<13>(c, src, rm, dst, rows, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_ntt_inv_rows(const ParamCtx &c, const uint32_t *src, uint64_t off, uint64_t G, uint64_t S,
                                uint64_t T, uint32_t *dst, uint64_t rows, cudaStream_t s) {
  if (rows == 0) return cudaSuccess;
  const RowMap rm = {off, G, S, T};
  switch (c.logn) {
    case 11: return inv_launch<11>(c, src, rm, dst, rows, s);
    case 12: return inv_launch<12>(c, src, rm, dst, rows, s);
    case 13: return inv_launch<13>(c, src, rm, dst, rows, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_ntt_fwd_rows_t(const ParamCtx &c, const uint32_t *src, uint64_t off, uint64_t G, uint64_t S,
                                  uint64_t T, uint32_t *dst, uint64_t rows, cudaStream_t s) {
  const RawSrc rs = {};
  const RowMap rm = {off, G, S, T};
  return fwd_any(c, src, rm, rs, dst, rows, s, false);
}

}  // namespace gbpir
