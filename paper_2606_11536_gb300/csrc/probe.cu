// probe.cu -- peak rate of the INT8 warp-level tensor instruction on this GPU, the
// denominator of the scalar-HE GEMM's roofline (the driver's measured peaks cover
// HBM copies and bf16 GEMMs only).  Every warp of a full grid issues eight
// independent chains of mma.sync m16n8k32 s8 x u8 -> s32 on register operands; the
// rate is 2 x 16 x 8 x 32 operations per instruction over the event-timed duration.
#include "common.cuh"

namespace gbpir {
namespace {

constexpr int kChains = 8;

__global__ void __launch_bounds__(256) k_probe_imma(uint32_t iters, uint32_t seed, int *__restrict__ sink) {
  uint32_t a[4], b0 = seed * 3u + threadIdx.x, b1 = seed ^ 0x9e3779b9u;
#pragma unroll
  for (int i = 0; i < 4; ++i) a[i] = seed + i * 0x01010101u + threadIdx.x;
  int d[kChains][4];
#pragma unroll
  for (int c = 0; c < kChains; ++c)
#pragma unroll
    for (int f = 0; f < 4; ++f) d[c][f] = 0;
  for (uint32_t it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c)
      asm volatile(
          "mma.sync.aligned.m16n8k32.row.col.s32.s8.u8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
          "{%0,%1,%2,%3};\n"
          : "+r"(d[c][0]), "+r"(d[c][1]), "+r"(d[c][2]), "+r"(d[c][3])
          : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
  }
  int s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += d[c][0] ^ d[c][1] ^ d[c][2] ^ d[c][3];
  if (s == 0x7fffffff) sink[0] = s;  // keeps the chains live
}

}  // namespace
}  // namespace gbpir

extern "C" pir_status_t pir_probe_int8_mma(void *stream, double *tops) {
  using namespace gbpir;
  if (!tops) return PIR_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return cuda_status(e);
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return cuda_status(e);
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_probe_imma, 256, 0)) != cudaSuccess)
    return cuda_status(e);
  int *sink = nullptr;
  if ((e = cudaMallocAsync(&sink, sizeof(int), s)) != cudaSuccess) return cuda_status(e);
  const unsigned grid = (unsigned)(sms * (per_sm > 0 ? per_sm : 1));
  const uint32_t iters = 4096;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  k_probe_imma<<<grid, 256, 0, s>>>(iters / 8, 1, sink);  // warm-up
  cudaEventRecord(e0, s);
  k_probe_imma<<<grid, 256, 0, s>>>(iters, 2, sink);
  cudaEventRecord(e1, s);
  e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFreeAsync(sink, s);
  if (e != cudaSuccess) return cuda_status(e);
  count_launches(2);
  const double ops = 2.0 * 16 * 8 * 32 * (double)kChains * iters * (grid * 8.0);  // 8 warps per block
  *tops = ops / (ms * 1e-3) / 1e12;
  return PIR_OK;
}
