// gemm_limb.cu -- the first-dimension modular GEMM on the INT8 tensor pipe.
// (Kernel follows; until then the limb layout answers PIR_ERR_CUDA / not supported.)
#include "common.cuh"

namespace gbpir {

uint32_t gemm_limb_tiles() { return 0; }

cudaError_t launch_gemm_limb(const ParamCtx &, const uint8_t *, uint32_t, uint32_t, const uint8_t *, uint32_t,
                             uint32_t, uint32_t, uint32_t, uint32_t *, int, uint32_t, cudaStream_t) {
  return cudaErrorNotSupported;
}

}  // namespace gbpir
