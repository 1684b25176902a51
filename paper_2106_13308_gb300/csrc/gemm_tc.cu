// tcgen05 tensor-core GEMM (BF16 operands, FP32 accumulation in tensor memory).
#include "gemm.cuh"

namespace vqmc {

bool gemm_tc_available() { return false; }

cudaError_t launch_gemm_tc_bf16(const GemmArgs<bf16>&, cudaStream_t) { return cudaErrorNotSupported; }

}  // namespace vqmc
