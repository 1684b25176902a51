// Sampler instantiations for FP32 weights.
#include "sampler_impl.cuh"

namespace vqmc {
template cudaError_t launch_sampler_wt<float>(const SamplerArgs& a, cudaStream_t st);
}  // namespace vqmc
