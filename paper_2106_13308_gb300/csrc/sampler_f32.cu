// Sampler instantiations for FP32 weights.
#include "sampler_impl.cuh"

namespace vqmc {
template cudaError_t launch_sampler_wt<float>(const SamplerArgs& a, cudaStream_t st);
template bool sampler_wt_supports<float>(int hp, bool wide);
}  // namespace vqmc
