// Sampler instantiations for BF16 weights.
#include "sampler_impl.cuh"

namespace vqmc {
template cudaError_t launch_sampler_wt<bf16>(const SamplerArgs& a, cudaStream_t st);
template bool sampler_wt_supports<bf16>(int hp, bool wide);
}  // namespace vqmc
