// Exact autoregressive sampling (Algorithm 1 of the paper, Sec. 2.3) from
// Philox4x32-10 uniforms (Sec. 4), and the dispatch between the two sampler
// kernels: the blocked tensor-core sampler (sampler_tc.cu) for the BF16
// models it covers, the per-step CUDA-core sampler (sampler_impl.cuh,
// instantiated in sampler_bf16.cu and sampler_f32.cu) for every other model.
//
// uniforms_kernel writes the same stream the samplers draw internally:
// u_{b,i} = word (i mod 4) of Philox4x32-10(counter (i/4, b0 + b, iteration),
// key = seed), as (x >> 8) 2^-24, with b0 the context's sample offset (0
// unless the context draws one shard of a batch spread over several GPUs).
#include <cstdio>

#include "sampler.cuh"

namespace vqmc {
namespace {

__global__ void uniforms_kernel(int B, int n, uint32_t k0, uint32_t k1, uint32_t it0, uint32_t it1, uint32_t boff,
                                float* __restrict__ u) {
  const int groups = (n + 3) / 4;
  const long long tot = (long long)B * groups;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < tot;
       q += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(q / groups), g = (int)(q % groups);
    const uint4 r = philox4x32_10(make_uint4((uint32_t)g, (uint32_t)b + boff, it0, it1), k0, k1);
    const uint32_t w[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int i = 4 * g + e;
      if (i < n) u[(size_t)b * n + i] = to_unit(w[e]);
    }
  }
}

}  // namespace

cudaError_t launch_uniforms(int B, int n, uint64_t seed, uint64_t iteration, float* d_u, cudaStream_t st,
                            uint32_t boff) {
  if (B <= 0 || n <= 0) return cudaSuccess;
  const long long work = (long long)B * ((n + 3) / 4);
  const int grid = (int)((work + 255) / 256 < 4096 ? (work + 255) / 256 : 4096);
  uniforms_kernel<<<grid, 256, 0, st>>>(B, n, (uint32_t)seed, (uint32_t)(seed >> 32), (uint32_t)iteration,
                                        (uint32_t)(iteration >> 32), boff, d_u);
  return cudaGetLastError();
}

cudaError_t launch_sampler(const vqmc_ctx* c, int B, const float* d_u, uint64_t iteration, int8_t* d_s,
                           float* d_logp, cudaStream_t st, const unsigned long long* it_dev) {
  if (B <= 0) return cudaSuccess;
  if (c->sampler == VQMC_SAMPLER_TENSOR_CORE)
    return launch_sampler_tc(c, B, d_u, iteration, d_s, d_logp, st, nullptr, nullptr, nullptr, it_dev);
  SamplerArgs a;
  a.n = c->n;
  a.h = c->h;
  a.hp = c->hp;
  a.B = B;
  a.wt = c->wt_s;
  a.v = c->v_s;
  a.b1 = c->b1;
  a.b2 = c->b2;
  a.u = d_u;
  a.key0 = (uint32_t)c->cfg.seed;
  a.key1 = (uint32_t)(c->cfg.seed >> 32);
  a.it0 = (uint32_t)iteration;
  a.it1 = (uint32_t)(iteration >> 32);
  a.boff = c->sample_offset;
  a.it_dev = it_dev;
  a.s_out = d_s;
  a.logp = d_logp;
  a.err = c->err;
  a.act = c->act;
  a.wide = c->sampler_wide;
  return c->prec == VQMC_PREC_BF16 ? launch_sampler_wt<bf16>(a, st) : launch_sampler_wt<float>(a, st);
}

}  // namespace vqmc
