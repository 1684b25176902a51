// Persistent autoregressive sampler (Algorithm 1 of the paper, Sec. 2.3) and
// the Philox4x32-10 uniforms it transforms into exact samples (Sec. 4).
//
// One CTA owns S = 4*SL samples for all n steps.  Hidden unit k's
// pre-activation a_k = b1_k + sum_{j <= m(k)} W1_kj s_j lives in registers for
// every sample of the CTA.  At step i the CTA
//   (1) adds W1[:, i-1] s_{i-1} to the units with m(k) >= i-1,
//   (2) applies act() to the units that just became complete (m(k) = i-1),
//   (3) accumulates z_i = b2_i + sum_{k : m(k) <= i-1} W2_ik act(a_k),
//   (4) reduces z_i over lanes (shuffles) and warps (shared memory + one
//       mbarrier phase per step), and every warp then draws
//       s_i = +1 iff u_{b,i} < sigma(z_i) for all samples of the CTA.
// Each unit does exactly one multiply-add per step and sample (an update
// while m(k) >= i, a dot term afterwards), so a sample costs h*n FMA.
// Rows of W1^T and W2 are streamed into a shared-memory ring by bulk
// asynchronous copies (cp.async.bulk + mbarrier transaction counts), SPS
// consecutive rows of each per copy, several stages ahead of use.
//
// Lane layout: lane = 8*sg + ug.  The 8 "unit groups" ug of a warp hold 8
// consecutive hidden units of each slot; the 4 "sample groups" sg hold SL
// samples each.  Slot r of warp w, lane ug holds unit k = r*8*NW + 8*w + ug.
// With sorted degrees, at any step every slot of a warp is either a pure dot
// slot, a pure update slot, or (at most one) mixed slot; a warp-uniform
// dispatch on the number of pure dot slots selects a fully unrolled body.
#include <cstdio>

#include "sampler.cuh"

namespace vqmc {
namespace {

__global__ void uniforms_kernel(int B, int n, uint32_t k0, uint32_t k1, uint32_t it0, uint32_t it1,
                                float* __restrict__ u) {
  const int groups = (n + 3) / 4;
  const long long tot = (long long)B * groups;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < tot;
       q += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(q / groups), g = (int)(q % groups);
    const uint4 r = philox4x32_10(make_uint4((uint32_t)g, (uint32_t)b, it0, it1), k0, k1);
    const uint32_t w[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int i = 4 * g + e;
      if (i < n) u[(size_t)b * n + i] = to_unit(w[e]);
    }
  }
}

}  // namespace

cudaError_t launch_uniforms(int B, int n, uint64_t seed, uint64_t iteration, float* d_u, cudaStream_t st) {
  if (B <= 0 || n <= 0) return cudaSuccess;
  const long long work = (long long)B * ((n + 3) / 4);
  const int grid = (int)((work + 255) / 256 < 4096 ? (work + 255) / 256 : 4096);
  uniforms_kernel<<<grid, 256, 0, st>>>(B, n, (uint32_t)seed, (uint32_t)(seed >> 32), (uint32_t)iteration,
                                        (uint32_t)(iteration >> 32), d_u);
  return cudaGetLastError();
}

cudaError_t launch_sampler(const vqmc_ctx* c, int B, const float* d_u, uint64_t iteration, int8_t* d_s,
                           float* d_logp, cudaStream_t st) {
  if (B <= 0) return cudaSuccess;
  if (c->sampler == VQMC_SAMPLER_TENSOR_CORE) return launch_sampler_tc(c, B, d_u, iteration, d_s, d_logp, st);
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
  a.s_out = d_s;
  a.logp = d_logp;
  a.err = c->err;
  a.act = c->act;
  return c->prec == VQMC_PREC_BF16 ? launch_sampler_wt<bf16>(a, st) : launch_sampler_wt<float>(a, st);
}

}  // namespace vqmc
