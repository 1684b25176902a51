// Declarations shared by the sampler's translation units: launch arguments,
// the per-weight-type launcher, and the Philox4x32-10 generator.
#pragma once

#include "common.cuh"

namespace vqmc {

struct SamplerArgs {
  int n, h, hp, B;
  int act;          // VQMC_ACT_*
  int nst;          // ring stages
  int wide;         // 1: the four-warp-group layout (4 samples per CTA) at any hp
  const void* wt;   // [n][hp]
  const void* v;    // [n][hp]
  const float* b1;  // [h]
  const float* b2;  // [n]
  const float* u;   // [B][n] or null (internal Philox)
  uint32_t key0, key1, it0, it1;
  uint32_t boff;    // index of sample 0 in the Philox counter (a shard's first global sample)
  const unsigned long long* it_dev;  // if not null: the Philox iteration, read on the device
  int8_t* s_out;    // [B][n]
  float* logp;      // [B] or null
  uint32_t* err;
};

// Launches the sampler for weights of type WT (float or bf16).
template <typename WT>
cudaError_t launch_sampler_wt(const SamplerArgs& a, cudaStream_t st);



namespace {

// ------------------------------------------------------------------ Philox

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11, Sec. 4.2): ten rounds of
// two 32x32->64 multiplies of (c0, c2) by the round multipliers, with the
// high halves xored into the other counter words and the round key, which
// advances by the Weyl constants between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
  }
  return c;
}

// 24 high bits -> [0, 1) on the 2^-24 grid (exact in float).
__device__ __forceinline__ float to_unit(uint32_t x) { return (float)(x >> 8) * (1.0f / 16777216.0f); }

// logit(u) = log(u / (1 - u)); -inf at u = 0.  u < sigma(z) iff z > logit(u).
__device__ __forceinline__ float logit(float u) { return logf(u) - log1pf(-u); }

__device__ __forceinline__ float act_f(int act, float x) {
  return act == VQMC_ACT_RELU ? fmaxf(x, 0.0f) : 1.0f / (1.0f + expf(-x));
}

// log sigma(x) without overflow.
__device__ __forceinline__ float log_sigmoid(float x) {
  return x >= 0.0f ? -log1pf(expf(-x)) : x - log1pf(expf(x));
}

}  // namespace

}  // namespace vqmc
