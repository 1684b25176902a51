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
// Row i-1 of W1^T and row i of W2 are streamed into a shared-memory ring by
// bulk asynchronous copies (cp.async.bulk + mbarrier transaction counts),
// NSTAGE steps ahead of use.
//
// Lane layout: lane = 8*sg + ug.  The 8 "unit groups" ug of a warp hold 8
// consecutive hidden units of each slot; the 4 "sample groups" sg hold SL
// samples each.  Slot r of warp w, lane ug holds unit k = r*8*NW + 8*w + ug.
// With sorted degrees, at any step every slot of a warp is either a pure dot
// slot, a pure update slot, or (at most one) mixed slot; a warp-uniform
// dispatch on the number of pure dot slots selects a fully unrolled body.
#include <cstdio>

#include "common.cuh"

namespace vqmc {
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

// ------------------------------------------------------- PTX: mbarrier/bulk

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: false (and the timeout bit set) if the phase never completed.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, uint32_t* err) {
  for (long long it = 0; it < kSpinLimit; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  atomicOr(err, kErrTimeout);
  return false;
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}

// ------------------------------------------------------------------ helpers

template <typename T>
__device__ __forceinline__ float ld_w(const T* p);
template <>
__device__ __forceinline__ float ld_w<float>(const float* p) { return *p; }
template <>
__device__ __forceinline__ float ld_w<bf16>(const bf16* p) { return __bfloat162float(*p); }

template <typename T>
__device__ __forceinline__ T from_f(float x);
template <>
__device__ __forceinline__ float from_f<float>(float x) { return x; }
template <>
__device__ __forceinline__ bf16 from_f<bf16>(float x) { return __float2bfloat16_rn(x); }

template <int ACT>
__device__ __forceinline__ float act_f(float x) {
  if constexpr (ACT == VQMC_ACT_RELU) return fmaxf(x, 0.0f);
  else return 1.0f / (1.0f + expf(-x));
}

// log sigma(x) without overflow.
__device__ __forceinline__ float log_sigmoid(float x) {
  return x >= 0.0f ? -log1pf(expf(-x)) : x - log1pf(expf(x));
}

constexpr int kBig = 0x3fffffff;

struct SamplerArgs {
  int n, h, hp, B;
  const void* wt;   // [n][hp]
  const void* v;    // [n][hp]
  const float* b1;  // [h]
  const float* b2;  // [n]
  const float* u;   // [B][n] or null (internal Philox)
  uint32_t key0, key1, it0, it1;
  int8_t* s_out;    // [B][n]
  float* logp;      // [B] or null
  void* sx;         // [B][ldsx] or null
  int ldsx;
  void* st;         // [n][ldst] or null
  int ldst;
  uint32_t* err;
};

template <typename WT, int NW, int UL, int SL, int ACT>
struct Sampler {
  static constexpr int S = 4 * SL;           // samples per CTA
  static constexpr int SLOTSTRIDE = 8 * NW;  // units between slots of a lane
  static constexpr int RL = 8 * NW * UL;     // row length held in shared memory
  static constexpr int NSTAGE = 8;

  struct State {
    float a[UL][SL];
    float acc[SL];
    float sgn[SL];
  };

  // Slots r < ND: all units complete -> dot; slot ND: mixed (per lane);
  // slots r > ND: all units still accumulating -> update.
  template <int ND>
  static __device__ __forceinline__ void body(State& st, const WT* __restrict__ wrow, const WT* __restrict__ vrow,
                                              int kbase, int i, int m_gen) {
#pragma unroll
    for (int r = 0; r < ND && r < UL; ++r) {
      const float w = ld_w(vrow + kbase + r * SLOTSTRIDE);
#pragma unroll
      for (int q = 0; q < SL; ++q) st.acc[q] = fmaf(w, st.a[r][q], st.acc[q]);
    }
    if constexpr (ND < UL) {
      const int k = kbase + ND * SLOTSTRIDE;
      if (i >= 2 && m_gen >= i - 1) {
        const float w = ld_w(wrow + k);
#pragma unroll
        for (int q = 0; q < SL; ++q) st.a[ND][q] = fmaf(w, st.sgn[q], st.a[ND][q]);
      }
      if (m_gen == i - 1) {
#pragma unroll
        for (int q = 0; q < SL; ++q) st.a[ND][q] = act_f<ACT>(st.a[ND][q]);
      }
      if (m_gen <= i - 1) {
        const float w = ld_w(vrow + k);
#pragma unroll
        for (int q = 0; q < SL; ++q) st.acc[q] = fmaf(w, st.a[ND][q], st.acc[q]);
      }
      if (i >= 2) {
#pragma unroll
        for (int r = ND + 1; r < UL; ++r) {
          const float w = ld_w(wrow + kbase + r * SLOTSTRIDE);
#pragma unroll
          for (int q = 0; q < SL; ++q) st.a[r][q] = fmaf(w, st.sgn[q], st.a[r][q]);
        }
      }
    }
  }

  template <int LO, int HI>
  static __device__ __forceinline__ void dispatch(int nd, State& st, const WT* wrow, const WT* vrow, int kbase,
                                                  int i, int m_gen) {
    if constexpr (LO == HI) {
      body<LO>(st, wrow, vrow, kbase, i, m_gen);
    } else {
      constexpr int MID = (LO + HI) / 2;
      if (nd <= MID) dispatch<LO, MID>(nd, st, wrow, vrow, kbase, i, m_gen);
      else dispatch<MID + 1, HI>(nd, st, wrow, vrow, kbase, i, m_gen);
    }
  }

  // Fallback when more than one slot of the warp is mixed (tiny n / large h).
  static __device__ __forceinline__ void body_general(State& st, const WT* __restrict__ wrow,
                                                      const WT* __restrict__ vrow, int kbase, int i, int n,
                                                      int h) {
#pragma unroll
    for (int r = 0; r < UL; ++r) {
      const int k = kbase + r * SLOTSTRIDE;
      const int m = k < h ? degree(k, n, h) : kBig;
      if (i >= 2 && m >= i - 1) {
        const float w = ld_w(wrow + k);
#pragma unroll
        for (int q = 0; q < SL; ++q) st.a[r][q] = fmaf(w, st.sgn[q], st.a[r][q]);
      }
      if (m == i - 1) {
#pragma unroll
        for (int q = 0; q < SL; ++q) st.a[r][q] = act_f<ACT>(st.a[r][q]);
      }
      if (m <= i - 1) {
        const float w = ld_w(vrow + k);
#pragma unroll
        for (int q = 0; q < SL; ++q) st.acc[q] = fmaf(w, st.a[r][q], st.acc[q]);
      }
    }
  }

  static __device__ __forceinline__ int deg_or_big(int k, int n, int h) { return k < h ? degree(k, n, h) : kBig; }

  static size_t smem_bytes() {
    return (size_t)NSTAGE * 2 * RL * sizeof(WT) + 128 + (size_t)2 * NW * S * sizeof(float) + 64;
  }
};

template <typename WT, int NW, int UL, int SL, int ACT>
__global__ void __launch_bounds__(NW * 32, 1) sampler_kernel(const SamplerArgs g) {
  using K = Sampler<WT, NW, UL, SL, ACT>;
  constexpr int S = K::S, RL = K::RL, NSTAGE = K::NSTAGE;
  extern __shared__ __align__(128) unsigned char smem[];
  WT* stages = reinterpret_cast<WT*>(smem);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + (size_t)NSTAGE * 2 * RL * sizeof(WT));
  uint64_t* redbar = full + NSTAGE;
  float* red = reinterpret_cast<float*>(full + NSTAGE + 2);  // [2][NW][S]

  const int n = g.n, h = g.h;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int sg = lane >> 3, ug = lane & 7;
  const int b0 = blockIdx.x * S;
  const uint32_t FULL = 0xffffffffu;

  // zero the row tails beyond the copied hp elements (never overwritten)
  for (int q = tid; q < NSTAGE * 2 * (RL - g.hp); q += NW * 32) {
    const int row = q / (RL - g.hp), col = q % (RL - g.hp);
    stages[(size_t)row * RL + g.hp + col] = from_f<WT>(0.0f);
  }
  if (tid == 0) {
    for (int s = 0; s < NSTAGE; ++s) mbar_init(smem_u32(&full[s]), 1);
    mbar_init(smem_u32(redbar), NW * 32);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();

  const uint32_t row_bytes = (uint32_t)(g.hp * sizeof(WT));
  const WT* gwt = reinterpret_cast<const WT*>(g.wt);
  const WT* gv = reinterpret_cast<const WT*>(g.v);
  // Stage for step j (1-based): W1^T row j-2 (input j-1, j >= 2) and W2 row j-1.
  auto issue = [&](int j) {
    const int s = (j - 1) % NSTAGE;
    const uint32_t bar = smem_u32(&full[s]);
    WT* dst = stages + (size_t)s * 2 * RL;
    mbar_expect_tx(bar, (j >= 2 ? row_bytes : 0u) + row_bytes);
    if (j >= 2) bulk_g2s(smem_u32(dst), gwt + (size_t)(j - 2) * g.hp, row_bytes, bar);
    bulk_g2s(smem_u32(dst + RL), gv + (size_t)(j - 1) * g.hp, row_bytes, bar);
  };
  int issued = 0, consumed = 0;  // steps whose copies were issued / waited for (thread 0)
  if (tid == 0)
    for (int j = 1; j <= n && j <= NSTAGE; ++j) issue(j), issued = j;

  typename K::State st;
  const int kbase = 8 * warp + ug;
#pragma unroll
  for (int r = 0; r < UL; ++r) {
    const int k = kbase + r * K::SLOTSTRIDE;
    const float bk = k < h ? g.b1[k] : 0.0f;
#pragma unroll
    for (int q = 0; q < SL; ++q) st.a[r][q] = bk;
  }
#pragma unroll
  for (int q = 0; q < SL; ++q) st.sgn[q] = 0.0f;

  // warp-uniform slot bookkeeping
  const int k7 = 8 * warp + 7, k0 = 8 * warp;
  int nd = 0, nt = 0;
  int thr_nd = K::deg_or_big(k7, n, h), thr_nt = K::deg_or_big(k0, n, h);
  int m_gen = K::deg_or_big(kbase, n, h);

  // per-sample inputs for the draw (lanes < S)
  const int my_b = b0 + (lane < S ? lane : 0);
  const bool my_valid = lane < S && my_b < g.B;
  float ucur[4] = {0.5f, 0.5f, 0.5f, 0.5f}, unxt[4] = {0.5f, 0.5f, 0.5f, 0.5f};
  const float* urow = g.u ? g.u + (size_t)my_b * n : nullptr;
  if (urow && my_valid)
    for (int e = 0; e < 4 && e < n; ++e) unxt[e] = __ldg(urow + e);
  float cval = __ldg(g.b2);
  float lp = 0.0f;
  bool ok = true;
  WT* sx = reinterpret_cast<WT*>(g.sx);
  WT* stt = reinterpret_cast<WT*>(g.st);

  for (int i = 1; i <= n; ++i) {
    const int t = i - 1;
    // uniforms for steps t..t+3
    if ((t & 3) == 0) {
      if (urow) {
#pragma unroll
        for (int e = 0; e < 4; ++e) ucur[e] = unxt[e];
        if (my_valid) {
#pragma unroll
          for (int e = 0; e < 4; ++e)
            if (t + 4 + e < n) unxt[e] = __ldg(urow + t + 4 + e);
        }
      } else {
        const uint4 r = philox4x32_10(make_uint4((uint32_t)(t >> 2), (uint32_t)my_b, g.it0, g.it1), g.key0, g.key1);
        ucur[0] = to_unit(r.x);
        ucur[1] = to_unit(r.y);
        ucur[2] = to_unit(r.z);
        ucur[3] = to_unit(r.w);
      }
    }
    const float cnext = (i < n) ? __ldg(g.b2 + i) : 0.0f;

    // slot bookkeeping (warp-uniform)
    while (nd < UL && thr_nd <= i - 2) {
      ++nd;
      thr_nd = nd < UL ? K::deg_or_big(k7 + nd * K::SLOTSTRIDE, n, h) : kBig;
      m_gen = nd < UL ? K::deg_or_big(kbase + nd * K::SLOTSTRIDE, n, h) : kBig;
    }
    while (nt < UL && thr_nt <= i - 1) {
      ++nt;
      thr_nt = nt < UL ? K::deg_or_big(k0 + nt * K::SLOTSTRIDE, n, h) : kBig;
    }

    const int s = t % NSTAGE;
    if (!mbar_wait(smem_u32(&full[s]), (uint32_t)((t / NSTAGE) & 1), g.err)) {
      ok = false;
      break;
    }
    consumed = i;
    const WT* wrow = stages + (size_t)s * 2 * RL;
    const WT* vrow = wrow + RL;
#pragma unroll
    for (int q = 0; q < SL; ++q) st.acc[q] = 0.0f;
    if (nt <= nd + 1) K::template dispatch<0, UL>(nd, st, wrow, vrow, kbase, i, m_gen);
    else K::body_general(st, wrow, vrow, kbase, i, n, h);

    // lane reduction over the 8 unit groups; lane ug == q keeps sample q
    const int buf = t & 1;
#pragma unroll
    for (int q = 0; q < SL; ++q) {
      float v = st.acc[q];
      v += __shfl_xor_sync(FULL, v, 1);
      v += __shfl_xor_sync(FULL, v, 2);
      v += __shfl_xor_sync(FULL, v, 4);
      if (ug == q) red[(buf * NW + warp) * S + sg * SL + q] = v;
    }
    mbar_arrive(smem_u32(redbar));
    if (!mbar_wait(smem_u32(redbar), (uint32_t)(t & 1), g.err)) {
      ok = false;
      break;
    }
    // stage s is free: every thread has finished reading it
    if (tid == 0 && i + NSTAGE <= n) issue(i + NSTAGE), issued = i + NSTAGE;

    // every warp draws s_i for all S samples (identical arithmetic)
    float z = cval;
    if (lane < S) {
#pragma unroll
      for (int w = 0; w < NW; ++w) z += red[(buf * NW + w) * S + lane];
    }
    const float p = 1.0f / (1.0f + expf(-z));
    const float u = (t & 3) == 0 ? ucur[0] : (t & 3) == 1 ? ucur[1] : (t & 3) == 2 ? ucur[2] : ucur[3];
    const bool up = lane < S && u < p;
    const uint32_t mask = __ballot_sync(FULL, up);
#pragma unroll
    for (int q = 0; q < SL; ++q) st.sgn[q] = ((mask >> (sg * SL + q)) & 1u) ? 1.0f : -1.0f;
    if (warp == 0 && my_valid) {
      lp += log_sigmoid(up ? z : -z);
      const float sv = up ? 1.0f : -1.0f;
      g.s_out[(size_t)my_b * n + t] = up ? (int8_t)1 : (int8_t)-1;
      if (sx) sx[(size_t)my_b * g.ldsx + t] = from_f<WT>(sv);
      if (stt) stt[(size_t)t * g.ldst + my_b] = from_f<WT>(sv);
    }
    cval = cnext;
  }

  if (!ok) {
    // Drain: the producer waits (bounded) for every copy it issued and no
    // thread consumed, so no bulk copy is in flight when the CTA exits.
    if (tid == 0)
      for (int j = consumed + 1; j <= issued; ++j)
        if (!mbar_wait(smem_u32(&full[(j - 1) % NSTAGE]), (uint32_t)(((j - 1) / NSTAGE) & 1), g.err)) break;
    return;
  }
  if (warp == 0 && my_valid && g.logp) g.logp[my_b] = lp;
}

template <typename WT, int NW, int UL, int SL, int ACT>
cudaError_t launch_cfg(const SamplerArgs& a, cudaStream_t st) {
  using K = Sampler<WT, NW, UL, SL, ACT>;
  const size_t smem = K::smem_bytes();
  auto kern = sampler_kernel<WT, NW, UL, SL, ACT>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int grid = (a.B + K::S - 1) / K::S;
  kern<<<grid, NW * 32, smem, st>>>(a);
  return cudaGetLastError();
}

template <typename WT, int ACT>
cudaError_t launch_shape(const SamplerArgs& a, cudaStream_t st) {
  // rows held in shared memory must cover hp = pad64(h)
  if (a.hp <= 64) return launch_cfg<WT, 1, 8, 4, ACT>(a, st);
  if (a.hp <= 512) return launch_cfg<WT, 8, 8, 4, ACT>(a, st);
  if (a.hp <= 1024) return launch_cfg<WT, 8, 16, 4, ACT>(a, st);
  if (a.hp <= 2048) return launch_cfg<WT, 8, 32, 4, ACT>(a, st);
  return cudaErrorNotSupported;
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
                           float* d_logp, void* Sx, void* St, cudaStream_t st) {
  if (B <= 0) return cudaSuccess;
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
  a.sx = Sx;
  a.ldsx = c->np;
  a.st = St;
  a.ldst = c->Bp;
  a.err = c->err;
  const bool bf = c->prec == VQMC_PREC_BF16;
  const bool relu = c->act == VQMC_ACT_RELU;
  if (bf) return relu ? launch_shape<bf16, VQMC_ACT_RELU>(a, st) : launch_shape<bf16, VQMC_ACT_SIGMOID>(a, st);
  return relu ? launch_shape<float, VQMC_ACT_RELU>(a, st) : launch_shape<float, VQMC_ACT_SIGMOID>(a, st);
}

}  // namespace vqmc
