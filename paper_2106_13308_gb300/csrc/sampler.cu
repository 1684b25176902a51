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
__device__ __forceinline__ bool mbar_test_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
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

// ---- packed FP32 pairs (fma.rn.f32x2: two IEEE FP32 FMAs in one instruction)
__device__ __forceinline__ uint64_t pack2(float lo, float hi) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void unpack2(uint64_t v, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ uint64_t fma2(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

// weights of units (2q, 2q+1) of a staged row as an FP32 pair
template <typename T>
__device__ __forceinline__ uint64_t ld_pair(const T* row, int q);
template <>
__device__ __forceinline__ uint64_t ld_pair<bf16>(const bf16* row, int q) {
  const uint32_t x = reinterpret_cast<const uint32_t*>(row)[q];
  return pack2(__uint_as_float(x << 16), __uint_as_float(x & 0xffff0000u));
}
template <>
__device__ __forceinline__ uint64_t ld_pair<float>(const float* row, int q) {
  return reinterpret_cast<const uint64_t*>(row)[q];
}

struct SamplerArgs {
  int n, h, hp, B;
  int nst;          // ring stages
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

// A CTA = NGRP groups of GW warps.  Group g owns
// SL samples; its GW*32 lanes split the hidden units: lane L of the group
// holds unit pairs q = r*GW*32 + L (units 2q, 2q+1), r = 0..U2-1, for all SL
// samples.  Per step a group reduces its partial sums with shuffles and one
// named barrier of its own warps; groups never wait for each other.  Lane 0
// of the last warp also keeps the weight ring filled: whenever every warp
// has released a stage it issues the copies for the block a full ring ahead.
template <typename WT, int GW, int NGRP, int U2, int SL, int ACT>
struct Sampler {
  static constexpr int NCW = GW * NGRP;      // warps
  static constexpr int NT = NCW * 32;        // threads
  static constexpr int S = SL * NGRP;        // samples per CTA
  static constexpr int GL = GW * 32;         // lanes per group
  static constexpr int RL = GL * 2 * U2;     // units covered (row length in smem)
  static constexpr int SPS = 4;              // steps per ring stage (rows per copy)
  static constexpr int UWIN = 128 / SL;      // steps per uniform window (32 lanes x 4 words)
  static_assert(SL >= 1 && SL <= 16 && (SL & (SL - 1)) == 0, "SL must be a power of two <= 16");

  struct State {
    uint64_t a[U2][SL];  // pre-activations of units (2q, 2q+1), or act() once complete
    uint64_t acc[SL];    // dot accumulators (even / odd units)
    uint64_t sg[SL];     // {s_{i-1}, s_{i-1}}
  };

  static __device__ __forceinline__ int deg(int k, int n, int h) { return k < h ? degree(k, n, h) : kBig; }

  // Mixed slot: the lane's two units may be in different roles.  Weights of
  // units that must not take part are zeroed, so the pair still runs as f32x2.
  static __device__ __forceinline__ void mixed(State& st, const WT* wrow, const WT* vrow, int r, int q, int i,
                                               int m0, int m1) {
    if (i >= 2 && (m0 >= i - 1 || m1 >= i - 1)) {
      float w0, w1;
      unpack2(ld_pair(wrow, q), w0, w1);
      const uint64_t w = pack2(m0 >= i - 1 ? w0 : 0.0f, m1 >= i - 1 ? w1 : 0.0f);
#pragma unroll
      for (int s = 0; s < SL; ++s) st.a[r][s] = fma2(w, st.sg[s], st.a[r][s]);
    }
    if (m0 == i - 1 || m1 == i - 1) {
#pragma unroll
      for (int s = 0; s < SL; ++s) {
        float a0, a1;
        unpack2(st.a[r][s], a0, a1);
        if (m0 == i - 1) a0 = act_f<ACT>(a0);
        if (m1 == i - 1) a1 = act_f<ACT>(a1);
        st.a[r][s] = pack2(a0, a1);
      }
    }
    if (m0 <= i - 1) {
      float v0, v1;
      unpack2(ld_pair(vrow, q), v0, v1);
      const uint64_t v = pack2(v0, m1 <= i - 1 ? v1 : 0.0f);
#pragma unroll
      for (int s = 0; s < SL; ++s) st.acc[s] = fma2(v, st.a[r][s], st.acc[s]);
    }
  }

  // Slots r < ND: every unit complete -> dot.  MIX: slot ND is mixed.
  // Remaining slots: every unit still accumulating -> update.
  template <int ND, bool MIX>
  static __device__ __forceinline__ void body(State& st, const WT* __restrict__ wrow, const WT* __restrict__ vrow,
                                              int lq, int i, int m0, int m1) {
#pragma unroll
    for (int r = 0; r < ND && r < U2; ++r) {
      const uint64_t w = ld_pair(vrow, lq + r * GL);
#pragma unroll
      for (int s = 0; s < SL; ++s) st.acc[s] = fma2(w, st.a[r][s], st.acc[s]);
    }
    constexpr int FIRST_UPD = MIX ? ND + 1 : ND;
    if constexpr (MIX && ND < U2) mixed(st, wrow, vrow, ND, lq + ND * GL, i, m0, m1);
    if (i >= 2) {
#pragma unroll
      for (int r = FIRST_UPD; r < U2; ++r) {
        const uint64_t w = ld_pair(wrow, lq + r * GL);
#pragma unroll
        for (int s = 0; s < SL; ++s) st.a[r][s] = fma2(w, st.sg[s], st.a[r][s]);
      }
    }
  }

  // code = 2*nd + mixed, nd in [0, U2]
  template <int LO, int HI>
  static __device__ __forceinline__ void dispatch(int code, State& st, const WT* wrow, const WT* vrow, int lq, int i,
                                                  int m0, int m1) {
    if constexpr (LO == HI) {
      body<LO / 2, (LO & 1) != 0>(st, wrow, vrow, lq, i, m0, m1);
    } else {
      constexpr int MID = (LO + HI) / 2;
      if (code <= MID) dispatch<LO, MID>(code, st, wrow, vrow, lq, i, m0, m1);
      else dispatch<MID + 1, HI>(code, st, wrow, vrow, lq, i, m0, m1);
    }
  }

  // every slot treated as mixed (small n or h >> n)
  static __device__ __forceinline__ void body_general(State& st, const WT* wrow, const WT* vrow, int lq, int i,
                                                      int n, int h) {
#pragma unroll
    for (int r = 0; r < U2; ++r) {
      const int q = lq + r * GL;
      mixed(st, wrow, vrow, r, q, i, deg(2 * q, n, h), deg(2 * q + 1, n, h));
    }
  }

  // Reduce SL values over the 32 lanes: afterwards lane l holds the warp sum
  // of sample q(l); lanes with (l & (32/SL - 1)) == 0 hold distinct samples.
  static __device__ __forceinline__ float reduce_scatter(float (&v)[SL], int lane, int& q) {
    q = 0;
    int cnt = SL;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
      if (cnt > 1) {
        const bool up = (lane & o) != 0;
        const int half = cnt / 2;
#pragma unroll
        for (int e = 0; e < SL / 2; ++e) {
          if (e < half) {
            const float keep = up ? v[e + half] : v[e];
            const float send = up ? v[e] : v[e + half];
            v[e] = keep + __shfl_xor_sync(0xffffffffu, send, o);
          }
        }
        q = 2 * q + (up ? 1 : 0);
        cnt = half;
      } else {
        v[0] += __shfl_xor_sync(0xffffffffu, v[0], o);
      }
    }
    return v[0];
  }

  // ring stages (each: SPS rows of W1^T and SPS rows of W2) that fit the
  // shared-memory budget, at most 8
  static int stages_for(int hp) {
    const size_t stage = (size_t)2 * SPS * hp * sizeof(WT);
    const size_t fixed = (size_t)RL * sizeof(WT) + 2 * 8 * 8 + (size_t)2 * NGRP * GW * SL * sizeof(float) + 256;
    int nst = (int)((200 * 1024 - fixed) / stage);
    return nst > 8 ? 8 : nst;
  }
  static size_t smem_bytes(int hp, int nst) {
    return (size_t)nst * 2 * SPS * hp * sizeof(WT) + (size_t)RL * sizeof(WT) + 2 * 8 * 8 +
           (size_t)2 * NGRP * GW * SL * sizeof(float) + 64;
  }
};

template <typename WT, int GW, int NGRP, int U2, int SL, int ACT>
__global__ void __launch_bounds__(GW * NGRP * 32, 1) sampler_kernel(const SamplerArgs g) {
  using K = Sampler<WT, GW, NGRP, U2, SL, ACT>;
  constexpr int RL = K::RL, SPS = K::SPS, NCW = K::NCW, GL = K::GL, UWIN = K::UWIN;
  extern __shared__ __align__(128) unsigned char smem[];
  const int nst = g.nst, hp = g.hp;
  const int stage_elems = 2 * SPS * hp;  // W1^T rows then W2 rows
  // ring, then RL elements of slack: lanes holding padding units (k >= hp)
  // read past their row, never past the ring
  const int ring_elems = nst * stage_elems + RL;
  WT* stages = reinterpret_cast<WT*>(smem);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + ((size_t)ring_elems * sizeof(WT) + 7) / 8 * 8);
  uint64_t* empty = full + 8;
  float* red = reinterpret_cast<float*>(empty + 8);  // [2][NGRP][GW][SL]

  const int n = g.n, h = g.h;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t FULL = 0xffffffffu;

  // zero the ring once: every value a lane may read must be finite
  for (int q = tid; q < ring_elems; q += K::NT) stages[q] = from_f<WT>(0.0f);
  if (tid == 0) {
    for (int s = 0; s < nst; ++s) {
      mbar_init(smem_u32(&full[s]), 1);
      mbar_init(smem_u32(&empty[s]), NCW);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncthreads();

  // ------------------------------------------------------------ producer
  const bool producer = warp == NCW - 1 && lane == 0;
  const WT* gwt = reinterpret_cast<const WT*>(g.wt);
  const WT* gv = reinterpret_cast<const WT*>(g.v);
  const int nblocks = (n + SPS - 1) / SPS;
  int issued = 0;  // ring blocks (SPS steps each) whose copies were issued (producer lane)
  // Block q covers steps q*SPS+1 .. q*SPS+SPS: rows q*SPS.. of wt_s (row j =
  // input j, row 0 zero) and of v_s (row i = output i+1), copied whole.
  const uint32_t block_bytes = (uint32_t)(SPS * hp * sizeof(WT));
  auto issue = [&](int q) {
    const int s = q % nst;
    const uint32_t bar = smem_u32(&full[s]);
    WT* dst = stages + (size_t)s * stage_elems;
    mbar_expect_tx(bar, 2 * block_bytes);
    bulk_g2s(smem_u32(dst), gwt + (size_t)q * SPS * hp, block_bytes, bar);
    bulk_g2s(smem_u32(dst + SPS * hp), gv + (size_t)q * SPS * hp, block_bytes, bar);
    issued = q + 1;
  };
  // refill every stage all warps have released (non-blocking)
  auto refill = [&]() {
    while (issued < nblocks) {
      const int q = issued;
      if (q >= nst && !mbar_test_wait(smem_u32(&empty[q % nst]), (uint32_t)((q / nst - 1) & 1))) break;
      issue(q);
    }
  };
  if (producer) refill();

  // ----------------------------------------------------------- consumers
  const int grp = warp / GW, wg = warp % GW;
  const int L = wg * 32 + lane;                  // lane within the group
  const int b0 = blockIdx.x * K::S + grp * SL;   // first sample of the group
  float* gred = red + (size_t)grp * GW * SL;     // + buf * NGRP*GW*SL

  typename K::State st;
#pragma unroll
  for (int r = 0; r < U2; ++r) {
    const int k = 2 * (r * GL + L);
    const float x0 = k < h ? __ldg(g.b1 + k) : 0.0f;
    const float x1 = k + 1 < h ? __ldg(g.b1 + k + 1) : 0.0f;
#pragma unroll
    for (int s = 0; s < SL; ++s) st.a[r][s] = pack2(x0, x1);
  }
#pragma unroll
  for (int s = 0; s < SL; ++s) st.sg[s] = pack2(0.0f, 0.0f);

  // warp-uniform slot bookkeeping: nd = #slots complete before this step,
  // nt = #slots with at least one unit complete at this step
  const int kw = 2 * wg * 32;  // first unit of the warp in slot 0
  int nd = 0, nt = 0;
  int thr_nd = K::deg(kw + 63, n, h), thr_nt = K::deg(kw, n, h);
  int m0 = K::deg(2 * L, n, h), m1 = K::deg(2 * L + 1, n, h);

  // uniforms: lane L (< 32) holds 4 words for sample L % SL, steps
  // win + 4*(L / SL) .. +3 of the current window
  const int us = lane % SL, ug = lane / SL;
  const int ub = b0 + us;
  const bool uvalid = ub < g.B;
  uint32_t uw[4] = {0, 0, 0, 0}, unx[4] = {0, 0, 0, 0};
  auto load_u = [&](int win, uint32_t (&dst)[4]) {
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int t = win + 4 * ug + e;
      dst[e] = (uvalid && t < n) ? __float_as_uint(__ldg(g.u + (size_t)ub * n + t)) : 0x3f000000u;
    }
  };
  if (g.u) load_u(0, unx);
  float cw = lane < n ? __ldg(g.b2 + lane) : 0.0f, cnx = 0.0f;
  if (32 + lane < n) cnx = __ldg(g.b2 + 32 + lane);

  const bool writer = wg == 0 && lane < SL && b0 + lane < g.B;
  const int my_b = b0 + lane;
  float lp = 0.0f;
  bool ok = true;
  WT* sx = reinterpret_cast<WT*>(g.sx);
  WT* stt = reinterpret_cast<WT*>(g.st);

  int cs = 0;         // ring stage of the current block
  uint32_t cpar = 0;  // phase parity of that stage's current fill
  for (int i = 1; i <= n; ++i) {
    const int t = i - 1;
    if (t % UWIN == 0) {
      if (g.u) {
#pragma unroll
        for (int e = 0; e < 4; ++e) uw[e] = unx[e];
        if (t + UWIN < n) load_u(t + UWIN, unx);
      } else {
        const uint4 r = philox4x32_10(make_uint4((uint32_t)((t + 4 * ug) >> 2), (uint32_t)ub, g.it0, g.it1), g.key0,
                                      g.key1);
        uw[0] = r.x, uw[1] = r.y, uw[2] = r.z, uw[3] = r.w;
      }
    }
    if ((t & 31) == 0 && t > 0) {
      cw = cnx;
      cnx = (t + 32 + lane < n) ? __ldg(g.b2 + t + 32 + lane) : 0.0f;
    }
    while (nd < U2 && thr_nd <= i - 2) {
      ++nd;
      thr_nd = nd < U2 ? K::deg(kw + nd * 2 * GL + 63, n, h) : kBig;
      m0 = nd < U2 ? K::deg(2 * (L + nd * GL), n, h) : kBig;
      m1 = nd < U2 ? K::deg(2 * (L + nd * GL) + 1, n, h) : kBig;
    }
    while (nt < U2 && thr_nt <= i - 1) {
      ++nt;
      thr_nt = nt < U2 ? K::deg(kw + nt * 2 * GL, n, h) : kBig;
    }

    const int ro = t % SPS;
    if (ro == 0 && t > 0 && ++cs == nst) cs = 0, cpar ^= 1u;
    const int s = cs;
    if (ro == 0) {
      const uint32_t fb = smem_u32(&full[s]), par = cpar;
      bool got = false;
      if (warp == NCW - 1) {
        // the producer's warp never suspends: lane 0 keeps refilling
        for (long long it = 0; it < kSpinLimit && !got; ++it) {
          if (producer) refill();
          got = mbar_test_wait(fb, par);
        }
      } else {
        for (long long it = 0; it < kSpinLimit && !got; ++it) got = mbar_try_wait(fb, par);
      }
      if (!got) {
        atomicOr(g.err, kErrTimeout);
        ok = false;
        break;
      }
    }
    const WT* wrow = stages + (size_t)s * stage_elems + ro * hp;
    const WT* vrow = wrow + SPS * hp;
#pragma unroll
    for (int q = 0; q < SL; ++q) st.acc[q] = pack2(0.0f, 0.0f);
    if (nt <= nd + 1) K::template dispatch<0, 2 * U2>(2 * nd + (nt - nd), st, wrow, vrow, L, i, m0, m1);
    else K::body_general(st, wrow, vrow, L, i, n, h);
    if (ro == SPS - 1 || i == n) {
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&empty[s]));
    }

    // z_i: lanes -> warp (shuffles) -> group (shared memory + named barrier)
    float v[SL];
#pragma unroll
    for (int q = 0; q < SL; ++q) {
      float lo, hi;
      unpack2(st.acc[q], lo, hi);
      v[q] = lo + hi;
    }
    int qs;
    const float ws = K::reduce_scatter(v, lane, qs);
    float* rb = gred + (size_t)(t & 1) * NGRP * GW * SL;
    if ((lane & (32 / SL - 1)) == 0) rb[wg * SL + qs] = ws;
    if constexpr (GW > 1) asm volatile("bar.sync %0, %1;" ::"r"(1 + grp), "r"(GW * 32) : "memory");
    else __syncwarp();
    float z = __shfl_sync(FULL, cw, t & 31);
    if (lane < SL) {
#pragma unroll
      for (int w = 0; w < GW; ++w) z += rb[w * SL + lane];
    }
    const int src = ((t % UWIN) >> 2) * SL + (lane < SL ? lane : 0);
    const int e = t & 3;
    const uint32_t wsel = e == 0 ? uw[0] : e == 1 ? uw[1] : e == 2 ? uw[2] : uw[3];
    const uint32_t uword = __shfl_sync(FULL, wsel, src);
    const float u = g.u ? __uint_as_float(uword) : to_unit(uword);
    const float p = 1.0f / (1.0f + expf(-z));
    const bool up = u < p;
    const uint32_t mask = __ballot_sync(FULL, up);
#pragma unroll
    for (int q = 0; q < SL; ++q) {
      const float sv = ((mask >> q) & 1u) ? 1.0f : -1.0f;
      st.sg[q] = pack2(sv, sv);
    }
    if (writer) {
      const float sv = up ? 1.0f : -1.0f;
      if (g.logp) lp += log_sigmoid(up ? z : -z);
      g.s_out[(size_t)my_b * n + t] = up ? (int8_t)1 : (int8_t)-1;
      if (sx) sx[(size_t)my_b * g.ldsx + t] = from_f<WT>(sv);
      if (stt) stt[(size_t)t * g.ldst + my_b] = from_f<WT>(sv);
    }
  }
  if (!ok && producer) {
    // drain: wait (bounded) for every copy still in flight before exiting
    for (int q = issued - nst > 0 ? issued - nst : 0; q < issued; ++q)
      if (!mbar_wait(smem_u32(&full[q % nst]), (uint32_t)((q / nst) & 1), g.err)) break;
  }
  if (ok && writer && g.logp) g.logp[my_b] = lp;
}

template <typename WT, int GW, int NGRP, int U2, int SL, int ACT>
cudaError_t launch_cfg(const SamplerArgs& a, cudaStream_t st) {
  using K = Sampler<WT, GW, NGRP, U2, SL, ACT>;
  SamplerArgs b = a;
  b.nst = K::stages_for(a.hp);
  if (b.nst < 2) return cudaErrorNotSupported;
  const size_t smem = K::smem_bytes(a.hp, b.nst);
  auto kern = sampler_kernel<WT, GW, NGRP, U2, SL, ACT>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int grid = (a.B + K::S - 1) / K::S;
  kern<<<grid, K::NT, smem, st>>>(b);
  return cudaGetLastError();
}

template <typename WT, int ACT>
cudaError_t launch_shape(const SamplerArgs& a, cudaStream_t st) {
  // units covered by a group (GW*32 lanes x 2*U2) must be >= hp
  if (a.hp <= 64) return launch_cfg<WT, 1, 2, 1, 8, ACT>(a, st);
  if (a.hp <= 512) return launch_cfg<WT, 1, 2, 8, 8, ACT>(a, st);
  if (a.hp <= 1024) return launch_cfg<WT, 2, 2, 8, 8, ACT>(a, st);
  if (a.hp <= 2048) return launch_cfg<WT, 2, 4, 16, 4, ACT>(a, st);
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
