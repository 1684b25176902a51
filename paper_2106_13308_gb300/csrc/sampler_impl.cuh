// Implementation of the persistent sampler kernel, included by one
// translation unit per weight type (sampler_bf16.cu, sampler_f32.cu).
#pragma once

#include "sampler.cuh"

namespace vqmc {

namespace {


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

// Weights of units (2q, 2q+1) of a staged row: raw (as stored) and as an
// FP32 pair.  BF16 widens exactly by a shift.
template <typename T>
struct Pair;
template <>
struct Pair<bf16> {
  using raw = uint32_t;
  static __device__ __forceinline__ raw ld(const bf16* row, int q) { return reinterpret_cast<const uint32_t*>(row)[q]; }
  static __device__ __forceinline__ uint64_t f32(raw x) {
    return pack2(__uint_as_float(x << 16), __uint_as_float(x & 0xffff0000u));
  }
};
template <>
struct Pair<float> {
  using raw = uint64_t;
  static __device__ __forceinline__ raw ld(const float* row, int q) { return reinterpret_cast<const uint64_t*>(row)[q]; }
  static __device__ __forceinline__ uint64_t f32(raw x) { return x; }
};
template <typename T>
__device__ __forceinline__ uint64_t ld_pair(const T* row, int q) {
  return Pair<T>::f32(Pair<T>::ld(row, q));
}



// A CTA = NGRP groups of GW warps.  Group g owns
// SL samples; its GW*32 lanes split the hidden units: lane L of the group
// holds unit pairs q = r*GW*32 + L (units 2q, 2q+1), r = 0..U2-1, for all SL
// samples.  Per step a group reduces its partial sums with shuffles and one
// named barrier of its own warps; groups never wait for each other.  Lane 0
// of the last warp also keeps the weight ring filled: whenever every warp
// has released a stage it issues the copies for the block a full ring ahead.
template <typename WT, int GW, int NGRP, int U2, int SL>
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

  // hidden activation as the output layer sees it: rounded to bfloat16 in
  // the BF16 model (as the BF16 forward GEMM stores it), exact in FP32
  static __device__ __forceinline__ float g1(int g_act, float a) {
    const float g = act_f(g_act, a);
    if constexpr (sizeof(WT) == 2) return __bfloat162float(__float2bfloat16_rn(g));
    else return g;
  }

  // Mixed slot: the lane's two units may be in different roles.  Weights of
  // units that must not take part are zeroed, so the pair still runs as f32x2.
  // (At i = 1 the spins are still zero, so the update adds nothing.)
  static __device__ __forceinline__ void mixed(State& st, uint64_t wpair, uint64_t vpair, int r, int i, int m0,
                                               int m1, int g_act) {
    if (m0 >= i - 1 || m1 >= i - 1) {
      float w0, w1;
      unpack2(wpair, w0, w1);
      const uint64_t w = pack2(m0 >= i - 1 ? w0 : 0.0f, m1 >= i - 1 ? w1 : 0.0f);
#pragma unroll
      for (int s = 0; s < SL; ++s) st.a[r][s] = fma2(w, st.sg[s], st.a[r][s]);
    }
    if (m0 == i - 1 || m1 == i - 1) {
#pragma unroll
      for (int s = 0; s < SL; ++s) {
        float a0, a1;
        unpack2(st.a[r][s], a0, a1);
        if (m0 == i - 1) a0 = g1(g_act, a0);
        if (m1 == i - 1) a1 = g1(g_act, a1);
        st.a[r][s] = pack2(a0, a1);
      }
    }
    if (m0 <= i - 1) {
      float v0, v1;
      unpack2(vpair, v0, v1);
      const uint64_t v = pack2(v0, m1 <= i - 1 ? v1 : 0.0f);
#pragma unroll
      for (int s = 0; s < SL; ++s) st.acc[s] = fma2(v, st.a[r][s], st.acc[s]);
    }
  }

  // Slots r < ND: every unit complete -> dot.  MIX: slot ND is mixed.
  // Remaining slots: every unit still accumulating -> update.  wp[r] holds
  // the W2 pair of a dot slot and the W1 pair of the others; wq the W2 pair
  // of the mixed slot.
  using PR = typename Pair<WT>::raw;
  template <int ND, bool MIX>
  static __device__ __forceinline__ void body(State& st, const PR (&wp)[U2], PR wq, int i, int m0, int m1,
                                              int g_act) {
#pragma unroll
    for (int r = 0; r < ND && r < U2; ++r) {
      const uint64_t w = Pair<WT>::f32(wp[r]);
#pragma unroll
      for (int s = 0; s < SL; ++s) st.acc[s] = fma2(w, st.a[r][s], st.acc[s]);
    }
    constexpr int FIRST_UPD = MIX ? ND + 1 : ND;
    if constexpr (MIX && ND < U2) mixed(st, Pair<WT>::f32(wp[ND]), Pair<WT>::f32(wq), ND, i, m0, m1, g_act);
#pragma unroll
    for (int r = FIRST_UPD; r < U2; ++r) {
      const uint64_t w = Pair<WT>::f32(wp[r]);
#pragma unroll
      for (int s = 0; s < SL; ++s) st.a[r][s] = fma2(w, st.sg[s], st.a[r][s]);
    }
  }

  // the pairs body<ND, MIX> reads, from the staged rows of its step
  template <int ND, bool MIX>
  static __device__ __forceinline__ void load(PR (&wp)[U2], PR& wq, const WT* wrow, const WT* vrow, int lq) {
#pragma unroll
    for (int r = 0; r < U2; ++r) wp[r] = Pair<WT>::ld(r < ND ? vrow : wrow, lq + r * GL);
    if constexpr (MIX && ND < U2) wq = Pair<WT>::ld(vrow, lq + ND * GL);
  }

  // every slot treated as mixed (small n or h >> n)
  static __device__ __forceinline__ void body_general(State& st, const WT* wrow, const WT* vrow, int lq, int i,
                                                      int n, int h, int g_act) {
#pragma unroll
    for (int r = 0; r < U2; ++r) {
      const int q = lq + r * GL;
      mixed(st, ld_pair(wrow, q), ld_pair(vrow, q), r, i, deg(2 * q, n, h), deg(2 * q + 1, n, h), g_act);
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

// The per-warp step loop.  Slot roles (how many slots are complete, whether
// one is mixed) change only every few hundred steps, so the kernel runs the
// steps of one phase in a loop specialised for that phase, and re-dispatches
// between phases.
template <typename WT, int GW, int NGRP, int U2, int SL>
struct Run {
  using K = Sampler<WT, GW, NGRP, U2, SL>;
  static constexpr int SPS = K::SPS, UWIN = K::UWIN, GL = K::GL, NCW = K::NCW;

  const SamplerArgs& g;
  typename K::State st;
  WT* stages;
  uint64_t* full;
  int* relcnt;
  int* fills;
  float* gred;
  const WT* gwt;
  const WT* gv;
  int stage_elems, hp, n, h, nst, nblocks;
  uint32_t block_bytes;
  int L, lane, wg, grp, b0, my_b, ub, ug;
  bool writer, uvalid, ok;
  float uw[4], unx[4];  // logits of this window / uniforms of the next (explicit mode)
  float cw, cnx;        // b2 of this / the next 32 steps, lane l holds step win+l
  float lp;
  uint32_t bits;        // drawn spins of the current 32-step window (writer lanes)
  int cs;               // ring stage holding the current step's rows
  uint32_t cpar;        // its fill parity
  int i;                // next step (1-based)
  int m0, m1;           // degrees of this lane's units in the mixed slot
  typename K::PR wp[U2], wq;  // this step's weight pairs, loaded one step ahead

  uint32_t it0, it1;    // Philox iteration words

  __device__ __forceinline__ Run(const SamplerArgs& a) : g(a) {
    const unsigned long long it = a.it_dev ? *a.it_dev : ((unsigned long long)a.it1 << 32 | a.it0);
    it0 = (uint32_t)it, it1 = (uint32_t)(it >> 32);
  }

  __device__ __forceinline__ void issue(int q) {
    const int s = q % nst;
    const uint32_t bar = smem_u32(&full[s]);
    WT* dst = stages + (size_t)s * stage_elems;
    fills[s] += 1;
    mbar_expect_tx(bar, 2 * block_bytes);
    bulk_g2s(smem_u32(dst), gwt + (size_t)q * SPS * hp, block_bytes, bar);
    bulk_g2s(smem_u32(dst + SPS * hp), gv + (size_t)q * SPS * hp, block_bytes, bar);
  }

  __device__ __forceinline__ const WT* wrow_of(int t) const { return stages + (size_t)cs * stage_elems + (t & (SPS - 1)) * hp; }

  // bounded wait for the current stage's copies
  __device__ __forceinline__ void wait_stage() {
    const uint32_t fb = smem_u32(&full[cs]);
    bool got = !ok;
    for (long long it = 0; it < kSpinLimit && !got; ++it) got = mbar_try_wait(fb, cpar);
    if (!got) {
      atomicOr(g.err, kErrTimeout);
      ok = false;  // run on without waiting: every warp still reaches every named barrier
    }
  }

  __device__ __forceinline__ void load_u(int win, float (&dst)[4]) {
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int t = win + 4 * ug + e;
      dst[e] = (uvalid && t < n) ? __ldg(g.u + (size_t)ub * n + t) : 0.5f;
    }
  }

  // writes the spins of the window ending at step t (0-based) as int8 +-1
  __device__ __forceinline__ void flush(int t) {
    const int w0 = t & ~31, len = t - w0 + 1;
    int8_t* dst = g.s_out + (size_t)my_b * n + w0;
    if (len == 32 && ((reinterpret_cast<uintptr_t>(dst) & 15) == 0)) {
      uint32_t wd[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        // byte e of word k = +1 if bit 4k+e is set, else -1 (0xFF)
        const uint32_t spread = (((bits >> (4 * k)) & 0xFu) * 0x00204081u) & 0x01010101u;
        wd[k] = 0xFFFFFFFFu - 0xFEu * spread;
      }
      reinterpret_cast<uint4*>(dst)[0] = make_uint4(wd[0], wd[1], wd[2], wd[3]);
      reinterpret_cast<uint4*>(dst)[1] = make_uint4(wd[4], wd[5], wd[6], wd[7]);
    } else {
      for (int e = 0; e < len; ++e) dst[e] = ((bits >> e) & 1u) ? (int8_t)1 : (int8_t)-1;
    }
  }

  // One step.  The weights of step i were loaded during step i-1; this step
  // loads those of step i+1 right after its own FMAs, so the shared-memory
  // latency hides behind the reduction and the draw.
  template <int ND, bool MIX, bool GEN>
  __device__ __forceinline__ void step() {
    const int t = i - 1;
    if ((t & (UWIN - 1)) == 0) {
      if (g.u) {
#pragma unroll
        for (int e = 0; e < 4; ++e) uw[e] = logit(unx[e]);
        if (t + UWIN < n) load_u(t + UWIN, unx);
      } else {
        const uint4 r = philox4x32_10(make_uint4((uint32_t)((t + 4 * ug) >> 2), (uint32_t)ub + g.boff, it0, it1), g.key0,
                                      g.key1);
        uw[0] = logit(to_unit(r.x)), uw[1] = logit(to_unit(r.y));
        uw[2] = logit(to_unit(r.z)), uw[3] = logit(to_unit(r.w));
      }
    }
    if ((t & 31) == 0 && t > 0) {
      cw = cnx;
      cnx = (t + 32 + lane < n) ? __ldg(g.b2 + t + 32 + lane) : 0.0f;
    }
    const int ro = t & (SPS - 1);
#pragma unroll
    for (int q = 0; q < SL; ++q) st.acc[q] = pack2(0.0f, 0.0f);
    if constexpr (GEN) {
      const WT* wrow = wrow_of(t);
      K::body_general(st, wrow, wrow + SPS * hp, L, i, n, h, g.act);
    } else {
      K::template body<ND, MIX>(st, wp, wq, i, m0, m1, g.act);
    }
    if (ro == SPS - 1 || i == n) {
      // done with the stage; the last warp to release it refills it
      __syncwarp();
      if (lane == 0) {
        __threadfence_block();
        if (atomicAdd(&relcnt[cs], 1) == NCW - 1) {
          __threadfence_block();
          relcnt[cs] = 0;
          const int q = t / SPS + nst;
          if (q < nblocks) issue(q);
        }
      }
    }
    if (i < n) {
      if (ro == SPS - 1) {
        if (++cs == nst) cs = 0, cpar ^= 1u;
        wait_stage();
      }
      if constexpr (!GEN) {
        // next step's pairs, with this phase's roles (a new phase reloads)
        const WT* wrow = wrow_of(t + 1);
        K::template load<ND, MIX>(wp, wq, wrow, wrow + SPS * hp, L);
      }
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
    const int e = t & 3;
    const float lsel = e == 0 ? uw[0] : e == 1 ? uw[1] : e == 2 ? uw[2] : uw[3];
    const float lg = __shfl_sync(0xffffffffu, lsel, ((t & (UWIN - 1)) >> 2) * SL + (lane & (SL - 1)));
    float z = __shfl_sync(0xffffffffu, cw, t & 31);
    if constexpr (GW > 1) asm volatile("barrier.sync %0, %1;" ::"r"(1 + grp), "r"(GW * 32) : "memory");
    else __syncwarp();
    // lanes >= SL compute a copy of lane (lane % SL)'s value; only bits < SL are used
#pragma unroll
    for (int w = 0; w < GW; ++w) z += rb[w * SL + (lane & (SL - 1))];
    const bool up = z > lg;  // u < sigma(z)
    const uint32_t mask = __ballot_sync(0xffffffffu, up);
#pragma unroll
    for (int q = 0; q < SL; ++q) {
      const float sv = ((mask >> q) & 1u) ? 1.0f : -1.0f;
      st.sg[q] = pack2(sv, sv);
    }
    bits |= (up ? 1u : 0u) << (t & 31);
    if (g.logp && writer) lp += log_sigmoid(up ? z : -z);
    if ((t & 31) == 31 || i == n) {
      if (writer) flush(t);
      bits = 0;
    }
    ++i;
  }

  template <int ND, bool MIX, bool GEN>
  __device__ __forceinline__ void steps(int i_end) {
    if constexpr (!GEN) {
      const WT* wrow = wrow_of(i - 1);
      K::template load<ND, MIX>(wp, wq, wrow, wrow + SPS * hp, L);
    }
    while (i < i_end) step<ND, MIX, GEN>();
  }

  // code = 2*nd + mixed, nd in [0, U2]
  template <int LO, int HI>
  __device__ __forceinline__ void dispatch(int code, int i_end) {
    if constexpr (LO == HI) {
      steps<LO / 2, (LO & 1) != 0, false>(i_end);
    } else {
      constexpr int MID = (LO + HI) / 2;
      if (code <= MID) dispatch<LO, MID>(code, i_end);
      else dispatch<MID + 1, HI>(code, i_end);
    }
  }
};

template <typename WT, int GW, int NGRP, int U2, int SL>
__global__ void __launch_bounds__(GW * NGRP * 32, 1) sampler_kernel(const SamplerArgs g) {
  using K = Sampler<WT, GW, NGRP, U2, SL>;
  constexpr int RL = K::RL, SPS = K::SPS, GL = K::GL;
  extern __shared__ __align__(128) unsigned char smem[];
  const int nst = g.nst, hp = g.hp;
  const int stage_elems = 2 * SPS * hp;  // W1^T rows then W2 rows
  // ring, then RL elements of slack: lanes holding padding units (k >= hp)
  // read past their row, never past the ring
  const int ring_elems = nst * stage_elems + RL;
  WT* stages = reinterpret_cast<WT*>(smem);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + ((size_t)ring_elems * sizeof(WT) + 7) / 8 * 8);
  int* relcnt = reinterpret_cast<int*>(full + 8);     // [8] warps that released each stage
  int* fills = relcnt + 8;                            // [8] copies issued into each stage
  int* failed = fills + 8;                            // some warp gave up a wait
  float* red = reinterpret_cast<float*>(fills + 12);  // [2][NGRP][GW][SL]

  const int n = g.n, h = g.h;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  // zero the ring once: every value a lane may read must be finite
  for (int q = tid; q < ring_elems; q += K::NT) stages[q] = from_f<WT>(0.0f);
  if (tid == 0) {
    for (int s = 0; s < nst; ++s) {
      mbar_init(smem_u32(&full[s]), 1);
      relcnt[s] = 0;
      fills[s] = 0;
    }
    *failed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncthreads();

  Run<WT, GW, NGRP, U2, SL> R(g);
  R.stages = stages, R.full = full, R.relcnt = relcnt, R.fills = fills;
  R.gwt = reinterpret_cast<const WT*>(g.wt);
  R.gv = reinterpret_cast<const WT*>(g.v);
  R.stage_elems = stage_elems, R.hp = hp, R.n = n, R.h = h, R.nst = nst;
  R.nblocks = (n + SPS - 1) / SPS;
  R.block_bytes = (uint32_t)(SPS * hp * sizeof(WT));
  // Stage q % nst holds block q: rows q*SPS.. of wt_s (row j = input j, row 0
  // zero) and of v_s (row i = output i+1), copied whole.  The warp that
  // releases a stage last issues the copies of the block a full ring ahead.
  if (tid == 0)
    for (int q = 0; q < nst && q < R.nblocks; ++q) R.issue(q);

  const int grp = warp / GW, wg = warp % GW;
  R.grp = grp, R.wg = wg, R.lane = lane;
  R.L = wg * 32 + lane;
  R.b0 = blockIdx.x * K::S + grp * SL;
  R.gred = red + (size_t)grp * GW * SL;
#pragma unroll
  for (int r = 0; r < U2; ++r) {
    const int k = 2 * (r * GL + R.L);
    const float x0 = k < h ? __ldg(g.b1 + k) : 0.0f;
    const float x1 = k + 1 < h ? __ldg(g.b1 + k + 1) : 0.0f;
#pragma unroll
    for (int s = 0; s < SL; ++s) R.st.a[r][s] = pack2(x0, x1);
  }
#pragma unroll
  for (int s = 0; s < SL; ++s) R.st.sg[s] = pack2(0.0f, 0.0f);
  // uniforms: lane l (< 32) holds 4 words for sample l % SL, steps
  // win + 4*(l / SL) .. +3 of the current window
  R.ug = lane / SL;
  R.ub = R.b0 + lane % SL;
  R.uvalid = R.ub < g.B;
#pragma unroll
  for (int e = 0; e < 4; ++e) R.uw[e] = 0.0f, R.unx[e] = 0.5f;
  if (g.u) R.load_u(0, R.unx);
  R.cw = lane < n ? __ldg(g.b2 + lane) : 0.0f;
  R.cnx = 32 + lane < n ? __ldg(g.b2 + 32 + lane) : 0.0f;
  R.my_b = R.b0 + lane;
  R.writer = wg == 0 && lane < SL && R.my_b < g.B;
  R.ok = true;
  R.lp = 0.0f;
  R.bits = 0;
  R.cs = 0, R.cpar = 0;
  R.i = 1;
  R.wait_stage();

  // warp-uniform slot bookkeeping: nd = #slots complete before step i, nt =
  // #slots with at least one unit complete at step i; thresholds are the
  // degrees of the next slot's last / first unit
  const int kw = 2 * wg * 32;  // first unit of the warp in slot 0
  int nd = 0, nt = 0;
  int thr_nd = K::deg(kw + 63, n, h), thr_nt = K::deg(kw, n, h);
  while (R.i <= n) {
    const int i = R.i;
    while (nd < U2 && thr_nd <= i - 2) {
      ++nd;
      thr_nd = nd < U2 ? K::deg(kw + nd * 2 * GL + 63, n, h) : kBig;
    }
    while (nt < U2 && thr_nt <= i - 1) {
      ++nt;
      thr_nt = nt < U2 ? K::deg(kw + nt * 2 * GL, n, h) : kBig;
    }
    // the phase lasts until nd or nt next changes
    long long end = (long long)n + 1;
    if (thr_nd < kBig && thr_nd + 2 < end) end = thr_nd + 2;
    if (thr_nt < kBig && thr_nt + 1 < end) end = thr_nt + 1;
    const int i_end = (int)end;
    R.m0 = nd < U2 ? K::deg(2 * (R.L + nd * GL), n, h) : kBig;
    R.m1 = nd < U2 ? K::deg(2 * (R.L + nd * GL) + 1, n, h) : kBig;
    if (nt <= nd + 1) R.template dispatch<0, 2 * U2>(2 * nd + (nt - nd), i_end);
    else R.template steps<0, false, true>(i_end);
  }

  // Every warp runs all n steps, so this barrier is reached by all.  After a
  // failed wait, copies may still be in flight: drain them before exiting.
  if (!R.ok) *failed = 1;
  __syncthreads();
  if (tid == 0 && *failed)
    for (int s = 0; s < nst; ++s)
      if (fills[s] > 0 && !mbar_wait(smem_u32(&full[s]), (uint32_t)((fills[s] - 1) & 1), g.err)) break;
  if (R.ok && R.writer && g.logp) g.logp[R.my_b] = R.lp;
}

template <typename WT, int GW, int NGRP, int U2, int SL>
cudaError_t launch_cfg(const SamplerArgs& a, cudaStream_t st) {
  using K = Sampler<WT, GW, NGRP, U2, SL>;
  SamplerArgs b = a;
  b.nst = K::stages_for(a.hp);
  if (b.nst < 2) return cudaErrorNotSupported;
  const size_t smem = K::smem_bytes(a.hp, b.nst);
  auto kern = sampler_kernel<WT, GW, NGRP, U2, SL>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int grid = (a.B + K::S - 1) / K::S;
  kern<<<grid, K::NT, smem, st>>>(b);
  return cudaGetLastError();
}

}  // namespace

// Shapes: a group covers GW*32 lanes x 2*U2 units >= hp; 16 samples per CTA
// up to hp = 2048.  Beyond, four warps per group and 2 samples per group (4
// per CTA) keep the pre-activations in about 140 registers per thread; the
// ring then holds two stages of SPS rows when they fit the shared memory
// (BF16 up to hp = 5120, FP32 up to hp = 2816).
template <typename WT>
cudaError_t launch_sampler_wt(const SamplerArgs& a, cudaStream_t st) {
  if (a.wide && a.hp <= 5120) return launch_cfg<WT, 4, 2, 20, 2>(a, st);
  if (a.hp <= 64) return launch_cfg<WT, 1, 2, 1, 8>(a, st);
  if (a.hp <= 1024) return launch_cfg<WT, 2, 2, 8, 8>(a, st);
  if (a.hp <= 2048) return launch_cfg<WT, 2, 4, 16, 4>(a, st);
  if (a.hp <= 5120) return launch_cfg<WT, 4, 2, 20, 2>(a, st);
  return cudaErrorNotSupported;
}

// Whether launch_sampler_wt<WT> runs models with hp padded hidden units.
template <typename WT>
bool sampler_wt_supports(int hp, bool wide) {
  if (hp <= 2048 && !wide) return true;
  if (hp <= 5120) return Sampler<WT, 4, 2, 20, 2>::stages_for(hp) >= 2;
  return false;
}

}  // namespace vqmc
