// Blocked autoregressive sampler on the tcgen05 tensor cores, for the BF16
// model (BF16 weights, hidden activations rounded to BF16, FP32 accumulation).
//
// Algorithm 1 draws s_1 .. s_n in order; with the incremental forward pass
// (Sec. 2.3) the logit of step i is
//     z_i = b2_i + sum_{k : m(k) < i} W2_ik g1_k,
//     g1_k = act(b1_k + sum_{j <= m(k)} W1_kj s_j),
// and with sorted degrees a hidden unit is complete once s_{m(k)} is drawn.
// This kernel processes the n steps in blocks of D (64 or 128).  For block
// [i0, i0 + D):
//   * units complete before the block (m(k) < i0, a prefix of the units)
//     feed every output of the block through one tensor-core GEMM,
//         Z[i][s] = sum_k W2[i][k] g1[k][s]     (M = 128 outputs, N = 16
//     samples, K = that prefix), with g1 kept in shared memory in BF16;
//   * the few units completing inside the block (m(k) in [i0, i0 + D), at
//     most 32: the "recent" units) are carried by a small sequential solver
//     that draws the D spins: z_i = Z[i] + b2_i + sum_recent W2_ik g1_k, with
//     each recent pre-activation extended by W1_ki s_i after every draw;
//   * the block's spins then update every unit still incomplete by a second
//     tensor-core GEMM, A[k][s] += sum_j W1[k][j] s_j over the block's inputs
//     (M = 128 units, N = 16, K = D), into FP32 accumulators that stay in
//     tensor memory for the whole run (16 columns per 128 units).
// The masks need no special handling: masked weights are stored as zeros, so
// an update adds nothing to a complete unit and an incomplete unit (g1 = 0
// in shared memory until it completes) adds nothing to any logit.
//
// CTA = 16 samples, 8 warps: warps 0-3 own TMEM lanes 32w..32w+31 (read Z
// and the recent pre-activations); warps 0, 1, 6 and 7 are the solver (8
// lanes per sample, each lane owning every 8th step of a segment and partial
// sums of all the block's recent units) and then write the block's spins as
// the update GEMM's operand; while they solve, warps 2-3 merge the previous
// block's recent g1 into the Z operand, prepare the next block's logits and
// recent-unit weights and write out the previous block's spins; warp 4 lane 0
// streams 128 x 64 BF16 weight tiles with TMA into a ring of six tiles,
// consumed in two slots of three; warp 5 lane 0 issues the MMAs.  Every wait is bounded; after a failed wait the CTA
// raises the timeout bit and runs on without waiting, so it still finishes.
#include <algorithm>
#include <type_traits>

#include "gemm.cuh"
#include "sampler.cuh"
#include "tc_ptx.cuh"

namespace vqmc {
namespace {

using namespace tc;

constexpr int kS = 16;                     // samples per CTA (MMA N)
constexpr int kRmax = 32;                  // recent units per block
constexpr int kNStage = 6;                 // weight tiles in the ring
constexpr int kTileBytes = 128 * 64 * 2;   // one 128 x 64 BF16 tile
// The ring is consumed in slots of up to three tiles (48 KB): one
// full-barrier wait and one commit per slot.  The single thread that issues
// the MMAs pays a fixed cost for every wait and every commit, comparable to
// the tensor work of an N = 16 tile, so grouping tiles cuts the time per
// tile.  A slot's tiles that are consecutive 64-column chunks of the same
// rows arrive in one copy: the copy engine's time goes by copies more than by
// bytes (a 32 KB box streams about twice as fast as two 16 KB boxes).
constexpr int kSlotTiles = 3;
constexpr int kNSlot = kNStage / kSlotTiles;
constexpr int kMaxHp = 2048;               // hidden units (padded) in TMEM
constexpr int kDmax = 128;
constexpr int kTmemCols = 512;             // A: 16 per 128 units (<= 256), Z at 256
constexpr int kZCol = 256;
constexpr int kThreads = 256;
// The solver: kLanes lanes per sample on warps 0, 1, 6 and 7 (one warp on
// each SM sub-partition).
constexpr int kLanes = 8;
constexpr int kSolverThreads = kS * kLanes;
// named barriers: 1 = warps 0-3 and the solver warps, 2 = warps 2-3 (arrive)
// with the solver warps (sync)
constexpr int kBar1Threads = 128 + 64;
constexpr int kBar2Threads = 64 + kSolverThreads;
constexpr int kZld = kS + 1;               // padded row of the Z buffer
constexpr uint32_t kIdesc = idesc_bf16(128, kS);

// shared memory map (offsets from a 1024-byte aligned base)
constexpr int kOffRing = 0;
constexpr int kOffH = kOffRing + kNStage * kTileBytes;         // g1, [hp/64] x (16 x 64) swizzled
constexpr int kOffS = kOffH + (kMaxHp / 64) * 2048;            // spins, [2][D/64] x (16 x 64) swizzled
// Per-step tables of the solver have kDrows = D + 4 rows (the rows past the
// block are zero) so that it reads up to 3 steps ahead without clamping.  In
// the recent-unit tables column kRmax is zero and stands for "no unit".
constexpr int kDrows = kDmax + 4;
constexpr int kLdW = kRmax + 8;                                // bf16 row of the recent-unit weight tables
constexpr int kLdP = kRmax + 4;                                // float row of the per-sample unit tables
constexpr int kOffHr = kOffS + 2 * (kDmax / 64) * 2048;        // g1 of the last block's recent units, 2 x (16 x 64)
constexpr int kOffZ = kOffHr + 2 * 2048;                       // Z + b2 [kDrows][kZld] float
constexpr int kOffLG = kOffZ + kDrows * kZld * 4;              // logit(u) [2][kDrows][16] float
constexpr int kOffP = kOffLG + 2 * kDrows * kS * 4;            // recent pre-activations at block start [32][16]
constexpr int kOffWr = kOffP + kRmax * kS * 4;                 // W1 of recent units [kDrows][kLdW] bf16
constexpr int kOffVr = kOffWr + kDrows * kLdW * 2;             // W2 of recent units [kDrows][kLdW] bf16
constexpr int kOffPS = kOffVr + kDrows * kLdW * 2;             // solver: g1 of the recent units [16][kLdP]
constexpr int kOffHF = kOffPS + kS * kLdP * 4;                 // (unused)
constexpr int kOffSB = kOffHF + kS * kLdP * 4;                 // drawn spins, bit e%32 of word [2][16][e/32]
constexpr int kOffCU = kOffSB + 2 * kS * (kDmax / 32) * 4;     // completion step of each recent unit, [kRmax] int
constexpr int kOffBar = kOffCU + (kDmax + 8) * 4;              // mbarriers + slots
constexpr int kSmemBytes = 1024 + kOffBar + 128;
static_assert(kSmemBytes <= 232448, "shared memory budget");

struct TcArgs {
  int n, h, hp, B, D, act;
  const bf16* w;      // w_s [h][np]: row k = W1[k] (column j-1 = input j)
  int np;
  const bf16* v;      // v_s  [rows][hp]: row r = W2[r] (output r + 1)
  const float* b1;
  const float* b2;
  const float* u;     // [B][n] or null (internal Philox)
  uint32_t key0, key1, it0, it1;
  uint32_t boff;      // index of sample 0 in the Philox counter (a shard's first global sample)
  const unsigned long long* it_dev;  // if not null: the Philox iteration, read on the device
  int8_t* s_out;      // [B][n]
  float* logp;        // [B] or null
  uint32_t* err;
  // optional copies of the spins for the rest of the step (null when absent):
  // GEMM operands Sx [B][ldsx] and St [n][ldst] (BF16 +-1) and the packed
  // layout of the sparse energy, bit l of 32-bit word [w][i] = [s_i of
  // sample 32 w + l is -1], written as 16-bit halves
  bf16* sx;
  int ldsx;
  bf16* stt;
  int ldst;
  uint16_t* sbits;
};

__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }
__device__ __forceinline__ float bf_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf_hi(uint32_t w) { return __uint_as_float(w & 0xffff0000u); }
// FP32 pairs for fma.rn.f32x2 (two IEEE FP32 FMAs per instruction)
__device__ __forceinline__ uint64_t pk2(float lo, float hi) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void upk2(uint64_t v, float& lo, float& hi) { asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v)); }
__device__ __forceinline__ uint64_t fma2(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
// the two BF16 weights of a word, widened (exactly) to an FP32 pair
__device__ __forceinline__ uint64_t bf2(uint32_t w) { return pk2(bf_lo(w), bf_hi(w)); }

// bounded wait that gives up at once after any failure in the CTA; with
// backoff the polling thread sleeps between tries so that it takes no issue
// slots from a busy warp on the same sub-partition
// The same wait polling with mbarrier.test_wait, which returns at once: for
// the MMA issuer's waits on landed tiles, which are usually already complete
// (a try_wait there costs the issuing thread about 190 cycles even then),
// and for the single threads of the producer and the MMA issuer on the
// block hand-offs, where a try_wait's suspension delays the reaction.
__device__ __forceinline__ bool test_or_abort(uint32_t bar, uint32_t parity, volatile int* abort, uint32_t* err) {
  for (long long it = 0; it < kSpinLimit; ++it) {
    if (mbar_test_wait(bar, parity)) return true;
    if ((it & 255) == 255 && *abort) return false;
  }
  atomicOr(err, kErrTimeout);
  *abort = 1;
  return false;
}
__device__ __forceinline__ bool wait_or_abort(uint32_t bar, uint32_t parity, volatile int* abort, uint32_t* err,
                                              bool backoff = false) {
  if (*abort) return false;
  for (long long it = 0; it < kSpinLimit; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 255) == 255 && *abort) return false;
    if (backoff) __nanosleep(64);
  }
  atomicOr(err, kErrTimeout);
  *abort = 1;
  return false;
}

template <int ACT>
__device__ __forceinline__ float g1f(float a) {
  if constexpr (ACT == VQMC_ACT_RELU) return fmaxf(a, 0.0f);
  else return 1.0f / (1.0f + expf(-a));
}

// The sequential part of a block: the draws of its D steps, carried for
// sample s by solver threads 8s .. 8s+7 (kLanes lanes of one warp of the
// solver warps 0, 1, 6 and 7).  With sorted degrees at most
// one hidden unit completes per step (h < n), and the logit of step e
// depends on the earlier spins only through the units completed before e:
//     z_e = (Z_e + b2) + sum_{recent r: t_r < e} W2_{e,r} g1_r,
// t_r the step whose spin is recent unit r's last input.  So the steps
// between two completions, (t_{r-1}, t_r], are conditionally independent
// given g1_0 .. g1_{r-1}: they form one segment, drawn in parallel.  Lane q
// of the sample's kLanes draws the steps e = q (mod kLanes) and keeps, for
// all 32 recent units, its own partial pre-activation sum over the spins it
// drew (lane 0 also holds the value at the start of the block).  When
// segment r ends, unit r's partials are added with log2(kLanes) shuffles,
// and g1_r = bf16(act(a_r)) enters
// the logits of the later segments.  The chain from one completion to the
// next is: the shuffle reduction, the activation and the rounding, one FMA
// with W2_{e,r} (the rest of the lane's next logit is summed before the
// reduction), the compare, and the lane's partial sum of unit r+1.  W2_{e,r}
// is zero for units not complete before step e and W1 for inputs after a
// unit's last one, so no masks are applied; g1 is zero (HH) until a unit
// completes.  HH holds each sample's recent g1 in shared memory (written by
// all the sample's lanes with the same value).
template <int ACT, bool LP>
__device__ __forceinline__ void solve(const float* Pr, const bf16* Vr, const bf16* Wr, const float* Zs,
                                      const float* LG, const int* TC, uint32_t* SB, float* HH, unsigned char* Hr,
                                      int s_me, int q, int klo, int R, int steps, float& lp) {
  float* hh = HH + s_me * kLdP;
  float P[kRmax];
#pragma unroll
  for (int k = 0; k < kRmax; ++k) P[k] = q == 0 ? Pr[k * kS + s_me] : 0.0f;
  static_assert(kLanes == 8 && kRmax == 32, "hh is zeroed as one float4 per lane");
  reinterpret_cast<float4*>(hh)[q] = make_float4(0.f, 0.f, 0.f, 0.f);
  __syncwarp();
  uint32_t w0 = 0, w1 = 0, w2 = 0, w3 = 0;  // this lane's drawn spins: bit e % 32 of word e / 32
  // The segments run in four phases by r / 8 (a template parameter PH of the
  // helpers below): in segment r only units 0 .. r-1 are complete (g1 != 0
  // in hh) and only units r .. 31 still need partial sums, so the logit's dot
  // product reads the 8-unit chunks 0 .. PH, the weight-row update writes the
  // chunks PH .. 3 and the completing unit's partial sum is one of 16 (8 in
  // the last phase).  The
  // skipped terms are zeros (g1 of incomplete units) or sums never read
  // again, so the draws are those of the full loops.
  // Z_e + b2 + the terms of the recent units completed so far (hh, chunks 0 .. PH)
  auto zdot = [&](auto ph, int e) -> float {
    constexpr int PH = decltype(ph)::value;
    const uint4* vr = reinterpret_cast<const uint4*>(Vr + e * kLdW);
    const float4* hv = reinterpret_cast<const float4*>(hh);
    // four FP32 accumulators a0..a3 as the pairs (a0, a1), (a2, a3)
    uint64_t a01 = pk2(Zs[e * kZld + s_me], 0.0f), a23 = pk2(0.0f, 0.0f);
#pragma unroll
    for (int c = 0; c <= PH; ++c) {
      const uint4 v = vr[c];
      const float4 x = hv[2 * c], y = hv[2 * c + 1];
      a01 = fma2(bf2(v.x), pk2(x.x, x.y), a01);
      a23 = fma2(bf2(v.y), pk2(x.z, x.w), a23);
      a01 = fma2(bf2(v.z), pk2(y.x, y.y), a01);
      a23 = fma2(bf2(v.w), pk2(y.z, y.w), a23);
    }
    float a0, a1, a2, a3;
    upk2(a01, a0, a1);
    upk2(a23, a2, a3);
    return (a0 + a1) + (a2 + a3);
  };
  // this lane's partial sums of the recent units of chunks PH .. 3 += sv * W1 of step row el
  auto wrow = [&](auto ph, int el, float sv) {
    constexpr int PH = decltype(ph)::value;
    const uint4* wr = reinterpret_cast<const uint4*>(Wr + el * kLdW);
    const uint64_t s2 = pk2(sv, sv);
#pragma unroll
    for (int c = PH; c < 4; ++c) {
      const uint4 w = wr[c];
      const uint32_t ww[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        uint64_t pp = pk2(P[8 * c + 2 * j], P[8 * c + 2 * j + 1]);
        pp = fma2(bf2(ww[j]), s2, pp);
        upk2(pp, P[8 * c + 2 * j], P[8 * c + 2 * j + 1]);
      }
    }
  };
  // draw of step e from its logit, and the spin into this lane's partial sums
  auto draw = [&](auto ph, int e, float z) {
    const bool up = z > LG[e * kS + s_me];  // u < sigma(z)
    const uint32_t m = up ? 1u << (e & 31) : 0u;
    const int wd = e >> 5;
    w0 |= wd == 0 ? m : 0u;
    w1 |= wd == 1 ? m : 0u;
    w2 |= wd == 2 ? m : 0u;
    w3 |= wd == 3 ? m : 0u;
    if constexpr (LP) lp += log_sigmoid(up ? z : -z);
    wrow(ph, e, up ? 1.0f : -1.0f);
  };
  // the partial sum of unit k among this lane's units 8 PH .. 8 PH + 15
  // (8 PH .. 31 in the last phase): a binary select by k - 8 PH
  auto extract = [&](auto ph, int k) -> float {
    constexpr int PH = decltype(ph)::value;
    constexpr int kB = 8 * PH, kN = PH < 3 ? 16 : 8;
    const int i = k - kB;
    float l1[kN / 2], l2[kN / 4], l3[kN / 8];
#pragma unroll
    for (int t = 0; t < kN / 2; ++t) l1[t] = (i & 1) ? P[kB + 2 * t + 1] : P[kB + 2 * t];
#pragma unroll
    for (int t = 0; t < kN / 4; ++t) l2[t] = (i & 2) ? l1[2 * t + 1] : l1[2 * t];
#pragma unroll
    for (int t = 0; t < kN / 8; ++t) l3[t] = (i & 4) ? l2[2 * t + 1] : l2[2 * t];
    if constexpr (kN == 16) return (i & 8) ? l3[1] : l3[0];
    else return l3[0];
  };
  auto wt = [&](int e, int r) { return r < kRmax ? __bfloat162float(Wr[e * kLdW + r]) : 0.0f; };
  auto vt = [&](int e, int r) { return r >= 0 ? __bfloat162float(Vr[e * kLdW + r]) : 0.0f; };
  auto allsum = [&](float x) {
#pragma unroll
    for (int d = 1; d < kLanes; d <<= 1) x += __shfl_xor_sync(0xffffffffu, x, d);
    return x;
  };
  // Prepared for this lane's step e of the current segment r (when the
  // segment has at most kLanes steps, a lane has at most one): its logit
  // without the unit completed last (zp), that unit's weight on it (vn),
  // logit(u) (lgn), unit r's weight on its spin (wn) and the lane's partial
  // sum of unit r over the earlier segments (xr).  Everything else of a
  // segment runs beside the chain of the completions.
  // The segment body below is free of lane-dependent branches: a lane
  // without a step in the segment (e past its end) draws nothing (sv = 0)
  // and reads row min(e, kDrows - 1) of the tables, so that the compiler can
  // move the next segment's loads ahead of the completion chain.
  using Ph0 = std::integral_constant<int, 0>;
  float g_last = 0.0f;  // g1 of the unit that completed last
  int lo = 0;
  int e = q;
  int hi = R > 0 ? TC[0] : steps - 1;  // last step of the current segment
  float zp = 0.0f, vn = 0.0f, lgn = 0.0f, wn = 0.0f, xr = 0.0f;
  if (e <= hi) zp = zdot(Ph0{}, e), lgn = LG[e * kS + s_me], wn = wt(e, 0);
  xr = extract(Ph0{}, 0);
  // segment r: steps [lo, hi], units 0 .. r-1 complete; true after the last (r = R)
  auto segment = [&](auto ph, int r) -> bool {
    const int nhi = r + 1 < R ? TC[r + 1] : steps - 1;  // last step of segment r + 1
    hh[r > 0 ? r - 1 : 0] = g_last;                     // (unit 0's entry is still zero at r = 0)
    float x;
    if (hi - lo + 1 <= kLanes) {
      // ---- at most one step per lane: the chain, then the rest
      const bool own = e <= hi;
      const int el = min(e, kDrows - 1);
      const float z = fmaf(vn, g_last, zp);
      const bool up = z > lgn;
      const float sv = own ? (up ? 1.0f : -1.0f) : 0.0f;
      x = allsum(fmaf(wn, sv, xr));
      const uint32_t m = (own && up) ? 1u << (e & 31) : 0u;
      const int wd = e >> 5;
      w0 |= wd == 0 ? m : 0u;
      w1 |= wd == 1 ? m : 0u;
      w2 |= wd == 2 ? m : 0u;
      w3 |= wd == 3 ? m : 0u;
      if constexpr (LP) lp += own ? log_sigmoid(up ? z : -z) : 0.0f;
      wrow(ph, el, sv);
    } else {
      // ---- a long segment: every step of the lane with its full logit,
      // then unit r's partial sums
      for (int ee = lo + ((q - lo) & (kLanes - 1)); ee <= hi; ee += kLanes) draw(ph, ee, zdot(ph, ee));
      x = allsum(extract(ph, r < kRmax ? r : kRmax - 1));
    }
    if (r == R) return true;
    // prepare this lane's step of segment r + 1 (hh holds units 0 .. r-1);
    // a lane without one (e > nhi) keeps values that its sv = 0 ignores
    const int nlo = hi + 1;
    e = nlo + ((q - nlo) & (kLanes - 1));
    {
      const int el = min(e, kDrows - 1);
      zp = zdot(ph, el);
      vn = vt(el, r);
      lgn = LG[el * kS + s_me];
      wn = wt(el, r + 1);
    }
    xr = extract(ph, r + 1 < kRmax ? r + 1 : kRmax - 1);
    g_last = bf16r(g1f<ACT>(x));
    lo = nlo;
    hi = nhi;
    return false;
  };
  bool last = false;
  int r = 0;
  for (; r < 8 && !last; ++r) last = segment(Ph0{}, r);
  for (; r < 16 && !last; ++r) last = segment(std::integral_constant<int, 1>{}, r);
  for (; r < 24 && !last; ++r) last = segment(std::integral_constant<int, 2>{}, r);
  for (; !last; ++r) last = segment(std::integral_constant<int, 3>{}, r);  // r <= R <= 32
  // the sample's spins: its lanes' words combined; lane q < 4 stores word q
#pragma unroll
  for (int d = 1; d < kLanes; d <<= 1) {
    w0 |= __shfl_xor_sync(0xffffffffu, w0, d);
    w1 |= __shfl_xor_sync(0xffffffffu, w1, d);
    w2 |= __shfl_xor_sync(0xffffffffu, w2, d);
    w3 |= __shfl_xor_sync(0xffffffffu, w3, d);
  }
  if (q < kDmax / 32) SB[s_me * (kDmax / 32) + q] = q == 0 ? w0 : q == 1 ? w1 : q == 2 ? w2 : w3;
  // every recent unit is complete: its g1 goes to the staging operand Hr
  // (2 chunks of 64 units from chunk klo / 64), once warps 2-3 have moved
  // the previous block's recent g1 out of it
  asm volatile("bar.sync 2, %0;" ::"n"(kBar2Threads) : "memory");
#pragma unroll
  for (int j = 0; j < kRmax / kLanes; ++j) {
    const int r = q + kLanes * j;
    if (r < R) {
      const int k = klo + r;
      *reinterpret_cast<bf16*>(Hr + ((k >> 6) - (klo >> 6)) * 2048 + sw128_offset(s_me, k & 63)) =
          __float2bfloat16_rn(hh[r]);
    }
  }
}

// The schedule of block b, computed alike by the producer, the MMA issuer
// and the compute warps.  Recent units of block b: [klo, khi).
struct Blk {
  int klo, khi;
  int crit0, crit1;  // update tiles needed before block b's solver (those of its recent units)
  int bulk0;         // further update tiles [bulk0, ntiles), overlapped with block b's solver
  int cor0, cor1;    // chunks of block b-1's recent units (Hr), added to Z of block b
  int np;            // chunks [0, np) of the Z GEMM of block b+1, run during block b's solver
  bool zinit;        // Z of block b was started during block b-1
  bool zvalid;       // Z of block b holds any term
};
__device__ __forceinline__ Blk blk_of(int b, int n, int h, int D, int ntiles, int nblk) {
  Blk r;
  r.klo = count_deg_le(b * D, n, h);
  r.khi = count_deg_le(b * D + D, n, h);
  const int kprev = b > 0 ? count_deg_le((b - 1) * D, n, h) : 0;
  if (b > 0 && r.khi > r.klo) r.crit0 = r.klo / 128, r.crit1 = (r.khi - 1) / 128 + 1;
  else r.crit0 = r.crit1 = r.klo / 128;
  r.bulk0 = (b > 0 && b + 1 < nblk) ? (r.crit1 > r.klo / 128 ? r.crit1 : r.klo / 128) : ntiles;
  if (b > 0 && r.klo > kprev) r.cor0 = kprev / 64, r.cor1 = (r.klo - 1) / 64 + 1;
  else r.cor0 = r.cor1 = 0;
  r.np = b + 1 < nblk ? (r.klo + 63) / 64 : 0;
  r.zinit = b > 0 && (kprev + 63) / 64 > 0;  // np of block b-1
  r.zvalid = r.zinit || r.cor1 > r.cor0;
  return r;
}

__global__ void __launch_bounds__(kThreads, 1)
    sampler_tc_kernel(const __grid_constant__ CUtensorMap mapV, const __grid_constant__ CUtensorMap mapW,
                      const __grid_constant__ CUtensorMap mapV2, const __grid_constant__ CUtensorMap mapV3,
                      const __grid_constant__ CUtensorMap mapW2, const TcArgs g) {
  extern __shared__ unsigned char smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  unsigned char* sm = smem_raw + (base - raw);
  unsigned char* Hs = sm + kOffH;
  unsigned char* Ss = sm + kOffS;
  unsigned char* Hr = sm + kOffHr;
  float* Zs = reinterpret_cast<float*>(sm + kOffZ);
  float* LG = reinterpret_cast<float*>(sm + kOffLG);
  float* Pr = reinterpret_cast<float*>(sm + kOffP);
  bf16* Wr = reinterpret_cast<bf16*>(sm + kOffWr);
  bf16* Vr = reinterpret_cast<bf16*>(sm + kOffVr);
  float* PreS = reinterpret_cast<float*>(sm + kOffPS);
  uint32_t* SB = reinterpret_cast<uint32_t*>(sm + kOffSB);
  int* CU = reinterpret_cast<int*>(sm + kOffCU);
  const unsigned long long it_all = g.it_dev ? *g.it_dev : ((unsigned long long)g.it1 << 32 | g.it0);
  const uint32_t it0 = (uint32_t)it_all, it1 = (uint32_t)(it_all >> 32);
  uint64_t* full = reinterpret_cast<uint64_t*>(sm + kOffBar);
  uint64_t* empty = full + kNStage;
  uint64_t* zfull = empty + kNStage;
  uint64_t* ready = zfull + 1;
  uint64_t* merged = ready + 1;
  uint64_t* drain = merged + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  volatile int* abort = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int n = g.n, h = g.h, D = g.D;
  const int nblk = (n + D - 1) / D;
  const int ntiles = (g.hp + 127) / 128;
  const int nkd = D / 64;
  const int b0 = blockIdx.x * kS;

  if (tid == 0) {
    for (int s = 0; s < kNStage; ++s) {
      mbar_init(smem_u32(&full[s]), 1);
      mbar_init(smem_u32(&empty[s]), 1);
    }
    mbar_init(smem_u32(zfull), 1);
    mbar_init(smem_u32(ready), kSolverThreads);
    mbar_init(smem_u32(merged), 64);
    mbar_init(smem_u32(drain), 1);
    *abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 5) tmem_alloc(smem_u32(tmem_slot), kTmemCols);
  // g1 of every unit is zero until the unit completes; spins start at zero
  // zero g1 (every unit is zero until it completes), the spins, and the
  // solver tables (their padding rows and "no unit" columns stay zero)
  for (int q = tid; q < (kOffSB - kOffH) / 16; q += kThreads) reinterpret_cast<uint4*>(Hs)[q] = make_uint4(0, 0, 0, 0);
  fence_proxy_async();
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;
  // A = b1 for every sample
  if (warp < 4) {
    for (int t = 0; t < ntiles; ++t) {
      const int k = 128 * t + 32 * warp + lane;
      const float x = k < h ? g.b1[k] : 0.0f;
      float v[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) v[q] = x;
      tmem_st16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(16 * t), v);
    }
  }
  fence_before();
  __syncthreads();
  fence_after();

  if (warp == 4) {
    // ----------------------------------------------------------- producer
    // Tiles in the MMA issuer's order; per block b: the update tiles needed
    // before its solver (W1, block b-1's inputs), the tiles of block b-1's
    // recent units (W2, block b's rows), the remaining update tiles, then the
    // Z GEMM of block b+1 over the units complete before block b (W2, block
    // b+1's rows).
    if (lane == 0) {
      int it = 0;  // slots issued
      // the tiles [i0, i1) of one phase, kSlotTiles per slot; yc(i, y, c)
      // gives tile i's first row and 64-column chunk.  A run of tiles with
      // the same rows and consecutive chunks (at most `most`) is one copy
      // through the chunked map of its length (m2: 2, m3: 3).
      auto load_phase = [&](const CUtensorMap* m1, const CUtensorMap* m2, const CUtensorMap* m3, int most, int i0,
                            int i1, auto yc) -> bool {
        for (int i = i0; i < i1; i += kSlotTiles) {
          const int cnt = min(kSlotTiles, i1 - i);
          const int s = it % kNSlot;
          if (it >= kNSlot &&
              !test_or_abort(smem_u32(&empty[s]), (uint32_t)((it / kNSlot - 1) & 1), abort, g.err))
            return false;
          const uint32_t bar = smem_u32(&full[s]);
          mbar_expect_tx(bar, (uint32_t)(cnt * kTileBytes));
          for (int j = 0; j < cnt;) {
            int y, c;
            yc(i + j, y, c);
            int run = 1;
            while (j + run < cnt && run < most) {
              int y2, c2;
              yc(i + j + run, y2, c2);
              if (y2 != y || c2 != c + run) break;
              ++run;
            }
            const uint32_t dst = base + kOffRing + (s * kSlotTiles + j) * kTileBytes;
            if (run == 1) tma_load_2d(dst, m1, 64 * c, y, bar);
            else tma_load_3d(dst, run == 2 ? m2 : m3, 0, y, c, bar);
            j += run;
          }
          ++it;
        }
        return true;
      };
      bool ok = true;
      for (int b = 0; b < nblk && ok; ++b) {
        const Blk B = blk_of(b, n, h, D, ntiles, nblk);
        // update tiles: index q -> unit tile q / nkd, K-chunk q % nkd of block b-1's inputs
        auto upd = [&](int q, int& y, int& c) { y = 128 * (q / nkd), c = (b - 1) * (D / 64) + q % nkd; };
        ok = load_phase(&mapW, &mapW2, &mapW2, 2, B.crit0 * nkd, B.crit1 * nkd, upd);
        if (ok)
          ok = load_phase(&mapV, &mapV2, &mapV3, 3, B.cor0, B.cor1, [&](int c, int& y, int& cc) { y = b * D, cc = c; });
        if (ok) ok = load_phase(&mapW, &mapW2, &mapW2, 2, B.bulk0 * nkd, ntiles * nkd, upd);
        if (ok)
          ok = load_phase(&mapV, &mapV2, &mapV3, 3, 0, B.np, [&](int c, int& y, int& cc) { y = (b + 1) * D, cc = c; });
      }
      // no copy may still be landing when the CTA exits (after a failure
      // some loaded tiles are never consumed)
      for (int p = it > kNSlot ? it - kNSlot : 0; p < it; ++p)
        mbar_wait(smem_u32(&full[p % kNSlot]), (uint32_t)((p / kNSlot) & 1), g.err);
    }
  } else if (warp == 5) {
    // --------------------------------------------------------- MMA issuer
    // Block b: after block b-1's solver, the update of block b's recent units
    // by block b-1's spins and the terms of block b-1's recent units in Z of
    // block b (commit -> zfull); then, while block b's solver runs, the rest
    // of the update and, once block b-1's recent g1 are in the operand, the Z
    // GEMM of block b+1 into the other Z buffer.
    if (lane == 0) {
      int it = 0;  // slots consumed
      bool ok = true, any = false;
      // the tiles [i0, i1) of one phase in the producer's slots; op(i, dcol,
      // bop, acc) gives tile i's accumulator column, B operand and whether it
      // accumulates.  Each 128 x 64 weight tile against a 16 x 64 operand is
      // 4 MMAs of K = 16; one commit releases the slot.
      auto mma_phase = [&](int i0, int i1, auto op) -> bool {
        for (int i = i0; i < i1; i += kSlotTiles) {
          const int cnt = min(kSlotTiles, i1 - i);
          const int s = it % kNSlot;
          if (!test_or_abort(smem_u32(&full[s]), (uint32_t)((it / kNSlot) & 1), abort, g.err)) return false;
          fence_after();
          for (int j = 0; j < cnt; ++j) {
            uint32_t dcol, bop;
            bool acc;
            op(i + j, dcol, bop, acc);
            const uint64_t da = smem_desc_sw128(base + kOffRing + (s * kSlotTiles + j) * kTileBytes);
            const uint64_t db = smem_desc_sw128(bop);
#pragma unroll
            for (int k = 0; k < 4; ++k)
              mma_bf16(tmem + dcol, da + (uint64_t)(2 * k), db + (uint64_t)(2 * k), kIdesc,
                       (acc || k > 0) ? 1u : 0u);
          }
          mma_commit(smem_u32(&empty[s]));
          ++it;
          any = true;
        }
        return true;
      };
      for (int b = 0; b < nblk; ++b) {
        const Blk B = blk_of(b, n, h, D, ntiles, nblk);
        const uint32_t s_prev = base + kOffS + ((b - 1) & 1) * (kDmax / 64) * 2048;
        if (b > 0 && ok) {
          ok = test_or_abort(smem_u32(ready), (uint32_t)((b - 1) & 1), abort, g.err);
          fence_after();
        }
        // update tiles: index q -> accumulator of unit tile q / nkd, K-chunk q % nkd of block b-1's spins
        auto upd = [&](int q, uint32_t& dcol, uint32_t& bop, bool& acc) {
          dcol = (uint32_t)(16 * (q / nkd)), bop = s_prev + (q % nkd) * 2048, acc = true;
        };
        if (ok) ok = mma_phase(B.crit0 * nkd, B.crit1 * nkd, upd);
        const uint32_t zcol = kZCol + 16 * (b & 1);
        if (ok)
          ok = mma_phase(B.cor0, B.cor1, [&](int c, uint32_t& dcol, uint32_t& bop, bool& acc) {
            dcol = zcol, bop = base + kOffHr + (c - B.cor0) * 2048, acc = B.zinit || c > B.cor0;
          });
        if (ok && any) mma_commit(smem_u32(zfull));  // also covers the previous block's work
        else mbar_arrive(smem_u32(zfull));
        if (ok) ok = mma_phase(B.bulk0 * nkd, ntiles * nkd, upd);
        if (B.np > 0 && ok) {
          ok = test_or_abort(smem_u32(merged), (uint32_t)(b & 1), abort, g.err);
          fence_after();
          const uint32_t zn = kZCol + 16 * ((b + 1) & 1);
          if (ok)
            ok = mma_phase(0, B.np, [&](int c, uint32_t& dcol, uint32_t& bop, bool& acc) {
              dcol = zn, bop = base + kOffH + c * 2048, acc = c > 0;
            });
        }
      }
      // every MMA has completed before tensor memory is released
      mma_commit(smem_u32(drain));
      mbar_wait(smem_u32(drain), 0u, g.err);
    }
  } else {
    // ---------------------------- warps 0-3 and 6-7: blocks, solver
    // Warps 0, 1, 6 and 7 are the solver, one warp on each SM sub-partition
    // (warp w runs on w % 4): the solver is issue-bound, and the producer and
    // MMA warps that share sub-partitions 0 and 1 with it issue little.
    // Warps 0-3 read tensor memory; warps 2-3 meanwhile prepare the next
    // block's logits and write out the previous block's spins.
    const bool solver = warp <= 1 || warp >= 6;
    const int sid = (warp <= 1 ? warp : warp - 4) * 32 + lane;  // solver thread
    const int ht = tid - 64;                                      // helper thread (warps 2-3)
    const int s_me = sid / kLanes, sub = sid % kLanes;
    float lp = 0.0f;
    const uint32_t tq = tmem + ((uint32_t)(32 * warp) << 16);
    // logit(u) of block b's steps into LG buffer b & 1; threads t0, t0 + nt, ...
    auto logits = [&](int b, int t0, int nt) {
      float* L = LG + (b & 1) * kDrows * kS;
      for (int q = t0; q < kS * (D / 4); q += nt) {
        const int s = q % kS, t = b * D + 4 * (q / kS);
        const int bb = b0 + s;
        float* dst = L + (size_t)(4 * (q / kS)) * kS + s;
        if (g.u) {
#pragma unroll
          for (int w = 0; w < 4; ++w)
            dst[w * kS] = (bb < g.B && t + w < n) ? logit(__ldg(g.u + (size_t)bb * n + t + w)) : 0.0f;
        } else {
          const uint4 r = philox4x32_10(make_uint4((uint32_t)(t >> 2), (uint32_t)bb + g.boff, it0, it1), g.key0, g.key1);
          dst[0] = logit(to_unit(r.x));
          dst[kS] = logit(to_unit(r.y));
          dst[2 * kS] = logit(to_unit(r.z));
          dst[3 * kS] = logit(to_unit(r.w));
        }
      }
    };
    // spins of block b (bits in SB buffer b & 1) to the outputs; threads t0,
    // t0 + nt, ...  Runs of 16 steps of one sample (s_out, sx) and the 16
    // samples of one step (stt) go out as 16-byte stores where the whole run
    // is inside the output and aligned, else element by element.
    auto write_spins = [&](int b, int t0, int nt) {
      const uint32_t* sb = SB + (b & 1) * kS * (kDmax / 32);
      const int steps = min(D, n - b * D);
      const bf16 one = __float2bfloat16_rn(1.0f), mone = __float2bfloat16_rn(-1.0f);
      // two spins as BF16 (+1 = 0x3F80, -1 = 0xBF80); bit set in dn: spin -1
      auto bf_pair = [](uint32_t dn) { return 0x3F803F80u | (dn & 1u) << 15 | (dn >> 1 & 1u) << 31; };
      for (int q = t0; q < kS * (kDmax / 16); q += nt) {
        const int s = q / (kDmax / 16), e0 = 16 * (q % (kDmax / 16));
        const int bb = b0 + s;
        if (bb >= g.B || e0 >= steps) continue;
        const uint32_t up = (sb[s * (kDmax / 32) + (e0 >> 5)] >> (e0 & 16)) & 0xFFFFu;  // bit k: step e0 + k is +1
        const int cnt = min(16, steps - e0);
        int8_t* so = g.s_out + (size_t)bb * n + b * D + e0;
        if (cnt == 16 && (reinterpret_cast<uintptr_t>(so) & 15) == 0) {
          uint32_t w[4];
#pragma unroll
          for (int p = 0; p < 4; ++p) {
            // the 4 bits spread to bit 0 of 4 bytes (the shifted copies do
            // not overlap), then +1 -> 0x01 and -1 -> 0xFF per byte
            const uint32_t m = ((up >> (4 * p)) & 0xFu) * 0x00204081u & 0x01010101u;
            w[p] = m | (m ^ 0x01010101u) * 0xFFu;
          }
          *reinterpret_cast<uint4*>(so) = make_uint4(w[0], w[1], w[2], w[3]);
        } else {
          for (int k = 0; k < cnt; ++k) so[k] = (up >> k) & 1u ? (int8_t)1 : (int8_t)-1;
        }
        if (g.sx) {
          bf16* dx = g.sx + (size_t)bb * g.ldsx + b * D + e0;
          if (cnt == 16 && (reinterpret_cast<uintptr_t>(dx) & 15) == 0) {
            const uint32_t dn = ~up;
            uint4* d4 = reinterpret_cast<uint4*>(dx);
            d4[0] = make_uint4(bf_pair(dn), bf_pair(dn >> 2), bf_pair(dn >> 4), bf_pair(dn >> 6));
            d4[1] = make_uint4(bf_pair(dn >> 8), bf_pair(dn >> 10), bf_pair(dn >> 12), bf_pair(dn >> 14));
          } else {
            for (int k = 0; k < cnt; ++k) dx[k] = (up >> k) & 1u ? one : mone;
          }
        }
      }
      // the 16 samples of each step (stt, sbits): a warp transposes a word of
      // 32 steps with ballots (lane s < 16 holds sample s's word; ballot j
      // collects step j's spins) and lane j keeps step j's column
      const uint32_t valid = b0 + kS <= g.B ? 0xFFFFu : (1u << (g.B - b0)) - 1u;  // samples inside B
      if (g.stt || g.sbits)
        for (int w = t0 >> 5; w < (steps + 31) / 32; w += nt >> 5) {
          const int ln = t0 & 31;
          const uint32_t word = ln < kS ? sb[ln * (kDmax / 32) + w] : 0u;
          uint32_t up = 0;
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const uint32_t col = __ballot_sync(0xffffffffu, (word >> j) & 1u);
            up = ln == j ? col : up;
          }
          const int e = 32 * w + ln;
          if (e >= steps) continue;
          const uint32_t dn = ~up & valid;  // bit s: sample b0 + s has spin -1 at step e
          if (g.stt) {
            bf16* dt = g.stt + (size_t)(b * D + e) * g.ldst + b0;
            if (b0 + kS <= g.B && (reinterpret_cast<uintptr_t>(dt) & 15) == 0) {
              uint4* d4 = reinterpret_cast<uint4*>(dt);
              d4[0] = make_uint4(bf_pair(dn), bf_pair(dn >> 2), bf_pair(dn >> 4), bf_pair(dn >> 6));
              d4[1] = make_uint4(bf_pair(dn >> 8), bf_pair(dn >> 10), bf_pair(dn >> 12), bf_pair(dn >> 14));
            } else {
              for (int s = 0; s < kS; ++s)
                if (b0 + s < g.B) dt[s] = (dn >> s) & 1u ? mone : one;
            }
          }
          if (g.sbits) g.sbits[((size_t)(b0 >> 5) * n + b * D + e) * 2 + ((b0 >> 4) & 1)] = (uint16_t)dn;
        }
    };
    // The recent units' weights of block bb (W2 rows of its steps, W1 of its
    // recent units), loaded by warps 2-3 (helper thread t < 64) into registers
    // during the previous block's solver and stored into Vr / Wr once the
    // solver is done.  Vr: thread t owns steps t and t + 64, 5 aligned
    // 16-byte pieces of W2 from unit klo & ~7; Wr: pieces (unit q % 32,
    // inputs 8 (q / 32) ..) for q = t + 64 j, so that a warp's transposing
    // stores hit 32 different units.
    uint4 gv[2][5], gw[8];
    auto gather_load = [&](int bb, int t) {
      const int klo = count_deg_le(bb * D, n, h), R = count_deg_le(bb * D + D, n, h) - klo;
      const int steps = min(D, n - bb * D), k8 = klo & ~7;
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const int e = t + 64 * i;
#pragma unroll
        for (int c = 0; c < 5; ++c)
          gv[i][c] = (e < steps && k8 + 8 * c < g.hp)
                         ? __ldg(reinterpret_cast<const uint4*>(g.v + (size_t)(bb * D + e) * g.hp + k8) + c)
                         : make_uint4(0, 0, 0, 0);
      }
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int q = t + 64 * j, r = q & 31, c = q >> 5;
        gw[j] = (8 * c < steps && r < R)  // pieces past the last step stay in [0, np)
                    ? __ldg(reinterpret_cast<const uint4*>(g.w + (size_t)(klo + r) * g.np + (size_t)bb * D) + c)
                    : make_uint4(0, 0, 0, 0);
      }
    };
    auto gather_store = [&](int bb, int t) {
      const int klo = count_deg_le(bb * D, n, h);
      const int steps = min(D, n - bb * D), off = klo & 7;
      // Vr[e][r] = W2 of step e, unit klo + r (r < 32; zero for units past the
      // block's recent ones: they complete after the block, masked in W2)
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const int e = t + 64 * i;
        if (e >= D) continue;
        uint32_t w[20];
#pragma unroll
        for (int c = 0; c < 5; ++c) w[4 * c] = gv[i][c].x, w[4 * c + 1] = gv[i][c].y, w[4 * c + 2] = gv[i][c].z,
                                    w[4 * c + 3] = gv[i][c].w;
        uint32_t d[16];
#pragma unroll
        for (int sh = 0; sh < 4; ++sh)
          if ((off >> 1) == sh) {
#pragma unroll
            for (int j = 0; j < 16; ++j) d[j] = (off & 1) ? __byte_perm(w[sh + j], w[sh + j + 1], 0x5432) : w[sh + j];
          }
        uint4* dst = reinterpret_cast<uint4*>(Vr + e * kLdW);
#pragma unroll
        for (int j = 0; j < 4; ++j) dst[j] = make_uint4(d[4 * j], d[4 * j + 1], d[4 * j + 2], d[4 * j + 3]);
      }
      // Wr[e][r] = W1 of unit klo + r, input of step e (zero for r >= R)
      unsigned short* sw = reinterpret_cast<unsigned short*>(Wr);
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int q = t + 64 * j, r = q & 31, c = q >> 5;
        if (8 * c >= D) continue;
        const uint32_t w[4] = {gw[j].x, gw[j].y, gw[j].z, gw[j].w};
#pragma unroll
        for (int tt = 0; tt < 8; ++tt) {
          const int e = 8 * c + tt;
          sw[e * kLdW + r] = e < steps ? (unsigned short)(w[tt >> 1] >> (16 * (tt & 1))) : (unsigned short)0;
        }
      }
    };
    if (warp < 4) logits(0, tid, 128);
    if (warp == 2 || warp == 3) {
      gather_load(0, ht);
      gather_store(0, ht);
    }
    for (int b = 0; b < nblk; ++b) {
      const Blk B = blk_of(b, n, h, D, ntiles, nblk);
      const int klo = B.klo, khi = B.khi;
      const int R = khi - klo;  // <= kRmax (checked by the host)
      const int steps = min(D, n - b * D);
      if (warp < 4) {
      // (a) the recent units' completion steps (their weights are in Vr / Wr)
      for (int q = tid; q < (kRmax - R) * kS; q += 128) Pr[R * kS + q] = 0.0f;
      // TC[r] = the block step whose spin is recent unit r's last input
      for (int r = tid; r < kRmax; r += 128) CU[r] = r < R ? degree(klo + r, n, h) - 1 - b * D : D;
      // (b) Z and the recent pre-activations from tensor memory
      wait_or_abort(smem_u32(zfull), (uint32_t)(b & 1), abort, g.err);
      __syncwarp();
      fence_after();
      // warp-uniform: tcgen05.ld is executed by all lanes of a warp or none
      const bool live = !__any_sync(0xffffffffu, *abort != 0);
      {
        float v[16];
        if (B.zvalid && live) {
          tmem_ld16(tq + kZCol + 16 * (b & 1), v);
        } else {
#pragma unroll
          for (int q = 0; q < 16; ++q) v[q] = 0.0f;
        }
        const int e = 32 * warp + lane;
        if (e < D) {
          const float c = e < steps ? __ldg(g.b2 + b * D + e) : 0.0f;
#pragma unroll
          for (int q = 0; q < 16; ++q) Zs[e * kZld + q] = v[q] + c;  // b2 folded in
        }
      }
      if (R > 0 && live) {
        for (int t = klo / 128; t <= (khi - 1) / 128; ++t) {
          float v[16];
          tmem_ld16(tq + (uint32_t)(16 * t), v);
          const int k = 128 * t + 32 * warp + lane;
          if (k >= klo && k < khi) {
#pragma unroll
            for (int q = 0; q < 16; ++q) Pr[(k - klo) * kS + q] = v[q];
          }
        }
      }
      fence_before();  // the tensor-memory reads precede the next MMAs into Z (after merged)
      }
      asm volatile("bar.sync 1, %0;" ::"n"(kBar1Threads) : "memory");
      // (c) the D draws of the block (the solver warps), then the block's
      // spins as the update GEMM's operand; warps 2-3 meanwhile
      if (solver) {
        const bool relu = g.act == VQMC_ACT_RELU;
        const float* L = LG + (b & 1) * kDrows * kS;
        uint32_t* sb = SB + (b & 1) * kS * (kDmax / 32);
        if (g.logp) {
          if (relu) solve<VQMC_ACT_RELU, true>(Pr, Vr, Wr, Zs, L, CU, sb, PreS, Hr, s_me, sub, klo, R, steps, lp);
          else solve<VQMC_ACT_SIGMOID, true>(Pr, Vr, Wr, Zs, L, CU, sb, PreS, Hr, s_me, sub, klo, R, steps, lp);
        } else {
          if (relu) solve<VQMC_ACT_RELU, false>(Pr, Vr, Wr, Zs, L, CU, sb, PreS, Hr, s_me, sub, klo, R, steps, lp);
          else solve<VQMC_ACT_SIGMOID, false>(Pr, Vr, Wr, Zs, L, CU, sb, PreS, Hr, s_me, sub, klo, R, steps, lp);
        }
        asm volatile("bar.sync 1, %0;" ::"n"(kBar1Threads) : "memory");
        // (d) 8 spins of one sample per 16-byte store (+1 = 0x3F80, -1 = 0xBF80)
        unsigned char* ss = Ss + (b & 1) * (kDmax / 64) * 2048;
        for (int q = sid; q < kS * (D / 8); q += kSolverThreads) {
          const int s = q / (D / 8), e = 8 * (q % (D / 8));
          const uint32_t bits = ~(sb[s * (kDmax / 32) + (e >> 5)] >> (e & 31));  // bit set: spin -1
          uint32_t w[4];
#pragma unroll
          for (int p = 0; p < 4; ++p)
            w[p] = 0x3F803F80u | ((bits >> (2 * p)) & 1u) << 15 | ((bits >> (2 * p + 1)) & 1u) << 31;
          *reinterpret_cast<uint4*>(ss + (e >> 6) * 2048 + sw128_offset(s, e & 63)) = make_uint4(w[0], w[1], w[2], w[3]);
        }
        fence_proxy_async();
        fence_before();
        mbar_arrive(smem_u32(ready));
      } else {
        // block b-1's recent g1 from the staging operand into the GEMM
        // operand (the block's Z GEMM has read Hr: zfull), then release Hr
        // to the solver and the operand to the next Z GEMM
        if (b > 0) {
          const int kprev = count_deg_le((b - 1) * D, n, h), cb = kprev >> 6;
          for (int q = ht; q < (klo - kprev) * kS; q += 64) {
            const int k = kprev + q / kS, s = q % kS;
            const uint32_t o = sw128_offset(s, k & 63);
            bf16* src = reinterpret_cast<bf16*>(Hr + ((k >> 6) - cb) * 2048 + o);
            *reinterpret_cast<bf16*>(Hs + (k >> 6) * 2048 + o) = *src;
            *src = __float2bfloat16_rn(0.0f);  // Hr is zero outside the current recent units
          }
        }
        fence_proxy_async();
        fence_before();
        mbar_arrive(smem_u32(merged));
        asm volatile("bar.arrive 2, %0;" ::"n"(kBar2Threads) : "memory");
        if (b + 1 < nblk) logits(b + 1, ht, 64);
        if (b > 0) write_spins(b - 1, ht, 64);
        if (b + 1 < nblk) gather_load(b + 1, ht);
        asm volatile("bar.sync 1, %0;" ::"n"(kBar1Threads) : "memory");
        if (b + 1 < nblk) gather_store(b + 1, ht);
      }
    }
    asm volatile("bar.sync 1, %0;" ::"n"(kBar1Threads) : "memory");
    if (warp < 4) write_spins(nblk - 1, tid, 128);
    if (solver) {  // the partial sums of log pi of the sample's lanes
#pragma unroll
      for (int d = 1; d < kLanes; d <<= 1) lp += __shfl_xor_sync(0xffffffffu, lp, d);
    }
    if (solver && sub == 0 && g.logp && b0 + s_me < g.B && !*abort) g.logp[b0 + s_me] = lp;
  }

  __syncwarp();
  fence_before();
  __syncthreads();
  if (warp == 5) {
    __syncwarp();
    fence_after();
    tmem_dealloc(tmem, kTmemCols);
  }
}

bool g_attr_set = false;

// largest number of units completing inside one block of D steps
int max_recent(int n, int h, int D) {
  int r = 0;
  for (int b = 0; b * D < n; ++b) r = std::max(r, count_deg_le(b * D + D, n, h) - count_deg_le(b * D, n, h));
  return r;
}

}  // namespace

// Block size the tensor-core sampler would use for this model, or 0 when it
// does not apply (FP32 weights, more than 2048 hidden units, or more than
// 32 units completing within every block size).
int sampler_tc_block(const vqmc_ctx* c) {
  // h < n: distinct degrees, at most one unit completes per step
  if (c->prec != VQMC_PREC_BF16 || c->hp > kMaxHp || c->h >= c->n) return 0;
  for (int D : {128, 64})
    if (max_recent(c->n, c->h, D) <= kRmax) return D;
  return 0;
}

cudaError_t launch_sampler_tc(const vqmc_ctx* c, int B, const float* d_u, uint64_t iteration, int8_t* d_s,
                              float* d_logp, cudaStream_t st, void* sx, void* stt, uint32_t* sbits,
                              const unsigned long long* it_dev) {
  const int D = sampler_tc_block(c);
  if (D == 0 || !gemm_tc_available()) return cudaErrorNotSupported;
  if (B <= 0) return cudaSuccess;
  // v_s [sampler_rows(n)][hp] and w_s [h][np] (hp, np multiples of 64): one
  // 128 x 64 tile per copy, or 2 or 3 consecutive chunks of the same rows
  CUtensorMap mapV, mapW, mapV2, mapV3, mapW2;
  if (!tc_encode_bf16(&mapV, c->v_s, sampler_rows(c->n), c->hp, c->hp, 128) ||
      !tc_encode_bf16(&mapW, c->w_s, c->h, c->np, c->np, 128) ||
      !tc_encode_bf16_chunks(&mapV2, c->v_s, sampler_rows(c->n), c->hp, c->hp, 128, 2) ||
      !tc_encode_bf16_chunks(&mapV3, c->v_s, sampler_rows(c->n), c->hp, c->hp, 128, 3) ||
      !tc_encode_bf16_chunks(&mapW2, c->w_s, c->h, c->np, c->np, 128, 2))
    return cudaErrorInvalidValue;
  if (!g_attr_set) {
    cudaError_t e = cudaFuncSetAttribute(sampler_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
    if (e != cudaSuccess) return e;
    g_attr_set = true;
  }
  TcArgs a;
  a.n = c->n;
  a.h = c->h;
  a.hp = c->hp;
  a.B = B;
  a.D = D;
  a.act = c->act;
  a.w = reinterpret_cast<const bf16*>(c->w_s);
  a.np = c->np;
  a.v = reinterpret_cast<const bf16*>(c->v_s);
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
  a.sx = reinterpret_cast<bf16*>(sx);
  a.ldsx = c->np;
  a.stt = reinterpret_cast<bf16*>(stt);
  a.ldst = c->Bp;
  a.sbits = reinterpret_cast<uint16_t*>(sbits);
  sampler_tc_kernel<<<(B + kS - 1) / kS, kThreads, kSmemBytes, st>>>(mapV, mapW, mapV2, mapV3, mapW2, a);
  return cudaGetLastError();
}

}  // namespace vqmc
