// column_tc.cu -- steps a1-a5 (ZC transform, LS division, DFT-CE) for N = 1024
// with both 1024-point DFTs on the tensor cores, in split FP16.
//
// Four-step form of a 1024-point DFT (1024 = 32 x 32), k = 32 k1 + k2,
// n = n1 + 32 n2, w_L = exp(+2 pi i / L):
//     Y[n1, k2] = sum_k1 x[32 k1 + k2] w_32^(n1 k1)        (32-point DFTs)
//     X[n1 + 32 n2] = sum_k2 (Y[n1, k2] w_1024^(n1 k2)) w_32^(n2 k2)
// Each 32-point stage is one matrix product per tile of 4 OFDM symbols:
// 128 rows (4 symbols x 32) by K = 64 (32 complex inputs as interleaved
// re, im) times the 64 x 64 real form of the 32-point DFT matrix, on
// tcgen05 (M = 128, N = 64, fp16 operands, fp32 accumulation in TMEM).  FP16
// alone would leave ~2^-11 relative error, which the LS division multiplies
// at small precoded cells, so every operand is split into hi + lo halves and
// the product is taken as A_hi B_hi + A_lo B_hi + A_hi B_lo (about 2^-21).
//
// The chain per tile (Sec. III-B, Eq. (16), Eqs. (20)-(22)):
//   stage 1-2  X_p = post . DFT(pre . A) / sqrt(N)    ZC transform, Eqs. (23)-(24)
//              (cells with |X_p|^2 < tau mean recomputed in double-float)
//              F = Y / X_p                            LS division, Eq. (16)
//   stage 3-4  h[n] = sum_k F[k] w_1024^(n k), n < 256 (the last stage
//              computes 8 of its 32 output rows: DFT-CE keeps n < L_cp)
//   stencil    g[r] = c0 h[r] + c1 (h[r-1] + h[r+1]) on the support rows.
// Rows are exchanged between stages through the shared-memory operand
// image: a thread that holds a whole operand row (stages 1, 3) stores it as
// 16-byte vectors, one that holds a column (stages 2, 4) as 4-byte (re, im)
// pairs; the K order (k, re/im) makes both conflict-free.
//
// Dynamic range: FP16 has a 5-bit exponent, so the inputs of stages 1 and 3
// are scaled per OFDM symbol by a power of two (exact) that brings the
// largest component to [1, 2); stages 2 and 4 take their inputs divided by
// 32 (folded into the twiddle table), which bounds them the same way.  The
// scales cancel in the division and the stencil.
//
// Work: persistent CTAs of two warpgroups of 8 warps, one CTA per SM.  Warp w
// of a warpgroup holds TMEM lane quarter w % 4 (one symbol of the tile) and
// column half w / 4 (16 complex values per thread).  Each warpgroup takes
// tiles of 4 consecutive symbols of one frame from a ticket counter, loads
// the tile's X and Y rows with 32 KB bulk copies (mbarrier completion) one
// tile ahead, and issues its own MMAs from one thread; the two warpgroups
// interleave on the tensor core.  Every wait is bounded: on a timeout the
// warpgroup marks its frame OFDM_STATUS_TIMEOUT, stops taking tiles, waits
// (bounded) for what it issued and the CTA releases its TMEM.
#include <cuda_fp16.h>

#include "fft.cuh"
#include "internal.h"
#include "refine.cuh"
#include "tc.cuh"

namespace ofdm {
namespace {

constexpr int kN = 1024;
constexpr int kWG = 2;                        // warpgroups per CTA
constexpr int kWgThreads = 256;               // 8 warps: lane quarter (symbol) x column half
constexpr int kThreads = kWgThreads * kWG;
constexpr uint32_t kSBO = 128;                // 8-row group stride of every operand image
constexpr uint32_t kLboA = 16 * 128 + 16;     // 128 rows; +16 B puts the 8 K-slices on distinct banks
constexpr uint32_t kLboB = 8 * 128;           // 64 rows
constexpr uint32_t kABytes = 8 * kLboA;       // 128 x 64 fp16 (K = 64: 8 slices)
constexpr uint32_t kBBytes = 8 * kLboB;       // 64 x 64 fp16
constexpr uint32_t kTileBytes = 4 * kN * 8;   // 4 rows of complex64
// Shared-memory map (bytes): B hi, B lo, twiddles, pre-chirp, then per warpgroup X, Y, A hi, A lo.
constexpr uint32_t kOffBhi = 0, kOffBlo = kBBytes, kOffT12 = 2 * kBBytes, kOffPre = kOffT12 + kN * 8;
constexpr uint32_t kOffWG = kOffPre + kN * 8;
constexpr uint32_t kWgX = 0, kWgY = kTileBytes, kWgAhi = 2 * kTileBytes, kWgAlo = 2 * kTileBytes + kABytes;
constexpr uint32_t kWgBytes = 2 * kTileBytes + 2 * kABytes;
constexpr uint32_t kSmemBytes = kOffWG + kWG * kWgBytes;
static_assert(kSmemBytes + 1024 <= 227u * 1024u, "shared memory");
static_assert(kABytes >= 258 * 4 * 8, "the strip exchange reuses the A image");

constexpr uint32_t kIdesc64 = tc::idesc_f16_f32(128, 64);
constexpr uint32_t kIdesc16 = tc::idesc_f16_f32(128, 16);

// named barrier of one warpgroup (ids 1, 2), OR-reduced predicate
__device__ __forceinline__ bool wg_sync_or(int wg, bool pred) {
  unsigned r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\tbar.red.or.pred q, %2, 256, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"((unsigned)pred), "r"(wg + 1)
      : "memory");
  return r != 0;
}

// Power of two that brings m (the largest |component|, >= 0) into [1, 2):
// 2^(127 - e) for the biased exponent e of m, clamped to the normal range.
__device__ __forceinline__ float pow2_scale(float m) {
  int e = (__float_as_int(m) >> 23) & 0xff;
  e = e < 1 ? 1 : (e > 253 ? 253 : e);
  return __int_as_float((254 - e) << 23);
}
__device__ __forceinline__ float rcp_fast(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// hi / lo fp16 halves of (re, im), packed as half2 bit patterns.
__device__ __forceinline__ void split2(float re, float im, uint32_t& hi, uint32_t& lo) {
  const __half2 h = __floats2half2_rn(re, im);
  const float2 hf = __half22float2(h);
  const __half2 l = __floats2half2_rn(re - hf.x, im - hf.y);
  hi = *reinterpret_cast<const uint32_t*>(&h);
  lo = *reinterpret_cast<const uint32_t*>(&l);
}

// Half an operand row: K values 32 h .. 32 h + 31 of row `row` from 16
// complex values times s (four 16-byte vectors for each of hi and lo).
__device__ __forceinline__ void store_row16(const float2* v, float s, unsigned char* ahi, unsigned char* alo, int row,
                                            int h) {
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    uint4 hv, lv;
    split2(v[4 * j].x * s, v[4 * j].y * s, hv.x, lv.x);
    split2(v[4 * j + 1].x * s, v[4 * j + 1].y * s, hv.y, lv.y);
    split2(v[4 * j + 2].x * s, v[4 * j + 2].y * s, hv.z, lv.z);
    split2(v[4 * j + 3].x * s, v[4 * j + 3].y * s, hv.w, lv.w);
    const uint32_t off = tc::kmajor_off((uint32_t)row, 32u * h + 8u * j, kLboA, kSBO);
    *reinterpret_cast<uint4*>(ahi + off) = hv;
    *reinterpret_cast<uint4*>(alo + off) = lv;
  }
}
// Operand column pair (K = 2c, 2c + 1) of rows row0 .. row0 + 15 from 16 complex values.
__device__ __forceinline__ void store_col16(const float2* v, unsigned char* ahi, unsigned char* alo, int row0, int c) {
#pragma unroll
  for (int n = 0; n < 16; ++n) {
    uint32_t hv, lv;
    split2(v[n].x, v[n].y, hv, lv);
    const uint32_t off = tc::kmajor_off((uint32_t)(row0 + n), 2u * c, kLboA, kSBO);
    *reinterpret_cast<uint32_t*>(ahi + off) = hv;
    *reinterpret_cast<uint32_t*>(alo + off) = lv;
  }
}

// One 32-point DFT stage: D = A_hi B_hi + A_lo B_hi + A_hi B_lo over K = 64.
// The descriptors of K-step j differ from step 0's only in the start address
// field (bits 0-13, in 16-byte units), so step 0's are built once per launch
// and advanced by 2 j LBO / 16.
struct StageDesc { uint64_t ah, al, bh, bl; };
__device__ __forceinline__ void issue_stage(uint32_t tmem, const StageDesc& d, uint32_t idesc) {
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const uint64_t da = (uint64_t)(2 * j * kLboA / 16), db = (uint64_t)(2 * j * kLboB / 16);
    tc::mma_f16(tmem, d.ah + da, d.bh + db, idesc, j > 0 ? 1u : 0u);
    tc::mma_f16(tmem, d.al + da, d.bh + db, idesc, 1u);
    tc::mma_f16(tmem, d.ah + da, d.bl + db, idesc, 1u);
  }
}

// 32 accumulator columns (16 complex) of this thread's TMEM lane.
__device__ __forceinline__ void load_acc32(uint32_t taddr, float2* v) {
  float* f = reinterpret_cast<float*>(v);
  tc::tmem_ld16(taddr, f);
  tc::tmem_ld16(taddr + 16, f + 16);
  tc::tmem_wait_ld();
}

// R1Q0: instantiated for r' = 1, q' = 0 (identity input permutation, post
// factor (-1)^i), without the per-point post-chirp table multiply that the
// unrolled division loop would otherwise issue predicated.
template <bool R1Q0>
__global__ void __launch_bounds__(kThreads, 1)
column_tc_kernel(const float2* __restrict__ Y, const float2* __restrict__ X, float2* __restrict__ strip,
                 uint32_t* __restrict__ wstatus, ColumnArgs a) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t s_bar[kWG][3];   // X landed, Y landed, MMAs done
  __shared__ uint32_t s_tmem;
  __shared__ long long s_first[kWG], s_next[kWG];
  __shared__ float s_red[kWG][3][8];                 // per-warp partials: stage-1 max, refine sum, stage-3 max
  const int tid = threadIdx.x, wg = tid / kWgThreads, wt = tid % kWgThreads;
  const int w = wt >> 5, q = w & 3, h = w >> 2, lane = tid & 31;   // symbol q of the tile, column half h

  {  // constant operand images, twiddles and the pre-chirp
    const uint4* src = a.tc_b;
    uint4* dst = reinterpret_cast<uint4*>(smem + kOffBhi);
    for (int i = tid; i < (int)(2 * kBBytes / 16); i += kThreads) dst[i] = __ldg(src + i);
    const float4* t = reinterpret_cast<const float4*>(a.tc_t12);
    float4* d = reinterpret_cast<float4*>(smem + kOffT12);
    for (int i = tid; i < kN * 8 / 16; i += kThreads) d[i] = __ldg(t + i);
    if (a.zc) {
      const float4* pr = reinterpret_cast<const float4*>(a.pre);
      float4* dp = reinterpret_cast<float4*>(smem + kOffPre);
      for (int i = tid; i < kN * 8 / 16; i += kThreads) dp[i] = __ldg(pr + i);
    }
  }
  if (tid == 0) {
    for (int g = 0; g < kWG; ++g)
      for (int b = 0; b < 3; ++b) tc::mbar_init(tc::smem_u32(&s_bar[g][b]), 1);
    tc::fence_mbar_init();
  }
  if (tid < 32) {
    tc::tmem_alloc(tc::smem_u32(&s_tmem), 128);   // 64 fp32 columns per warpgroup
    tc::tmem_relinquish();
  }
  tc::fence_proxy_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();

  const uint32_t tmem = s_tmem + 64u * wg;
  const uint32_t tacc = tmem + ((uint32_t)(32 * q) << 16);   // this warp's lane quarter
  unsigned char* wb = smem + kOffWG + wg * kWgBytes;
  const float2* Xs = reinterpret_cast<const float2*>(wb + kWgX) + q * kN;   // symbol q of the tile
  const float2* Ys = reinterpret_cast<const float2*>(wb + kWgY) + q * kN;
  unsigned char* ahi = wb + kWgAhi;
  unsigned char* alo = wb + kWgAlo;
  StageDesc sd;
  sd.ah = tc::smem_desc(tc::smem_u32(ahi), kLboA, kSBO);
  sd.al = tc::smem_desc(tc::smem_u32(alo), kLboA, kSBO);
  sd.bh = tc::smem_desc(tc::smem_u32(smem + kOffBhi), kLboB, kSBO);
  sd.bl = tc::smem_desc(tc::smem_u32(smem + kOffBlo), kLboB, kSBO);
  const uint32_t barX = tc::smem_u32(&s_bar[wg][0]), barY = tc::smem_u32(&s_bar[wg][1]),
                 barM = tc::smem_u32(&s_bar[wg][2]);
  const float2* T12 = reinterpret_cast<const float2*>(smem + kOffT12);
  const float2* pre = reinterpret_cast<const float2*>(smem + kOffPre);
  const int tiles_per_frame = a.M >> 2;
  const long tiles = (long)a.frames * tiles_per_frame;
  const uint64_t pol = tc::evict_first();
  auto tile_off = [&](long t) -> long {   // complex offset of the tile's first row in Y and X
    const long f = t / tiles_per_frame, l0 = (t % tiles_per_frame) * 4;
    return (a.frame_off ? (long)a.frame_off[f] : f * (long)a.M * kN) + l0 * kN;
  };
  auto draw = [&]() -> long { return (long)(atomicAdd(a.work_ctr, 1ull) - a.work_base); };
  auto issue = [&](const float2* g, long t, uint32_t dst, uint32_t bar) {
    tc::mbar_arrive_expect_tx(bar, kTileBytes);
    tc::bulk_load(dst, g + tile_off(t), kTileBytes, bar, pol);
  };
  const uint32_t u_xs = tc::smem_u32(wb + kWgX), u_ys = tc::smem_u32(wb + kWgY);
  // the symbol-wide value of a per-warp partial: the partner warp (other column half) holds the rest
  // (each use has its own slot, so no warp overwrites a partial its partner has yet to read)
  auto symbol_max = [&](float v, int slot) -> float {
    v = warp_max(v);
    if (lane == 0) s_red[wg][slot][w] = v;
    wg_sync_or(wg, false);
    return fmaxf(s_red[wg][slot][q], s_red[wg][slot][q + 4]);
  };

  // thread 0 of the warpgroup: what it has issued and not yet seen complete
  int pendX = 0, pendY = 0, pendM = 0;
  uint32_t px = 0, py = 0, pm = 0;
  bool bad = false;
  if (wt == 0) {
    const long t0 = draw();
    s_first[wg] = t0;
    if (t0 < tiles) {
      issue(X, t0, u_xs, barX);
      issue(Y, t0, u_ys, barY);
      pendX = pendY = 1;
    }
  }
  wg_sync_or(wg, false);
  long tile = s_first[wg];
  const float sgn0 = (a.post_sign && (lane & 1)) ? -1.f : 1.f;   // (-1)^i, i = lane + 32 n2

  while (tile < tiles) {
    const int f = (int)(tile / tiles_per_frame);
    const int l0 = (int)(tile % tiles_per_frame) * 4;
    long next = 0;
    if (wt == 0) {
      next = draw();
      s_next[wg] = next;
    }
    uint32_t flags = 0;
    float2 v[16];
    float bscale;   // v holds DFT(pre . A) * bscale after the ZC stages
    if (a.zc) {
      bad |= !tc::mbar_wait(barX, px);
      px ^= 1;
      if (wt == 0) pendX = 0;
      // ---- stage 1: rows (symbol q, k2 = lane), K = (k1, re/im), k1 = 16 h + i
      float mx = 0.f;
      if (R1Q0 || a.rinv == 1) {
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int k = 32 * (16 * h + i) + lane;
          v[i] = cmul(Xs[k], pre[k]);
        }
      } else {
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int s = (int)(((unsigned)a.rinv * (unsigned)(32 * (16 * h + i) + lane)) & (kN - 1));
          v[i] = cmul(Xs[s], pre[s]);
        }
      }
#pragma unroll
      for (int i = 0; i < 16; ++i) mx = fmaxf(mx, fmaxf(fabsf(v[i].x), fabsf(v[i].y)));
      const float s1 = pow2_scale(symbol_max(mx, 0));
      store_row16(v, s1, ahi, alo, 32 * q + lane, h);
      tc::fence_proxy_async();
      tc::fence_before_sync();
      if (wg_sync_or(wg, bad)) break;
      if (wt == 0) {
        if (next < tiles) { issue(X, next, u_xs, barX); pendX = 1; }   // X rows consumed
        tc::fence_after_sync();
        issue_stage(tmem, sd, kIdesc64);
        tc::mma_commit(barM);
        pendM = 1;
      }
      bad |= !tc::mbar_wait(barM, pm);
      pm ^= 1;
      if (wt == 0) pendM = 0;
      tc::fence_after_sync();
      // ---- stage 2: twiddle w_1024^(n1 k2) / 32; rows (q, n1), K = (k2 = lane, re/im), n1 = 16 h + i
      load_acc32(tacc + 32 * h, v);
#pragma unroll
      for (int i = 0; i < 16; ++i) v[i] = cmul(v[i], T12[(16 * h + i) * 32 + lane]);
      store_col16(v, ahi, alo, 32 * q + 16 * h, lane);
      tc::fence_proxy_async();
      tc::fence_before_sync();
      if (wg_sync_or(wg, bad)) break;
      if (wt == 0) {
        tc::fence_after_sync();
        issue_stage(tmem, sd, kIdesc64);
        tc::mma_commit(barM);
        pendM = 1;
      }
      bad |= !tc::mbar_wait(barM, pm);
      pm ^= 1;
      if (wt == 0) pendM = 0;
      tc::fence_after_sync();
      load_acc32(tacc + 32 * h, v);   // row (q, n1 = lane): DFT(pre . A)[lane + 32 n2] s1 / 32, n2 = 16 h + i
      bscale = s1 * (1.f / 32.f);
      if (a.refine_tau > 0.f) {
        // precoded cells with |X_p|^2 < tau * (symbol mean) are recomputed in double-float
        float s2 = 0.f;
#pragma unroll
        for (int i = 0; i < 16; ++i) s2 += v[i].x * v[i].x + v[i].y * v[i].y;
        s2 = warp_sum(s2);
        if (lane == 0) s_red[wg][1][w] = s2;
        wg_sync_or(wg, false);
        const float thr = a.refine_tau * (s_red[wg][1][q] + s_red[wg][1][q + 4]) * (1.f / kN);
        unsigned fl = 0;
#pragma unroll
        for (int i = 0; i < 16; ++i) fl |= (v[i].x * v[i].x + v[i].y * v[i].y < thr) ? (1u << i) : 0u;
        unsigned pending = __ballot_sync(0xffffffffu, fl != 0);
        const float2* xrow = X + tile_off(tile) + q * kN;
        while (pending) {
          const int src = __ffs(pending) - 1;
          const unsigned fm = __shfl_sync(0xffffffffu, fl, src);
          const int i = __ffs(fm) - 1;
          float2 val = refine_cell<kN>(xrow, src + 32 * (16 * h + i), a, lane);
          if (lane == src) {
#pragma unroll
            for (int ii = 0; ii < 16; ++ii)
              if (ii == i) v[ii] = make_float2(val.x * bscale, val.y * bscale);
            fl &= ~(1u << i);
          }
          pending = __ballot_sync(0xffffffffu, fl != 0);
        }
      }
    } else {
      bad |= !tc::mbar_wait(barX, px);
      px ^= 1;
      if (wt == 0) pendX = 0;
#pragma unroll
      for (int i = 0; i < 16; ++i) v[i] = Xs[lane + 32 * (16 * h + i)];
      bscale = 1.f;
    }
    // ---- LS division F = Y / X_p (Eq. (16)), i = lane + 32 n2, n2 = 16 h + j
    bad |= !tc::mbar_wait(barY, py);
    py ^= 1;
    if (wt == 0) pendY = 0;
    {
      const float mul = a.zc ? sgn0 * a.sqrtN * bscale : 1.f;
      float mx = 0.f;
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int i = lane + 32 * (16 * h + j);
        float2 yv = Ys[i];
        if (!R1Q0 && a.zc && !a.post_sign) yv = cmul(yv, __ldg(a.post_conj + i));
        const float d2 = v[j].x * v[j].x + v[j].y * v[j].y;
        flags |= (d2 == 0.f) ? OFDM_STATUS_ZERO_X : 0u;
        const float inv = (d2 > 0.f) ? mul * rcp_fast(d2) : 0.f;
        v[j] = cscale(cmulc(yv, v[j]), inv);
        mx = fmaxf(mx, fmaxf(fabsf(v[j].x), fabsf(v[j].y)));
      }
      // ---- stage 3: rows (q, k2 = lane), K = (k1 = n2, re/im)
      const float s3 = pow2_scale(symbol_max(mx, 2));
      store_row16(v, s3, ahi, alo, 32 * q + lane, h);
      tc::fence_proxy_async();
      tc::fence_before_sync();
      if (wg_sync_or(wg, bad)) break;
      next = s_next[wg];
      if (wt == 0) {
        if (next < tiles) {   // Y (and X, without the ZC stages) rows consumed
          issue(Y, next, u_ys, barY);
          pendY = 1;
          if (!a.zc) { issue(X, next, u_xs, barX); pendX = 1; }
        }
        tc::fence_after_sync();
        issue_stage(tmem, sd, kIdesc64);
        tc::mma_commit(barM);
        pendM = 1;
      }
      bad |= !tc::mbar_wait(barM, pm);
      pm ^= 1;
      if (wt == 0) pendM = 0;
      tc::fence_after_sync();
      // ---- stage 4: twiddle; rows (q, m1), K = (k2 = lane, re/im); 8 output rows (n < 256)
      load_acc32(tacc + 32 * h, v);
#pragma unroll
      for (int i = 0; i < 16; ++i) v[i] = cmul(v[i], T12[(16 * h + i) * 32 + lane]);
      store_col16(v, ahi, alo, 32 * q + 16 * h, lane);
      tc::fence_proxy_async();
      tc::fence_before_sync();
      if (wg_sync_or(wg, bad)) break;
      if (wt == 0) {
        tc::fence_after_sync();
        issue_stage(tmem, sd, kIdesc16);
        tc::mma_commit(barM);
        pendM = 1;
      }
      bad |= !tc::mbar_wait(barM, pm);
      pm ^= 1;
      if (wt == 0) pendM = 0;
      tc::fence_after_sync();
      float hf[16];
      tc::tmem_ld16(tacc, hf);   // row (q, m1 = lane): h[lane + 32 m2] * s3 / 32, m2 < 8
      tc::tmem_wait_ld();
      // ---- keep taps n < L_cp (Eq. (21)); g[r] = c0 h[r] + c1 (h[r-1] + h[r+1]) (Eqs. (17), (22))
      const float un = 32.f / s3;
      float2 hh[8];
#pragma unroll
      for (int m2 = 0; m2 < 8; ++m2) {
        const int n = lane + 32 * m2;
        hh[m2] = n < a.L_cp ? make_float2(hf[2 * m2] * un, hf[2 * m2 + 1] * un) : make_float2(0.f, 0.f);
      }
      float2* ex = reinterpret_cast<float2*>(ahi);   // [rows][4] exchange (the A image is free now)
#pragma unroll
      for (int m2 = 0; m2 < 8; ++m2) {
        const float2 lo_prev = make_float2(__shfl_sync(0xffffffffu, hh[m2 > 0 ? m2 - 1 : 0].x, 31),
                                           __shfl_sync(0xffffffffu, hh[m2 > 0 ? m2 - 1 : 0].y, 31));
        const float2 hi_next = make_float2(__shfl_sync(0xffffffffu, hh[m2 < 7 ? m2 + 1 : 7].x, 0),
                                           __shfl_sync(0xffffffffu, hh[m2 < 7 ? m2 + 1 : 7].y, 0));
        float2 hm = make_float2(__shfl_up_sync(0xffffffffu, hh[m2].x, 1), __shfl_up_sync(0xffffffffu, hh[m2].y, 1));
        float2 hp = make_float2(__shfl_down_sync(0xffffffffu, hh[m2].x, 1),
                                __shfl_down_sync(0xffffffffu, hh[m2].y, 1));
        if (lane == 0) hm = m2 > 0 ? lo_prev : make_float2(0.f, 0.f);
        if (lane == 31) hp = m2 < 7 ? hi_next : make_float2(0.f, 0.f);
        const int r = lane + 32 * m2;
        const int ri = (r - a.row0) & (kN - 1);
        if ((m2 >> 2) == h && ri < a.rows) {   // the two column halves write alternate row blocks
          float2 g;
          g.x = a.c0 * hh[m2].x + a.c1 * (hm.x + hp.x);
          g.y = a.c0 * hh[m2].y + a.c1 * (hm.y + hp.y);
          flags |= (isfinite(g.x) && isfinite(g.y)) ? 0u : OFDM_STATUS_NONFINITE;
          ex[ri * 4 + q] = g;
        }
      }
      if (h == 0 && lane == 0 && a.row0 != 0) {   // r = N - 1: the window's spill of tap 0 (h[N-1] = h[N-2] = 0)
        const int ri = (kN - 1 - a.row0) & (kN - 1);
        const float2 g = make_float2(a.c1 * hh[0].x, a.c1 * hh[0].y);
        flags |= (isfinite(g.x) && isfinite(g.y)) ? 0u : OFDM_STATUS_NONFINITE;
        ex[ri * 4 + q] = g;
      }
      wg_sync_or(wg, false);
      // each row's 4 consecutive symbols are 32 contiguous bytes of the strip
      for (int ri = wt; ri < a.rows; ri += kWgThreads) {
        const float4* e4 = reinterpret_cast<const float4*>(ex + ri * 4);
        float4* d = reinterpret_cast<float4*>(strip + ((long)f * a.rows + ri) * a.M + l0);
        d[0] = e4[0];
        d[1] = e4[1];
      }
    }
    flags = __reduce_or_sync(0xffffffffu, flags);
    if (lane == 0 && flags) atomicOr(wstatus + f, flags);
    if (wg_sync_or(wg, bad)) break;   // the exchange has been read before the next tile's operands
    tile = next;
  }
  if (bad && wt == 0) {
    // A wait ran out.  Report it on the frames this warpgroup leaves
    // unprocessed: the current tile's, the one drawn for next, and every
    // tile it still draws until the counter runs past the end (which keeps
    // the ticket count of the launch exact for the next one).  Then wait
    // (bounded) for the copies and products it issued before TMEM is released.
    const uint32_t to = (uint32_t)OFDM_STATUS_TIMEOUT;
    if (tile < tiles) atomicOr(wstatus + (int)(tile / tiles_per_frame), to);
    long t = s_next[wg];
    while (t < tiles) {
      atomicOr(wstatus + (int)(t / tiles_per_frame), to);
      t = draw();
    }
    if (pendX) tc::mbar_wait(barX, px);
    if (pendY) tc::mbar_wait(barY, py);
    if (pendM) tc::mbar_wait(barM, pm);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (tid < 32) tc::tmem_dealloc(s_tmem, 128);
}

}  // namespace

size_t tc_table_bytes() { return kBBytes; }

// The real form of the 32-point DFT w_32^(+n k) as the B operand image:
// row (n, c) (output n, component c), column (k, c') (input k, component
// c'), K-major, split into fp16 hi and lo halves (exact FP64 cos / sin).
void build_tc_tables(unsigned char* b, float2* t12) {
  for (int n = 0; n < 32; ++n)
    for (int k = 0; k < 32; ++k) {
      const double th = 2.0 * M_PI * (double)((n * k) % 32) / 32.0, c = cos(th), s = sin(th);
      // out_re = in_re c - in_im s, out_im = in_re s + in_im c
      const double e[2][2] = {{c, -s}, {s, c}};   // e[out c][in c']
      for (int co = 0; co < 2; ++co)
        for (int ci = 0; ci < 2; ++ci) {
          const double val = e[co][ci];
          const __half hi = __float2half_rn((float)val);
          const __half lo = __float2half_rn((float)(val - (double)__half2float(hi)));
          const uint32_t off = tc::kmajor_off(2 * n + co, 2 * k + ci, kLboB, kSBO);
          memcpy(b + off, &hi, 2);
          memcpy(b + kBBytes + off, &lo, 2);
        }
    }
  for (int n1 = 0; n1 < 32; ++n1)
    for (int k2 = 0; k2 < 32; ++k2) {
      const double th = 2.0 * M_PI * (double)(n1 * k2) / 1024.0;
      t12[n1 * 32 + k2] = make_float2((float)(cos(th) / 32.0), (float)(sin(th) / 32.0));
    }
}

cudaError_t launch_column_tc(const float2* Y, const float2* X, float2* strip, uint32_t* wstatus, const ColumnArgs& a,
                             cudaStream_t s, unsigned long long* tickets) {
  *tickets = 0;
  auto kern = (a.rinv == 1 && a.post_sign) ? column_tc_kernel<true> : column_tc_kernel<false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const long tiles = (long)a.frames * (a.M / 4);
  long blocks = sms;
  const long need = (tiles + kWG - 1) / kWG;
  if (blocks > need) blocks = need;
  kern<<<(unsigned)blocks, kThreads, kSmemBytes, s>>>(Y, X, strip, wstatus, a);
  *tickets = (unsigned long long)tiles + (unsigned long long)blocks * kWG;
  return cudaGetLastError();
}

}  // namespace ofdm
