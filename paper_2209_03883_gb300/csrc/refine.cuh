// refine.cuh -- double-float recomputation of ill-conditioned precoded cells
// (shared by the FP32 and the tensor-core column kernels).
#pragma once
#include "fft.cuh"
#include "internal.h"

namespace ofdm {

// Precoded cells with |X_p|^2 below this fraction of the symbol's mean power
// are recomputed in double-float (about 5e-5 of the cells for a ZC-precoded
// QAM grid), which keeps the FP32 chain's map error within half of the 1e-5
// gate even when the LS division meets a near-zero precoded cell.  Each
// recomputed cell costs an N-term double-float sum, so the threshold trades
// the column stage's time against that margin.
#ifndef OFDM_REFINE_TAU
#define OFDM_REFINE_TAU 5e-5f
#endif
constexpr float kRefineTau = OFDM_REFINE_TAU;

// B_i = sum_k pre_k A_k exp(+2 pi i r' i k / N) in double-float by the whole
// warp (lane handles k = lane, lane + 32, ...), rounded once to float.  Used
// for precoded cells so small that the FP32 FFT's normwise rounding would be
// amplified by the LS division (|X_p|^2 < tau * mean).
template <int N>
__device__ __noinline__ float2 refine_cell(const float2* __restrict__ x, int i, const ColumnArgs& a, int lane) {
  cdf acc = {{0.f, 0.f}, {0.f, 0.f}};
  for (int k = lane; k < N; k += 32) {
    const cdf b = cdf_mulf(cdf_ld(a.pre_df + k), __ldg(x + k));
    const unsigned m = ((unsigned)a.rprime * (unsigned)i * (unsigned)k) & (unsigned)(N - 1);
    acc = cdf_add(acc, cdf_mul(b, cdf_ld(a.w_df + m)));
  }
#pragma unroll
  for (int off = 16; off; off >>= 1) {
    acc.re = df_add(acc.re, df_shfl_xor(acc.re, off));
    acc.im = df_add(acc.im, df_shfl_xor(acc.im, off));
  }
  return make_float2(acc.re.hi + acc.re.lo, acc.im.hi + acc.im.lo);
}

// After the ZC FFT: find this warp's ill-conditioned cells and recompute them.
// Thread t of a T-thread group holds positions i = t + T q.
// `scale` multiplies the recomputed value: the caller's v may hold the
// transform scaled by a power of two.
template <int N, int T, int E>
__device__ __forceinline__ void refine_small_cells(float2* v, const float2* __restrict__ x, const ColumnArgs& a,
                                                   int t, int lane, float scale = 1.f) {
  float s2 = 0.f;
#pragma unroll
  for (int q = 0; q < E; ++q) s2 += v[q].x * v[q].x + v[q].y * v[q].y;
#pragma unroll
  for (int off = 16; off; off >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, off);
  const float thr = a.refine_tau * s2 * (1.f / (32.f * E));
  unsigned flags = 0;
#pragma unroll
  for (int q = 0; q < E; ++q) flags |= (v[q].x * v[q].x + v[q].y * v[q].y < thr) ? (1u << q) : 0u;
  unsigned pending = __ballot_sync(0xffffffffu, flags != 0);
  while (pending) {
    const int src = __ffs(pending) - 1;
    const unsigned fm = __shfl_sync(0xffffffffu, flags, src);
    const int q = __ffs(fm) - 1;
    const int tsrc = __shfl_sync(0xffffffffu, t, src);
    float2 val = refine_cell<N>(x, tsrc + T * q, a, lane);
    val.x *= scale;
    val.y *= scale;
    if (lane == src) {
#pragma unroll
      for (int qq = 0; qq < E; ++qq)
        if (qq == q) v[qq] = val;
      flags &= ~(1u << q);
    }
    pending = __ballot_sync(0xffffffffu, flags != 0);
  }
}

}  // namespace ofdm
