// range_pad.cu -- the range transform of Eq. (17) with zero padding N' > N.
//
// Without padding, the DFT back of DFT-CE followed by the windowed range IDFT
// collapses to a 3-tap stencil of the kept taps, so only L_cp + 2 rows can be
// non-zero.  On a padded grid (N' = P N) the range IDFT interpolates between
// bins and every one of the N' rows carries signal, so each OFDM symbol's
// range profile is computed in full from the kept taps N h[n] (which the
// column kernel writes with a rect stencil):
//   H'[k] = sum_{n < L_cp} h[n] e^{-2 pi i n k / N}        (the DFT back, Eq. (22))
//   g[r]  = sum_{k < N} w_k H'[k] e^{+2 pi i k r / N'}     (r < N', Eq. (17))
// One group of T threads per symbol runs the N-point DFT and the N'-point
// inverse DFT in registers (layout t + T q: the first N / T slots of the
// N'-point transform are exactly the bins k < N, the rest are the padding).
#include "fft.cuh"
#include "internal.h"

namespace ofdm {

template <int NP>
struct PadCfg {
  static constexpr int T = NP <= 1024 ? 32 : NP / 32;
  static constexpr int GROUPS = NP <= 1024 ? 8 : (NP == 2048 ? 4 : 2);
  static constexpr int THREADS = T * GROUPS;
  static constexpr size_t SMEM = (size_t)GROUPS * smem_elems(NP) * sizeof(float2);
};

template <int N, int NP>
__global__ void __launch_bounds__(PadCfg<NP>::THREADS)
range_pad_kernel(const float2* __restrict__ taps, float2* __restrict__ strip, PadArgs a) {
  using C = PadCfg<NP>;
  constexpr int T = C::T, EN = N / T, EP = NP / T;
  static_assert(EN >= 2 && EP >= EN, "padding factor");
  extern __shared__ float2 pad_smem[];
  const int group = threadIdx.x / T, t = threadIdx.x % T;
  float2* sm = pad_smem + (size_t)group * smem_elems(NP);
  const long total = (long)a.frames * a.M;
  const float invN = 1.f / (float)N;
  for (long sym = (long)blockIdx.x * C::GROUPS + group; sym < total; sym += (long)gridDim.x * C::GROUPS) {
    const long f = sym / a.M;
    const int l = (int)(sym % a.M);
    float2 v[EP];
#pragma unroll
    for (int q = 0; q < EN; ++q) {
      const int n = t + T * q;
      v[q] = n < a.L_cp ? cscale(__ldg(taps + ((size_t)f * a.L_cp + n) * a.M + l), invN) : make_float2(0.f, 0.f);
    }
    group_fft<N, T, -1>(v, sm, a.twN, t, group);            // H'[k], k = t + T q
#pragma unroll
    for (int q = 0; q < EN; ++q) v[q] = cscale(v[q], __ldg(a.wk + t + T * q));
#pragma unroll
    for (int q = EN; q < EP; ++q) v[q] = make_float2(0.f, 0.f);
    group_sync<T>(group);                                    // the N-point pass is done with sm
    group_fft<NP, T, +1>(v, sm, a.twP, t, group);           // g[r], r = t + T q
    float2* out = strip + (size_t)f * NP * a.M + l;
#pragma unroll
    for (int q = 0; q < EP; ++q) out[(size_t)(t + T * q) * a.M] = v[q];
    group_sync<T>(group);                                    // sm is reused by the next symbol
  }
}

int pad_threads(int NP) { return NP <= 1024 ? 32 : NP / 32; }

template <int N, int NP>
static cudaError_t launch_pad_n(const float2* taps, float2* strip, const PadArgs& a, cudaStream_t s) {
  using C = PadCfg<NP>;
  cudaError_t e = cudaFuncSetAttribute(range_pad_kernel<N, NP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)C::SMEM);
  if (e != cudaSuccess) return e;
  const long total = (long)a.frames * a.M;
  long blocks = (total + C::GROUPS - 1) / C::GROUPS;
  if (blocks > 152L * 16) blocks = 152L * 16;
  range_pad_kernel<N, NP><<<(unsigned)blocks, C::THREADS, C::SMEM, s>>>(taps, strip, a);
  return cudaGetLastError();
}

template <int N>
static cudaError_t launch_pad_np(int NP, const float2* taps, float2* strip, const PadArgs& a, cudaStream_t s) {
  if constexpr (N * 2 <= 4096) {
    if (NP == 2 * N) return launch_pad_n<N, 2 * N>(taps, strip, a, s);
  }
  if constexpr (N * 4 <= 4096) {
    if (NP == 4 * N) return launch_pad_n<N, 4 * N>(taps, strip, a, s);
  }
  if constexpr (N * 8 <= 4096) {
    if (NP == 8 * N) return launch_pad_n<N, 8 * N>(taps, strip, a, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_range_pad(int N, int NP, const float2* taps, float2* strip, const PadArgs& a, cudaStream_t s,
                             int* launches) {
  ++*launches;
  switch (N) {
    case 64: return launch_pad_np<64>(NP, taps, strip, a, s);
    case 128: return launch_pad_np<128>(NP, taps, strip, a, s);
    case 256: return launch_pad_np<256>(NP, taps, strip, a, s);
    case 512: return launch_pad_np<512>(NP, taps, strip, a, s);
    case 1024: return launch_pad_np<1024>(NP, taps, strip, a, s);
    case 2048: return launch_pad_np<2048>(NP, taps, strip, a, s);
    default: --*launches; return cudaErrorInvalidValue;
  }
}

}  // namespace ofdm
