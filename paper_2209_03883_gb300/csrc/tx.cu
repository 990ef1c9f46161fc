// tx.cu -- the transmit side of Sec. III-B on the GPU: the PAPR (Eq. (25))
// of the oversampled OFDM time signal and the out-of-band power that the
// power amplifier's nonlinearity adds (the adjacent-channel interference of
// the paper's spectrum study).
//
// Per OFDM symbol (one thread group, T threads, E = LN / T points each):
//   1. place the N subcarriers of the transmitted grid on an L N-point
//      frequency grid (subcarrier k at bin k for k < N/2, at k + (L-1) N
//      otherwise) and take x[n] = sum_f Z[f] e^{+2 pi i f n / (L N)};
//   2. PAPR = max |x|^2 / mean |x|^2;
//   3. amplifier: |y| = |x| / sqrt(1 + (|x| / (x_bar 10^(q/10)))^2), phase
//      kept, x_bar the mean modulus of the symbol's samples;
//   4. Y = DFT(y); ACI = power outside the N occupied bins / total power.
#include "fft.cuh"
#include "internal.h"

namespace ofdm {

template <int LN>
struct TxCfg {
  static constexpr int T = LN <= 1024 ? 32 : LN / 32;
  static constexpr int E = LN / T;
  static constexpr int GROUPS = 4;
  static constexpr int THREADS = T * GROUPS;
  static constexpr int WARPS = T / 32;
};

// Sum (op 0) or maximum (op 1) over the T threads of a group.
template <int T>
__device__ __forceinline__ float group_reduce(float v, int op, float* part, int group, int t) {
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    const float u = __shfl_xor_sync(0xffffffffu, v, o);
    v = op ? fmaxf(v, u) : v + u;
  }
  if constexpr (T > 32) {
    group_sync<T>(group);                 // earlier readers of part are done
    if ((t & 31) == 0) part[t >> 5] = v;
    group_sync<T>(group);
    v = part[0];
#pragma unroll
    for (int w = 1; w < T / 32; ++w) v = op ? fmaxf(v, part[w]) : v + part[w];
  }
  return v;
}

template <int LN>
__global__ void __launch_bounds__(TxCfg<LN>::THREADS)
tx_kernel(const float2* __restrict__ S, float* __restrict__ papr, float* __restrict__ aci, TxArgs a) {
  using C = TxCfg<LN>;
  constexpr int T = C::T, E = C::E;
  extern __shared__ float2 tx_smem[];
  __shared__ float s_part[C::GROUPS][C::WARPS > 0 ? C::WARPS : 1];
  const int group = threadIdx.x / T, t = threadIdx.x % T;
  float2* sm = tx_smem + (size_t)group * smem_elems(LN);
  const int N = a.N, half = N / 2;
  const long total = (long)a.frames * a.M;
  for (long sym = (long)blockIdx.x * C::GROUPS + group; sym < total; sym += (long)gridDim.x * C::GROUPS) {
    const float2* s = S + sym * N;
    float2 v[E];
#pragma unroll
    for (int q = 0; q < E; ++q) {
      const int f = t + T * q;
      v[q] = f < half ? s[f] : (f >= LN - half ? s[f - (LN - N)] : make_float2(0.f, 0.f));
    }
    group_fft<LN, T, +1>(v, sm, a.tw, t, group);
    float pmax = 0.f, psum = 0.f, asum = 0.f;
#pragma unroll
    for (int q = 0; q < E; ++q) {
      const float p = v[q].x * v[q].x + v[q].y * v[q].y;
      pmax = fmaxf(pmax, p);
      psum += p;
      asum += sqrtf(p);
    }
    pmax = group_reduce<T>(pmax, 1, s_part[group], group, t);
    psum = group_reduce<T>(psum, 0, s_part[group], group, t);
    asum = group_reduce<T>(asum, 0, s_part[group], group, t);
    const float sat = asum / (float)LN * a.sat_factor;
    const float inv_sat2 = sat > 0.f ? 1.f / (sat * sat) : 0.f;
#pragma unroll
    for (int q = 0; q < E; ++q) {
      const float p = v[q].x * v[q].x + v[q].y * v[q].y;
      v[q] = cscale(v[q], rsqrtf(1.f + p * inv_sat2));
    }
    group_fft<LN, T, -1>(v, sm, a.tw, t, group);
    float oob = 0.f, all = 0.f;
#pragma unroll
    for (int q = 0; q < E; ++q) {
      const int f = t + T * q;
      const float p = v[q].x * v[q].x + v[q].y * v[q].y;
      all += p;
      oob += (f >= half && f < LN - half) ? p : 0.f;
    }
    oob = group_reduce<T>(oob, 0, s_part[group], group, t);
    all = group_reduce<T>(all, 0, s_part[group], group, t);
    if (t == 0) {
      if (papr) papr[sym] = psum > 0.f ? pmax / (psum / (float)LN) : 0.f;
      if (aci) aci[sym] = all > 0.f ? oob / all : 0.f;
    }
    group_sync<T>(group);   // sm and s_part are reused by the next symbol
  }
}

template <int LN>
static cudaError_t launch_tx_n(const float2* S, float* papr, float* aci, const TxArgs& a, cudaStream_t s) {
  using C = TxCfg<LN>;
  const size_t smem = (size_t)C::GROUPS * smem_elems(LN) * sizeof(float2);
  cudaError_t e = cudaFuncSetAttribute(tx_kernel<LN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const long total = (long)a.frames * a.M;
  long blocks = (total + C::GROUPS - 1) / C::GROUPS;
  if (blocks > 152L * 8) blocks = 152L * 8;
  tx_kernel<LN><<<(unsigned)blocks, C::THREADS, smem, s>>>(S, papr, aci, a);
  return cudaGetLastError();
}

int tx_points_per_thread(int LN) { return LN <= 1024 ? LN / 32 : 32; }

cudaError_t launch_tx(int LN, const float2* S, float* papr, float* aci, const TxArgs& a, cudaStream_t s,
                      int* launches) {
  ++*launches;
  switch (LN) {
    case 64: return launch_tx_n<64>(S, papr, aci, a, s);
    case 128: return launch_tx_n<128>(S, papr, aci, a, s);
    case 256: return launch_tx_n<256>(S, papr, aci, a, s);
    case 512: return launch_tx_n<512>(S, papr, aci, a, s);
    case 1024: return launch_tx_n<1024>(S, papr, aci, a, s);
    case 2048: return launch_tx_n<2048>(S, papr, aci, a, s);
    case 4096: return launch_tx_n<4096>(S, papr, aci, a, s);
    default: --*launches; return cudaErrorInvalidValue;
  }
}

}  // namespace ofdm
