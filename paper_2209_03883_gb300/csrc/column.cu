// column.cu -- the per-OFDM-symbol half of the chain (steps a1-a5) and the
// stand-alone ZC transform.
//
// One thread group (a warp for N <= 1024, N/32 threads above) owns one OFDM
// symbol l of one frame at a time:
//   1. load the known grid X[l, :] (coalesced, streaming) and apply the ZC
//      transform of Sec. III-B, X_p = Z_m A / sqrt(N), written as
//      pre-chirp -> N-point DFT (+) -> post factor (Eqs. (23)-(24));
//   2. load Y[l, :] and divide, F = Y / X_p (Eq. (16));
//   3. DFT-CE's IDFT over subcarriers (Eq. (20)) by a second N-point DFT (+);
//   4. keep the first L_cp taps (Eq. (21)).  The DFT back (Eq. (22)) followed
//      by the windowed range IDFT of Eq. (17) collapses to a 3-tap circular
//      stencil of the kept taps (periodic Hann/Hamming) or to the taps
//      themselves (rect), so only the L_cp(+2) support rows are produced;
//   5. write those rows g[r, l] into the range-profile strip.
// Both 1/N and N factors of Eqs. (20)/(22) and the range sum cancel.
#include "fft.cuh"
#include "internal.h"

namespace ofdm {

template <int N>
struct ColCfg {
  static constexpr int T = N <= 1024 ? 32 : N / 32;   // threads per symbol
  static constexpr int E = N / T;                     // points per thread
  static constexpr int GROUPS = N <= 1024 ? 8 : (N == 2048 ? 4 : 2);
  static constexpr int THREADS = T * GROUPS;
  static constexpr size_t SMEM = (size_t)GROUPS * smem_elems(N) * sizeof(float2);
};

template <int N>
__global__ void __launch_bounds__(ColCfg<N>::THREADS)
column_kernel(const float2* __restrict__ Y, const float2* __restrict__ X, float2* __restrict__ strip,
              uint32_t* __restrict__ wstatus, ColumnArgs a) {
  using C = ColCfg<N>;
  constexpr int T = C::T, E = C::E;
  extern __shared__ float2 smem[];
  const int group = threadIdx.x / T;
  const int t = threadIdx.x % T;
  float2* sm = smem + group * smem_elems(N);
  const long total = (long)a.frames * a.M;

  for (long sym = (long)blockIdx.x * C::GROUPS + group; sym < total; sym += (long)gridDim.x * C::GROUPS) {
    const int f = (int)(sym / a.M);
    const int l = (int)(sym % a.M);
    const float2* x = X + sym * N;
    const float2* y = Y + sym * N;
    float2 v[E];
    uint32_t flags = 0;

    if (a.zc) {
      // b~[k'] = pre[s] A[s], s = r'^{-1} k' mod N, so that the DFT below
      // yields B[r' i] = sum_k pre_k A_k e^{+2 pi i r' i k / N} at position i.
#pragma unroll
      for (int q = 0; q < E; ++q) {
        const int k = t + T * q;
        const int s = (a.rinv == 1) ? k : (int)(((unsigned)a.rinv * (unsigned)k) & (N - 1));
        const float2 xv = (a.rinv == 1) ? ld_stream(x + s) : __ldg(x + s);
        v[q] = cmul(xv, __ldg(a.pre + s));
      }
      group_fft<N, T, +1>(v, sm, a.tw, t, group);
      // F_i = Y_i / X_p,i with X_p,i = post_i B / sqrt(N):
      //     F_i = Y_i conj(post_i) sqrt(N) conj(B) / |B|^2.
#pragma unroll
      for (int q = 0; q < E; ++q) {
        const int i = t + T * q;
        const float2 yv = cmul(ld_stream(y + i), __ldg(a.post_conj + i));
        const float d2 = v[q].x * v[q].x + v[q].y * v[q].y;
        flags |= (d2 == 0.f) ? OFDM_STATUS_ZERO_X : 0u;
        const float inv = (d2 > 0.f) ? a.sqrtN / d2 : 0.f;
        v[q] = cscale(cmulc(yv, v[q]), inv);
      }
    } else {
#pragma unroll
      for (int q = 0; q < E; ++q) {
        const int i = t + T * q;
        const float2 xv = ld_stream(x + i);
        const float2 yv = ld_stream(y + i);
        const float d2 = xv.x * xv.x + xv.y * xv.y;
        flags |= (d2 == 0.f) ? OFDM_STATUS_ZERO_X : 0u;
        const float inv = (d2 > 0.f) ? 1.f / d2 : 0.f;
        v[q] = cscale(cmulc(yv, xv), inv);
      }
    }

    // N h[n] = sum_i F_i e^{+2 pi i n i / N}   (Eq. (20) times N)
    group_fft<N, T, +1>(v, sm, a.tw, t, group);

    group_sync<T>(group);  // the last FFT pass finished reading sm
#pragma unroll
    for (int q = 0; q < E; ++q) {
      const int n = t + T * q;
      if (n < a.L_cp) sm[pad32(n)] = v[q];
    }
    group_sync<T>(group);

    // g[r] = c0 h[r] + c1 (h[r-1] + h[r+1]), h zero beyond the kept taps.
    for (int ri = t; ri < a.rows; ri += T) {
      const int r = (a.row0 + ri) & (N - 1);
      const int rm = (r - 1) & (N - 1), rp = (r + 1) & (N - 1);
      const float2 z = make_float2(0.f, 0.f);
      const float2 h0 = r < a.L_cp ? sm[pad32(r)] : z;
      const float2 hm = rm < a.L_cp ? sm[pad32(rm)] : z;
      const float2 hp = rp < a.L_cp ? sm[pad32(rp)] : z;
      float2 g;
      g.x = a.c0 * h0.x + a.c1 * (hm.x + hp.x);
      g.y = a.c0 * h0.y + a.c1 * (hm.y + hp.y);
      flags |= (isfinite(g.x) && isfinite(g.y)) ? 0u : OFDM_STATUS_NONFINITE;
      strip[((long)f * a.rows + ri) * a.M + l] = g;
    }

    // One atomic per group and only when something was flagged.
    if constexpr (T <= 32) {
      flags = __reduce_or_sync(0xffffffffu, flags);
      if (t == 0 && flags) atomicOr(wstatus + f, flags);
    } else {
      if (flags) atomicOr(wstatus + f, flags);
    }
  }
}

template <int N>
__global__ void __launch_bounds__(ColCfg<N>::THREADS)
zct_kernel(const float2* __restrict__ in, float2* __restrict__ out, ZctArgs a) {
  using C = ColCfg<N>;
  constexpr int T = C::T, E = C::E;
  extern __shared__ float2 smem[];
  const int group = threadIdx.x / T;
  const int t = threadIdx.x % T;
  float2* sm = smem + group * smem_elems(N);
  const long total = (long)a.frames * a.M;
  for (long sym = (long)blockIdx.x * C::GROUPS + group; sym < total; sym += (long)gridDim.x * C::GROUPS) {
    const float2* x = in + sym * N;
    float2* o = out + sym * N;
    float2 v[E];
#pragma unroll
    for (int q = 0; q < E; ++q) {
      const int k = t + T * q;
      const int s = (int)(((unsigned)a.rinv * (unsigned)k) & (N - 1));
      v[q] = cmul(__ldg(x + s), __ldg(a.in_tab + s));
    }
    if (a.dir > 0)
      group_fft<N, T, +1>(v, sm, a.tw, t, group);
    else
      group_fft<N, T, -1>(v, sm, a.tw, t, group);
#pragma unroll
    for (int q = 0; q < E; ++q) {
      const int i = t + T * q;
      o[i] = cscale(cmul(v[q], __ldg(a.out_tab + i)), a.scale);
    }
  }
}

template <int N>
static cudaError_t launch_column_n(const float2* Y, const float2* X, float2* strip, uint32_t* wstatus,
                                   const ColumnArgs& a, cudaStream_t s) {
  using C = ColCfg<N>;
  cudaError_t e = cudaFuncSetAttribute(column_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)C::SMEM);
  if (e != cudaSuccess) return e;
  const long total = (long)a.frames * a.M;
  const long blocks = (total + C::GROUPS - 1) / C::GROUPS;
  column_kernel<N><<<(unsigned)blocks, C::THREADS, C::SMEM, s>>>(Y, X, strip, wstatus, a);
  return cudaGetLastError();
}

template <int N>
static cudaError_t launch_zct_n(const float2* in, float2* out, const ZctArgs& a, cudaStream_t s) {
  using C = ColCfg<N>;
  cudaError_t e =
      cudaFuncSetAttribute(zct_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
  if (e != cudaSuccess) return e;
  const long total = (long)a.frames * a.M;
  const long blocks = (total + C::GROUPS - 1) / C::GROUPS;
  zct_kernel<N><<<(unsigned)blocks, C::THREADS, C::SMEM, s>>>(in, out, a);
  return cudaGetLastError();
}

cudaError_t launch_column(int N, const float2* Y, const float2* X, float2* strip, uint32_t* wstatus,
                          const ColumnArgs& a, cudaStream_t s, int* launches) {
  ++*launches;
  switch (N) {
    case 64: return launch_column_n<64>(Y, X, strip, wstatus, a, s);
    case 128: return launch_column_n<128>(Y, X, strip, wstatus, a, s);
    case 256: return launch_column_n<256>(Y, X, strip, wstatus, a, s);
    case 512: return launch_column_n<512>(Y, X, strip, wstatus, a, s);
    case 1024: return launch_column_n<1024>(Y, X, strip, wstatus, a, s);
    case 2048: return launch_column_n<2048>(Y, X, strip, wstatus, a, s);
    case 4096: return launch_column_n<4096>(Y, X, strip, wstatus, a, s);
    default: --*launches; return cudaErrorInvalidValue;
  }
}

cudaError_t launch_zct(int N, const float2* in, float2* out, const ZctArgs& a, cudaStream_t s,
                       int* launches) {
  ++*launches;
  switch (N) {
    case 64: return launch_zct_n<64>(in, out, a, s);
    case 128: return launch_zct_n<128>(in, out, a, s);
    case 256: return launch_zct_n<256>(in, out, a, s);
    case 512: return launch_zct_n<512>(in, out, a, s);
    case 1024: return launch_zct_n<1024>(in, out, a, s);
    case 2048: return launch_zct_n<2048>(in, out, a, s);
    case 4096: return launch_zct_n<4096>(in, out, a, s);
    default: --*launches; return cudaErrorInvalidValue;
  }
}

}  // namespace ofdm
