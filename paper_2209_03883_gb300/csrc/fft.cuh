// fft.cuh -- register/shared-memory FFT building blocks for sm_103a.
//
// A transform of N = 2^p points is computed by T cooperating threads, each
// holding E = N / T points in registers in the layout
//     thread t holds x[t + T q],  q = 0 .. E-1,
// which is also the coalesced global-memory pattern (for every q the T
// threads touch T consecutive complex values).  The transform is a sequence
// of Stockham auto-sort passes of radix R <= E; inside a pass every thread
// runs G = E / R radix-R DFTs fully in registers (compile-time twiddles),
// and passes exchange data through a padded shared-memory buffer.  The first
// pass reads its operands straight from the registers and the last pass
// leaves its results in registers in the same layout, so only
// (passes - 1) shared-memory exchanges happen (one for N = 1024).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <utility>

namespace ofdm {

// ---------------------------------------------------------------- constexpr math
constexpr double kPi = 3.14159265358979323846264338327950288;

constexpr double cx_reduce(double x) {
  while (x > kPi) x -= 2.0 * kPi;
  while (x < -kPi) x += 2.0 * kPi;
  return x;
}
constexpr double cx_sin(double x) {
  x = cx_reduce(x);
  double term = x, sum = x;
  for (int n = 1; n < 24; ++n) {
    term *= -x * x / ((2.0 * n) * (2.0 * n + 1.0));
    sum += term;
  }
  return sum;
}
constexpr double cx_cos(double x) {
  x = cx_reduce(x);
  double term = 1.0, sum = 1.0;
  for (int n = 1; n < 24; ++n) {
    term *= -x * x / ((2.0 * n - 1.0) * (2.0 * n));
    sum += term;
  }
  return sum;
}
constexpr int cx_log2(int n) { return n <= 1 ? 0 : 1 + cx_log2(n / 2); }
constexpr int cx_brev(int i, int bits) {
  int r = 0;
  for (int b = 0; b < bits; ++b) r = (r << 1) | ((i >> b) & 1);
  return r;
}

// ---------------------------------------------------------------- pass schedule
// Radix of pass p for an N-point transform with E points per thread: as many
// radix-E passes as divide N, then the remainder.  Shared by the host table
// builder and the kernels.
__host__ __device__ constexpr int pass_radix(int N, int E, int p) {
  int rem = N, r = 1;
  for (int i = 0; i <= p; ++i) {
    r = E < rem ? E : rem;
    while (rem % r) r /= 2;
    rem /= r;
  }
  return r;
}
__host__ __device__ constexpr int num_passes(int N, int E) {
  int rem = N, n = 0;
  while (rem > 1) {
    int r = E < rem ? E : rem;
    while (rem % r) r /= 2;
    rem /= r;
    ++n;
  }
  return n;
}
__host__ __device__ constexpr int pass_ns(int N, int E, int p) {
  int ns = 1;
  for (int i = 0; i < p; ++i) ns *= pass_radix(N, E, i);
  return ns;
}
// Twiddle table offset of pass p (pass 0 needs none):
// tab[off(p) + r * Ns + u] = exp(+2 pi i u r / (Ns R)), u < Ns, r < R.
__host__ __device__ constexpr int tw_offset(int N, int E, int p) {
  int off = 0;
  for (int i = 1; i < p; ++i) off += pass_ns(N, E, i) * pass_radix(N, E, i);
  return off;
}
__host__ __device__ constexpr int tw_size(int N, int E) { return tw_offset(N, E, num_passes(N, E)); }

// Padded shared-memory index: one spare slot per 32 elements keeps the
// stride-32 writes of the first pass free of bank conflicts.  Exchange
// buffers hold N + N / 16 elements, room for either padding below.
__host__ __device__ constexpr int smem_elems(int N) { return N + N / 16; }
__device__ __forceinline__ int pad32(int i) { return i + (i >> 5); }
// Exchange-buffer position of element i.  With 16 points per thread the
// first pass writes at stride 16, which the stride-32 padding leaves 2-way
// bank-conflicted; one spare slot per 16 elements spreads those writes over
// all banks, keeps 16 consecutive elements (a 16-aligned half-warp) on
// distinct banks, and stays linear in i, so constant offsets fold into the
// load and store instructions.
template <int E>
__device__ __forceinline__ int xidx(int i) {
  if constexpr (E == 16) return i + (i >> 4);
  else return pad32(i);
}

// ---------------------------------------------------------------- complex helpers
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {  // a * conj(b)
  return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }

// Streaming load for data read exactly once (keeps L2 for the workspace).
__device__ __forceinline__ float2 ld_stream(const float2* p) { return __ldcs(p); }

// ---------------------------------------------------------------- register DFT
template <int LEN, int K, int DIR>
__device__ __forceinline__ float2 tw_const_mul(float2 b) {
  if constexpr (K == 0) {
    return b;
  } else if constexpr (4 * K == LEN) {  // exp(DIR i pi / 2) = DIR * i
    return DIR > 0 ? make_float2(-b.y, b.x) : make_float2(b.y, -b.x);
  } else {
    constexpr float c = (float)cx_cos(2.0 * kPi * K / LEN);
    constexpr float s = (float)(DIR * cx_sin(2.0 * kPi * K / LEN));
    return make_float2(b.x * c - b.y * s, b.x * s + b.y * c);
  }
}

// Radix-2 butterflies (a, b) -> (a + w b, a - w b), w = exp(DIR 2 pi i K / LEN).
// A twiddle other than 1 or +-i is applied in the FMA form of Linzer and
// Feig ("Modified FFTs for fused multiply-add architectures", Math. Comp.
// 1993): with w = c + i s and |c| >= |s|, w b = c (b.x - t b.y, b.y + t b.x),
// t = s / c, so both outputs take six FMAs instead of eight operations
// (|s| > |c|: w b = s (t b.x - b.y, b.x + t b.y), t = c / s).
template <int R, int LEN, int K, int DIR>
__device__ __forceinline__ void bfly_k(float2* v) {
  constexpr bool kTrivial = K == 0 || 4 * K == LEN;
  constexpr double cd = cx_cos(2.0 * kPi * K / LEN), sd = DIR * cx_sin(2.0 * kPi * K / LEN);
  constexpr bool kCosMajor = (cd < 0 ? -cd : cd) >= (sd < 0 ? -sd : sd);
#pragma unroll
  for (int i = 0; i < R; i += LEN) {
    const float2 a = v[i + K];
    const float2 b = v[i + K + LEN / 2];
    if constexpr (kTrivial) {
      const float2 wb = tw_const_mul<LEN, K, DIR>(b);
      v[i + K] = cadd(a, wb);
      v[i + K + LEN / 2] = csub(a, wb);
    } else if constexpr (kCosMajor) {
      constexpr float t = (float)(sd / cd), c = (float)cd;
      const float u = __fmaf_rn(-t, b.y, b.x), w = __fmaf_rn(t, b.x, b.y);
      v[i + K] = make_float2(__fmaf_rn(c, u, a.x), __fmaf_rn(c, w, a.y));
      v[i + K + LEN / 2] = make_float2(__fmaf_rn(-c, u, a.x), __fmaf_rn(-c, w, a.y));
    } else {
      constexpr float t = (float)(cd / sd), sn = (float)sd;
      const float u = __fmaf_rn(t, b.x, -b.y), w = __fmaf_rn(t, b.y, b.x);
      v[i + K] = make_float2(__fmaf_rn(sn, u, a.x), __fmaf_rn(sn, w, a.y));
      v[i + K + LEN / 2] = make_float2(__fmaf_rn(-sn, u, a.x), __fmaf_rn(-sn, w, a.y));
    }
  }
}
template <int R, int LEN, int DIR, int... Ks>
__device__ __forceinline__ void dit_stage(float2* v, std::integer_sequence<int, Ks...>) {
  (bfly_k<R, LEN, Ks, DIR>(v), ...);
}
template <int R, int DIR, int LEN>
__device__ __forceinline__ void dit_stages(float2* v) {
  if constexpr (LEN <= R) {
    dit_stage<R, LEN, DIR>(v, std::make_integer_sequence<int, LEN / 2>{});
    dit_stages<R, DIR, LEN * 2>(v);
  }
}
template <int I, int B>
struct Brev { static constexpr int value = cx_brev(I, B); };

template <int R, int... Is>
__device__ __forceinline__ void brev_perm(float2* v, std::integer_sequence<int, Is...>) {
  float2 t[R];
  ((t[Is] = v[Brev<Is, cx_log2(R)>::value]), ...);
  ((v[Is] = t[Is]), ...);
}

// In-place R-point DFT  v[b] <- sum_a v[a] exp(DIR 2 pi i a b / R), natural order.
template <int R, int DIR>
__device__ __forceinline__ void dft_reg(float2* v) {
  if constexpr (R > 1) {
    brev_perm<R>(v, std::make_integer_sequence<int, R>{});
    dit_stages<R, DIR, 2>(v);
  }
}

// ---------------------------------------------------------------- output-pruned DFT
// a + w b with w = exp(DIR 2 pi i K / LEN) a compile-time twiddle.
template <int LEN, int K, int DIR>
__device__ __forceinline__ float2 cmac_const(float2 a, float2 b) {
  if constexpr (K == 0 || 4 * K == LEN) {
    return cadd(a, tw_const_mul<LEN, K, DIR>(b));
  } else {
    constexpr float c = (float)cx_cos(2.0 * kPi * K / LEN);
    constexpr float s = (float)(DIR * cx_sin(2.0 * kPi * K / LEN));
    return make_float2(__fmaf_rn(c, b.x, __fmaf_rn(-s, b.y, a.x)), __fmaf_rn(c, b.y, __fmaf_rn(s, b.x, a.y)));
  }
}
template <int L, int DIR, int... Ks>
__device__ __forceinline__ void pruned_combine(float2* y, const float2* e, const float2* o,
                                               std::integer_sequence<int, Ks...>) {
  ((y[Ks] = cmac_const<L, Ks, DIR>(e[Ks], o[Ks])), ...);
}
// The first QO outputs y[k] = sum_m x[OFF + STRIDE m] exp(DIR 2 pi i m k / L),
// k < QO <= L, by radix-2 decimation in time that drops the outputs it does
// not need: X[k] = E[k] + exp(DIR 2 pi i k / L) O[k] for k < QO <= L / 2.
template <int L, int QO, int OFF, int STRIDE, int DIR>
__device__ __forceinline__ void pruned_dft(const float2* x, float2* y) {
  if constexpr (L <= QO) {
    float2 t[L];
#pragma unroll
    for (int m = 0; m < L; ++m) t[m] = x[OFF + STRIDE * m];
    dft_reg<L, DIR>(t);
#pragma unroll
    for (int k = 0; k < L; ++k) y[k] = t[k];
  } else {
    float2 e[QO], o[QO];
    pruned_dft<L / 2, QO, OFF, 2 * STRIDE, DIR>(x, e);
    pruned_dft<L / 2, QO, OFF + STRIDE, 2 * STRIDE, DIR>(x, o);
    pruned_combine<L, DIR>(y, e, o, std::make_integer_sequence<int, QO>{});
  }
}

// ---------------------------------------------------------------- group barrier
// T threads of one transform group; groups are warp-aligned.
template <int T>
__device__ __forceinline__ void group_sync(int group) {
  if constexpr (T <= 32) {
    __syncwarp();
  } else {
    asm volatile("bar.sync %0, %1;" ::"r"(group + 1), "r"(T) : "memory");
  }
}

// ---------------------------------------------------------------- Stockham passes
template <int N, int T, int DIR, int P, bool TW_SHARED = false>
__device__ __forceinline__ void stockham_pass(float2* v, float2* sm, const float2* __restrict__ tw,
                                              int t, int group) {
  constexpr int E = N / T;
  constexpr int R = pass_radix(N, E, P);
  constexpr int NS = pass_ns(N, E, P);
  constexpr int G = E / R;
  constexpr int NP = num_passes(N, E);
  static_assert(G * R == E, "pass does not tile the thread's points");
  if constexpr (P > 0) {
#pragma unroll
    for (int g = 0; g < G; ++g)
#pragma unroll
      for (int r = 0; r < R; ++r) v[g + r * G] = sm[xidx<E>(t + T * g + r * (N / R))];
  }
#pragma unroll
  for (int g = 0; g < G; ++g) {
    float2 w[R];
#pragma unroll
    for (int r = 0; r < R; ++r) w[r] = v[g + r * G];
    if constexpr (P > 0) {
      const int u = (t + T * g) & (NS - 1);
#pragma unroll
      for (int r = 1; r < R; ++r) {
        float2 tv = TW_SHARED ? tw[tw_offset(N, E, P) + r * NS + u] : __ldg(tw + tw_offset(N, E, P) + r * NS + u);
        if (DIR < 0) tv.y = -tv.y;
        w[r] = cmul(w[r], tv);
      }
    }
    dft_reg<R, DIR>(w);
#pragma unroll
    for (int r = 0; r < R; ++r) v[g + r * G] = w[r];
  }
  if constexpr (P < NP - 1) {
    group_sync<T>(group);  // previous readers of sm are done
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const int j = t + T * g;
      const int u = j & (NS - 1);
      const int base = (j / NS) * NS * R + u;
#pragma unroll
      for (int r = 0; r < R; ++r) sm[xidx<E>(base + r * NS)] = v[g + r * G];
    }
    group_sync<T>(group);
  }
}

template <int N, int T, int DIR, bool TW_SHARED, int... Ps>
__device__ __forceinline__ void run_passes(float2* v, float2* sm, const float2* __restrict__ tw, int t,
                                           int group, std::integer_sequence<int, Ps...>) {
  (stockham_pass<N, T, DIR, Ps, TW_SHARED>(v, sm, tw, t, group), ...);
}

// Unnormalised N-point DFT  X[m] = sum_n x[n] exp(DIR 2 pi i m n / N)
// on the group's registers (layout t + T q in and out).  `sm` holds
// smem_elems(N) float2 private to the group; `tw` is the host-built table
// for DIR = +1 (conjugated on the fly for DIR = -1).  TW_SHARED: `tw` is a
// copy of the table in shared memory (plain loads instead of __ldg).
template <int N, int T, int DIR, bool TW_SHARED = false>
__device__ __forceinline__ void group_fft(float2* v, float2* sm, const float2* __restrict__ tw, int t,
                                          int group) {
  static_assert(N % T == 0 && N / T >= 2, "at least two points per thread");
  run_passes<N, T, DIR, TW_SHARED>(v, sm, tw, t, group, std::make_integer_sequence<int, num_passes(N, N / T)>{});
}

// Output-pruned form of group_fft: the last pass produces only the outputs
// t + T q with q < QO (the others are left unset), which is all that is read
// when the transform's later use keeps a prefix of its outputs.  QO must not
// exceed the last pass's G = E / R, so each kept output is the r = 0 output of
// its radix-R butterfly group: the plain sum of the R twiddled inputs.
template <int N, int T, int DIR, int P, bool TW_SHARED, int QO>
__device__ __forceinline__ void stockham_last_pruned(float2* v, const float2* sm, const float2* __restrict__ tw,
                                                     int t) {
  constexpr int E = N / T;
  constexpr int R = pass_radix(N, E, P);
  constexpr int NS = pass_ns(N, E, P);
  constexpr int G = E / R;
  static_assert(P > 0 && P == num_passes(N, E) - 1, "the last pass");
  static_assert(QO >= 1 && QO <= G, "kept outputs are r = 0 outputs");
#pragma unroll
  for (int g = 0; g < QO; ++g) {
    const int u = (t + T * g) & (NS - 1);
    float2 acc = sm[xidx<E>(t + T * g)];
#pragma unroll
    for (int r = 1; r < R; ++r) {
      float2 tv = TW_SHARED ? tw[tw_offset(N, E, P) + r * NS + u] : __ldg(tw + tw_offset(N, E, P) + r * NS + u);
      if (DIR < 0) tv.y = -tv.y;
      acc = cadd(acc, cmul(sm[xidx<E>(t + T * g + r * (N / R))], tv));
    }
    v[g] = acc;
  }
}
template <int N, int T, int DIR, bool TW_SHARED, int QO, int... Ps>
__device__ __forceinline__ void run_passes_pruned(float2* v, float2* sm, const float2* __restrict__ tw, int t,
                                                  int group, std::integer_sequence<int, Ps...>) {
  (stockham_pass<N, T, DIR, Ps, TW_SHARED>(v, sm, tw, t, group), ...);
  stockham_last_pruned<N, T, DIR, (int)sizeof...(Ps), TW_SHARED, QO>(v, sm, tw, t);
}
template <int N, int T, int DIR, bool TW_SHARED, int QO>
__device__ __forceinline__ void group_fft_pruned(float2* v, float2* sm, const float2* __restrict__ tw, int t,
                                                 int group) {
  run_passes_pruned<N, T, DIR, TW_SHARED, QO>(v, sm, tw, t, group,
                                              std::make_integer_sequence<int, num_passes(N, N / T) - 1>{});
}

// ---------------------------------------------------------------- double-float
// Unevaluated pairs hi + lo of floats (about 48-bit significands) built from
// the error-free transformations TwoSum (Knuth) and TwoProd (via FMA), after
// Dekker, "A floating-point technique for extending the available precision"
// (1971).  Used only to recompute the rare ill-conditioned precoded cells.
struct dfl { float hi, lo; };
struct cdf { dfl re, im; };

__device__ __forceinline__ dfl df_quick(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ dfl df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ dfl df_add(dfl a, dfl b) {
  dfl s = df_two_sum(a.hi, b.hi);
  return df_quick(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ dfl df_neg(dfl a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ dfl df_mul(dfl a, dfl b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return df_quick(p, e);
}
__device__ __forceinline__ dfl df_mulf(dfl a, float b) {
  const float p = __fmul_rn(a.hi, b);
  const float e = __fmaf_rn(a.lo, b, __fmaf_rn(a.hi, b, -p));
  return df_quick(p, e);
}
__device__ __forceinline__ cdf cdf_mul(cdf a, cdf b) {
  return {df_add(df_mul(a.re, b.re), df_neg(df_mul(a.im, b.im))),
          df_add(df_mul(a.re, b.im), df_mul(a.im, b.re))};
}
__device__ __forceinline__ cdf cdf_mulf(cdf a, float2 b) {
  return {df_add(df_mulf(a.re, b.x), df_neg(df_mulf(a.im, b.y))),
          df_add(df_mulf(a.re, b.y), df_mulf(a.im, b.x))};
}
__device__ __forceinline__ cdf cdf_add(cdf a, cdf b) { return {df_add(a.re, b.re), df_add(a.im, b.im)}; }
__device__ __forceinline__ cdf cdf_ld(const float4* p) {
  const float4 v = __ldg(p);
  return {{v.x, v.y}, {v.z, v.w}};
}
__device__ __forceinline__ dfl df_shfl_xor(dfl a, int m) {
  return {__shfl_xor_sync(0xffffffffu, a.hi, m), __shfl_xor_sync(0xffffffffu, a.lo, m)};
}

}  // namespace ofdm
