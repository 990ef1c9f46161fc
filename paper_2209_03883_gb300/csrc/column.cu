// column.cu -- the per-OFDM-symbol half of the chain (steps a1-a5) and the
// stand-alone ZC transform.
//
// One thread group owns one OFDM symbol l of one frame at a time: a warp for
// N <= 512 (and the one-warp form at N = 1024), N/16 threads with 16 points
// each for N >= 1024 (the default), N/32 threads in the no-allocation path.
// The group kernel is instantiated for the default ZC parameters (r' = 1,
// q' = 0) and for the output-pruned inverse DFT (L_cp <= 2 T) as well as in
// general form, so that its unrolled loops carry no per-point runtime choice.
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
#include "refine.cuh"

namespace ofdm {

template <int N>
struct ColCfg {
  static constexpr int T = N <= 1024 ? 32 : N / 32;   // threads per symbol
  static constexpr int E = N / T;                     // points per thread
  static constexpr int GROUPS = N <= 1024 ? 8 : (N == 2048 ? 4 : 2);
  static constexpr int THREADS = T * GROUPS;
  static constexpr size_t SMEM = (size_t)GROUPS * smem_elems(N) * sizeof(float2);
};

// Pipelined configuration for N <= 1024 (one warp per symbol): each warp
// owns a ring of three padded row buffers in shared memory.  At any time one
// holds the current symbol's A row (then serves as the FFT exchange buffer),
// one its Y row, and one receives the next symbol's A row by cp.async; the
// next Y row is issued as soon as the current one has been consumed.
template <int N, int W = 0>
struct PipeCfg {
  static constexpr int E = N / 32;
  static constexpr int BUF = smem_elems(N);  // float2 per row buffer
  static constexpr int FIT = (int)((227u * 1024u) / (3u * BUF * sizeof(float2)));
  static constexpr int WMAX = FIT < 10 ? FIT : 10;
  // N = 1024, widest variant: the pre-chirp and pass-1 twiddle tables (16 KB)
  // live in shared memory, which leaves room for 8 warps instead of 9.
  static constexpr bool SMEM_TABLES = (N == 1024 && W == 0);
  static constexpr int TABLE_BYTES = SMEM_TABLES ? 2 * N * (int)sizeof(float2) : 0;
  static constexpr int WFIT = (int)((227u * 1024u - TABLE_BYTES) / (3u * BUF * sizeof(float2)));
  static constexpr int WMAX2 = WFIT < WMAX ? WFIT : WMAX;
  static constexpr int WARPS = W > 0 && W < WMAX2 ? W : WMAX2;
  static constexpr int THREADS = 32 * WARPS;
  static constexpr size_t SMEM = (size_t)WARPS * 3 * BUF * sizeof(float2) + TABLE_BYTES;
};

__device__ __forceinline__ uint64_t evict_first_policy() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src, uint64_t pol) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2;" ::"r"(s), "l"(gmem_src), "l"(pol)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int K>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(K) : "memory"); }

__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// True if `pred` holds on any thread of the group (named barrier reduction;
// every thread of the group must call it).
template <int T>
__device__ __forceinline__ bool group_any(int group, bool pred) {
  unsigned r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\tbar.red.or.pred q, %2, %3, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"((unsigned)pred), "r"(group + 1), "r"(T)
      : "memory");
  return r != 0;
}

constexpr int kRefineList = 64;  // flagged cells refined per symbol; more set OFDM_STATUS_UNREFINED

// Group form of refine_small_cells for T > 32: the same cells (a warp-local
// mean sets the threshold) are recomputed by all T threads of the group, each
// summing N / T terms, so no warp idles at the group's next barrier while
// another recomputes a cell alone.
template <int N, int T, int E>
__device__ __forceinline__ uint32_t refine_small_cells_group(float2* v, const float2* __restrict__ x,
                                                             const ColumnArgs& a, int t, int lane, int group,
                                                             int* cnt, int* list, cdf* part) {
  float s2 = 0.f;
#pragma unroll
  for (int q = 0; q < E; ++q) s2 += v[q].x * v[q].x + v[q].y * v[q].y;
#pragma unroll
  for (int off = 16; off; off >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, off);
  const float thr = a.refine_tau * s2 * (1.f / (32.f * E));
  unsigned flags = 0;
#pragma unroll
  for (int q = 0; q < E; ++q) flags |= (v[q].x * v[q].x + v[q].y * v[q].y < thr) ? (1u << q) : 0u;
  if (!group_any<T>(group, flags != 0)) return 0u;
  for (unsigned m = flags; m; m &= m - 1) {
    const int pos = atomicAdd(cnt, 1);
    if (pos < kRefineList) list[pos] = (t << 8) | (__ffs(m) - 1);
  }
  group_sync<T>(group);
  const int n_flagged = *cnt;
  const int n = min(n_flagged, kRefineList);
  for (int j = 0; j < n; ++j) {
    const int code = list[j], tt = code >> 8, qq = code & 255;
    const int i = tt + T * qq;
    cdf acc = {{0.f, 0.f}, {0.f, 0.f}};
    for (int k = t; k < N; k += T) {
      const cdf b = cdf_mulf(cdf_ld(a.pre_df + k), __ldg(x + k));
      const unsigned mi = ((unsigned)a.rprime * (unsigned)i * (unsigned)k) & (unsigned)(N - 1);
      acc = cdf_add(acc, cdf_mul(b, cdf_ld(a.w_df + mi)));
    }
#pragma unroll
    for (int off = 16; off; off >>= 1) {
      acc.re = df_add(acc.re, df_shfl_xor(acc.re, off));
      acc.im = df_add(acc.im, df_shfl_xor(acc.im, off));
    }
    if (lane == 0) part[(t >> 5)] = acc;
    group_sync<T>(group);
    if (t == tt) {
      cdf tot = part[0];
#pragma unroll
      for (int w = 1; w < T / 32; ++w) tot = cdf_add(tot, part[w]);
      const float2 val = make_float2(tot.re.hi + tot.re.lo, tot.im.hi + tot.im.lo);
#pragma unroll
      for (int q = 0; q < E; ++q)
        if (q == qq) v[q] = val;
    }
    group_sync<T>(group);  // part[] is rewritten by the next cell
  }
  if (t == 0) *cnt = 0;    // the next symbol appends after its group_any barrier
  // more flagged cells than the list holds: the rest stay FP32, and the frame says so
  return n_flagged > kRefineList ? (uint32_t)OFDM_STATUS_UNREFINED : 0u;
}

// F_i = Y_i / X_p,i with X_p,i = post_i B_i / sqrt(N), B in v:
//   F_i = Y_i conj(post_i) sqrt(N) conj(B_i) / |B_i|^2   (Eq. (16)).
// R1Q0: r' = 1 and q' = 0 known at compile time, so the post factor is (-1)^i
// (no table) -- the form the group kernel is instantiated for when the
// plan's ZC parameters allow it.
template <int T, int E, bool R1Q0 = false>
__device__ __forceinline__ uint32_t divide_precoded(float2* v, const float2* yrow, bool y_in_smem,
                                                    const ColumnArgs& a, int t) {
  uint32_t flags = 0;
  const float sgn = (a.post_sign && (t & 1)) ? -a.sqrtN : a.sqrtN;
#pragma unroll
  for (int q = 0; q < E; ++q) {
    const int i = t + T * q;
    float2 yv = y_in_smem ? yrow[i] : ld_stream(yrow + i);
    if (!R1Q0 && !a.post_sign) yv = cmul(yv, __ldg(a.post_conj + i));
    const float d2 = v[q].x * v[q].x + v[q].y * v[q].y;
    flags |= (d2 == 0.f) ? OFDM_STATUS_ZERO_X : 0u;
    const float inv = (d2 > 0.f) ? sgn * rcp_approx(d2) : 0.f;
    v[q] = cscale(cmulc(yv, v[q]), inv);
  }
  return flags;
}

template <int T, int E>
__device__ __forceinline__ uint32_t divide_plain(float2* v, const float2* xrow, const float2* yrow, bool in_smem,
                                                 int t) {
  uint32_t flags = 0;
#pragma unroll
  for (int q = 0; q < E; ++q) {
    const int i = t + T * q;
    const float2 xv = in_smem ? xrow[i] : ld_stream(xrow + i);
    const float2 yv = in_smem ? yrow[i] : ld_stream(yrow + i);
    const float d2 = xv.x * xv.x + xv.y * xv.y;
    flags |= (d2 == 0.f) ? OFDM_STATUS_ZERO_X : 0u;
    const float inv = (d2 > 0.f) ? rcp_approx(d2) : 0.f;
    v[q] = cscale(cmulc(yv, xv), inv);
  }
  return flags;
}

// Keep taps n < L_cp (Eq. (21)) and write the support rows of the windowed
// range profile, g[r] = c0 h[r] + c1 (h[r-1] + h[r+1]) (Eqs. (17), (22)).
// QMAX: only v[q], q < QMAX, can hold kept taps (E, or 2 after an
// output-pruned inverse DFT).
template <int N, int T, int E, int QMAX = E>
__device__ __forceinline__ uint32_t stencil_write(const float2* v, float2* sm, float2* __restrict__ strip,
                                                  const ColumnArgs& a, int f, int l, int t, int group) {
  group_sync<T>(group);  // the last FFT pass finished reading sm
#pragma unroll
  for (int q = 0; q < QMAX; ++q) {
    const int n = t + T * q;
    if (n < a.L_cp) sm[pad32(n)] = v[q];
  }
  group_sync<T>(group);
  uint32_t flags = 0;
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
  return flags;
}

// ---------------------------------------------------------------- N <= 1024: pipelined, one warp per symbol
template <int N, int W>
__global__ void __launch_bounds__(PipeCfg<N, W>::THREADS, 1)
column_pipe_kernel(const float2* __restrict__ Y, const float2* __restrict__ X, float2* __restrict__ strip,
                   uint32_t* __restrict__ wstatus, ColumnArgs a) {
  using C = PipeCfg<N, W>;
  constexpr int E = C::E;
  extern __shared__ float2 smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float2* ring = smem + (size_t)warp * 3 * C::BUF;
  const long total = (long)a.frames * a.M;
  const uint64_t pol = evict_first_policy();
  const float2* pre = a.pre;
  const float2* tw1 = a.tw;   // pass-1 table: tw1[r * 32 + u] for N = 1024
  if constexpr (C::SMEM_TABLES) {
    float2* tab = smem + (size_t)C::WARPS * 3 * C::BUF;
    for (int i = threadIdx.x; i < N; i += C::THREADS) {
      tab[i] = __ldg(a.pre + i);
      tab[N + i] = __ldg(a.tw + i);
    }
    __syncthreads();
    pre = tab;
    tw1 = tab + N;
  }

  auto issue_row = [&](const float2* g, float2* dst) {
    const char* gs = reinterpret_cast<const char*>(g);
    char* ds = reinterpret_cast<char*>(dst);
#pragma unroll
    for (int c = lane; c < N / 2; c += 32) cp_async16(ds + 16 * c, gs + 16 * c, pol);
  };

  // Dynamic scheduling: each warp draws symbol tickets from a monotonic
  // counter and stops after its first ticket past the end, so one launch
  // advances the counter by exactly (symbols + warps).  The next ticket is
  // drawn one symbol ahead so that its rows can be prefetched.
  auto ticket = [&]() -> long {
    unsigned long long v = 0;
    if (lane == 0) v = atomicAdd(a.work_ctr, 1ull);
    v = __shfl_sync(0xffffffffu, v, 0);
    return (long)(v - a.work_base);
  };
  // Offset of symbol `sm`'s row in Y and X (frames may be scattered).
  auto row_off = [&](long sm) -> long {
    if (!a.frame_off) return sm * N;
    return (long)a.frame_off[sm / a.M] + (sm % a.M) * N;
  };
  int ia = 0, iy = 1, ifree = 2;
  long sym = ticket();
  if (sym < total) issue_row(X + row_off(sym), ring + ia * C::BUF);
  cp_async_commit();
  if (sym < total) issue_row(Y + row_off(sym), ring + iy * C::BUF);
  cp_async_commit();
  long nxt = sym < total ? ticket() : total;
  for (; sym < total; sym = nxt, nxt = (nxt < total ? ticket() : total)) {
    if (nxt < total) issue_row(X + row_off(nxt), ring + ifree * C::BUF);
    cp_async_commit();
    const int f = (int)(sym / a.M);
    const int l = (int)(sym % a.M);
    float2* sa = ring + ia * C::BUF;        // A row, then the FFT exchange buffer
    const float2* sy = ring + iy * C::BUF;  // Y row
    float2 v[E];
    uint32_t flags = 0;
    int pass0 = 0;
    if (a.zc) {
      cp_async_wait<2>();                   // A(sym) has landed
      __syncwarp();
#pragma unroll
      for (int q = 0; q < E; ++q) {
        const int k = lane + 32 * q;
        const int s = (a.rinv == 1) ? k : (int)(((unsigned)a.rinv * (unsigned)k) & (N - 1));
        v[q] = cmul(sa[s], pre[s]);
      }
    } else {
      cp_async_wait<1>();                   // A(sym) and Y(sym)
      __syncwarp();
      flags |= divide_plain<32, E>(v, sa, sy, true, lane);
      __syncwarp();
      if (nxt < total) issue_row(Y + row_off(nxt), ring + iy * C::BUF);
      cp_async_commit();
      pass0 = 1;
    }
    // Both N-point DFTs run through one copy of the FFT code: pass 0 is the ZC
    // transform, pass 1 the DFT-CE IDFT, N h[n] = sum_i F_i e^{+2 pi i n i / N} (Eq. (20)).
    if constexpr (N == 1024) {
      // Four radix-32 Stockham half-passes through ONE register DFT body
      // (instruction-cache footprint): even h reads the registers and writes
      // the transposed exchange, odd h reads it back and applies the
      // exp(+2 pi i lane r / 1024) twiddles (pass-1 table, u = lane).
      // DFT-CE keeps taps n = lane + 32 q < L_cp only, so for L_cp <= 128 the
      // last half-pass needs outputs q < 4 alone (pruned transform).
      const bool prune4 = a.L_cp <= 128;
#pragma unroll 1
      for (int h = 2 * pass0; h < 4; ++h) {
        if (h & 1) {
#pragma unroll
          for (int r = 0; r < 32; ++r) v[r] = sa[pad32(lane + 32 * r)];
#pragma unroll
          for (int r = 1; r < 32; ++r) v[r] = cmul(v[r], tw1[r * 32 + lane]);
        }
        if (h == 3 && prune4) {
          float2 y[4];
          pruned_dft<32, 4, 0, 1, +1>(v, y);
#pragma unroll
          for (int q = 0; q < 4; ++q) v[q] = y[q];
          break;
        }
        dft_reg<32, +1>(v);
        if (!(h & 1)) {
          __syncwarp();
#pragma unroll
          for (int r = 0; r < 32; ++r) sa[pad32(32 * lane + r)] = v[r];
          __syncwarp();
        } else if (h == 1) {
          if (a.refine_tau > 0.f) refine_small_cells<N, 32, E>(v, X + row_off(sym), a, lane, lane);
          cp_async_wait<1>();               // Y(sym)
          __syncwarp();
          flags |= divide_precoded<32, E>(v, sy, true, a, lane);
          __syncwarp();
          if (nxt < total) issue_row(Y + row_off(nxt), ring + iy * C::BUF);
          cp_async_commit();
        }
      }
    } else {
#pragma unroll 1
      for (int pass = pass0; pass < 2; ++pass) {
        group_fft<N, 32, +1>(v, sa, a.tw, lane, 0);
        if (pass == 0) {
          if (a.refine_tau > 0.f) refine_small_cells<N, 32, E>(v, X + row_off(sym), a, lane, lane);
          cp_async_wait<1>();               // Y(sym)
          __syncwarp();
          flags |= divide_precoded<32, E>(v, sy, true, a, lane);
          __syncwarp();
          if (nxt < total) issue_row(Y + row_off(nxt), ring + iy * C::BUF);
          cp_async_commit();
        }
      }
    }
    flags |= stencil_write<N, 32, E>(v, sa, strip, a, f, l, lane, 0);
    flags = __reduce_or_sync(0xffffffffu, flags);
    if (lane == 0 && flags) atomicOr(wstatus + f, flags);
    __syncwarp();  // every lane is done with sa before it is refilled
    const int t = ia;
    ia = ifree;
    ifree = t;
  }
  cp_async_wait<0>();
}

// ---------------------------------------------------------------- N >= 2048: pipelined multi-warp groups
// The same ring-of-three-rows pipeline as above, with a symbol owned by a
// group of T = N / 32 threads (2 warps for N = 2048, 4 for 4096) that meets
// at a named barrier (id = group + 1) wherever one warp would use __syncwarp.
// T = N / 32 (32 points per thread) for N >= 2048; N = 1024 also has a
// 2-warp form (T = 64, 16 points per thread, at most 512 threads per CTA so
// that 128 registers per thread fit).
template <int N, int TT = N / 32>
struct GroupPipeCfg {
  static constexpr int T = TT;
  static constexpr int E = N / T;
  static constexpr int BUF = smem_elems(N);
  // Row buffers per group.  Three (A, Y, next A) give every copy a whole
  // symbol of lead.  With 16 points per thread and N >= 2048 two buffers are
  // used instead (next A lands in the Y slot after the division, next Y in
  // the A slot after the stencil: half a symbol of lead, several
  // microseconds), so that the tables fit in shared memory beside them.
  static constexpr int RING = (E < 32 && N >= 2048) ? 2 : 3;
  static constexpr int FIT = (int)((227u * 1024u) / (RING * BUF * sizeof(float2)));
  static constexpr int GROUPS = (E < 32 && FIT > 512 / T) ? 512 / T : FIT;
  static constexpr int THREADS = T * GROUPS;
  // 16 points per thread: the pre-chirp and the pass twiddles live in shared
  // memory behind the rings (18 KB for N = 1024, 34 KB for 2048, 68 KB for 4096)
  static constexpr size_t RING_BYTES = (size_t)GROUPS * RING * BUF * sizeof(float2);
  static constexpr bool SMEM_TABLES =
      E < 32 && RING_BYTES + (size_t)(N + tw_size(N, E)) * sizeof(float2) + 4096 <= 227u * 1024u;
  static constexpr int TABLE_ELEMS = SMEM_TABLES ? N + tw_size(N, E) : 0;
  static constexpr size_t SMEM = RING_BYTES + (size_t)TABLE_ELEMS * sizeof(float2);
  static_assert(GROUPS >= 1 && GROUPS <= 15, "named barriers 1..15");
  static_assert(SMEM <= 227u * 1024u, "shared memory");
  static_assert(T % 32 == 0, "whole warps");
};

// R1Q0: instantiated for r' = 1, q' = 0 (the ZC transform's input permutation
// is the identity and its post factor is (-1)^i): the per-point index and
// table branches, which the unrolled loops would otherwise issue predicated,
// are gone.  PRUNE: L_cp <= 2 T with 16 points per thread, so the DFT-CE
// inverse DFT computes only the outputs q < 2 (the launcher picks the form).
template <int N, int TT = N / 32, bool R1Q0 = false, bool PRUNE = false>
__global__ void __launch_bounds__(GroupPipeCfg<N, TT>::THREADS, 1)
column_group_pipe_kernel(const float2* __restrict__ Y, const float2* __restrict__ X, float2* __restrict__ strip,
                         uint32_t* __restrict__ wstatus, ColumnArgs a) {
  using C = GroupPipeCfg<N, TT>;
  constexpr int T = C::T, E = C::E;
  extern __shared__ float2 smem[];
  __shared__ long long s_tk[C::GROUPS][2];
  __shared__ int s_rcnt[C::GROUPS];
  __shared__ int s_rlist[C::GROUPS][kRefineList];
  __shared__ cdf s_rpart[C::GROUPS][T / 32];
  const int group = threadIdx.x / T, t = threadIdx.x % T, lane = threadIdx.x & 31;
  if (t == 0) s_rcnt[group] = 0;
  const float2* pre = a.pre;
  const float2* tw = a.tw;
  if constexpr (C::SMEM_TABLES) {
    float2* tab = smem + (size_t)C::GROUPS * C::RING * C::BUF;
    for (int i = threadIdx.x; i < N; i += C::THREADS) tab[i] = __ldg(a.pre + i);
    for (int i = threadIdx.x; i < tw_size(N, E); i += C::THREADS) tab[N + i] = __ldg(a.tw + i);
    pre = tab;
    tw = tab + N;
  }
  __syncthreads();
  float2* ring = smem + (size_t)group * C::RING * C::BUF;
  const long total = (long)a.frames * a.M;
  const uint64_t pol = evict_first_policy();

  auto issue_row = [&](const float2* g, float2* dst) {
    const char* gs = reinterpret_cast<const char*>(g);
    char* ds = reinterpret_cast<char*>(dst);
#pragma unroll
    for (int c = t; c < N / 2; c += T) cp_async16(ds + 16 * c, gs + 16 * c, pol);
  };
  // Group-wide ticket: thread 0 of the group draws it, the group's barrier
  // publishes it.  Two slots alternate so that a slot is rewritten only after
  // every thread has passed the barrier that follows its last read.
  int slot = 0;
  auto ticket = [&]() -> long {
    if (t == 0) s_tk[group][slot] = (long long)(atomicAdd(a.work_ctr, 1ull) - a.work_base);
    group_sync<T>(group);
    const long v = (long)s_tk[group][slot];
    slot ^= 1;
    return v;
  };
  auto row_off = [&](long sm) -> long {
    if (!a.frame_off) return sm * N;
    return (long)a.frame_off[sm / a.M] + (sm % a.M) * N;
  };
  // Commit groups in flight at the top of a symbol, oldest first: A(sym),
  // Y(sym) with two buffers; A(sym), Y(sym), A(next) with three.
  constexpr int R2 = C::RING == 2 ? 1 : 0;
  int ia = 0, iy = 1, ifree = 2;
  long sym = ticket();
  if (sym < total) issue_row(X + row_off(sym), ring + ia * C::BUF);
  cp_async_commit();
  if (sym < total) issue_row(Y + row_off(sym), ring + iy * C::BUF);
  cp_async_commit();
  long nxt = sym < total ? ticket() : total;
  for (; sym < total; sym = nxt, nxt = (nxt < total ? ticket() : total)) {
    if constexpr (!R2) {
      if (nxt < total) issue_row(X + row_off(nxt), ring + ifree * C::BUF);
      cp_async_commit();
    }
    const int f = (int)(sym / a.M);
    const int l = (int)(sym % a.M);
    float2* sa = ring + ia * C::BUF;        // A row, then the FFT exchange buffer
    const float2* sy = ring + iy * C::BUF;  // Y row
    float2 v[E];
    uint32_t flags = 0;
    if (a.zc) {
      cp_async_wait<2 - R2>();              // A(sym) has landed (this thread's copies) ...
      group_sync<T>(group);                 // ... and every thread's
#pragma unroll
      for (int q = 0; q < E; ++q) {
        const int k = t + T * q;
        const int s2 = (R1Q0 || a.rinv == 1) ? k : (int)(((unsigned)a.rinv * (unsigned)k) & (N - 1));
        v[q] = cmul(sa[s2], C::SMEM_TABLES ? pre[s2] : __ldg(pre + s2));   // the row lands unpadded
      }
      group_fft<N, T, +1, C::SMEM_TABLES>(v, sa, tw, t, group);
      if (a.refine_tau > 0.f)
        flags |= refine_small_cells_group<N, T, E>(v, X + row_off(sym), a, t, lane, group, &s_rcnt[group],
                                                   s_rlist[group], s_rpart[group]);
      cp_async_wait<1 - R2>();              // Y(sym)
      group_sync<T>(group);
      flags |= divide_precoded<T, E, R1Q0>(v, sy, true, a, t);
    } else {
      cp_async_wait<1 - R2>();              // A(sym) and Y(sym)
      group_sync<T>(group);
      flags |= divide_plain<T, E>(v, sa, sy, true, t);
    }
    group_sync<T>(group);                   // every thread is done with the Y row
    if (nxt < total) issue_row((R2 ? X : Y) + row_off(nxt), ring + iy * C::BUF);   // next A (two) or Y (three)
    cp_async_commit();
    // DFT-CE keeps taps n = t + T q < L_cp only: for N = 1024 in two-warp
    // groups and L_cp <= 128 that is q < 2, so the last pass is pruned.
    // (same for N = 2048 in four-warp groups, whose last pass is radix 8, G = 2)
    if constexpr (PRUNE) {
      group_fft_pruned<N, T, +1, C::SMEM_TABLES, 2>(v, sa, tw, t, group);
      flags |= stencil_write<N, T, E, 2>(v, sa, strip, a, f, l, t, group);
    } else {
      group_fft<N, T, +1, C::SMEM_TABLES>(v, sa, tw, t, group);
      flags |= stencil_write<N, T, E>(v, sa, strip, a, f, l, t, group);
    }
    flags = __reduce_or_sync(0xffffffffu, flags);
    if (lane == 0 && flags) atomicOr(wstatus + f, flags);
    group_sync<T>(group);                   // every thread is done with sa before it is refilled
    if constexpr (R2) {
      if (nxt < total) issue_row(Y + row_off(nxt), ring + ia * C::BUF);   // next Y into the A slot
      cp_async_commit();
      const int tmp = ia;                   // next symbol: A in the old Y slot, Y in the old A slot
      ia = iy;
      iy = tmp;
    } else {
      const int tmp = ia;
      ia = ifree;
      ifree = tmp;
    }
  }
  cp_async_wait<0>();
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

template <int N, int W>
static cudaError_t launch_pipe(const float2* Y, const float2* X, float2* strip, uint32_t* wstatus,
                               const ColumnArgs& a, cudaStream_t s, unsigned long long* tickets, int sms,
                               long total) {
  using C = PipeCfg<N, W>;
  cudaError_t e = cudaFuncSetAttribute(column_pipe_kernel<N, W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)C::SMEM);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, column_pipe_kernel<N, W>, C::THREADS, C::SMEM);
  if (e != cudaSuccess) return e;
  long blocks = (long)sms * (per_sm > 0 ? per_sm : 1);
  const long need = (total + C::WARPS - 1) / C::WARPS;
  if (blocks > need) blocks = need;
  column_pipe_kernel<N, W><<<(unsigned)blocks, C::THREADS, C::SMEM, s>>>(Y, X, strip, wstatus, a);
  *tickets = (unsigned long long)total + (unsigned long long)blocks * C::WARPS;
  return cudaGetLastError();
}

template <int N, int TT = N / 32>
static cudaError_t launch_group_pipe(const float2* Y, const float2* X, float2* strip, uint32_t* wstatus,
                                     const ColumnArgs& a, cudaStream_t s, unsigned long long* tickets, int sms,
                                     long total) {
  using C = GroupPipeCfg<N, TT>;
  constexpr int E = N / TT;
  constexpr bool CAN_PRUNE = E == 16 && E / pass_radix(N, E, num_passes(N, E) - 1) >= 2;
  const bool r1q0 = a.rinv == 1 && a.post_sign;
  auto kern = r1q0 ? column_group_pipe_kernel<N, TT, true> : column_group_pipe_kernel<N, TT, false>;
  if constexpr (CAN_PRUNE) {
    if (a.L_cp <= 2 * TT)
      kern = r1q0 ? column_group_pipe_kernel<N, TT, true, true> : column_group_pipe_kernel<N, TT, false, true>;
  }
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, C::THREADS, C::SMEM);
  if (e != cudaSuccess) return e;
  long blocks = (long)sms * (per_sm > 0 ? per_sm : 1);
  const long need = (total + C::GROUPS - 1) / C::GROUPS;
  if (blocks > need) blocks = need;
  kern<<<(unsigned)blocks, C::THREADS, C::SMEM, s>>>(Y, X, strip, wstatus, a);
  *tickets = (unsigned long long)total + (unsigned long long)blocks * C::GROUPS;
  return cudaGetLastError();
}

template <int N>
static cudaError_t launch_column_n(const float2* Y, const float2* X, float2* strip, uint32_t* wstatus,
                                   const ColumnArgs& a, cudaStream_t s, unsigned long long* tickets) {
  *tickets = 0;
  const long total = (long)a.frames * a.M;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if constexpr (N == 1024) {
    if (a.tc_b) return launch_column_tc(Y, X, strip, wstatus, a, s, tickets);
  }
  if constexpr (N <= 1024) {
    if (a.pipe_warps == 4) return launch_pipe<N, 4>(Y, X, strip, wstatus, a, s, tickets, sms, total);
    if constexpr (N == 1024) {
      if (a.pipe_warps == 2 && a.tw_group) {
        ColumnArgs g = a;
        g.tw = a.tw_group;
        return launch_group_pipe<N, 64>(Y, X, strip, wstatus, g, s, tickets, sms, total);
      }
    }
    return launch_pipe<N, 0>(Y, X, strip, wstatus, a, s, tickets, sms, total);
  } else {
    if (a.pipe_warps == 2 && a.tw_group) {   // groups of N / 16 threads, 16 points each
      ColumnArgs g = a;
      g.tw = a.tw_group;
      return launch_group_pipe<N, N / 16>(Y, X, strip, wstatus, g, s, tickets, sms, total);
    }
    return launch_group_pipe<N>(Y, X, strip, wstatus, a, s, tickets, sms, total);
  }
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
                          const ColumnArgs& a, cudaStream_t s, int* launches, unsigned long long* tk) {
  ++*launches;
  switch (N) {
    case 64: return launch_column_n<64>(Y, X, strip, wstatus, a, s, tk);
    case 128: return launch_column_n<128>(Y, X, strip, wstatus, a, s, tk);
    case 256: return launch_column_n<256>(Y, X, strip, wstatus, a, s, tk);
    case 512: return launch_column_n<512>(Y, X, strip, wstatus, a, s, tk);
    case 1024: return launch_column_n<1024>(Y, X, strip, wstatus, a, s, tk);
    case 2048: return launch_column_n<2048>(Y, X, strip, wstatus, a, s, tk);
    case 4096: return launch_column_n<4096>(Y, X, strip, wstatus, a, s, tk);
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
