// fps.cu -- FPS-SFT (Sec. III-C): the sparse alternative to the 2D
// periodogram, on the DFT-CE channel estimate H' (or, for plain LS
// estimation without precoding, on F = Y / X itself).
//
// The slice positions of every iteration are inputs, so the samples and
// their Q-point DFTs do not depend on what earlier iterations recover; only
// the peeling and the decoding do.  The work is therefore split by what it
// depends on:
//   1. fps_sample_taps_kernel / fps_sample_direct_kernel (all frames, all
//      iterations and slices at once, spread over the GPU):
//        s_j[n] = H'[(a0 n + t0_j) mod N, (a1 n + t1_j) mod M],  n < Q
//      from the kept DFT-CE taps of the strip (rect stencil, N h[n]):
//        H'[k, l] = (1/N) sum_{n < L_cp} (N h[n, l]) e^{-2 pi i n k / N}  (Eq. (22)),
//      one CTA per 8 columns l (every slice visits each column Q / M times),
//      or, when F is cell-local (no ZC division to undo and L_cp = N), the
//      sampled cells of Y and X alone: s = Y / X (Eq. (16)) -- the regime in
//      which FPS-SFT reads a small fraction of the frame;
//   2. fps_fft_kernel: the Q-point DFT of every slice (one warp each);
//   3. fps_decode_kernel (one CTA per frame, iterations in order): removal of
//      the recovered frequencies from every slice, bin energies, the median
//      threshold, ML decoding along each surviving bin's projection line
//      with the coherence (1-sparsity) test, and the recovered list.
#include <float.h>

#include "fft.cuh"
#include "internal.h"

namespace ofdm {

constexpr int kFpsThreads = 256;
constexpr int kFpsMaxT = 8;        // slices per iteration
constexpr int kFpsMaxRec = 64;     // recovered frequencies per frame
constexpr int kFpsMaxCand = 256;   // candidate bins decoded per iteration
constexpr int kFpsCols = 8;        // columns per CTA of the sampling kernel

struct FpsRec { int f0, f1; float2 a; };

__device__ __forceinline__ float2 ptab_at(const float2* ptab, int m, int sign) {
  float2 w = ptab[m];
  if (sign < 0) w.y = -w.y;
  return w;
}
__device__ __forceinline__ int inv_mod_pow2(int a1, int M) {   // a1^{-1} mod M (a1 odd, M a power of two)
  unsigned inv = 1u;
  for (int k = 0; k < 5; ++k) inv = inv * (2u - (unsigned)a1 * inv);
  return (int)(inv & (unsigned)(M - 1));
}

// ---------------------------------------------------------------- 1. samples from the taps
// CTA = (8 consecutive columns, frame); warp w owns column l0 + w and loops
// over its (iteration, slice, repeat) items, one per lane.
__global__ void __launch_bounds__(kFpsThreads)
fps_sample_taps_kernel(const float2* __restrict__ strip, const int32_t* __restrict__ slices,
                       float2* __restrict__ S, FpsArgs a) {
  extern __shared__ __align__(16) unsigned char fps_smem[];
  float2* taps = reinterpret_cast<float2*>(fps_smem);   // [rows][kFpsCols]
  const int f = blockIdx.y, l0 = blockIdx.x * kFpsCols;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int N = a.N, M = a.M, T = a.T, rows = a.rows, Q = a.Q;
  const float2* g = strip + (size_t)f * rows * M;
  for (int e = tid; e < rows * kFpsCols; e += kFpsThreads) {
    const int n = e / kFpsCols, c = e % kFpsCols;
    taps[e] = (l0 + c < M) ? g[(size_t)n * M + l0 + c] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  const int l = l0 + warp;
  if (l >= M) return;
  const int reps = Q / M;
  const int items = a.iterations * T * reps;
  for (int item = lane; item < items; item += 32) {
    const int rep = item % reps, rest = item / reps;
    const int j = rest % T, it = rest / T;
    const int32_t* sp = slices + ((size_t)f * a.iterations + it) * (2 + 2 * T);
    const int a0 = sp[0], a1 = sp[1], t0 = sp[2 + 2 * j], t1 = sp[3 + 2 * j];
    const int n0 = (int)(((unsigned)inv_mod_pow2(a1, M) * (unsigned)((l - t1) & (M - 1))) & (unsigned)(M - 1));
    const int n = n0 + M * rep;
    const int k = (int)((((long)a0 * n + t0) % N + N) % N);
    float2 acc = make_float2(0.f, 0.f);
    for (int nn = 0; nn < rows; ++nn) {
      const float4 w4 = __ldg(a.w_df + (int)(((unsigned)nn * (unsigned)k) & (unsigned)(N - 1)));
      const float2 w = make_float2(w4.x, -w4.z);   // exp(-2 pi i nn k / N)
      acc = cadd(acc, cmul(taps[nn * kFpsCols + warp], w));
    }
    S[(((size_t)f * a.iterations + it) * T + j) * Q + n] = cscale(acc, a.invN);
  }
}

// ---------------------------------------------------------------- 1'. samples of F = Y / X
// Thread per sample; the only bytes read are the sampled cells of Y and X.
__global__ void __launch_bounds__(kFpsThreads)
fps_sample_direct_kernel(const float2* __restrict__ Y, const float2* __restrict__ X,
                         const int32_t* __restrict__ slices, float2* __restrict__ S,
                         uint32_t* __restrict__ wstatus, FpsArgs a) {
  const int N = a.N, M = a.M, T = a.T, Q = a.Q;
  const long per_frame = (long)a.iterations * T * Q;
  const long total = per_frame * a.frames;
  for (long e = (long)blockIdx.x * kFpsThreads + threadIdx.x; e < total; e += (long)gridDim.x * kFpsThreads) {
    const int f = (int)(e / per_frame);
    const long r = e % per_frame;
    const int n = (int)(r % Q);
    const int j = (int)((r / Q) % T), it = (int)(r / ((long)Q * T));
    const int32_t* sp = slices + ((size_t)f * a.iterations + it) * (2 + 2 * T);
    const int k = (int)((((long)sp[0] * n + sp[2 + 2 * j]) % N + N) % N);
    const int l = (int)((((long)sp[1] * n + sp[3 + 2 * j]) % M + M) % M);
    const size_t cell = ((size_t)f * M + l) * N + k;
    const float2 yv = __ldcs(Y + cell), xv = __ldcs(X + cell);
    const float d2 = xv.x * xv.x + xv.y * xv.y;
    if (d2 == 0.f) atomicOr(wstatus + f, (uint32_t)OFDM_STATUS_ZERO_X);
    S[e] = d2 > 0.f ? cscale(cmulc(yv, xv), 1.f / d2) : make_float2(0.f, 0.f);
  }
}

// ---------------------------------------------------------------- 2. slice DFTs
template <int Q>
__global__ void __launch_bounds__(kFpsThreads)
fps_fft_kernel(float2* __restrict__ S, long nslices, const float2* __restrict__ twQ) {
  extern __shared__ __align__(16) unsigned char fps_smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float2* sm = reinterpret_cast<float2*>(fps_smem) + (size_t)warp * smem_elems(Q);
  const long sl = (long)blockIdx.x * (kFpsThreads / 32) + warp;
  if (sl >= nslices) return;
  float2* s = S + sl * Q;
  constexpr int E = Q / 32;
  float2 v[E];
#pragma unroll
  for (int q = 0; q < E; ++q) v[q] = s[lane + 32 * q];
  group_fft<Q, 32, -1>(v, sm, twQ, lane, 0);
#pragma unroll
  for (int q = 0; q < E; ++q) s[lane + 32 * q] = v[q];
}

// ---------------------------------------------------------------- 3. iterations of one frame
template <int Q>
__global__ void __launch_bounds__(kFpsThreads)
fps_decode_kernel(const float2* __restrict__ Sg, const int32_t* __restrict__ slices, ofdm_target* __restrict__ out,
                  int32_t* __restrict__ n_out, uint32_t* __restrict__ wstatus, FpsArgs a) {
  extern __shared__ __align__(16) unsigned char fps_smem[];
  float2* S = reinterpret_cast<float2*>(fps_smem);                 // T slices of this iteration
  float2* ptab = S + (size_t)kFpsMaxT * Q;                          // exp(+2 pi i m / Q)
  float* E = reinterpret_cast<float*>(ptab + Q);                    // bin energy
  float* srt = E + Q;                                               // sorted copy
  FpsRec* rec = reinterpret_cast<FpsRec*>(srt + Q);                 // recovered list
  FpsRec* fnd = rec + kFpsMaxRec;                                   // found this iteration
  int* cand = reinterpret_cast<int*>(fnd + kFpsMaxCand);            // candidate bins
  __shared__ int s_nrec, s_ncand, s_nfnd;
  __shared__ float s_peak;

  const int f = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int N = a.N, M = a.M, T = a.T;
  const int qn = Q / N, qm = Q / M;

  for (int m = tid; m < Q; m += kFpsThreads) {
    double s, c;
    sincospi(2.0 * m / Q, &s, &c);
    ptab[m] = make_float2((float)c, (float)s);
  }
  if (tid == 0) { s_nrec = 0; s_peak = 0.f; }
  __syncthreads();

  for (int it = 0; it < a.iterations; ++it) {
    const int32_t* sp = slices + ((size_t)f * a.iterations + it) * (2 + 2 * T);
    const int a0 = sp[0], a1 = sp[1];
    const int a1inv = inv_mod_pow2(a1, M);
    const float4* src = reinterpret_cast<const float4*>(Sg + ((size_t)f * a.iterations + it) * T * Q);
    for (int e = tid; e < T * Q / 2; e += kFpsThreads) reinterpret_cast<float4*>(S)[e] = src[e];
    __syncthreads();
    // ---- remove the recovered frequencies (serial per slice: bins may coincide)
    if (tid < T) {
      const int j = tid;
      float2* sj = S + (size_t)j * Q;
      const int t0 = sp[2 + 2 * j], t1 = sp[3 + 2 * j];
      for (int r = 0; r < s_nrec; ++r) {
        const int f0 = rec[r].f0, f1 = rec[r].f1;
        const int m = (int)(((long)a0 * f0 * qn + (long)a1 * f1 * qm) % Q);
        const int ph = (int)(((long)f0 * t0 * qn + (long)f1 * t1 * qm) % Q);
        const float2 c = cscale(cmul(rec[r].a, ptab_at(ptab, ph, +1)), (float)Q * a.invNM);
        sj[m] = csub(sj[m], c);
      }
    }
    __syncthreads();

    // ---- bin energies, median threshold, running peak
    for (int m = tid; m < Q; m += kFpsThreads) {
      float e = 0.f;
      for (int j = 0; j < T; ++j) {
        const float2 v = S[(size_t)j * Q + m];
        e += v.x * v.x + v.y * v.y;
      }
      E[m] = e / (float)T;
      srt[m] = E[m];
    }
    __syncthreads();
    for (int k = 2; k <= Q; k <<= 1)
      for (int jj = k >> 1; jj > 0; jj >>= 1) {
        for (int i = tid; i < Q; i += kFpsThreads) {
          const int p = i ^ jj;
          if (p > i) {
            const float x = srt[i], y = srt[p];
            const bool up = (i & k) == 0;
            if (up ? (x > y) : (x < y)) { srt[i] = y; srt[p] = x; }
          }
        }
        __syncthreads();
      }
    if (tid == 0) {
      s_peak = fmaxf(s_peak, srt[Q - 1]);
      s_ncand = 0;
      s_nfnd = 0;
    }
    __syncthreads();
    const float thr = fmaxf(srt[(Q - 1) / 2] * a.median_factor, a.dynamic_range * s_peak);
    for (int m = tid; m < Q; m += kFpsThreads)
      if (E[m] > thr) {
        const int slot = atomicAdd(&s_ncand, 1);
        if (slot < kFpsMaxCand) cand[slot] = m;
      }
    __syncthreads();
    const int ncand = min(s_ncand, kFpsMaxCand);
    if (ncand == 0) break;  // nothing above the noise: done (uniform: shared value)

    // ---- ML decoding along each candidate bin's line (one warp per bin)
    for (int ci = warp; ci < ncand; ci += kFpsThreads / 32) {
      const int m = cand[ci];
      float best = -1.f;
      int bf0 = -1, bf1 = 0;
      float2 bacc = make_float2(0.f, 0.f);
      for (int f0 = lane; f0 < N; f0 += 32) {
        const int rest = (int)((((long)m - (long)a0 * f0 * qn) % Q + Q) % Q);
        if (rest % qm) continue;
        const int f1 = (int)(((unsigned)a1inv * (unsigned)(rest / qm)) & (unsigned)(M - 1));
        float2 acc = make_float2(0.f, 0.f);
        for (int j = 0; j < T; ++j) {
          const int t0 = sp[2 + 2 * j], t1 = sp[3 + 2 * j];
          const int ph = (int)(((long)f0 * t0 * qn + (long)f1 * t1 * qm) % Q);
          acc = cadd(acc, cmul(S[(size_t)j * Q + m], ptab_at(ptab, ph, -1)));
        }
        const float mag = acc.x * acc.x + acc.y * acc.y;
        if (mag > best) { best = mag; bf0 = f0; bf1 = f1; bacc = acc; }
      }
      // warp argmax; ties go to the smaller f0 (first maximum in f0 order)
      for (int off = 16; off; off >>= 1) {
        const float ob = __shfl_xor_sync(0xffffffffu, best, off);
        const int o0 = __shfl_xor_sync(0xffffffffu, bf0, off);
        const int o1 = __shfl_xor_sync(0xffffffffu, bf1, off);
        const float ox = __shfl_xor_sync(0xffffffffu, bacc.x, off);
        const float oy = __shfl_xor_sync(0xffffffffu, bacc.y, off);
        if (ob > best || (ob == best && o0 >= 0 && (bf0 < 0 || o0 < bf0))) {
          best = ob; bf0 = o0; bf1 = o1; bacc = make_float2(ox, oy);
        }
      }
      if (lane == 0 && bf0 >= 0) {
        float sumabs = 0.f;
        for (int j = 0; j < T; ++j) {
          const float2 v = S[(size_t)j * Q + m];
          sumabs += sqrtf(v.x * v.x + v.y * v.y);
        }
        if (sqrtf(best) >= a.coherence_min * sumabs) {
          const int slot = atomicAdd(&s_nfnd, 1);
          fnd[slot].f0 = bf0;
          fnd[slot].f1 = bf1;
          fnd[slot].a = cscale(bacc, a.NMoverQ / (float)T);
        }
      }
    }
    __syncthreads();
    // ---- merge into the recovered list (in bin order, like a serial decoder)
    if (tid == 0) {
      const int nf = s_nfnd;
      for (int i = 1; i < nf; ++i) {  // order the found entries by their bin
        const FpsRec x = fnd[i];
        const int mx = (int)(((long)a0 * x.f0 * qn + (long)a1 * x.f1 * qm) % Q);
        int j = i - 1;
        while (j >= 0 && (int)(((long)a0 * fnd[j].f0 * qn + (long)a1 * fnd[j].f1 * qm) % Q) > mx) {
          fnd[j + 1] = fnd[j];
          --j;
        }
        fnd[j + 1] = x;
      }
      for (int i = 0; i < nf; ++i) {
        int r = 0;
        while (r < s_nrec && !(rec[r].f0 == fnd[i].f0 && rec[r].f1 == fnd[i].f1)) ++r;
        if (r < s_nrec) rec[r].a = cadd(rec[r].a, fnd[i].a);
        else if (s_nrec < a.max_recover) rec[s_nrec++] = fnd[i];
      }
    }
    __syncthreads();
  }

  // ---- output: strongest first, then map index (r = -f0 mod N, s centred)
  if (tid == 0) {
    const int nr = s_nrec;
    uint64_t keys[kFpsMaxRec];
    for (int r = 0; r < nr; ++r) {
      const float p = (rec[r].a.x * rec[r].a.x + rec[r].a.y * rec[r].a.y) * a.invNM;
      const int rr = (N - rec[r].f0) & (N - 1);
      const int s = rec[r].f1 >= M / 2 ? rec[r].f1 - M : rec[r].f1;
      const uint32_t idx = (uint32_t)rr * M + (uint32_t)(s + M / 2);
      keys[r] = ((uint64_t)__float_as_uint(p) << 32) | (uint64_t)(~idx);
    }
    for (int i = 1; i < nr; ++i) {
      const uint64_t x = keys[i];
      int j = i - 1;
      while (j >= 0 && keys[j] < x) { keys[j + 1] = keys[j]; --j; }
      keys[j + 1] = x;
    }
    const int nv = nr < a.K ? nr : a.K;
    for (int i = 0; i < nv; ++i) {
      const uint32_t idx = ~(uint32_t)(keys[i] & 0xffffffffu);
      ofdm_target tg;
      tg.r = (int32_t)(idx / (uint32_t)M);
      tg.s = (int32_t)(idx % (uint32_t)M) - M / 2;
      tg.power = __uint_as_float((uint32_t)(keys[i] >> 32));
      tg.range_m = (float)tg.r * a.dd;
      tg.vel_mps = (float)tg.s * a.dv;
      if (out) out[(size_t)f * a.K + i] = tg;
    }
    if (n_out) n_out[f] = nv;
    if (wstatus) wstatus[f] = 0u;
  }
}

size_t fps_workspace_elems(int frames, int iterations, int T, int Q) {
  return (size_t)frames * iterations * T * Q;
}

template <int Q>
static cudaError_t launch_fps_q(const float2* strip, const float2* Y, const float2* X, const int32_t* slices,
                                float2* S, ofdm_target* out, int32_t* n_out, uint32_t* wstatus, const FpsArgs& a,
                                cudaStream_t s, int* launches) {
  cudaError_t e;
  if (a.direct) {
    const long total = (long)a.frames * a.iterations * a.T * Q;
    long blocks = (total + kFpsThreads - 1) / kFpsThreads;
    if (blocks > 152 * 16) blocks = 152 * 16;
    fps_sample_direct_kernel<<<(unsigned)blocks, kFpsThreads, 0, s>>>(Y, X, slices, S, wstatus, a);
  } else {
    const size_t smem = (size_t)a.rows * kFpsCols * sizeof(float2);
    e = cudaFuncSetAttribute(fps_sample_taps_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)((a.M + kFpsCols - 1) / kFpsCols), (unsigned)a.frames);
    fps_sample_taps_kernel<<<grid, kFpsThreads, smem, s>>>(strip, slices, S, a);
  }
  ++*launches;
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  {
    const long nsl = (long)a.frames * a.iterations * a.T;
    const size_t smem = (size_t)(kFpsThreads / 32) * smem_elems(Q) * sizeof(float2);
    e = cudaFuncSetAttribute(fps_fft_kernel<Q>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const long blocks = (nsl + kFpsThreads / 32 - 1) / (kFpsThreads / 32);
    fps_fft_kernel<Q><<<(unsigned)blocks, kFpsThreads, smem, s>>>(S, nsl, a.twQ);
    ++*launches;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  const size_t smem = (size_t)kFpsMaxT * Q * sizeof(float2) + Q * sizeof(float2) + 2 * Q * sizeof(float) +
                      (kFpsMaxRec + kFpsMaxCand) * sizeof(FpsRec) + kFpsMaxCand * sizeof(int);
  e = cudaFuncSetAttribute(fps_decode_kernel<Q>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  fps_decode_kernel<Q><<<a.frames, kFpsThreads, smem, s>>>(S, slices, out, n_out, wstatus, a);
  ++*launches;
  return cudaGetLastError();
}

cudaError_t launch_fps(int Q, const float2* strip, const float2* Y, const float2* X, const int32_t* slices,
                       float2* S, ofdm_target* out, int32_t* n_out, uint32_t* wstatus, const FpsArgs& a,
                       cudaStream_t s, int* launches) {
  switch (Q) {
    case 64: return launch_fps_q<64>(strip, Y, X, slices, S, out, n_out, wstatus, a, s, launches);
    case 128: return launch_fps_q<128>(strip, Y, X, slices, S, out, n_out, wstatus, a, s, launches);
    case 256: return launch_fps_q<256>(strip, Y, X, slices, S, out, n_out, wstatus, a, s, launches);
    case 512: return launch_fps_q<512>(strip, Y, X, slices, S, out, n_out, wstatus, a, s, launches);
    case 1024: return launch_fps_q<1024>(strip, Y, X, slices, S, out, n_out, wstatus, a, s, launches);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace ofdm
