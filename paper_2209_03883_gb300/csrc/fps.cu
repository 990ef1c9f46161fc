// fps.cu -- FPS-SFT (Sec. III-C): the sparse alternative to the 2D
// periodogram, on the DFT-CE channel estimate H'.
//
// One CTA per frame runs every iteration (peeling needs the previous
// iteration's result, so the frame stays on one SM):
//   1. slice samples s_j[n] = H'[(a0 n + t0_j) mod N, (a1 n + t1_j) mod M]
//      evaluated straight from the kept DFT-CE taps (the strip written by the
//      column kernel with a rect stencil holds N h[n]):
//      H'[k, l] = (1/N) sum_{n < L_cp} (N h[n, l]) e^{-2 pi i n k / N}  (Eq. (22));
//   2. one warp per slice: Q-point DFT (Q = lcm(N, M) = max(N, M) here);
//   3. removal of the frequencies already recovered from every slice;
//   4. bin energy test against the median of the bin energies;
//   5. ML decoding along each surviving bin's projection line with a
//      coherence test (1-sparsity), amplitude from the coherent sum.
#include <float.h>

#include "fft.cuh"
#include "internal.h"

namespace ofdm {

constexpr int kFpsThreads = 256;
constexpr int kFpsMaxT = 8;        // slices per iteration
constexpr int kFpsMaxRec = 64;     // recovered frequencies per frame
constexpr int kFpsMaxCand = 256;   // candidate bins decoded per iteration

struct FpsRec { int f0, f1; float2 a; };

template <int Q>
struct FpsLayout {
  static constexpr int SL = smem_elems(Q);  // float2 per slice (padded for the FFT exchange)
};

__device__ __forceinline__ float2 ptab_at(const float2* ptab, int m, int sign) {
  float2 w = ptab[m];
  if (sign < 0) w.y = -w.y;
  return w;
}

template <int Q>
__global__ void __launch_bounds__(kFpsThreads)
fps_kernel(const float2* __restrict__ strip, const int32_t* __restrict__ slices, ofdm_target* __restrict__ out,
           int32_t* __restrict__ n_out, uint32_t* __restrict__ wstatus, FpsArgs a) {
  using Lay = FpsLayout<Q>;
  extern __shared__ __align__(16) unsigned char fps_smem[];
  float2* S = reinterpret_cast<float2*>(fps_smem);                 // T slices
  float2* ptab = S + (size_t)kFpsMaxT * Lay::SL;                    // exp(+2 pi i m / Q)
  float* E = reinterpret_cast<float*>(ptab + Q);                    // bin energy
  float* srt = E + Q;                                               // sorted copy
  FpsRec* rec = reinterpret_cast<FpsRec*>(srt + Q);                 // recovered list
  FpsRec* fnd = rec + kFpsMaxRec;                                   // found this iteration
  int* cand = reinterpret_cast<int*>(fnd + kFpsMaxCand);            // candidate bins
  float2* taps = reinterpret_cast<float2*>(cand + kFpsMaxCand);     // [rows][CB] batch of tap columns
  __shared__ int s_nrec, s_ncand, s_nfnd;
  __shared__ float s_peak;

  const int f = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int N = a.N, M = a.M, T = a.T, rows = a.rows;
  const int qn = Q / N, qm = Q / M;
  const float2* g = strip + (size_t)f * rows * M;

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
    unsigned inv = 1u;  // a1^{-1} mod 2^32 by Newton's iteration (a1 odd), then mod M
    for (int k = 0; k < 5; ++k) inv = inv * (2u - (unsigned)a1 * inv);
    const int a1inv = (int)(inv & (unsigned)(M - 1));

    // ---- 1. slice samples, CB tap columns at a time
    for (int l0 = 0; l0 < M; l0 += a.CB) {
      __syncthreads();
      for (int e = tid; e < rows * a.CB; e += kFpsThreads) {
        const int n = e / a.CB, cb = e % a.CB;
        taps[e] = (l0 + cb < M) ? g[(size_t)n * M + l0 + cb] : make_float2(0.f, 0.f);
      }
      __syncthreads();
      // items (column, slice, repeat) handled by quads of lanes
      const int reps = Q / M;
      const int items = a.CB * T * reps;
      for (int it4 = tid >> 2; it4 < items; it4 += kFpsThreads >> 2) {
        const int cb = it4 % a.CB, rest = it4 / a.CB;
        const int j = rest % T, rep = rest / T;
        const int l = l0 + cb;
        if (l >= M) continue;
        const int t0 = sp[2 + 2 * j], t1 = sp[3 + 2 * j];
        const int n0 = (int)(((unsigned)a1inv * (unsigned)((l - t1) & (M - 1))) & (unsigned)(M - 1));
        const int n = n0 + M * rep;
        const int k = (int)(((long)a0 * n + t0) % N + N) % N;
        float2 acc = make_float2(0.f, 0.f);
        for (int nn = (tid & 3); nn < rows; nn += 4) {
          const float4 w4 = __ldg(a.w_df + (int)(((unsigned)nn * (unsigned)k) & (unsigned)(N - 1)));
          const float2 w = make_float2(w4.x, -w4.z);  // exp(-2 pi i nn k / N)
          acc = cadd(acc, cmul(taps[nn * a.CB + cb], w));
        }
        const unsigned qmask = 0xfu << (lane & ~3);  // the four lanes of this item
        acc.x += __shfl_xor_sync(qmask, acc.x, 1);
        acc.y += __shfl_xor_sync(qmask, acc.y, 1);
        acc.x += __shfl_xor_sync(qmask, acc.x, 2);
        acc.y += __shfl_xor_sync(qmask, acc.y, 2);
        if ((tid & 3) == 0) S[(size_t)j * Lay::SL + n] = cscale(acc, a.invN);
      }
    }
    __syncthreads();

    // ---- 2. Q-point DFT of each slice (warp j), natural order in and out
    for (int j = warp; j < T; j += kFpsThreads / 32) {
      float2* sj = S + (size_t)j * Lay::SL;
      constexpr int E2 = Q / 32;
      float2 v[E2];
#pragma unroll
      for (int q = 0; q < E2; ++q) v[q] = sj[lane + 32 * q];
      group_fft<Q, 32, -1>(v, sj, a.twQ, lane, 0);
      __syncwarp();
#pragma unroll
      for (int q = 0; q < E2; ++q) sj[lane + 32 * q] = v[q];
      __syncwarp();
      // ---- 3. remove the recovered frequencies (serial per slice: bins may coincide)
      if (lane == 0) {
        const int t0 = sp[2 + 2 * j], t1 = sp[3 + 2 * j];
        for (int r = 0; r < s_nrec; ++r) {
          const int f0 = rec[r].f0, f1 = rec[r].f1;
          const int m = (int)(((long)a0 * f0 * qn + (long)a1 * f1 * qm) % Q);
          const int ph = (int)(((long)f0 * t0 * qn + (long)f1 * t1 * qm) % Q);
          const float2 c = cscale(cmul(rec[r].a, ptab_at(ptab, ph, +1)), (float)Q * a.invNM);
          sj[m] = csub(sj[m], c);
        }
      }
    }
    __syncthreads();

    // ---- 4. bin energies, median threshold, running peak
    for (int m = tid; m < Q; m += kFpsThreads) {
      float e = 0.f;
      for (int j = 0; j < T; ++j) {
        const float2 v = S[(size_t)j * Lay::SL + m];
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

    // ---- 5. ML decoding along each candidate bin's line (one warp per bin)
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
          acc = cadd(acc, cmul(S[(size_t)j * Lay::SL + m], ptab_at(ptab, ph, -1)));
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
          const float2 v = S[(size_t)j * Lay::SL + m];
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

template <int Q>
static cudaError_t launch_fps_q(const float2* strip, const int32_t* slices, ofdm_target* out, int32_t* n_out,
                                uint32_t* wstatus, const FpsArgs& a, cudaStream_t s) {
  const size_t smem = (size_t)kFpsMaxT * FpsLayout<Q>::SL * sizeof(float2) + Q * sizeof(float2) +
                      2 * Q * sizeof(float) + (kFpsMaxRec + kFpsMaxCand) * sizeof(FpsRec) +
                      kFpsMaxCand * sizeof(int) + (size_t)a.rows * a.CB * sizeof(float2);
  cudaError_t e = cudaFuncSetAttribute(fps_kernel<Q>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  fps_kernel<Q><<<a.frames, kFpsThreads, smem, s>>>(strip, slices, out, n_out, wstatus, a);
  return cudaGetLastError();
}

cudaError_t launch_fps(int Q, const float2* strip, const int32_t* slices, ofdm_target* out, int32_t* n_out,
                       uint32_t* wstatus, const FpsArgs& a, cudaStream_t s, int* launches) {
  ++*launches;
  switch (Q) {
    case 64: return launch_fps_q<64>(strip, slices, out, n_out, wstatus, a, s);
    case 128: return launch_fps_q<128>(strip, slices, out, n_out, wstatus, a, s);
    case 256: return launch_fps_q<256>(strip, slices, out, n_out, wstatus, a, s);
    case 512: return launch_fps_q<512>(strip, slices, out, n_out, wstatus, a, s);
    case 1024: return launch_fps_q<1024>(strip, slices, out, n_out, wstatus, a, s);
    default: --*launches; return cudaErrorInvalidValue;
  }
}

}  // namespace ofdm
