// learned.cu -- the learned proposal path (not in the paper; its conclusion
// names machine learning as future work).
//
// coarse_kernel: one warp per (frame, support row): an M/4-point Doppler DFT
//   of the first M/4 symbols of the range-profile strip (window over those
//   symbols), |.|^2, max-pooled 4x over range rows with atomicMax on the
//   float bits (P >= 0 orders like unsigned).
// coarse_norm_kernel: x = log(1 + C / mean_frame(C)) -- the CNN input.
// refine_select_kernel: coarse cells whose logit exceeds the threshold
//   become candidates (ascending cell order); a frame with more than the cap
//   is flagged for the full periodogram (the fallback and judge).
// refine_cand_kernel: one CTA per (frame, candidate): the exact periodogram
//   value (Eq. (17): full M-term Doppler sum of the strip, |.|^2 / (N M)) on
//   the 8 x 8 fine block around the candidate, local maxima of its inner 6 x 6.
// refine_merge_kernel: per frame, the strongest K distinct local maxima.
#include "fft.cuh"
#include "internal.h"

namespace ofdm {

constexpr int kRefThreads = 512;

struct CoarseArgs {
  int rows, M, frames, Hc;
  const float* w4;    // window over the first M/4 symbols
  const float2* tw;   // M/4-point pass twiddles
};

template <int MC>
__global__ void __launch_bounds__(256) coarse_kernel(const float2* __restrict__ strip, unsigned* __restrict__ cpow,
                                                     CoarseArgs a) {
  constexpr int E = MC / 32;
  __shared__ float2 smem[8][smem_elems(MC)];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long task = (long)blockIdx.x * 8 + warp;
  if (task >= (long)a.frames * a.rows) return;
  const int f = (int)(task / a.rows), ri = (int)(task % a.rows);
  const float2* g = strip + task * a.M;
  float2 v[E];
#pragma unroll
  for (int q = 0; q < E; ++q) v[q] = cscale(g[lane + 32 * q], __ldg(a.w4 + lane + 32 * q));
  group_fft<MC, 32, -1>(v, smem[warp], a.tw, lane, 0);
  unsigned* row = cpow + ((long)f * a.Hc + ri / 4) * MC;
#pragma unroll
  for (int q = 0; q < E; ++q) {
    const int s = lane + 32 * q;
    atomicMax(row + ((s + MC / 2) & (MC - 1)), __float_as_uint(v[q].x * v[q].x + v[q].y * v[q].y));
  }
}

__global__ void coarse_norm_kernel(const unsigned* __restrict__ cpow, float* __restrict__ x, int cells) {
  __shared__ float red[32];
  const int f = blockIdx.x;
  const unsigned* c = cpow + (long)f * cells;
  float s = 0.f;
  for (int i = threadIdx.x; i < cells; i += blockDim.x) s += __uint_as_float(c[i]);
  for (int off = 16; off; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    float t = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.f;
    for (int off = 16; off; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
    if (threadIdx.x == 0) red[0] = t;
  }
  __syncthreads();
  const float inv_mean = red[0] > 0.f ? (float)cells / red[0] : 0.f;
  for (int i = threadIdx.x; i < cells; i += blockDim.x)
    x[(long)f * cells + i] = log1pf(__uint_as_float(c[i]) * inv_mean);
}

// Candidate selection (one CTA per frame): coarse cells above the logit
// threshold, in a fixed order (ascending cell index) so that the result does
// not depend on thread timing; more than `cap` sends the frame to the fallback.
__global__ void __launch_bounds__(kRefThreads)
refine_select_kernel(const float* __restrict__ logits, int* __restrict__ cand, int* __restrict__ ncand,
                     int* __restrict__ mask, RefineArgs a) {
  __shared__ int s_n;
  const int f = blockIdx.x, tid = threadIdx.x, lane = tid & 31;
  const int cells = a.Hc * a.Mc;
  const float* z = logits + (long)f * cells;
  if (tid == 0) s_n = 0;
  __syncthreads();
  for (int c0 = 0; c0 < cells; c0 += kRefThreads) {
    const int i = c0 + tid;
    const bool hit = i < cells && z[i] > a.zthr;
    const unsigned m = __ballot_sync(0xffffffffu, hit);
    // warp-ordered compaction: warps append in warp order within the chunk
    __shared__ int s_wcount[kRefThreads / 32];
    if (lane == 0) s_wcount[tid >> 5] = __popc(m);
    __syncthreads();
    int base = s_n;
    for (int w = 0; w < (tid >> 5); ++w) base += s_wcount[w];
    const int pos = base + __popc(m & ((1u << lane) - 1u));
    if (hit && pos < a.cap) cand[(long)f * a.cap + pos] = i;
    __syncthreads();
    if (tid == 0) {
      int t = 0;
      for (int w = 0; w < kRefThreads / 32; ++w) t += s_wcount[w];
      s_n += t;
    }
    __syncthreads();
  }
  if (tid == 0) {
    ncand[f] = s_n;
    mask[f] = s_n > a.cap ? 1 : 0;
  }
}

// One CTA per (frame, candidate): exact P on the 8 x 8 fine block, keys of
// the local maxima of its inner 6 x 6 (36 slots, 0 = none).
__global__ void __launch_bounds__(kRefThreads)
refine_cand_kernel(const float2* __restrict__ strip, const int* __restrict__ cand, const int* __restrict__ ncand,
                   uint64_t* __restrict__ keys, RefineArgs a) {
  extern __shared__ __align__(16) unsigned char ref_smem[];
  float2* tw = reinterpret_cast<float2*>(ref_smem);            // exp(-2 pi i m / M), from the plan
  float2* rows8 = tw + a.M;                                    // 8 windowed strip rows
  float* blk = reinterpret_cast<float*>(rows8 + 8 * a.M);      // 8 x 8 block of P
  const int f = blockIdx.y, ci = blockIdx.x, tid = threadIdx.x;
  uint64_t* kout = keys + ((long)f * a.cap + ci) * 36;
  const int nc = ncand[f];
  if (nc > a.cap || ci >= nc) {  // fallback frame or unused slot
    if (tid < 36) kout[tid] = 0;
    return;
  }
  for (int m = tid; m < a.M; m += kRefThreads) tw[m] = __ldg(a.rootsM + m);
  const float2* g = strip + (long)f * a.rows * a.M;
  const int cell = cand[(long)f * a.cap + ci];
  const int rc = cell / a.Mc, col = cell % a.Mc;
  const int r0 = 4 * rc - 2;                        // first fine support row of the block
  const int s0 = 4 * (col - a.Mc / 2) - 4;          // first fine (centred) Doppler bin
  for (int e = tid; e < 8 * a.M; e += kRefThreads) {
    const int u = e / a.M, l = e % a.M, ri = r0 + u;
    rows8[e] = (ri >= 0 && ri < a.rows) ? cscale(g[(long)ri * a.M + l], __ldg(a.wl + l)) : make_float2(0.f, 0.f);
  }
  __syncthreads();
  {  // 64 cells, 8 lanes each: P = |sum_l w_l g[r, l] e^{-2 pi i l s / M}|^2 / (N M)  (Eq. (17))
    const int cidx = tid >> 3, part = tid & 7;
    const int u = cidx >> 3, vv = cidx & 7;
    const int sb = (s0 + vv) & (a.M - 1);
    float2 acc = make_float2(0.f, 0.f);
    for (int l = part; l < a.M; l += 8) acc = cadd(acc, cmul(rows8[u * a.M + l], tw[(l * sb) & (a.M - 1)]));
    const unsigned m8 = 0xffu << (threadIdx.x & 24);
    for (int off = 4; off; off >>= 1) {
      acc.x += __shfl_xor_sync(m8, acc.x, off);
      acc.y += __shfl_xor_sync(m8, acc.y, off);
    }
    if (part == 0) blk[cidx] = (acc.x * acc.x + acc.y * acc.y) * a.inv_nm;
  }
  __syncthreads();
  if (tid < 36) {  // inner 6 x 6: local maxima with the map's key order
    const int u = 1 + tid / 6, vv = 1 + tid % 6, ri = r0 + u;
    const float p = blk[u * 8 + vv];
    uint64_t key = 0;
    if (ri >= 0 && ri < a.rows && p > 0.f) {
      auto idx_of = [&](int uu, int w) -> uint32_t {
        const int r = (a.row0 + r0 + uu) & (a.N - 1);
        const int s = ((s0 + w + a.M / 2) & (a.M - 1));   // map column of the centred bin
        return (uint32_t)r * a.M + (uint32_t)s;
      };
      key = ((uint64_t)__float_as_uint(p) << 32) | (uint64_t)(~idx_of(u, vv));
      bool ok = true;
      for (int du = -1; du <= 1; ++du)
        for (int dv = -1; dv <= 1; ++dv) {
          if (!du && !dv) continue;
          const int rn = r0 + u + du;
          const float pn = (rn >= 0 && rn < a.rows) ? blk[(u + du) * 8 + vv + dv] : 0.f;
          const uint64_t kn = ((uint64_t)__float_as_uint(pn) << 32) | (uint64_t)(~idx_of(u + du, vv + dv));
          ok &= key > kn;
        }
      if (!ok) key = 0;
    }
    kout[tid] = key;
  }
}

// One CTA per frame: sort the candidates' keys, drop repeats (overlapping
// blocks), report the strongest K.
__global__ void __launch_bounds__(kRefThreads)
refine_merge_kernel(const uint64_t* __restrict__ keys, const int* __restrict__ ncand, ofdm_target* __restrict__ out,
                    int32_t* __restrict__ n_out, uint32_t* __restrict__ status, uint32_t* __restrict__ wstatus,
                    RefineArgs a) {
  extern __shared__ uint64_t buf[];   // next power of two >= cap * 36 keys
  const int f = blockIdx.x, tid = threadIdx.x;
  const int nc = ncand[f];
  if (nc > a.cap) return;  // fallback frame: the full path reports it
  const int n = min(nc, a.cap) * 36;
  int sort_n = 32;
  while (sort_n < n) sort_n <<= 1;
  for (int i = tid; i < sort_n; i += kRefThreads) buf[i] = i < n ? keys[(long)f * a.cap * 36 + i] : 0;
  __syncthreads();
  for (int k = 2; k <= sort_n; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = tid; i < sort_n; i += kRefThreads) {
        const int p = i ^ j;
        if (p > i) {
          const uint64_t x = buf[i], y = buf[p];
          const bool desc = (i & k) == 0;
          if (desc ? (x < y) : (x > y)) { buf[i] = y; buf[p] = x; }
        }
      }
      __syncthreads();
    }
  if (tid == 0) {
    int nv = 0;
    uint64_t prev = 0;
    for (int i = 0; i < n && nv < a.K; ++i) {
      const uint64_t k = buf[i];
      if (k == 0 || k == prev) continue;
      prev = k;
      const uint32_t idx = ~(uint32_t)(k & 0xffffffffu);
      ofdm_target tg;
      tg.r = (int32_t)(idx / (uint32_t)a.M);
      tg.s = (int32_t)(idx % (uint32_t)a.M) - a.M / 2;
      tg.power = __uint_as_float((uint32_t)(k >> 32));
      tg.range_m = (float)tg.r * a.dd;
      tg.vel_mps = (float)tg.s * a.dv;
      if (out) out[(long)f * a.K + nv] = tg;
      ++nv;
    }
    if (n_out) n_out[f] = nv;
    uint32_t st = wstatus[f];
    if (nv < a.K) st |= OFDM_STATUS_FEW_PEAKS;
    if (status) status[f] = st;
    wstatus[f] = 0u;
  }
}

template <int MC>
static cudaError_t launch_coarse_m(const float2* strip, unsigned* cpow, float* x, const CoarseArgs& a,
                                   cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(cpow, 0, (size_t)a.frames * a.Hc * MC * sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  const long tasks = (long)a.frames * a.rows;
  coarse_kernel<MC><<<(unsigned)((tasks + 7) / 8), 256, 0, s>>>(strip, cpow, a);
  coarse_norm_kernel<<<a.frames, 256, 0, s>>>(cpow, x, a.Hc * MC);
  return cudaGetLastError();
}

cudaError_t launch_coarse(const float2* strip, unsigned* cpow, float* x, int rows, int M, int frames,
                          const float* w4, const float2* tw, cudaStream_t s, int* launches) {
  CoarseArgs a;
  a.rows = rows; a.M = M; a.frames = frames; a.Hc = (rows + 3) / 4; a.w4 = w4; a.tw = tw;
  *launches += 2;
  switch (M / 4) {
    case 64: return launch_coarse_m<64>(strip, cpow, x, a, s);
    case 128: return launch_coarse_m<128>(strip, cpow, x, a, s);
    case 256: return launch_coarse_m<256>(strip, cpow, x, a, s);
    default: *launches -= 2; return cudaErrorInvalidValue;
  }
}

cudaError_t launch_refine(const float2* strip, const float* logits, ofdm_target* out, int32_t* n_out,
                          uint32_t* status, uint32_t* wstatus, int* mask, int* cand, int* ncand, uint64_t* keys,
                          const RefineArgs& a, cudaStream_t s, int* launches) {
  *launches += 3;
  refine_select_kernel<<<a.frames, kRefThreads, 0, s>>>(logits, cand, ncand, mask, a);
  const size_t smem = (size_t)a.M * sizeof(float2) * 9 + 64 * sizeof(float);
  cudaError_t e = cudaFuncSetAttribute(refine_cand_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  refine_cand_kernel<<<dim3(a.cap, a.frames), kRefThreads, smem, s>>>(strip, cand, ncand, keys, a);
  int pow2 = 32;
  while (pow2 < a.cap * 36) pow2 <<= 1;
  const size_t msmem = (size_t)pow2 * sizeof(uint64_t);
  e = cudaFuncSetAttribute(refine_merge_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)msmem);
  if (e != cudaSuccess) return e;
  refine_merge_kernel<<<a.frames, kRefThreads, msmem, s>>>(keys, ncand, out, n_out, status, wstatus, a);
  return cudaGetLastError();
}

}  // namespace ofdm
