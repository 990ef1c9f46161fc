// doppler_general.cu -- the Doppler stage and detection for a Doppler grid M'
// that is not a power of two (Table I's M = M' = 560 = 2^4 5 7).
//
// Doppler (Eq. (17)): the windowed DFT over the M OFDM symbols of every
// support row of the range profile,
//     D[r, s] = sum_{l < M} (w_l g[r, l]) e^{-2 pi i l s / M'},   P = |D|^2 / (N M),
// as a power-of-two-length DFT and an odd-length DFT (M' = P Q).
//
// Detection (Eq. (18)): 8-neighbour local maxima (circular), optionally above
// the global threshold or the CFAR one, ordered by power then map index:
// each CTA sorts the candidates of its block of cells and keeps its best K;
// one CTA per frame merges the block lists.
#include "fft.cuh"
#include "internal.h"

namespace ofdm {

constexpr int kGThreads = 256;

// Doppler (Eq. (17)) for M' = P Q with P the largest power of two dividing M'
// and Q odd (Table I: 560 = 16 x 35), by two smaller DFTs (Good-Thomas is not
// needed: the twiddles are applied between the stages):
//   l = Q l1 + l2,  s = s1 + P s2,  w = e^{-2 pi i / M'}:
//   A[s1][l2] = w^(l2 s1) sum_{l1 < P} x[Q l1 + l2] w^(Q l1 s1)          (P-point DFTs)
//   D[s1 + P s2] = sum_{l2 < Q} A[s1][l2] w^(P l2 s2)                    (Q-point DFTs)
// with x[l] = w_l g[r, l] for l < M and 0 up to M'.  M'(P + Q) complex
// multiply-adds per row instead of M'^2 (28.6k instead of 313.6k for 560).
// One CTA per (row, frame); the row and the intermediate A live in shared
// memory; the roots w^m come from a table (all exponents reduced mod M').
__global__ void __launch_bounds__(kGThreads)
doppler_2factor_kernel(const float2* __restrict__ strip, float* __restrict__ map, float* __restrict__ pow,
                       DopplerArgs d, const float2* __restrict__ roots, int P, int Q) {
  extern __shared__ float2 dg_smem[];
  float2* x = dg_smem;             // [M'] windowed row, zero-padded
  float2* A = dg_smem + d.Mp;      // [P][Q] after the first stage
  float2* w = A + d.Mp;            // [M'] roots
  const int ri = blockIdx.x, f = blockIdx.y, tid = threadIdx.x;
  const int M = d.M, Mp = d.Mp;
  const float2* g = strip + ((size_t)f * d.rows + ri) * M;
  for (int l = tid; l < Mp; l += kGThreads) {
    x[l] = l < M ? cscale(g[l], __ldg(d.wl + l)) : make_float2(0.f, 0.f);
    w[l] = __ldg(roots + l);
  }
  __syncthreads();
  for (int e = tid; e < Mp; e += kGThreads) {     // e = s1 Q + l2
    const int s1 = e / Q, l2 = e % Q;
    const int step = (int)(((long)Q * s1) % Mp);
    float2 acc = make_float2(0.f, 0.f);
    int m = 0;
    for (int l1 = 0; l1 < P; ++l1) {
      acc = cadd(acc, cmul(x[Q * l1 + l2], w[m]));
      m += step;
      if (m >= Mp) m -= Mp;
    }
    A[e] = cmul(acc, w[(int)(((long)l2 * s1) % Mp)]);
  }
  __syncthreads();
  const int row = (d.row0 + ri) % d.Np;
  float* mrow = map ? map + (d.map_off ? (long)d.map_off[f] : (long)f * d.Np * Mp) + (long)row * Mp : nullptr;
  float* prow = pow ? pow + ((size_t)f * d.rows + ri) * Mp : nullptr;
  for (int e = tid; e < Mp; e += kGThreads) {     // e = s1 + P s2
    const int s1 = e % P, s2 = e / P;
    const int step = (int)(((long)P * s2) % Mp);
    const float2* a = A + s1 * Q;
    float2 acc = make_float2(0.f, 0.f);
    int m = 0;
    for (int l2 = 0; l2 < Q; ++l2) {
      acc = cadd(acc, cmul(a[l2], w[m]));
      m += step;
      if (m >= Mp) m -= Mp;
    }
    const float p = (acc.x * acc.x + acc.y * acc.y) * d.inv_nm;
    const int c = (e + Mp / 2) % Mp;   // column of Doppler bin e (e >= M'/2 is negative)
    if (mrow) mrow[c] = p;
    if (prow) prow[c] = p;
  }
}

// ---------------------------------------------------------------- detection
constexpr int kGCells = 8;                      // cells per thread
constexpr int kGBlockCells = kGThreads * kGCells;

__device__ __forceinline__ float gval(const float* base, const DetectArgs& a, int rj, int c) {
  return base[(long)(a.compact ? rj : (a.row0 + rj) % a.Np) * a.Mp + c];
}

// CFAR statistic test (same rule as the power-of-two path, general M').
__device__ bool gcfar(const float* base, const DetectArgs& a, int ri, int c, float p) {
  const int g = a.cfar_guard, w = g + a.cfar_train, Mp = a.Mp;
  float sum = 0.f;
  int n = 0;
  for (int dr = -w; dr <= w; ++dr) {
    int rj = ri + dr;
    if (a.full) rj = ((rj % a.rows) + a.rows) % a.rows;
    else if (rj < 0 || rj >= a.rows) continue;
    for (int dc = -w; dc <= w; ++dc) {
      if (dr >= -g && dr <= g && dc >= -g && dc <= g) continue;
      sum += gval(base, a, rj, ((c + dc) % Mp + Mp) % Mp);
      ++n;
    }
  }
  return n > 0 && p >= a.cfar_alpha[n] * (sum / (float)n);
}

// Block b of a frame's support cells: candidates, sorted, best K to keys[f][b][0..K).
__global__ void __launch_bounds__(kGThreads)
detect_general_block_kernel(const float* __restrict__ src, DetectArgs a, int blocks, unsigned* __restrict__ counts) {
  __shared__ uint64_t buf[kGBlockCells];
  __shared__ unsigned s_n;
  const int b = blockIdx.x, f = blockIdx.y, tid = threadIdx.x;
  const float* base = src + (long)f * a.frame_stride;
  const int Mp = a.Mp;
  const long cells = (long)a.rows * Mp;
  const bool thr = a.mode == OFDM_DETECT_THRESHOLD, cfar = a.mode == OFDM_DETECT_CFAR;
  const float eta = thr ? (a.use_fixed_eta ? a.eta_fixed : a.eta[f]) : 0.f;
  if (tid == 0) s_n = 0;
  for (int i = tid; i < kGBlockCells; i += kGThreads) buf[i] = 0ull;
  __syncthreads();
  for (int k = 0; k < kGCells; ++k) {
    const long e = (long)b * kGBlockCells + (long)k * kGThreads + tid;
    if (e >= cells) break;
    const int ri = (int)(e / Mp), c = (int)(e % Mp);
    const int r = (a.row0 + ri) % a.Np;
    const float p = gval(base, a, ri, c);
    if (!(p > 0.f) || (thr && !(p >= eta))) continue;
    const uint32_t idx = (uint32_t)r * (uint32_t)Mp + (uint32_t)c;
    bool lm = true;
    for (int dr = -1; dr <= 1 && lm; ++dr) {
      int rj = ri + dr;
      float q;
      int rn = (r + dr + a.Np) % a.Np;
      if (a.full) { rj = (rj + a.rows) % a.rows; }
      for (int dc = -1; dc <= 1; ++dc) {
        if (dr == 0 && dc == 0) continue;
        const int cn = (c + dc + Mp) % Mp;
        q = (rj >= 0 && rj < a.rows) ? gval(base, a, rj, cn) : 0.f;   // rows off the support are zero
        const uint32_t nidx = (uint32_t)rn * (uint32_t)Mp + (uint32_t)cn;
        if (q > p || (q == p && nidx < idx)) { lm = false; break; }
      }
    }
    if (!lm || (cfar && !gcfar(base, a, ri, c, p))) continue;
    const unsigned slot = atomicAdd(&s_n, 1u);
    buf[slot] = ((uint64_t)__float_as_uint(p) << 32) | (uint64_t)(~idx);
  }
  __syncthreads();
  if (tid == 0 && s_n) atomicAdd(counts + f, s_n);
  // sort the block's candidates, keys descending (bitonic over the filled
  // prefix rounded up to a power of two; the rest of buf is zero)
  int n = 32;
  while (n < (int)s_n) n <<= 1;
  for (int k = 2; k <= n; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = tid; i < n; i += kGThreads) {
        const int p2 = i ^ j;
        if (p2 > i) {
          const uint64_t x = buf[i], y = buf[p2];
          const bool desc = (i & k) == 0;
          if (desc ? (x < y) : (x > y)) { buf[i] = y; buf[p2] = x; }
        }
      }
      __syncthreads();
    }
  uint64_t* out = a.part_keys + ((size_t)f * blocks + b) * 32;
  if (tid < 32) out[tid] = tid < a.K ? buf[tid] : 0ull;
}

// One CTA per frame: the K largest keys of the block lists (each sorted
// descending) by K rounds of a block-wide maximum over the lists' heads; then
// the targets and status.
__global__ void __launch_bounds__(kGThreads)
detect_general_merge_kernel(DetectArgs a, int blocks, unsigned* __restrict__ counts, ofdm_target* __restrict__ out,
                            int32_t* __restrict__ n_out, uint32_t* __restrict__ status,
                            uint32_t* __restrict__ wstatus) {
  extern __shared__ int heads[];                 // [blocks] position of each list's head
  __shared__ uint64_t s_key[kGThreads / 32];
  __shared__ int s_list[kGThreads / 32];
  __shared__ uint64_t s_top[32];
  const int f = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint64_t* src = a.part_keys + (size_t)f * blocks * 32;
  const int K = a.K;
  for (int b = tid; b < blocks; b += kGThreads) heads[b] = 0;
  __syncthreads();
  for (int k = 0; k < K; ++k) {
    uint64_t best = 0;
    int bl = -1;
    for (int b = tid; b < blocks; b += kGThreads) {
      const uint64_t v = heads[b] < 32 ? src[b * 32 + heads[b]] : 0ull;
      if (v > best) { best = v; bl = b; }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      const uint64_t ov = __shfl_xor_sync(0xffffffffu, best, o);
      const int ob = __shfl_xor_sync(0xffffffffu, bl, o);
      if (ov > best) { best = ov; bl = ob; }
    }
    if (lane == 0) { s_key[warp] = best; s_list[warp] = bl; }
    __syncthreads();
    if (tid == 0) {
      uint64_t m = s_key[0];
      int mb = s_list[0];
      for (int w = 1; w < kGThreads / 32; ++w)
        if (s_key[w] > m) { m = s_key[w]; mb = s_list[w]; }
      s_top[k] = m;
      if (m != 0 && mb >= 0) ++heads[mb];
    }
    __syncthreads();
  }
  if (tid == 0) {
    const unsigned total = counts[f];
    const int nv = (int)(total < (unsigned)K ? total : (unsigned)K);
    const int oi = a.out_idx ? a.out_idx[f] : f;
    for (int i = 0; i < nv; ++i) {
      const uint32_t idx = ~(uint32_t)(s_top[i] & 0xffffffffu);
      ofdm_target t;
      t.r = (int32_t)(idx / (uint32_t)a.Mp);
      t.s = (int32_t)(idx % (uint32_t)a.Mp) - a.Mp / 2;
      t.power = __uint_as_float((uint32_t)(s_top[i] >> 32));
      t.range_m = (float)t.r * a.dd;
      t.vel_mps = (float)t.s * a.dv;
      if (out) out[(size_t)oi * K + i] = t;
    }
    uint32_t st = wstatus ? wstatus[f] : 0u;
    if (a.mode == OFDM_DETECT_TOPK && total < (unsigned)K) st |= OFDM_STATUS_FEW_PEAKS;
    if (a.mode != OFDM_DETECT_TOPK && total > (unsigned)K) st |= OFDM_STATUS_OVERFLOW;
    if (n_out) n_out[oi] = nv;
    if (status) status[oi] = st;
    if (wstatus) wstatus[f] = 0u;
    counts[f] = 0u;
  }
}

// Threshold mode without a given noise level: the lower median of P over the
// frame's support cells (radix select on the float bits), times -ln(P_fa) / ln 2.
__global__ void __launch_bounds__(1024) median_general_kernel(const float* __restrict__ src, DetectArgs a) {
  __shared__ uint32_t hist[256];
  __shared__ uint32_t s_prefix, s_rank;
  const int f = blockIdx.x, tid = threadIdx.x;
  const float* base = src + (long)f * a.frame_stride;
  const long n = (long)a.rows * a.Mp;
  if (tid == 0) { s_prefix = 0; s_rank = (uint32_t)((n - 1) / 2); }
  uint32_t mask = 0;
  for (int shift = 24; shift >= 0; shift -= 8) {
    for (int i = tid; i < 256; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    const uint32_t prefix = s_prefix;
    for (long e = tid; e < n; e += blockDim.x) {
      const uint32_t u = __float_as_uint(gval(base, a, (int)(e / a.Mp), (int)(e % a.Mp)));
      if ((u & mask) == prefix) atomicAdd(&hist[(u >> shift) & 255u], 1u);
    }
    __syncthreads();
    if (tid == 0) {
      uint32_t rank = s_rank, d = 0;
      for (; d < 255; ++d) {
        if (hist[d] > rank) break;
        rank -= hist[d];
      }
      s_rank = rank;
      s_prefix = prefix | (d << shift);
    }
    mask |= 255u << shift;
    __syncthreads();
  }
  if (tid == 0) a.eta[f] = __fmul_rn(__uint_as_float(s_prefix), a.eta_factor);
}

cudaError_t launch_doppler_general(const float2* strip, float* map, float* pow, const DopplerArgs& a,
                                   const float2* roots, cudaStream_t s, int* launches) {
  int P = 1;
  while (a.Mp % (2 * P) == 0) P *= 2;
  const int Q = a.Mp / P;
  const size_t smem = (size_t)3 * a.Mp * sizeof(float2);
  ++*launches;
  doppler_2factor_kernel<<<dim3((unsigned)a.rows, (unsigned)a.frames), kGThreads, smem, s>>>(strip, map, pow, a, roots,
                                                                                            P, Q);
  return cudaGetLastError();
}

int detect_general_blocks(int rows, int Mp) { return (int)(((long)rows * Mp + kGBlockCells - 1) / kGBlockCells); }

cudaError_t launch_detect_general(const float* pow, ofdm_target* out, int32_t* n_out, uint32_t* status,
                                  uint32_t* wstatus, const DetectArgs& a, cudaStream_t s, int* launches) {
  const int blocks = detect_general_blocks(a.rows, a.Mp);
  if (a.mode == OFDM_DETECT_THRESHOLD && !a.use_fixed_eta) {
    median_general_kernel<<<a.frames, 1024, 0, s>>>(pow, a);
    ++*launches;
  }
  detect_general_block_kernel<<<dim3((unsigned)blocks, (unsigned)a.frames), kGThreads, 0, s>>>(pow, a, blocks,
                                                                                              a.counts);
  ++*launches;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const size_t smem = (size_t)blocks * sizeof(int);
  e = cudaFuncSetAttribute(detect_general_merge_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  detect_general_merge_kernel<<<a.frames, kGThreads, smem, s>>>(a, blocks, a.counts, out, n_out, status, wstatus);
  ++*launches;
  return cudaGetLastError();
}

}  // namespace ofdm
