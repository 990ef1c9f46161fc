// doppler_detect.cu -- the per-range-row half of the chain (steps a6-a7).
//
// doppler_kernel: one warp per (frame, support row r): the window over l,
//   the M'-point Doppler DFT  D[s] = sum_l w_l g[r, l] e^{-2 pi i l s / M'}
//   and P = |D|^2 / (N M) (Eq. (17)); column c = s + M'/2 (mod M').  Each row
//   goes to the compact power strip used by detection and, when asked, to the
//   full map.
// zero_rows_kernel: the map rows outside the DFT-CE support are exactly zero.
// detect_kernel: one CTA per frame: 8-neighbour local maxima (circular in r
//   and s), optional threshold eta = -sigma^2 ln(P_fa) with sigma^2 from the
//   lower median (Eq. (18)), top-K by (power desc, map index asc), Eq. (19).
#include <float.h>

#include "fft.cuh"
#include "internal.h"

namespace ofdm {

constexpr int kDopWarps = 8;

template <int MP>
__global__ void __launch_bounds__(32 * kDopWarps)
doppler_kernel(const float2* __restrict__ strip, float* __restrict__ map, float* __restrict__ pow,
               DopplerArgs a) {
  const int warp = threadIdx.x >> 5, t = threadIdx.x & 31;
  const long task = (long)blockIdx.x * kDopWarps + warp;
  if (task >= (long)a.frames * a.rows) return;
  const int f = (int)(task / a.rows);
  if (a.frame_mask && !a.frame_mask[f]) return;
  const int ri = (int)(task % a.rows);
  const int r = (a.row0 + ri) % a.Np;
  const float2* g = strip + task * a.M;
  float* prow = pow + task * MP;
  float* mrow = map ? map + (a.map_off ? (long)a.map_off[f] : (long)f * a.Np * MP) + (long)r * MP : nullptr;

  if constexpr (MP <= 32) {
    // Direct DFT: lane s computes one bin; g[l] is broadcast by shuffles.
    float2 gl = make_float2(0.f, 0.f);
    if (t < a.M) gl = cscale(g[t], __ldg(a.wl + t));
    float2 acc = make_float2(0.f, 0.f);
    for (int l = 0; l < a.M; ++l) {
      float2 x;
      x.x = __shfl_sync(0xffffffffu, gl.x, l);
      x.y = __shfl_sync(0xffffffffu, gl.y, l);
      float2 w = __ldg(a.tw + ((l * t) & (MP - 1)));
      w.y = -w.y;
      acc = cadd(acc, cmul(x, w));
    }
    if (t < MP) {
      const int c = (t + MP / 2) & (MP - 1);
      const float p = (acc.x * acc.x + acc.y * acc.y) * a.inv_nm;
      prow[c] = p;
      if (mrow) mrow[c] = p;
    }
  } else {
    constexpr int E = MP / 32;
    extern __shared__ float2 smem[];
    float2* sm = smem + warp * smem_elems(MP);
    float2 v[E];
#pragma unroll
    for (int q = 0; q < E; ++q) {
      const int l = t + 32 * q;
      v[q] = (l < a.M) ? cscale(g[l], __ldg(a.wl + l)) : make_float2(0.f, 0.f);
    }
    group_fft<MP, 32, -1>(v, sm, a.tw, t, 0);
#pragma unroll
    for (int q = 0; q < E; ++q) {
      const int s = t + 32 * q;
      const int c = (s + MP / 2) & (MP - 1);
      const float p = (v[q].x * v[q].x + v[q].y * v[q].y) * a.inv_nm;
      prow[c] = p;
      if (mrow) __stcs(mrow + c, p);
    }
  }
}

__global__ void zero_rows_kernel(float* __restrict__ map, int frames, long frame_floats, long z_off,
                                 long z_floats, const long long* __restrict__ map_off) {
  // z_off, z_floats and the frame offsets are multiples of 4 floats (M' >= 16).
  const long per = z_floats / 4;
  const long total = per * frames;
  const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
    const long f = i / per, j = i % per;
    const long base = map_off ? (long)map_off[f] : f * frame_floats;
    __stcs(reinterpret_cast<float4*>(map + base + z_off) + j, z);
  }
}

// ---------------------------------------------------------------- detection
// detect_band_kernel: grid (bands, frames).  Each CTA stages its band of
// scanned rows plus one halo row on each side in shared memory, finds the
// 8-neighbour local maxima (circular in r and s; equal powers broken by the
// smaller map index) and keeps its K strongest as keys
//   (float bits of P) << 32 | ~(flat map index)
// (descending key order = power descending, then index ascending).  The last
// CTA of a frame (atomic ticket, no waiting) merges the bands' keys, writes
// the targets and status, and resets the frame's ticket and counter.
// median_kernel: threshold mode without a given noise level -- the lower
// median of P over the scanned rows (radix select on the float bits).
constexpr int kDetThreads = 256;
constexpr int kBandCap = 1024;          // keys kept per band before compaction

__device__ __forceinline__ float det_value(const float* base, const DetectArgs& a, int ri, int c) {
  const int row = a.compact ? ri : ((a.row0 + ri) & (a.Np - 1));
  return base[((long)row << a.logMp) + c];
}

// Block-wide bitonic sort of buf[0..n) (n a power of two), keys descending.
__device__ void bitonic_desc(uint64_t* buf, int n) {
  for (int k = 2; k <= n; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < n; i += kDetThreads) {
        const int p = i ^ j;
        if (p > i) {
          const uint64_t a = buf[i], b = buf[p];
          const bool desc = (i & k) == 0;
          if (desc ? (a < b) : (a > b)) { buf[i] = b; buf[p] = a; }
        }
      }
      __syncthreads();
    }
  }
}

// Key of the cell at tile row i (1..tr) and column c, or 0.  Fast path: float
// comparisons with the eight neighbours; the map-index tie-break runs only
// when a neighbour has exactly the same power.
__device__ __forceinline__ uint64_t band_key(const float* tile, const DetectArgs& a, int t0, int i, int c,
                                             float eta) {
  const float p = tile[(i << a.logMp) + c];
  if (!(p > 0.f) || (a.mode == OFDM_DETECT_THRESHOLD && !(p >= eta))) return 0;
  const int cm = (c - 1) & (a.Mp - 1), cp = (c + 1) & (a.Mp - 1);
  const float* up = tile + ((i - 1) << a.logMp);
  const float* mid = tile + (i << a.logMp);
  const float* dn = tile + ((i + 1) << a.logMp);
  const float n0 = up[cm], n1 = up[c], n2 = up[cp], n3 = mid[cm], n4 = mid[cp], n5 = dn[cm], n6 = dn[c],
              n7 = dn[cp];
  const bool larger = (n0 > p) | (n1 > p) | (n2 > p) | (n3 > p) | (n4 > p) | (n5 > p) | (n6 > p) | (n7 > p);
  if (larger) return 0;
  const int r = (a.row0 + t0 + i - 1) & (a.Np - 1);
  const uint32_t idx = ((uint32_t)r << a.logMp) + c;
  const bool equal = (n0 == p) | (n1 == p) | (n2 == p) | (n3 == p) | (n4 == p) | (n5 == p) | (n6 == p) | (n7 == p);
  if (equal) {
    const float nb[8] = {n0, n1, n2, n3, n4, n5, n6, n7};
    const int dr[8] = {-1, -1, -1, 0, 0, 1, 1, 1}, dc[8] = {-1, 0, 1, -1, 1, -1, 0, 1};
    for (int k = 0; k < 8; ++k)
      if (nb[k] == p) {
        const uint32_t in_idx = ((uint32_t)((r + dr[k]) & (a.Np - 1)) << a.logMp) + ((c + dc[k]) & (a.Mp - 1));
        if (in_idx < idx) return 0;
      }
  }
  return ((uint64_t)__float_as_uint(p) << 32) | (uint64_t)(~idx);
}

__global__ void __launch_bounds__(kDetThreads)
detect_band_kernel(const float* __restrict__ src, ofdm_target* __restrict__ out, int32_t* __restrict__ n_out,
                   uint32_t* __restrict__ status, uint32_t* __restrict__ wstatus, DetectArgs a) {
  extern __shared__ __align__(16) unsigned char det_smem[];
  __shared__ uint64_t buf[kBandCap];
  __shared__ uint32_t bits[8192 / 32 + 32];
  __shared__ unsigned s_n, s_cnt;
  __shared__ int s_last;
  float* tile = reinterpret_cast<float*>(det_smem);
  const int band = blockIdx.x, f = blockIdx.y;
  if (a.frame_mask && !a.frame_mask[f]) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int K = a.K;
  const int t0 = band * a.band_rows;
  const int tr = min(a.band_rows, a.rows - t0);
  const float* base = src + (long)f * a.frame_stride;
  const float eta = a.mode == OFDM_DETECT_THRESHOLD ? (a.use_fixed_eta ? a.eta_fixed : a.eta[f]) : 0.f;

  // stage rows t0 - 1 .. t0 + tr; rows outside a partial support are zero, a full support wraps
  const int n4 = ((tr + 2) << a.logMp) >> 2;
  for (int v = tid; v < n4; v += kDetThreads) {
    const int idx = v << 2;
    const int i = idx >> a.logMp, c = idx & (a.Mp - 1);
    int rj = t0 - 1 + i;
    float4 val = make_float4(0.f, 0.f, 0.f, 0.f);
    if (a.full) rj &= (a.rows - 1);
    if (rj >= 0 && rj < a.rows) {
      const int row = a.compact ? rj : ((a.row0 + rj) & (a.Np - 1));
      val = *reinterpret_cast<const float4*>(base + ((long)row << a.logMp) + c);
    }
    *reinterpret_cast<float4*>(tile + idx) = val;
  }
  if (tid == 0) { s_n = 0; s_cnt = 0; }
  __syncthreads();

  // scan 1: candidate bits, count, each thread's best key
  const int nt = tr << a.logMp;
  uint64_t best = 0;
  unsigned cnt = 0;
  for (int e0 = 0; e0 < nt; e0 += kDetThreads) {
    const int e = e0 + tid;
    const uint64_t key = e < nt ? band_key(tile, a, t0, 1 + (e >> a.logMp), e & (a.Mp - 1), eta) : 0;
    const unsigned m = __ballot_sync(0xffffffffu, key != 0);
    if (lane == 0) bits[(e0 >> 5) + warp] = m;
    cnt += key ? 1u : 0u;
    best = key > best ? key : best;
  }
  cnt = __reduce_add_sync(0xffffffffu, cnt);
  if (lane == 0) atomicAdd(&s_cnt, cnt);
  buf[tid] = best;
  __syncthreads();
  bitonic_desc(buf, kDetThreads);      // the K-th best per-thread key is a floor for the band's top K
  const uint64_t floor_key = buf[K - 1];
  __syncthreads();
  for (int i = tid; i < kBandCap; i += kDetThreads) buf[i] = 0;
  __syncthreads();
  // scan 2: keys >= floor (only cells with their candidate bit set)
  for (int e0 = 0; e0 < nt; e0 += kDetThreads) {
    const int e = e0 + tid;
    uint64_t key = 0;
    if (e < nt && ((bits[e >> 5] >> (e & 31)) & 1u))
      key = band_key(tile, a, t0, 1 + (e >> a.logMp), e & (a.Mp - 1), eta);
    const bool keep = key != 0 && key >= floor_key;
    const unsigned km = __ballot_sync(0xffffffffu, keep);
    if (km) {
      unsigned wb = 0;
      if (lane == 0) wb = atomicAdd(&s_n, (unsigned)__popc(km));
      wb = __shfl_sync(0xffffffffu, wb, 0);
      const unsigned pos = wb + __popc(km & ((1u << lane) - 1u));
      if (keep && pos < kBandCap) buf[pos] = key;
    }
  }
  __syncthreads();
  // At most K threads have a best key at or above the floor and each scans at
  // most 8192 / kDetThreads = 32 cells, so s_n <= 32 K <= kBandCap.
  int sn = min((int)s_n, kBandCap), sort_n = 32;
  while (sort_n < sn) sort_n <<= 1;
  bitonic_desc(buf, sort_n);
  uint64_t* pk = a.part_keys + ((long)f * a.bands + band) * 32;
  if (tid < 32) pk[tid] = tid < K ? buf[tid] : 0;
  if (tid == 0) atomicAdd(a.counts + f, s_cnt);
  __threadfence();
  __syncthreads();
  if (tid == 0) s_last = atomicAdd(a.tickets + f, 1u) == (unsigned)(a.bands - 1);
  __syncthreads();
  if (!s_last) return;

  // last CTA of the frame: merge the bands
  __threadfence();
  uint64_t* mbuf = reinterpret_cast<uint64_t*>(det_smem);
  const int nk = a.bands * 32;
  int mn = 32;
  while (mn < nk) mn <<= 1;
  const volatile uint64_t* all = a.part_keys + (long)f * a.bands * 32;
  for (int i = tid; i < mn; i += kDetThreads) mbuf[i] = i < nk ? all[i] : 0;
  __syncthreads();
  bitonic_desc(mbuf, mn);
  if (tid < 32) {
    const uint64_t key = lane < K ? mbuf[lane] : 0;
    const bool valid = key != 0;
    const int nv = __popc(__ballot_sync(0xffffffffu, valid));
    const long g = a.out_idx ? (long)a.out_idx[f] : (long)f;  // index into the caller's outputs
    if (valid && out) {
      const uint32_t idx = ~(uint32_t)(key & 0xffffffffu);
      ofdm_target tg;
      tg.r = (int32_t)(idx >> a.logMp);
      tg.s = (int32_t)(idx & (uint32_t)(a.Mp - 1)) - a.Mp / 2;
      tg.power = __uint_as_float((uint32_t)(key >> 32));
      tg.range_m = (float)tg.r * a.dd;
      tg.vel_mps = (float)tg.s * a.dv;
      out[g * K + lane] = tg;
    }
    if (lane == 0) {
      const unsigned total = atomicExch(a.counts + f, 0u);
      uint32_t st = wstatus ? wstatus[f] : 0u;
      if (a.mode == OFDM_DETECT_TOPK && total < (unsigned)K) st |= OFDM_STATUS_FEW_PEAKS;
      if (a.mode == OFDM_DETECT_THRESHOLD && total > (unsigned)K) st |= OFDM_STATUS_OVERFLOW;
      if (status) status[g] = st;
      if (n_out) n_out[g] = nv;
      if (wstatus) wstatus[f] = 0u;  // ready for the next call
      a.tickets[f] = 0u;
    }
  }
}

__global__ void __launch_bounds__(1024) median_kernel(const float* __restrict__ src, DetectArgs a) {
  __shared__ uint32_t hist[256];
  __shared__ uint32_t s_prefix, s_rank;
  const int f = blockIdx.x, tid = threadIdx.x;
  if (a.frame_mask && !a.frame_mask[f]) return;
  const float* base = src + (long)f * a.frame_stride;
  const int n = a.rows << a.logMp;
  if (tid == 0) { s_prefix = 0; s_rank = (uint32_t)(n - 1) / 2; }
  uint32_t mask = 0;
  for (int shift = 24; shift >= 0; shift -= 8) {
    for (int i = tid; i < 256; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    const uint32_t prefix = s_prefix;
    for (int e = tid; e < n; e += blockDim.x) {
      const uint32_t u = __float_as_uint(det_value(base, a, e >> a.logMp, e & (a.Mp - 1)));
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

// ---------------------------------------------------------------- launchers
template <int MP>
static cudaError_t launch_doppler_m(const float2* strip, float* map, float* pow, const DopplerArgs& a,
                                    cudaStream_t s) {
  size_t smem = MP <= 32 ? 0 : (size_t)kDopWarps * smem_elems(MP) * sizeof(float2);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(doppler_kernel<MP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
  }
  const long tasks = (long)a.frames * a.rows;
  const long blocks = (tasks + kDopWarps - 1) / kDopWarps;
  doppler_kernel<MP><<<(unsigned)blocks, 32 * kDopWarps, smem, s>>>(strip, map, pow, a);
  return cudaGetLastError();
}

cudaError_t launch_doppler(int Mp, const float2* strip, float* map, float* pow, const DopplerArgs& a,
                           cudaStream_t s, int* launches) {
  ++*launches;
  switch (Mp) {
    case 16: return launch_doppler_m<16>(strip, map, pow, a, s);
    case 32: return launch_doppler_m<32>(strip, map, pow, a, s);
    case 64: return launch_doppler_m<64>(strip, map, pow, a, s);
    case 128: return launch_doppler_m<128>(strip, map, pow, a, s);
    case 256: return launch_doppler_m<256>(strip, map, pow, a, s);
    case 512: return launch_doppler_m<512>(strip, map, pow, a, s);
    case 1024: return launch_doppler_m<1024>(strip, map, pow, a, s);
    default: --*launches; return cudaErrorInvalidValue;
  }
}

cudaError_t launch_zero_rows(float* map, int frames, int Np, int Mp, int z0, int nz, cudaStream_t s,
                             int* launches, const long long* map_off) {
  if (nz <= 0) return cudaSuccess;
  ++*launches;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const long frame_floats = (long)Np * Mp;
  zero_rows_kernel<<<sms * 4, 256, 0, s>>>(map, frames, frame_floats, (long)z0 * Mp, (long)nz * Mp, map_off);
  return cudaGetLastError();
}

cudaError_t launch_detect(const float* pow, ofdm_target* out, int32_t* n_out, uint32_t* status,
                          uint32_t* wstatus, const DetectArgs& a_in, cudaStream_t s, int* launches) {
  DetectArgs a = a_in;
  detect_bands(a.rows, a.Mp, &a.band_rows, &a.bands);
  if (a.mode == OFDM_DETECT_THRESHOLD && !a.use_fixed_eta) {
    ++*launches;
    median_kernel<<<a.frames, 1024, 0, s>>>(pow, a);
  }
  const size_t tile = (size_t)(a.band_rows + 2) * a.Mp * sizeof(float);
  int mn = 32;
  while (mn < a.bands * 32) mn <<= 1;
  const size_t smem = tile > (size_t)mn * sizeof(uint64_t) ? tile : (size_t)mn * sizeof(uint64_t);
  cudaError_t e = cudaFuncSetAttribute(detect_band_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  ++*launches;
  detect_band_kernel<<<dim3(a.bands, a.frames), kDetThreads, smem, s>>>(pow, out, n_out, status, wstatus, a);
  return cudaGetLastError();
}

}  // namespace ofdm
