// doppler_detect.cu -- the per-range-row half of the chain (steps a6-a7).
//
// doppler_kernel: one warp per (frame, support row r) at a time: the window
//   over l, the M'-point Doppler DFT  D[s] = sum_l w_l g[r, l] e^{-2 pi i l s / M'}
//   and P = |D|^2 / (N M) (Eq. (17)); column c = s + M'/2 (mod M').  Each row
//   goes to the compact power strip used by detection and, when asked, to the
//   full map.
// zero_rows_kernel: the map rows outside the DFT-CE support are exactly zero
//   (the standalone Doppler step; the full chain has the detection launch
//   write them).
// detect_band_kernel: one CTA per band of rows: 8-neighbour local maxima
//   (circular in r and s), optional threshold eta = -sigma^2 ln(P_fa) with
//   sigma^2 from the lower median (Eq. (18)), top-K by (power desc, map index
//   asc), Eq. (19).
#include <float.h>

#include "fft.cuh"
#include "internal.h"
#include "keys.cuh"

namespace ofdm {

constexpr int kDopWarps = 4;

// Each warp transforms rows task, task + stride, ... (stride = all warps of
// the grid); for M' <= 512 the next row's loads are issued before the
// current row's transform so that their latency is hidden.
template <int MP>
__global__ void __launch_bounds__(32 * kDopWarps)
doppler_kernel(const float2* __restrict__ strip, float* __restrict__ map, float* __restrict__ pow,
               DopplerArgs a) {
  const int warp = threadIdx.x >> 5, t = threadIdx.x & 31;
  const long nt = (long)a.frames * a.rows;
  const long stride = (long)gridDim.x * kDopWarps;
  long task = (long)blockIdx.x * kDopWarps + warp;
  auto map_row = [&](int f, int r) -> float* {
    return map ? map + (a.map_off ? (long)a.map_off[f] : (long)f * a.Np * MP) + (long)r * MP : nullptr;
  };

  if constexpr (MP <= 32) {
    for (; task < nt; task += stride) {
      const int f = (int)(task / a.rows);
      if (a.frame_mask && !a.frame_mask[f]) continue;
      const int r = (a.row0 + (int)(task % a.rows)) % a.Np;
      const float2* g = strip + task * a.M;
      float* prow = pow + task * MP;
      float* mrow = map_row(f, r);
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
    }
  } else {
    constexpr int E = MP / 32;
    constexpr bool PF = E <= 16;
    extern __shared__ float2 smem[];
    float2* sm = smem + warp * smem_elems(MP);
    float w[E];
#pragma unroll
    for (int q = 0; q < E; ++q) w[q] = (t + 32 * q < a.M) ? __ldg(a.wl + t + 32 * q) : 0.f;
    auto load = [&](long tk, float2* d) {
      const float2* g = strip + tk * a.M;
#pragma unroll
      for (int q = 0; q < E; ++q) d[q] = (t + 32 * q < a.M) ? g[t + 32 * q] : make_float2(0.f, 0.f);
    };
    // rows of frames outside the mask are neither loaded nor transformed
    auto wanted = [&](long tk) { return !a.frame_mask || a.frame_mask[tk / a.rows] != 0; };
    float2 cur[E], nxt[PF ? E : 1];
    if (PF && task < nt && wanted(task)) load(task, cur);
    for (; task < nt; task += stride) {
      const long nx = task + stride;
      const bool want = wanted(task);
      if constexpr (PF) {
        if (nx < nt && wanted(nx)) load(nx, nxt);
      } else {
        if (want) load(task, cur);
      }
      const int f = (int)(task / a.rows);
      if (want) {
        const int r = (a.row0 + (int)(task % a.rows)) % a.Np;
        float* prow = pow + task * MP;
        float* mrow = map_row(f, r);
        float2 v[E];
#pragma unroll
        for (int q = 0; q < E; ++q) v[q] = cscale(cur[q], w[q]);
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
      if constexpr (PF) {
#pragma unroll
        for (int q = 0; q < E; ++q) cur[q] = nxt[q];
      }
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
constexpr int kCells = kDetBandCells / kDetThreads;   // cells scanned per thread (16)
static_assert(kCells <= 32 && (kCells & (kCells - 1)) == 0, "one candidate bit per cell");
constexpr int kBandCap = 1024;          // keys kept per band before compaction

__device__ __forceinline__ float det_value(const float* base, const DetectArgs& a, int ri, int c) {
  const int row = a.compact ? ri : ((a.row0 + ri) & (a.Np - 1));
  return base[((long)row << a.logMp) + c];
}

// CFAR test of the local maximum at input row ri (support-row index), column
// c, power p: alpha(n) times the mean of the n training cells -- within
// guard + train rows and columns, outside the guard square, on support rows
// (circular when the support is the whole map) -- read from the detection's
// input rows `base`.
__device__ __noinline__ bool cfar_pass(const float* __restrict__ base, const DetectArgs& a, int ri, int c, float p) {
  const int g = a.cfar_guard, w = g + a.cfar_train, Mp = a.Mp;
  float sum = 0.f;
  int n = 0;
  for (int dr = -w; dr <= w; ++dr) {
    int rj = ri + dr;
    if (a.full) rj &= (a.rows - 1);
    else if (rj < 0 || rj >= a.rows) continue;   // off the support: zero by construction, not noise
    const float* rp = base + ((long)(a.compact ? rj : ((a.row0 + rj) & (a.Np - 1))) << a.logMp);
    const bool in_guard_rows = dr >= -g && dr <= g;
    for (int dc = -w; dc <= w; ++dc) {
      if (in_guard_rows && dc >= -g && dc <= g) continue;
      sum += __ldg(rp + ((c + dc) & (Mp - 1)));
      ++n;
    }
  }
  return n > 0 && p >= a.cfar_alpha[n] * (sum / (float)n);
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

// A local maximum with an 8-neighbour of exactly the same power keeps its
// place only if its flat map index is the smaller one (the order of the
// output).  `ti` is the cell's tile row, r its map row.  Kept out of line:
// the scan calls it only for cells that have such a neighbour.
__device__ __noinline__ bool tie_lost(const float* tile, int logMp, int Np, int r, int ti, int c, float p) {
  const int Mp = 1 << logMp;
  const uint32_t idx = ((uint32_t)r << logMp) + (uint32_t)c;
  for (int dr = -1; dr <= 1; ++dr)
    for (int dc = -1; dc <= 1; ++dc) {
      if (dr == 0 && dc == 0) continue;
      const int cc = (c + dc) & (Mp - 1);
      if (tile[((ti + dr) << logMp) + cc] == p) {
        const uint32_t nidx = ((uint32_t)((r + dr) & (Np - 1)) << logMp) + (uint32_t)cc;
        if (nidx < idx) return true;
      }
    }
  return false;
}

// Warp-wide bitonic sort of one key per lane, descending (lane 0 the largest).
__device__ __forceinline__ uint64_t warp_sort_desc(uint64_t v, int lane) {
#pragma unroll
  for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
      const uint64_t o = __shfl_xor_sync(0xffffffffu, v, j);
      const bool keep_max = ((lane & j) == 0) == ((lane & k) == 0);
      v = keep_max ? (v > o ? v : o) : (v < o ? v : o);
    }
  }
  return v;
}

// LOGC = log2 of the columns each thread scans: 0 for M' <= 256, 1 for 512,
// 2 for 1024 (the band always holds kDetBandCells / M' rows, kCells cells
// per thread).
// Everything after the band's power rows are in `tile` (tile row i = band row
// i - 1; this thread's own writes to it complete): the zero map rows, the
// scan, the floor, the band's top K and the last CTA's merge.  Shared by the
// detection kernel (which stages the rows from the power strip) and the fused
// Doppler + detection kernel (which computes them).
template <int LOGC, bool CFAR = false>
__device__ __forceinline__ void band_detect(float* tile, ofdm_target* __restrict__ out, int32_t* __restrict__ n_out,
                                            uint32_t* __restrict__ status, uint32_t* __restrict__ wstatus,
                                            const DetectArgs& a, int band, int f, int t0, int tr,
                                            const float* __restrict__ base) {
  constexpr int C = 1 << LOGC, NR = kCells >> LOGC;
  __shared__ uint64_t buf[kBandCap];
  __shared__ unsigned s_n, s_cnt;
  __shared__ uint64_t s_floor;
  __shared__ int s_last;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int K = a.K, Mp = a.Mp, logMp = a.logMp;
  const bool thr = a.mode == OFDM_DETECT_THRESHOLD;
  const float eta = thr ? (a.use_fixed_eta ? a.eta_fixed : a.eta[f]) : 0.f;
  if (tid == 0) { s_n = 0; s_cnt = 0; }

  // The map rows outside the support are zero: this CTA's share of its
  // frame, two streaming stores per scanned row and the rest after the scan.
  float4* zp = nullptr;
  long zj = 0, zj1 = 0;
  if (a.zmap) {
    const long per = a.z_floats >> 2;
    zj = per * band / a.bands + tid;
    zj1 = per * (band + 1) / a.bands;
    zp = reinterpret_cast<float4*>(a.zmap + (a.zmap_off ? (long)a.zmap_off[f] : (long)f * a.zframe) + a.z_off);
  }
  const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
  __syncthreads();

  // Scan: each thread walks down C columns c0 + 256 q over NR band rows from
  // i0, keeping the 3-wide maxima of the rows above and below in registers.
  // Bit q NR + k of `mine` marks a local maximum at band row i0 + k.  Rows at
  // or past tr read tile rows that were not staged and are masked out.
  const int c0 = LOGC == 0 ? (tid & (Mp - 1)) : tid;
  const int i0 = LOGC == 0 ? (tid >> logMp) * NR : 0;
  const uint32_t rbase = (uint32_t)(a.row0 + t0);
  uint32_t mine = 0;
  unsigned cnt = 0;
  uint64_t best = 0;
#pragma unroll
  for (int q = 0; q < C; ++q) {
    const int c = c0 + (q << 8);
    const int cm = (c - 1) & (Mp - 1), cp = (c + 1) & (Mp - 1);
    const float* row = tile + (i0 << logMp);          // tile row i0 = band row i0 - 1
    float up3 = fmaxf(row[c], fmaxf(row[cm], row[cp]));
    row += Mp;
    float ml = row[cm], mc = row[c], mr = row[cp];
#pragma unroll 8
    for (int k = 0; k < NR; ++k) {
      const int i = i0 + k;
      row += Mp;                                      // band row i + 1
      const float dl = row[cm], dc = row[c], dr = row[cp];
      const float mid2 = fmaxf(ml, mr);
      const float nmax = fmaxf(up3, fmaxf(mid2, fmaxf(dc, fmaxf(dl, dr))));
      const float p = mc;
      // fmaxf skips NaN, so this is "no neighbour compares greater"
      bool cand = i < tr && p > 0.f && !(nmax > p) && (!thr || p >= eta) &&
                  (!CFAR || cfar_pass(base, a, t0 + i, c, p));   // CFAR: base holds the frame's input rows
      const uint32_t r = (rbase + (uint32_t)i) & (uint32_t)(a.Np - 1);
      if (cand && nmax == p) cand = !tie_lost(tile, logMp, a.Np, (int)r, i + 1, c, p);
      const uint64_t key =
          cand ? ((uint64_t)__float_as_uint(p) << 32) | (uint64_t)(~((r << logMp) + (uint32_t)c)) : 0ull;
      best = key > best ? key : best;
      mine |= (uint32_t)cand << (q * NR + k);
      cnt += cand ? 1u : 0u;
      up3 = fmaxf(mid2, mc);
      ml = dl; mc = dc; mr = dr;
      if (zj < zj1) { __stcs(zp + zj, zero4); zj += kDetThreads; }
      if (zj < zj1) { __stcs(zp + zj, zero4); zj += kDetThreads; }
    }
  }
  for (; zj < zj1; zj += kDetThreads) __stcs(zp + zj, zero4);
  cnt = __reduce_add_sync(0xffffffffu, cnt);
  if (lane == 0) atomicAdd(&s_cnt, cnt);

  // Floor = the K-th best of the 256 per-thread best keys: each warp sorts its
  // 32, warp 0 merges the eight sorted lists for K steps.  Every key of the
  // band's top K is at or above it, and at most K threads hold keys there.
  if (K <= 8) {  // the warp's K best, largest first, by repeated maximum
    uint64_t v = best;
    for (int r = 0; r < K; ++r) {
      const uint64_t m = warp_max_key(v);
      if (lane == 0) buf[(warp << 5) + r] = m;
      if (v == m) v = 0;
    }
  } else {
    buf[tid] = warp_sort_desc(best, lane);
  }
  __syncthreads();
  if (warp == 0) {  // 0 when fewer than K threads found a maximum
    const uint64_t m = warp_merge_lists(buf, kDetThreads / 32, K, lane);
    if (lane == K - 1) s_floor = m;
  }
  __syncthreads();
  const uint64_t floor_key = s_floor;
  // keys at or above the floor (at most kCells K <= kBandCap)
  if (best != 0 && best >= floor_key) {
    for (uint32_t m = mine; m; m &= m - 1) {
      const int b = __ffs(m) - 1;
      const int q = b / NR, i = i0 + (b % NR), c = c0 + (q << 8);
      const float p = tile[((i + 1) << logMp) + c];
      const uint32_t r = (rbase + (uint32_t)i) & (uint32_t)(a.Np - 1);
      const uint64_t key = ((uint64_t)__float_as_uint(p) << 32) | (uint64_t)(~((r << logMp) + (uint32_t)c));
      if (key >= floor_key) {
        const unsigned pos = atomicAdd(&s_n, 1u);
        if (pos < (unsigned)kBandCap) buf[pos] = key;
      }
    }
  }
  __syncthreads();
  const int sn = min((int)s_n, kBandCap);
  uint64_t* pk = a.part_keys + ((long)f * a.bands + band) * 32;
  if (sn <= 32) {
    if (warp == 0) {
      const uint64_t v = warp_sort_desc(lane < sn ? buf[lane] : 0, lane);
      pk[lane] = lane < K ? v : 0;
    }
  } else {
    int sort_n = 64;
    while (sort_n < sn) sort_n <<= 1;
    for (int i = sn + tid; i < sort_n; i += kDetThreads) buf[i] = 0;
    __syncthreads();
    bitonic_desc(buf, sort_n);
    if (tid < 32) pk[tid] = tid < K ? buf[tid] : 0;
  }
  if (tid == 0) atomicAdd(a.counts + f, s_cnt);
  __threadfence();
  __syncthreads();
  if (tid == 0) s_last = atomicAdd(a.tickets + f, 1u) == (unsigned)(a.bands - 1);
  __syncthreads();
  if (!s_last) return;

  // last CTA of the frame: merge the bands' sorted top-K lists (stride 32),
  // directly for up to 32 bands, else per group of 32 bands and then the groups
  __threadfence();
  const volatile uint64_t* all = a.part_keys + (long)f * a.bands * 32;
  uint64_t key = 0;
  if (a.bands <= 32) {
    for (int i = tid; i < (a.bands << 5); i += kDetThreads) buf[i] = all[i];
    __syncthreads();
    if (warp == 0) key = warp_merge_lists(buf, a.bands, K, lane);
  } else {
    const int groups = (a.bands + 31) >> 5;             // at most 32 (bands <= 1024)
    for (int g = warp; g < groups; g += kDetThreads / 32) {
      const uint64_t v = warp_merge_lists(all + ((long)g << 10), min(32, a.bands - (g << 5)), K, lane);
      buf[(g << 5) + lane] = lane < K ? v : 0;
    }
    __syncthreads();
    if (warp == 0) key = warp_merge_lists(buf, groups, K, lane);
  }
  if (warp == 0) {
    const bool valid = lane < K && key != 0;
    const int nv = __popc(__ballot_sync(0xffffffffu, valid));
    const long g = a.out_idx ? (long)a.out_idx[f] : (long)f;  // index into the caller's outputs
    if (valid && out) {
      const uint32_t idx = ~(uint32_t)(key & 0xffffffffu);
      ofdm_target tg;
      tg.r = (int32_t)(idx >> logMp);
      tg.s = (int32_t)(idx & (uint32_t)(Mp - 1)) - Mp / 2;
      tg.power = __uint_as_float((uint32_t)(key >> 32));
      tg.range_m = (float)tg.r * a.dd;
      tg.vel_mps = (float)tg.s * a.dv;
      out[g * K + lane] = tg;
    }
    if (lane == 0) {
      const unsigned total = atomicExch(a.counts + f, 0u);
      uint32_t st = wstatus ? wstatus[f] : 0u;
      if (a.mode == OFDM_DETECT_TOPK && total < (unsigned)K) st |= OFDM_STATUS_FEW_PEAKS;
      if (a.mode != OFDM_DETECT_TOPK && total > (unsigned)K) st |= OFDM_STATUS_OVERFLOW;
      if (status) status[g] = st;
      if (n_out) n_out[g] = nv;
      if (wstatus) wstatus[f] = 0u;  // ready for the next call
      a.tickets[f] = 0u;
    }
  }
}


template <int LOGC, bool CFAR>
__global__ void __launch_bounds__(kDetThreads)
detect_band_kernel(const float* __restrict__ src, ofdm_target* __restrict__ out, int32_t* __restrict__ n_out,
                   uint32_t* __restrict__ status, uint32_t* __restrict__ wstatus, DetectArgs a) {
  extern __shared__ __align__(16) unsigned char det_smem[];
  float* tile = reinterpret_cast<float*>(det_smem);  // (kDetBandCells / M' + 2) rows of M'
  const int band = blockIdx.x, f = blockIdx.y;
  if (a.frame_mask && !a.frame_mask[f]) return;
  const int tid = threadIdx.x;
  const int Mp = a.Mp, logMp = a.logMp;
  const int t0 = band * a.band_rows;
  const int tr = min(a.band_rows, a.rows - t0);
  const float* base = src + (long)f * a.frame_stride;

  // stage rows t0 - 1 .. t0 + tr; rows outside a partial support are zero, a full support wraps
  const int n4 = ((tr + 2) << logMp) >> 2;
  for (int v = tid; v < n4; v += kDetThreads) {
    const int idx = v << 2;
    const int i = idx >> logMp, c = idx & (Mp - 1);
    int rj = t0 - 1 + i;
    if (a.full) rj &= (a.rows - 1);
    if (rj >= 0 && rj < a.rows) {
      const int row = a.compact ? rj : ((a.row0 + rj) & (a.Np - 1));
      const unsigned d = (unsigned)__cvta_generic_to_shared(tile + idx);
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(base + ((long)row << logMp) + c)
                   : "memory");
    } else {
      *reinterpret_cast<float4*>(tile + idx) = make_float4(0.f, 0.f, 0.f, 0.f);
    }
  }
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  asm volatile("cp.async.wait_all;\n" ::: "memory");
  band_detect<LOGC, CFAR>(tile, out, n_out, status, wstatus, a, band, f, t0, tr, base);
}

// Fused Doppler stage and detection (top-K mode, 64 <= M' <= 256; frames
// outside an optional mask are skipped): each CTA computes
// the M'-point Doppler transforms of its band's support rows and the two halo
// rows (the neighbouring bands compute those too) straight into its tile,
// writes its own rows to the map, and detects.  Same arithmetic as
// doppler_kernel; the power strip is not written.
template <int MP>
__global__ void __launch_bounds__(kDetThreads)
doppler_band_kernel(const float2* __restrict__ strip, float* __restrict__ map, ofdm_target* __restrict__ out,
                    int32_t* __restrict__ n_out, uint32_t* __restrict__ status, uint32_t* __restrict__ wstatus,
                    DetectArgs a, DopplerArgs d) {
  constexpr int LOGC = MP <= 256 ? 0 : (MP == 512 ? 1 : 2);
  constexpr int E = MP / 32;
  constexpr int TILE = (kDetBandCells / MP + 2) * MP;   // floats
  extern __shared__ __align__(16) unsigned char det_smem[];
  float* tile = reinterpret_cast<float*>(det_smem);
  const int band = blockIdx.x, f = blockIdx.y;
  if (a.frame_mask && !a.frame_mask[f]) return;   // the whole CTA, before any barrier
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  float2* sm = reinterpret_cast<float2*>(det_smem + (size_t)TILE * sizeof(float)) + warp * smem_elems(MP);
  const int t0 = band * a.band_rows;
  const int tr = min(a.band_rows, a.rows - t0);
  float w[E];
#pragma unroll
  for (int q = 0; q < E; ++q) w[q] = (lane + 32 * q < d.M) ? __ldg(d.wl + lane + 32 * q) : 0.f;
  float* fmap = map ? map + (d.map_off ? (long)d.map_off[f] : (long)f * d.Np * MP) : nullptr;
  for (int i = warp; i < tr + 2; i += kDetThreads / 32) {   // tile row i = band row i - 1
    float* trow = tile + i * MP;
    int rj = t0 - 1 + i;
    if (a.full) rj &= (a.rows - 1);
    if (rj < 0 || rj >= a.rows) {
#pragma unroll
      for (int q = 0; q < E; ++q) trow[lane + 32 * q] = 0.f;
      continue;
    }
    const float2* g = strip + ((long)f * a.rows + rj) * d.M;
    float2 v[E];
#pragma unroll
    for (int q = 0; q < E; ++q)
      v[q] = (lane + 32 * q < d.M) ? cscale(g[lane + 32 * q], w[q]) : make_float2(0.f, 0.f);
    group_fft<MP, 32, -1>(v, sm, d.tw, lane, 0);
    float* mrow = (fmap && i >= 1 && i <= tr) ? fmap + (long)((d.row0 + rj) % d.Np) * MP : nullptr;
#pragma unroll
    for (int q = 0; q < E; ++q) {
      const int c = (lane + 32 * q + MP / 2) & (MP - 1);
      const float p = (v[q].x * v[q].x + v[q].y * v[q].y) * d.inv_nm;
      trow[c] = p;
      if (mrow) __stcs(mrow + c, p);
    }
  }
  band_detect<LOGC, false>(tile, out, n_out, status, wstatus, a, band, f, t0, tr, nullptr);
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
  // One wave of CTAs, each warp taking about the same number of rows.
  static int per_sm = 0, sms = 0;
  if (!per_sm) {
    int dev = 0, n = 0, occ = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, doppler_kernel<MP>, 32 * kDopWarps, smem);
    if (e != cudaSuccess) return e;
    sms = n;
    per_sm = occ > 0 ? occ : 1;
  }
  const long tasks = (long)a.frames * a.rows;
  const long slots = (long)sms * per_sm * kDopWarps;
  const long rows_per_warp = (tasks + slots - 1) / slots;
  const long blocks = (tasks + kDopWarps * rows_per_warp - 1) / (kDopWarps * rows_per_warp);
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
  // the scan reads up to kDetBandCells / M' + 2 tile rows whatever the band's height
  const int full_rows = kDetBandCells / a.Mp > 1 ? kDetBandCells / a.Mp : 1;
  const size_t tile = (size_t)(full_rows + 2) * a.Mp * sizeof(float);
  const size_t smem = tile;
  if (a.logMp > 10 || a.bands > 1024) return cudaErrorInvalidValue;
  const bool cfar = a.mode == OFDM_DETECT_CFAR;
  auto kern = a.logMp <= 8 ? (cfar ? detect_band_kernel<0, true> : detect_band_kernel<0, false>)
            : a.logMp == 9 ? (cfar ? detect_band_kernel<1, true> : detect_band_kernel<1, false>)
                           : (cfar ? detect_band_kernel<2, true> : detect_band_kernel<2, false>);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  ++*launches;
  kern<<<dim3(a.bands, a.frames), kDetThreads, smem, s>>>(pow, out, n_out, status, wstatus, a);
  return cudaGetLastError();
}

template <int MP>
static cudaError_t launch_doppler_band_m(const float2* strip, float* map, ofdm_target* out, int32_t* n_out,
                                        uint32_t* status, uint32_t* wstatus, const DetectArgs& a,
                                        const DopplerArgs& d, cudaStream_t s) {
  const size_t smem = (size_t)(kDetBandCells / MP + 2) * MP * sizeof(float) +
                      (size_t)(kDetThreads / 32) * smem_elems(MP) * sizeof(float2);
  cudaError_t e = cudaFuncSetAttribute(doppler_band_kernel<MP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  doppler_band_kernel<MP><<<dim3(a.bands, a.frames), kDetThreads, smem, s>>>(strip, map, out, n_out, status,
                                                                              wstatus, a, d);
  return cudaGetLastError();
}

cudaError_t launch_doppler_detect(int Mp, const float2* strip, float* map, ofdm_target* out, int32_t* n_out,
                                  uint32_t* status, uint32_t* wstatus, const DetectArgs& a_in, const DopplerArgs& d,
                                  cudaStream_t s, int* launches) {
  DetectArgs a = a_in;
  detect_bands(a.rows, a.Mp, &a.band_rows, &a.bands);
  if (a.mode != OFDM_DETECT_TOPK || a.frame_mask != d.frame_mask || a.bands > 1024 || !a.compact)
    return cudaErrorInvalidValue;
  ++*launches;
  switch (Mp) {
    case 64: return launch_doppler_band_m<64>(strip, map, out, n_out, status, wstatus, a, d, s);
    case 128: return launch_doppler_band_m<128>(strip, map, out, n_out, status, wstatus, a, d, s);
    case 256: return launch_doppler_band_m<256>(strip, map, out, n_out, status, wstatus, a, d, s);
    default: --*launches; return cudaErrorInvalidValue;
  }
}

}  // namespace ofdm
