// doppler_general.cu -- the Doppler stage and detection for a Doppler grid M'
// that is not a power of two (Table I's M = M' = 560 = 2^4 5 7).
//
// Doppler (Eq. (17)): the windowed DFT over the M OFDM symbols of every
// support row of the range profile,
//     D[r, s] = sum_{l < M} (w_l g[r, l]) e^{-2 pi i l s / M'},   P = |D|^2 / (N M),
// by a mixed-radix FFT when M' = 2^a 3^b 5^c 7^d, else as a power-of-two-length
// DFT and an odd-length DFT (M' = P Q).
//
// Detection (Eq. (18)): 8-neighbour local maxima (circular), optionally above
// the global threshold or the CFAR one, ordered by power then map index:
// each CTA takes a band of support rows, keeps its best K and zeroes its
// share of the map rows outside the support; the last CTA of a frame merges
// the band lists.
#include "fft.cuh"
#include "internal.h"
#include "keys.cuh"

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

// ---------------------------------------------------------------- mixed radix
// M' = 2^a 3^b 5^c 7^d (Table I: 560 = 7 x 5 x 16): a Stockham auto-sort
// transform, natural order in and out, with passes of radix 7, 5, 3 and then
// 16, 8, 4, 2.  Pass p (radix R, Ns = product of the earlier radices) takes
// butterfly j < M'/R with k = j mod Ns:
//   a[m] = x[j + m M'/R] w^(m k M'/(Ns R)),  a <- DFT_R(a),
//   y[(j / Ns) Ns R + k + m Ns] = a[m],      w = e^{-2 pi i / M'}.
// One warp per (support row, frame) with two shared-memory row buffers; the
// CTA shares the table of the M' roots.  At M' = 560 this is about 35 real
// operations per point against 4 (P + Q) = 204 for the two-factor form, and
// the operands of the small DFTs stay in registers.
constexpr int kMixWarps = 4;

template <int R, int K>
struct Trig {
  static constexpr float c = (float)cx_cos(2.0 * kPi * K / R);
  static constexpr float s = (float)cx_sin(2.0 * kPi * K / R);
};

// Odd R, X[b] = sum_a v[a] e^{DIR 2 pi i a b / R}: with s_a = v_a + v_{R-a} and
// d_a = v_a - v_{R-a} (a = 1 .. (R-1)/2), X[b] = A_b + DIR i C_b and
// X[R-b] = A_b - DIR i C_b, where A_b = v_0 + sum_a s_a cos(2 pi a b / R) and
// C_b = sum_a d_a sin(2 pi a b / R).
template <int R, int DIR, int B, int... As>
__device__ __forceinline__ void odd_pair(const float2* s, const float2* d, float2 v0, float2* X,
                                         std::integer_sequence<int, As...>) {
  float2 A = v0, C = make_float2(0.f, 0.f);
  ((A.x = __fmaf_rn(Trig<R, ((As + 1) * B) % R>::c, s[As].x, A.x),
    A.y = __fmaf_rn(Trig<R, ((As + 1) * B) % R>::c, s[As].y, A.y),
    C.x = __fmaf_rn(Trig<R, ((As + 1) * B) % R>::s, d[As].x, C.x),
    C.y = __fmaf_rn(Trig<R, ((As + 1) * B) % R>::s, d[As].y, C.y)),
   ...);
  X[B] = make_float2(A.x - DIR * C.y, A.y + DIR * C.x);
  X[R - B] = make_float2(A.x + DIR * C.y, A.y - DIR * C.x);
}
template <int R, int DIR, int... Bs>
__device__ __forceinline__ void odd_all(const float2* s, const float2* d, float2 v0, float2* X,
                                        std::integer_sequence<int, Bs...>) {
  (odd_pair<R, DIR, Bs + 1>(s, d, v0, X, std::make_integer_sequence<int, (R - 1) / 2>{}), ...);
}
template <int R, int DIR>
__device__ __forceinline__ void dft_odd(float2* v) {
  constexpr int H = (R - 1) / 2;
  float2 s[H], d[H], X[R];
  float2 x0 = v[0];
#pragma unroll
  for (int a = 0; a < H; ++a) {
    s[a] = cadd(v[a + 1], v[R - 1 - a]);
    d[a] = csub(v[a + 1], v[R - 1 - a]);
    x0 = cadd(x0, s[a]);
  }
  odd_all<R, DIR>(s, d, v[0], X, std::make_integer_sequence<int, H>{});
  X[0] = x0;
#pragma unroll
  for (int b = 0; b < R; ++b) v[b] = X[b];
}

template <int R>
__device__ __forceinline__ void mixed_pass(const float2* __restrict__ x, float2* __restrict__ y, int L, int Ns,
                                           const float2* __restrict__ roots, int lane) {
  const int nb = L / R, step = L / (Ns * R);
  int jq = lane / Ns, k = lane - (lane / Ns) * Ns;                // j = jq Ns + k, stepped by 32
  const int dq = 32 / Ns, dk = 32 % Ns;
  for (int j = lane; j < nb; j += 32) {
    float2 a[R];
#pragma unroll
    for (int m = 0; m < R; ++m) a[m] = x[j + m * nb];
    if (Ns > 1) {
      const int e = k * step;
#pragma unroll
      for (int m = 1; m < R; ++m) a[m] = cmul(a[m], roots[m * e]);
    }
    if constexpr (R == 3 || R == 5 || R == 7) dft_odd<R, -1>(a);
    else dft_reg<R, -1>(a);
    const int o = j + jq * Ns * (R - 1);
#pragma unroll
    for (int m = 0; m < R; ++m) y[o + m * Ns] = a[m];
    jq += dq;
    k += dk;
    if (k >= Ns) { k -= Ns; ++jq; }
  }
}

__global__ void __launch_bounds__(32 * kMixWarps)
doppler_mixed_kernel(const float2* __restrict__ strip, float* __restrict__ map, float* __restrict__ pow,
                     DopplerArgs d, const float2* __restrict__ roots, MixedSchedule sch) {
  extern __shared__ float2 mx_smem[];
  const int Mp = d.Mp, M = d.M;
  float2* w = mx_smem;                                            // [M'] roots
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float2* b0 = mx_smem + Mp + (size_t)warp * 2 * Mp;
  float2* b1 = b0 + Mp;
  for (int i = threadIdx.x; i < Mp; i += 32 * kMixWarps) w[i] = __ldg(roots + i);
  __syncthreads();
  const int f = blockIdx.y;
  const int ri = blockIdx.x * kMixWarps + warp;
  if (ri >= d.rows) return;                                       // no CTA-wide barrier below
  const float2* g = strip + ((size_t)f * d.rows + ri) * M;
  constexpr int kLd = 8;                                          // loads in flight per lane
  for (int l0 = 0; l0 < Mp; l0 += 32 * kLd) {
    float2 t[kLd];
    float wv[kLd];
#pragma unroll
    for (int u = 0; u < kLd; ++u) {
      const int l = l0 + lane + 32 * u;
      t[u] = l < M ? g[l] : make_float2(0.f, 0.f);
      wv[u] = l < M ? __ldg(d.wl + l) : 0.f;
    }
#pragma unroll
    for (int u = 0; u < kLd; ++u) {
      const int l = l0 + lane + 32 * u;
      if (l < Mp) b0[l] = cscale(t[u], wv[u]);
    }
  }
  __syncwarp();
  float2* x = b0;
  float2* y = b1;
  int Ns = 1;
  for (int p = 0; p < sch.n; ++p) {
    const int R = sch.r[p];
    switch (R) {
      case 2: mixed_pass<2>(x, y, Mp, Ns, w, lane); break;
      case 3: mixed_pass<3>(x, y, Mp, Ns, w, lane); break;
      case 4: mixed_pass<4>(x, y, Mp, Ns, w, lane); break;
      case 5: mixed_pass<5>(x, y, Mp, Ns, w, lane); break;
      case 7: mixed_pass<7>(x, y, Mp, Ns, w, lane); break;
      case 8: mixed_pass<8>(x, y, Mp, Ns, w, lane); break;
      default: mixed_pass<16>(x, y, Mp, Ns, w, lane); break;
    }
    __syncwarp();
    Ns *= R;
    float2* t = x;
    x = y;
    y = t;
  }
  const int row = (d.row0 + ri) % d.Np;
  float* mrow = map ? map + (d.map_off ? (long)d.map_off[f] : (long)f * d.Np * Mp) + (long)row * Mp : nullptr;
  float* prow = pow ? pow + ((size_t)f * d.rows + ri) * Mp : nullptr;
  const int half = Mp / 2;
  for (int c = lane; c < Mp; c += 32) {                           // column c holds bin c - M'/2 (mod M')
    const float2 v = x[c < half ? c + half : c - half];
    const float pw = (v.x * v.x + v.y * v.y) * d.inv_nm;
    if (mrow) __stcs(mrow + c, pw);
    if (prow) prow[c] = pw;
  }
}

// ---------------------------------------------------------------- detection

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

// A band of support rows per CTA (kGBandCells cells, at least one row): the
// rows and a halo row on each side are staged in shared memory (rows off a
// partial support are zero, a full support wraps), every cell is tested
// against its 8 neighbours (circular in s), the candidates go to a shared
// list, and K rounds of a block-wide maximum write the band's best K keys,
// descending, to keys[f][band][0..32).
constexpr int kGBandCells = 4096;
constexpr int kGListCap = kGBandCells / 4 + 64;   // strict local maxima are never 8-adjacent

int detect_general_band_rows(int Mp) { return Mp >= kGBandCells ? 1 : kGBandCells / Mp; }

// A neighbour with the same power and a smaller map index wins the tie (G).
__device__ __noinline__ bool gtie_lost(const float* row, int Mp, int Np, uint32_t r, int c, float p) {
  const uint32_t idx = r * (uint32_t)Mp + (uint32_t)c;
  for (int dr = -1; dr <= 1; ++dr)
    for (int dc = -1; dc <= 1; ++dc) {
      if (dr == 0 && dc == 0) continue;
      const int cn = c + dc < 0 ? Mp - 1 : (c + dc >= Mp ? 0 : c + dc);
      if (row[dr * Mp + cn] == p) {
        const uint32_t rn = (uint32_t)(((int)r + dr + Np) % Np);
        if (rn * (uint32_t)Mp + (uint32_t)cn < idx) return true;
      }
    }
  return false;
}

__global__ void __launch_bounds__(kGThreads)
detect_general_band_kernel(const float* __restrict__ src, DetectArgs a, int blocks, int band_rows,
                           unsigned* __restrict__ counts, ofdm_target* __restrict__ out_t,
                           int32_t* __restrict__ n_out, uint32_t* __restrict__ status,
                           uint32_t* __restrict__ wstatus) {
  extern __shared__ __align__(16) float gtile[];   // (band_rows + 2) rows of M'
  __shared__ uint64_t s_list[kGListCap];
  __shared__ uint64_t s_wk[kGThreads / 32][32];   // each warp's K best, descending
  __shared__ unsigned s_n;
  const int b = blockIdx.x, f = blockIdx.y, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int Mp = a.Mp;
  const int t0 = b * band_rows;
  const int tr = min(band_rows, a.rows - t0);
  const float* base = src + (long)f * a.frame_stride;
  const bool thr = a.mode == OFDM_DETECT_THRESHOLD, cfar = a.mode == OFDM_DETECT_CFAR;
  const float eta = thr ? (a.use_fixed_eta ? a.eta_fixed : a.eta[f]) : 0.f;
  if (tid == 0) s_n = 0;
  const int q4 = Mp >> 2;                            // float4 per row (M' % 4 == 0)
  {
    int i = tid / q4, c4 = tid - (tid / q4) * q4;    // stepped without divisions
    const int di = kGThreads / q4, dc4 = kGThreads % q4;
    for (int v = tid; v < (tr + 2) * q4; v += kGThreads) {
      int rj = t0 - 1 + i;
      if (a.full) rj = rj < 0 ? rj + a.rows : (rj >= a.rows ? rj - a.rows : rj);
      float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
      if (rj >= 0 && rj < a.rows) {
        const int row = a.compact ? rj : (a.row0 + rj) % a.Np;
        x = __ldg(reinterpret_cast<const float4*>(base + (long)row * Mp) + c4);
      }
      reinterpret_cast<float4*>(gtile)[v] = x;
      i += di;
      c4 += dc4;
      if (c4 >= q4) { c4 -= q4; ++i; }
    }
  }
  // The map rows outside the support are zero: this CTA's share of its frame
  // (streaming stores, issued before the scan so that they overlap it).
  if (a.zmap) {
    const long per = a.z_floats >> 2;
    float4* zp = reinterpret_cast<float4*>(a.zmap + (a.zmap_off ? (long)a.zmap_off[f] : (long)f * a.zframe) +
                                           a.z_off);
    for (long j = per * b / blocks + tid; j < per * (b + 1) / blocks; j += kGThreads)
      __stcs(zp + j, make_float4(0.f, 0.f, 0.f, 0.f));
  }
  __syncthreads();
  // Scan: a task is (column c, segment of the band rows); it walks down the
  // segment keeping the 3-wide maxima of the rows above and below in
  // registers.  With few columns the rows are split into segments so that
  // every thread has a task.
  unsigned cnt = 0;
  const int segs = max(1, min(tr, kGThreads / Mp));
  const int seg_len = (tr + segs - 1) / segs;
  const uint32_t Np = (uint32_t)a.Np;
  for (int task = tid; task < segs * Mp; task += kGThreads) {
    const int sg = task / Mp, c = task - sg * Mp;
    const int ia = sg * seg_len, ib = min(tr, ia + seg_len);
    if (ia >= ib) continue;
    const int cm = c == 0 ? Mp - 1 : c - 1, cp = c == Mp - 1 ? 0 : c + 1;
    const float* row = gtile + ia * Mp;               // tile row ia = band row ia - 1
    float up3 = fmaxf(row[c], fmaxf(row[cm], row[cp]));
    row += Mp;
    float ml = row[cm], mc = row[c], mr = row[cp];
    uint32_t r = (uint32_t)((a.row0 + t0 + ia) % a.Np);
    for (int i = ia; i < ib; ++i) {
      row += Mp;                                       // band row i + 1
      const float dl = row[cm], dc = row[c], dr = row[cp];
      const float mid2 = fmaxf(ml, mr);
      // fmaxf skips NaN, so this is "no neighbour compares greater"
      const float nmax = fmaxf(up3, fmaxf(mid2, fmaxf(dc, fmaxf(dl, dr))));
      const float p = mc;
      bool cand = p > 0.f && !(nmax > p) && (!thr || p >= eta);
      if (cand && nmax == p) cand = !gtie_lost(row - Mp, Mp, a.Np, r, c, p);
      if (cand && cfar) cand = gcfar(base, a, t0 + i, c, p);
      if (cand) {
        ++cnt;
        const uint32_t idx = r * (uint32_t)Mp + (uint32_t)c;
        const unsigned pos = atomicAdd(&s_n, 1u);
        if (pos < (unsigned)kGListCap) s_list[pos] = ((uint64_t)__float_as_uint(p) << 32) | (uint64_t)(~idx);
      }
      up3 = fmaxf(mid2, mc);
      ml = dl;
      mc = dc;
      mr = dr;
      r = r + 1 == Np ? 0u : r + 1;
    }
  }
  cnt = __reduce_add_sync(0xffffffffu, cnt);
  if (lane == 0 && cnt) atomicAdd(counts + f, cnt);
  __syncthreads();
  // The band's K best, descending: each warp takes the K best of its slice
  // of the list by repeated warp maxima (keys in registers, no block
  // barriers), then warp 0 merges the eight sorted lists.
  const int n = min((int)s_n, kGListCap);
  constexpr int kPer = (kGListCap + kGThreads - 1) / kGThreads;   // keys per lane
  const int per_w = (n + kGThreads / 32 - 1) / (kGThreads / 32);
  const int j0 = warp * per_w, j1 = min(n, j0 + per_w);
  uint64_t v[kPer];
#pragma unroll
  for (int q = 0; q < kPer; ++q) {
    const int j = j0 + lane + 32 * q;
    v[q] = j < j1 ? s_list[j] : 0ull;
  }
  for (int k = 0; k < a.K; ++k) {
    uint64_t best = v[0];
#pragma unroll
    for (int q = 1; q < kPer; ++q) best = v[q] > best ? v[q] : best;
    const uint64_t m = warp_max_key(best);
    if (lane == 0) s_wk[warp][k] = m;
#pragma unroll
    for (int q = 0; q < kPer; ++q) v[q] = v[q] == m ? 0ull : v[q];   // keys are unique (the map index)
  }
  __syncthreads();
  if (warp == 0) {
    uint64_t* out = a.part_keys + ((size_t)f * blocks + b) * 32;
    int h = 0;
    uint64_t head = lane < kGThreads / 32 ? s_wk[lane][0] : 0ull, key = 0;
    for (int k = 0; k < a.K; ++k) {
      const uint64_t m = warp_max_key(head);
      if (lane == k) key = m;
      if (m != 0 && head == m) { ++h; head = h < a.K ? s_wk[lane][h] : 0ull; }
    }
    out[lane] = lane < a.K ? key : 0ull;
  }

  // The last CTA of the frame (atomic ticket, no waiting) merges the band
  // lists: directly for up to 32 bands, else per group of 32 bands and then
  // the groups (at most 1024 bands: band_rows >= 4 rows of at most 4096).
  __shared__ int s_last;
  __threadfence();
  __syncthreads();
  if (tid == 0) s_last = atomicAdd(a.tickets + f, 1u) == (unsigned)(blocks - 1);
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  const volatile uint64_t* all = a.part_keys + (size_t)f * blocks * 32;
  uint64_t key = 0;
  if (blocks <= 32) {
    if (warp == 0) key = warp_merge_lists(all, blocks, a.K, lane);
  } else {
    const int groups = (blocks + 31) >> 5;
    for (int g = warp; g < groups; g += kGThreads / 32) {
      const uint64_t v = warp_merge_lists(all + ((size_t)g << 10), min(32, blocks - (g << 5)), a.K, lane);
      s_list[(g << 5) + lane] = lane < a.K ? v : 0ull;
    }
    __syncthreads();
    if (warp == 0) key = warp_merge_lists(s_list, groups, a.K, lane);
  }
  if (warp == 0) {
    const bool valid = lane < a.K && key != 0;
    const int nv = __popc(__ballot_sync(0xffffffffu, valid));
    const int oi = a.out_idx ? a.out_idx[f] : f;
    if (valid && out_t) {
      const uint32_t idx = ~(uint32_t)(key & 0xffffffffu);
      ofdm_target t;
      t.r = (int32_t)(idx / (uint32_t)Mp);
      t.s = (int32_t)(idx % (uint32_t)Mp) - Mp / 2;
      t.power = __uint_as_float((uint32_t)(key >> 32));
      t.range_m = (float)t.r * a.dd;
      t.vel_mps = (float)t.s * a.dv;
      out_t[(size_t)oi * a.K + lane] = t;
    }
    if (lane == 0) {
      const unsigned total = atomicExch(counts + f, 0u);
      uint32_t st = wstatus ? wstatus[f] : 0u;
      if (a.mode == OFDM_DETECT_TOPK && total < (unsigned)a.K) st |= OFDM_STATUS_FEW_PEAKS;
      if (a.mode != OFDM_DETECT_TOPK && total > (unsigned)a.K) st |= OFDM_STATUS_OVERFLOW;
      if (status) status[oi] = st;
      if (n_out) n_out[oi] = nv;
      if (wstatus) wstatus[f] = 0u;   // ready for the next call
      a.tickets[f] = 0u;
    }
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

// Radices of the mixed-radix transform (7, 5, 3 first, then 16, 8, 4, 2), or
// n = 0 when M' has a prime factor above 7.
MixedSchedule mixed_schedule(int Mp) {
  MixedSchedule m{};
  int q = Mp;
  for (int p : {7, 5, 3})
    while (q % p == 0 && m.n < kMixedMaxPasses) { m.r[m.n++] = (int8_t)p; q /= p; }
  while (q > 1 && m.n < kMixedMaxPasses) {
    int r = (q % 16 == 0 && q != 32) ? 16 : (q % 8 == 0 ? 8 : (q % 4 == 0 ? 4 : (q % 2 == 0 ? 2 : 0)));
    if (!r) break;
    m.r[m.n++] = (int8_t)r;
    q /= r;
  }
  if (q != 1) m.n = 0;
  return m;
}

cudaError_t launch_doppler_general(const float2* strip, float* map, float* pow, const DopplerArgs& a,
                                   const float2* roots, cudaStream_t s, int* launches) {
  const MixedSchedule sch = mixed_schedule(a.Mp);
  if (sch.n > 0) {
    const size_t smem = (size_t)(1 + 2 * kMixWarps) * a.Mp * sizeof(float2);
    cudaError_t e = cudaFuncSetAttribute(doppler_mixed_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    ++*launches;
    doppler_mixed_kernel<<<dim3((unsigned)((a.rows + kMixWarps - 1) / kMixWarps), (unsigned)a.frames), 32 * kMixWarps,
                           smem, s>>>(strip, map, pow, a, roots, sch);
    return cudaGetLastError();
  }
  int P = 1;
  while (a.Mp % (2 * P) == 0) P *= 2;
  const int Q = a.Mp / P;
  const size_t smem = (size_t)3 * a.Mp * sizeof(float2);
  ++*launches;
  doppler_2factor_kernel<<<dim3((unsigned)a.rows, (unsigned)a.frames), kGThreads, smem, s>>>(strip, map, pow, a, roots,
                                                                                            P, Q);
  return cudaGetLastError();
}

int detect_general_blocks(int rows, int Mp) {
  const int br = detect_general_band_rows(Mp);
  return (rows + br - 1) / br;
}

cudaError_t launch_detect_general(const float* pow, ofdm_target* out, int32_t* n_out, uint32_t* status,
                                  uint32_t* wstatus, const DetectArgs& a, cudaStream_t s, int* launches) {
  const int blocks = detect_general_blocks(a.rows, a.Mp);
  if (a.mode == OFDM_DETECT_THRESHOLD && !a.use_fixed_eta) {
    median_general_kernel<<<a.frames, 1024, 0, s>>>(pow, a);
    ++*launches;
  }
  const int br = detect_general_band_rows(a.Mp);
  const size_t tsm = (size_t)(br + 2) * a.Mp * sizeof(float);
  cudaError_t e = cudaFuncSetAttribute(detect_general_band_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tsm);
  if (e != cudaSuccess) return e;
  detect_general_band_kernel<<<dim3((unsigned)blocks, (unsigned)a.frames), kGThreads, tsm, s>>>(
      pow, a, blocks, br, a.counts, out, n_out, status, wstatus);
  ++*launches;
  return cudaGetLastError();
}

}  // namespace ofdm
