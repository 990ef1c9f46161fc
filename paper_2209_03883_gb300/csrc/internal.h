// internal.h -- plan layout and kernel launchers shared by the library's
// translation units (not part of the public ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <nvtx3/nvToolsExt.h>

#include "../../include/ofdm_radar.h"

namespace ofdm {

// Names the host-side span of an entry point for profilers (NVTX range;
// free when no tool is attached).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// Arguments of the column kernel (steps a1-a5 on every OFDM symbol).
struct ColumnArgs {
  int M, L_cp, rows, row0, full;  // support rows; full = rows cover all N bins (circular stencil)
  int frames;
  int zc;       // 1: apply the ZC transform to X
  int rinv;     // r'^{-1} mod N (the ZC transform's output permutation, moved to the input)
  float c0, c1; // range-window stencil: g[r] = c0 h[r] + c1 (h[r-1] + h[r+1])
  float sqrtN;
  const float2* pre;       // [N] pre-chirp exp(i pi r'(k^2 + 2q'k)/N^2)
  const float2* post_conj; // [N] conj of the post factor (-1)^{r'i} exp(i 2 pi r'q' i/N)
  const float2* tw;        // N-point pass twiddles (DIR = +1)
  int post_sign;           // 1: q' = 0, the post factor is (-1)^i (r' odd) and no table is read
  int rprime;              // r'
  float refine_tau;        // recompute precoded cells with |X_p|^2 < tau * mean in double-float; 0 = off
  const float4* pre_df;    // [N] pre-chirp as double-float (re.hi, re.lo, im.hi, im.lo)
  const float4* w_df;      // [N] exp(+2 pi i m / N) as double-float
  unsigned long long* work_ctr;  // monotonic symbol ticket counter (pipelined kernel)
  unsigned long long work_base;  // counter value at the start of this launch
  const long long* frame_off;    // per-frame complex offset of the Y / X rows, or null (f * M * N)
  int pipe_warps;                // pipelined kernel variant: 0 = most warps that fit, 4 = 4 warps per CTA,
                                 // 2 = groups of N / 16 threads, 16 points each (N >= 1024, needs tw_group)
  const float2* tw_group = nullptr;  // N >= 1024: pass twiddles for 16 points per thread, or null
  // Split-FP16 tensor-core form (N = 1024): the 32-point DFT operand tables
  // (hi and lo halves, tc_table_bytes() each) and the 32 x 32 inter-stage
  // twiddles exp(+2 pi i n1 k2 / 1024) / 32.  Null: the FP32 kernels.
  const uint4* tc_b = nullptr;
  const float2* tc_t12 = nullptr;
};

struct ZctArgs {
  int frames, M, rinv, dir;
  float scale;
  const float2* in_tab;   // multiplies the (permuted) input
  const float2* out_tab;  // multiplies the output
  const float2* tw;
};

struct DopplerArgs {
  int N, Np, M, Mp, rows, row0, frames;
  float inv_nm;           // 1 / (N M)
  const float* wl;        // [M] window over l
  const long long* map_off;  // per-frame float offset of the map, or null (f * N' * M')
  const int* frame_mask;     // process only frames with mask != 0, or null (all)
  const float2* tw;       // Mp-point pass twiddles (DIR = +1), or the Mp roots for Mp <= 32
};

struct DetectArgs {
  int Np, Mp, rows, row0, full;   // rows scanned, starting at range bin row0 (circular)
  int logMp;                      // log2(M'); N' and M' are powers of two
  int bit_words;                  // set by the launcher: candidate bit-mask words in shared memory
  int tile_rows;                  // set by the launcher: scanned rows per shared-memory tile
  const int* out_idx;             // per-frame index into out / n_out / status, or null (f)
  const int* frame_mask;          // process only frames with mask != 0, or null (all)
  long frame_stride;              // floats between frames of the input
  int compact;                    // 1: input rows are the support strip; 0: full map rows
  int frames;
  int mode, K;
  int use_fixed_eta;
  float eta_fixed, eta_factor;
  float dd, dv;                   // metres / (m/s) per bin, Eq. (19)
  // workspace (zero-initialised tickets / counts; the last CTA of a frame resets them)
  uint64_t* part_keys;            // [frames][bands][32] best keys of each band
  unsigned* tickets;              // [frames]
  unsigned* counts;               // [frames] candidates found
  float* eta;                     // [frames] threshold from the median pre-pass
  int bands, band_rows;           // set by detect_bands()
  // CFAR mode: guard and training half-widths and alpha(n) for n training cells (host-built table)
  int cfar_guard = 0, cfar_train = 0;
  const float* cfar_alpha = nullptr;
  // optional: the detection launch also zeroes map rows [z0, z0 + nz) of each frame
  float* zmap = nullptr;          // the map, or null (no zeroing)
  const long long* zmap_off = nullptr;  // per-frame float offset of the map, or null (f * zframe)
  long zframe = 0, z_off = 0, z_floats = 0;  // floats per frame, z0 * M', nz * M' (multiples of 4)
};

// Row bands of the detection grid: kDetBandCells cells per CTA.
#ifndef OFDM_DET_BAND_CELLS
#define OFDM_DET_BAND_CELLS 4096
#endif
constexpr int kDetBandCells = OFDM_DET_BAND_CELLS;
// The rows are spread evenly over the fewest bands of at most
// kDetBandCells / M' rows (130 rows at M' = 256: 9 bands of 15 or 10, not 16
// and a last band of 2), so that no CTA carries much more than the others.
inline void detect_bands(int rows, int Mp, int* band_rows, int* bands) {
  int br = kDetBandCells / Mp;
  if (br < 1) br = 1;
  if (br > rows) br = rows;
  const int nb = (rows + br - 1) / br;
  br = (rows + nb - 1) / nb;
  *band_rows = br;
  *bands = (rows + br - 1) / br;
}

// *tickets receives how far the launch advances a.work_ctr (symbols + warps
// for the pipelined kernel, 0 otherwise); the caller adds it to work_base.
struct FpsArgs {
  int N, M, Q, T, rows, iterations, frames, K, max_recover;
  int direct;                       // 1: samples are Y / X at the sampled cells (F is cell-local)
  float invN, invNM, NMoverQ;       // 1/N, 1/(N M), N M / Q
  float median_factor;             // bin threshold = median energy * (-ln pfa) / ln 2
  float dynamic_range, coherence_min;
  float dd, dv;                    // Eq. (19) bin widths
  const float4* w_df;              // exp(+2 pi i m / N), double-float (hi parts used)
  const float2* twQ;               // Q-point pass twiddles
};

struct RefineArgs {
  int N, M, rows, row0, Hc, Mc, frames, K, cap;
  float zthr, inv_nm, dd, dv;
  const float* wl;
  const float2* rootsM;   // exp(-2 pi i m / M), m < M
};

cudaError_t launch_coarse(const float2* strip, unsigned* cpow, float* x, int rows, int M, int frames,
                          const float* w4, const float2* tw, cudaStream_t s, int* launches);
cudaError_t launch_refine(const float2* strip, const float* logits, ofdm_target* out, int32_t* n_out,
                          uint32_t* status, uint32_t* wstatus, int* mask, int* cand, int* ncand, uint64_t* keys,
                          const RefineArgs& a, cudaStream_t s, int* launches);

cudaError_t cnn_forward(const float* th, int bf16, const float* x, int B, int H, int W, float* a1, float* a2,
                        float* z, cudaStream_t s);

// FPS-SFT: sampling (from the strip's taps, or from Y and X when a.direct),
// slice DFTs into the workspace S (fps_workspace_elems float2), decoding.
size_t fps_workspace_elems(int frames, int iterations, int T, int Q);
cudaError_t launch_fps(int Q, const float2* strip, const float2* Y, const float2* X, const int32_t* slices,
                       float2* S, ofdm_target* out, int32_t* n_out, uint32_t* wstatus, const FpsArgs& a,
                       cudaStream_t s, int* launches);

// Range transform on a zero-padded grid N' > N (range_pad.cu).
struct PadArgs {
  int M, L_cp, frames;
  const float* wk;         // [N] window over k
  const float2* twN;       // N-point pass twiddles for N / pad_threads(N') points per thread
  const float2* twP;       // N'-point pass twiddles for N' / pad_threads(N') points per thread
};
int pad_threads(int NP);
cudaError_t launch_range_pad(int N, int NP, const float2* taps, float2* strip, const PadArgs& a, cudaStream_t s,
                             int* launches);

// Doppler grid M' that is not a power of two (doppler_general.cu): the
// windowed Doppler DFT by a mixed-radix FFT (radices 2, 3, 4, 5, 7, 8, 16) or,
// for other M', a P-point then a Q-point DFT, M' = P Q (roots = e^{-2 pi i m / M'});
// detection by bands of support rows whose sorted top-K lists the last CTA
// of each frame merges (a.part_keys holds detect_general_blocks lists of 32
// keys per frame); the detection launch also zeroes the map rows outside the
// support (a.zmap).
constexpr int kMixedMaxPasses = 12;
struct MixedSchedule {
  int n;                       // passes (0: M' has a prime factor above 7)
  int8_t r[kMixedMaxPasses];   // radix of each pass
};
MixedSchedule mixed_schedule(int Mp);
cudaError_t launch_doppler_general(const float2* strip, float* map, float* pow, const DopplerArgs& a,
                                   const float2* roots, cudaStream_t s, int* launches);
int detect_general_blocks(int rows, int Mp);
cudaError_t launch_detect_general(const float* pow, ofdm_target* out, int32_t* n_out, uint32_t* status,
                                  uint32_t* wstatus, const DetectArgs& a, cudaStream_t s, int* launches);

// Transmit side (tx.cu): PAPR and amplifier out-of-band power per symbol.
struct TxArgs {
  int N, M, frames;
  float sat_factor;        // 10^(q/10): amplifier saturation / mean modulus
  const float2* tw;        // LN-point pass twiddles for tx_points_per_thread(LN) points per thread
};
int tx_points_per_thread(int LN);
cudaError_t launch_tx(int LN, const float2* S, float* papr, float* aci, const TxArgs& a, cudaStream_t s,
                      int* launches);

// Tensor-core column kernel (N = 1024, M % 4 == 0, L_cp <= 256, 16-byte
// aligned Y, X and frame offsets; the caller checks these).
cudaError_t launch_column_tc(const float2* Y, const float2* X, float2* strip, uint32_t* wstatus, const ColumnArgs& a,
                             cudaStream_t s, unsigned long long* tickets);
// Host tables of the tensor-core form: `b` receives the hi and lo operand
// images (2 * tc_table_bytes() bytes), `t12` the 1024 inter-stage twiddles.
size_t tc_table_bytes();
void build_tc_tables(unsigned char* b, float2* t12);

cudaError_t launch_column(int N, const float2* Y, const float2* X, float2* strip, uint32_t* wstatus,
                          const ColumnArgs& a, cudaStream_t s, int* launches,
                          unsigned long long* tickets);
cudaError_t launch_zct(int N, const float2* in, float2* out, const ZctArgs& a, cudaStream_t s,
                       int* launches);
cudaError_t launch_doppler(int Mp, const float2* strip, float* map, float* pow, const DopplerArgs& a,
                           cudaStream_t s, int* launches);
cudaError_t launch_zero_rows(float* map, int frames, int Np, int Mp, int z0, int nz, cudaStream_t s,
                             int* launches, const long long* map_off = nullptr);
cudaError_t launch_detect(const float* pow, ofdm_target* out, int32_t* n_out, uint32_t* status,
                          uint32_t* wstatus, const DetectArgs& a, cudaStream_t s, int* launches);
// Doppler stage and top-K detection in one launch (64 <= M' <= 256, compact
// strip; the Doppler and detection arguments carry the same frame mask, if
// any): the power strip is not written.  For M' >= 512 the fused kernel needs
// too many registers per thread and the two kernels were measured faster.
inline bool doppler_detect_fusable(const DetectArgs& a, int Mp) {
  return a.mode == OFDM_DETECT_TOPK && Mp >= 64 && Mp <= 256 && a.compact;   // (CFAR reads its own input rows)
}
cudaError_t launch_doppler_detect(int Mp, const float2* strip, float* map, ofdm_target* out, int32_t* n_out,
                                  uint32_t* status, uint32_t* wstatus, const DetectArgs& a, const DopplerArgs& d,
                                  cudaStream_t s, int* launches);

}  // namespace ofdm
