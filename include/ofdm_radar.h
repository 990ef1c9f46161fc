/*
 * ofdm_radar.h -- C ABI of the GB300 OFDM monostatic radar receive chain.
 *
 * The chain follows Delamou, Noubir, Dang, Amhoud, "An Efficient OFDM-Based
 * Monostatic Radar Design for Multitarget Detection" (arXiv 2209.03883):
 * the radar knows the transmitted grid and receives its echo (Sec. II-A), so
 * every call takes the received grid Y and the known transmit grid X and
 * returns the range-Doppler map and the detected targets.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Grids are complex64 (interleaved re, im), laid out [frame][l][k]: for each
 *   frame, M OFDM symbols l of N subcarriers k each, k contiguous.
 * - Unless a function says "host", every pointer is a DEVICE pointer owned by
 *   the caller; the plan owns only its tables and workspace.
 * - Device grids (Y, X, transmit grids), maps and range-profile strips must
 *   start on a 16-byte boundary (cudaMalloc and PyTorch allocations do): they
 *   are moved in 16-byte pieces.  A misaligned one is rejected with
 *   OFDM_ERR_INVALID_ARG; so is a batch frame whose yx_offset is odd.
 * - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *   Calls are asynchronous on it; no output is valid before the caller syncs.
 * - Return value: OFDM_OK (0) or a negative OFDM_ERR_* code.  Invalid sizes
 *   or pointers are rejected before anything is launched.
 * - No entry point allocates device memory except ofdm_radar_plan_create,
 *   ofdm_radar_learned_prepare, the *_host helpers and the batch creation,
 *   and, on their first use, the workspace of ofdm_fps_sft and the twiddle
 *   table of ofdm_tx_amplifier.
 * - Per-frame `status` words carry OFDM_STATUS_* bits.
 */
#ifndef OFDM_RADAR_H
#define OFDM_RADAR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct { float re, im; } ofdm_c32;

enum {
  OFDM_OK = 0,
  OFDM_ERR_INVALID_ARG = -1,      /* NULL plan/pointer, bad enum, frames out of range */
  OFDM_ERR_UNSUPPORTED_SIZE = -2, /* N, M, padding or L_cp outside what is built */
  OFDM_ERR_CUDA = -3,             /* a CUDA runtime call failed (message via strerror) */
  OFDM_ERR_TIMEOUT = -4,          /* a bounded device wait ran out */
  OFDM_ERR_NO_MEMORY = -5         /* plan workspace allocation failed */
};

enum { OFDM_WINDOW_RECT = 0, OFDM_WINDOW_HANN = 1, OFDM_WINDOW_HAMMING = 2 };
/* Detection (Eq. (18)): the max_targets strongest 8-neighbour local maxima
 * (TOPK), those at or above the global threshold eta = -sigma^2 ln P_fa
 * (THRESHOLD), or those at or above a locally estimated threshold (CFAR:
 * alpha(n) times the mean of the n training cells around the cell, within
 * cfar_guard + cfar_train rows and columns but outside the guard square, on
 * support rows; alpha(n) = n (P_fa^(-1/n) - 1) gives P_fa exactly for
 * exponential noise). */
enum { OFDM_DETECT_TOPK = 0, OFDM_DETECT_THRESHOLD = 1, OFDM_DETECT_CFAR = 2 };
/* Arithmetic of the two N-point DFTs of the column stage (the ZC transform
 * and DFT-CE's inverse DFT):
 *   OFDM_PREC_FP32        FP32 FFTs on the CUDA cores (any supported size);
 *   OFDM_PREC_SPLIT_BF16  not built: BF16's 8-bit significand needs three
 *                         pieces per operand (six products) for FP32-level
 *                         accuracy, twice the products of split FP16;
 *   OFDM_PREC_SPLIT_FP16  32-point DFT matrix products on the tensor cores
 *                         with FP16 hi + lo operands (three products, FP32
 *                         accumulation; about 2^-21 relative).  N = 1024,
 *                         M a multiple of 4, L_cp <= 256.  Everything after
 *                         the column stage is the FP32 path's. */
enum { OFDM_PREC_FP32 = 0, OFDM_PREC_SPLIT_BF16 = 1, OFDM_PREC_SPLIT_FP16 = 2 };

enum {
  OFDM_STATUS_ZERO_X = 1u,     /* a precoded transmit cell was exactly 0; its F was set to 0 */
  OFDM_STATUS_NONFINITE = 2u,  /* a non-finite value reached the range profile */
  OFDM_STATUS_OVERFLOW = 4u,   /* threshold mode: more targets than max_targets */
  OFDM_STATUS_FEW_PEAKS = 8u,  /* top-K mode: fewer than max_targets local maxima */
  OFDM_STATUS_UNREFINED = 32u, /* an OFDM symbol had more ill-conditioned precoded cells than are
                                  recomputed in double-float (64); the rest kept FP32 rounding */
  OFDM_STATUS_TIMEOUT = 64u    /* a bounded wait inside a kernel ran out (the split-FP16 column kernel's
                                  copy and tensor-core completions): this frame's outputs are invalid */
};

/* Parameters of one plan.  ofdm_radar_default_params fills the paper's
 * Table I physical constants and the defaults noted here. */
typedef struct {
  int32_t N, M;          /* subcarriers, OFDM symbols; powers of two, N in [64, 4096], M in [16, 1024] */
  int32_t N_pad, M_pad;  /* N', M' of Eq. (17); 0 -> N, M.  N' = N, 2N, 4N or 8N (<= 4096), M' a power of 2 >= M */
  int32_t L_cp;          /* DFT-CE taps kept (Eq. (21)), 1..N; L_cp == N is plain LS estimation */
  int32_t n_cp;          /* physical CP length for T_s in Eq. (19); 0 -> L_cp */
  int32_t zc_root;       /* ZC root r' of Sec. III-B (odd, so coprime to N^2); 0 -> no precoding */
  int32_t zc_q;          /* ZC shift q' (default 0) */
  int32_t x_is_precoded; /* 1 -> X already holds the precoded grid Z_m A / sqrt(N) */
  int32_t window;        /* OFDM_WINDOW_*, periodic, applied in both dimensions (Eq. (17)) */
  int32_t detect_mode;   /* OFDM_DETECT_* */
  int32_t max_targets;   /* 1..32: K of top-K mode, or the cap of threshold mode */
  int32_t max_frames;    /* workspace capacity: frames per call, >= 1 */
  int32_t precision;     /* OFDM_PREC_*; OFDM_PREC_FP32 is the plain FP32 FFT path */
  float pfa;             /* false-alarm probability of Eq. (18), default 1e-2 */
  float noise_var;       /* per-cell noise power of the map; <= 0 -> estimate from the map */
  double fc_hz, df_hz;   /* carrier and subcarrier spacing (Table I: 77 GHz, 240 kHz) */
  int32_t cfar_guard;    /* OFDM_DETECT_CFAR: guard cells on each side of the cell (default 1) */
  int32_t cfar_train;    /* OFDM_DETECT_CFAR: training cells beyond the guard on each side (default 4);
                            guard + train <= 8 */
} ofdm_radar_params;

/* One detection.  r = range bin 0..N'-1, s = Doppler bin -M'/2..M'/2-1,
 * power = P at that cell, range_m / vel_mps from Eq. (19). */
typedef struct { int32_t r, s; float power, range_m, vel_mps; } ofdm_target;

typedef struct ofdm_radar_plan ofdm_radar_plan;

/* Fill *p with defaults: window Hann, top-K detection, 8 targets, zc_root 1,
 * pfa 1e-2, fc 77 GHz, df 240 kHz, max_frames 1.  Sizes are left 0. */
void ofdm_radar_default_params(ofdm_radar_params* p);

/* Validate *p, build the FP64-derived tables (ZC chirps, twiddles, windows)
 * and allocate the workspace for max_frames frames on the CURRENT device.
 * On success *out owns them; release with ofdm_radar_plan_destroy. */
int ofdm_radar_plan_create(const ofdm_radar_params* p, ofdm_radar_plan** out);

/* Free the plan's device memory (after the caller's work on it finished). */
void ofdm_radar_plan_destroy(ofdm_radar_plan* plan);

/* Number of range rows that can be non-zero (the DFT-CE support of Eqs.
 * (17), (21)) and, if rows != NULL, their range bins in workspace order. */
int ofdm_radar_support_rows(const ofdm_radar_plan* plan, int32_t* rows);

/* Whole receive chain on `frames` frames (Sec. II-B.2, III-A, III-B):
 * ZC precoding of X, F = Y / X_p (Eq. (16)), DFT-CE (Eqs. (20)-(22)), the
 * windowed periodogram (Eq. (17)), detection (Eq. (18)) and the estimates of
 * Eq. (19).
 *   Y, X         [frames][M][N] complex64 (X = QAM grid, or X_p if x_is_precoded)
 *   out_map      [frames][N'][M'] float32, column c holds Doppler bin c - M'/2; may be NULL
 *   out_targets  [frames][max_targets]; may be NULL
 *   n_targets    [frames] number of valid entries of out_targets; may be NULL
 *   status       [frames] OFDM_STATUS_* bits; may be NULL
 * 1 <= frames <= max_frames. */
int ofdm_radar_process(ofdm_radar_plan* plan, const ofdm_c32* Y, const ofdm_c32* X,
                       int32_t frames, float* out_map, ofdm_target* out_targets,
                       int32_t* n_targets, uint32_t* status, void* stream);

/* Same as ofdm_radar_process with HOST buffers (pinned memory gives
 * asynchronous, overlapped copies).  The plan allocates device staging for
 * max_frames on the first call.  The frames go in up to 16 chunks through
 * three internal streams ordered after `stream`: uploads back to back on
 * one, each chunk's kernels on a second once its upload is done, and its
 * results back on a third.  The call returns after everything, copies
 * included, has finished.  NULL outputs are skipped. */
int ofdm_radar_process_host(ofdm_radar_plan* plan, const ofdm_c32* Y_host,
                            const ofdm_c32* X_host, int32_t frames, float* map_host,
                            ofdm_target* targets_host, int32_t* n_targets_host,
                            uint32_t* status_host, void* stream);

/* ZC precoding of Sec. III-B on every symbol: Xp = Z_m A / sqrt(N)
 * (inverse = 0) or A = (Z_m A / sqrt(N))^{-1} applied to Xp (inverse = 1,
 * undoing the precoding as the paper's receiver does with Z_m^{-1}).
 * in, out: [frames][M][N] complex64; in == out is not allowed. */
int ofdm_zc_precode(ofdm_radar_plan* plan, const ofdm_c32* in, ofdm_c32* out,
                    int32_t frames, int32_t inverse, void* stream);

/* Steps a1-a5 only: the windowed range profile
 *   g[r, l] = sum_k w_k H'[k, l] e^{+j 2 pi k r / N}   (inner range sum of Eq. (17))
 * on the support rows, written as strip[frames][rows][M] complex64 with rows
 * in ofdm_radar_support_rows order.  No Doppler window is applied. */
int ofdm_radar_range_profile(ofdm_radar_plan* plan, const ofdm_c32* Y, const ofdm_c32* X,
                             int32_t frames, ofdm_c32* strip, void* stream);

/* Step a6 only: Doppler DFT with the window over l, |.|^2 / (N M) (Eq. (17))
 * of a strip from ofdm_radar_range_profile into out_map (full map, zero rows
 * included). */
int ofdm_radar_doppler(ofdm_radar_plan* plan, const ofdm_c32* strip, int32_t frames,
                       float* out_map, void* stream);

/* Step a7 only: detection (Eq. (18)) and estimates (Eq. (19)) on full maps
 * [frames][N'][M'] float32 given by the caller. */
int ofdm_radar_detect(ofdm_radar_plan* plan, const float* map, int32_t frames,
                      ofdm_target* out_targets, int32_t* n_targets, uint32_t* status,
                      void* stream);

/* FPS-SFT (Sec. III-C): the sparse alternative to the periodogram.  The
 * paper outlines it (iterations of three or more Q-length slices, Q =
 * lcm(N, M), a Q-point DFT per slice, frequencies recovered in one iteration
 * removed from the next) and defers its details to its FPS-SFT reference;
 * this is a restatement from the projection-slice theorem:
 *   - slice j of an iteration samples the DFT-CE estimate H' along
 *     (a0 n + t0_j mod N, a1 n + t1_j mod M), n < Q, and is transformed;
 *   - recovered frequencies are removed from every slice;
 *   - bins whose energy (mean over the slices) exceeds the median bin energy
 *     times -ln(bin_pfa)/ln 2, and dynamic_range times the strongest bin seen
 *     so far, are decoded by a maximum-likelihood search along their
 *     projection line, kept when the coherence |sum_j S_j e^{-i theta_j}| /
 *     sum_j |S_j| reaches coherence_min (a 1-sparse bin);
 *   - iterations stop early once no bin passes the energy test. */
typedef struct {
  int32_t iterations;     /* I, 1..16 (default 4) */
  int32_t offsets;        /* T slices per iteration, 3..8 (default 8) */
  int32_t max_recover;    /* recovered frequencies kept per frame, 1..64 (default 32) */
  float bin_pfa;          /* default 1e-6 */
  float coherence_min;    /* default 0.95 */
  float dynamic_range;    /* default 1e-10 */
} ofdm_fps_params;

void ofdm_fps_default_params(ofdm_fps_params* fp);

/* FPS-SFT on `frames` frames.  The random slice geometry is an input:
 * slices is a DEVICE int32 array [frames][iterations][2 + 2 * offsets] holding
 * a0, a1 (odd) and then (t0_j, t1_j) for every slice.  Uses the plan's
 * ZC precoding, division and DFT-CE (any window setting: slices read the
 * un-windowed H'); requires Q = max(N, M) <= 1024 and M' = M.  Writes the
 * strongest min(recovered, max_targets) as targets with the periodogram's
 * conventions: r = -f0 mod N, s centred, power |X[f]|^2 / (N M) (the rect-
 * window periodogram value of that bin, Eq. (17)), ordered by power then
 * map index. */
int ofdm_fps_sft(ofdm_radar_plan* plan, const ofdm_c32* Y, const ofdm_c32* X, int32_t frames,
                 const ofdm_fps_params* fp, const int32_t* slices, ofdm_target* out_targets,
                 int32_t* n_targets, void* stream);

/* Batched frames of uneven shape (one launch of many frames).  Frames are
 * described one by one; frames of equal (N, M, L_cp) form a group with its
 * own plan (the base parameters give everything else; N_pad = M_pad = 0).
 * Y and X are packed arrays in which frame f's M x N grid starts at
 * desc[f].yx_offset complex elements; its N x M map starts at
 * desc[f].map_offset floats of out_map (a multiple of 4).  Targets, target
 * counts and status words are indexed by the frame's position in desc
 * (targets: [nframes][base->max_targets]). */
typedef struct {
  int32_t N, M, L_cp;
  int32_t reserved;
  int64_t yx_offset;
  int64_t map_offset;
} ofdm_frame_desc;

typedef struct ofdm_radar_batch ofdm_radar_batch;

enum { OFDM_BATCH_NO_GRAPH = 1u, OFDM_BATCH_NO_TUNE = 2u };

/* Group the frames, create one plan per group (allocates), upload the
 * per-frame offset tables.  flags: OFDM_BATCH_NO_GRAPH launches on the
 * stream instead of replaying a CUDA graph; OFDM_BATCH_NO_TUNE skips the
 * launch-shape tuner. */
int ofdm_radar_batch_create(const ofdm_radar_params* base, const ofdm_frame_desc* desc, int32_t nframes,
                            uint32_t flags, ofdm_radar_batch** out);

/* Whole chain on every frame of the batch.  Groups run concurrently (one
 * stream each, joined back into `stream`).  The first call on a batch tunes
 * the column kernel's launch shape of each group on these inputs (cached per
 * (N, M, L_cp) for the process) and, unless OFDM_BATCH_NO_GRAPH, captures the
 * launches into a CUDA graph that later calls with the same buffers replay
 * (other buffers are captured anew).  A capture that cannot be made -- e.g.
 * on the legacy NULL stream -- falls back to direct launches.  out_map may be
 * NULL. */
int ofdm_radar_batch_process(ofdm_radar_batch* b, const ofdm_c32* Y, const ofdm_c32* X, float* out_map,
                             ofdm_target* out_targets, int32_t* n_targets, uint32_t* status, void* stream);

/* Number of groups and, if shapes != NULL, [groups][5] = N, M, L_cp, frames,
 * chosen column-kernel variant: for N <= 1024, 0 = one warp per symbol in the
 * widest CTA, 4 = one warp per symbol in 4-warp CTAs, 2 = groups of N / 16
 * threads (N = 1024); for N >= 2048, 2 = groups of N / 16 threads (16 points
 * each), 0 = groups of N / 32 threads (32 points each); -1 = not tuned yet.
 * Returns the group count. */
int ofdm_radar_batch_groups(const ofdm_radar_batch* b, int32_t* shapes);

/* 1 if the last ofdm_radar_batch_process replayed or captured a graph, 0 if
 * it launched directly. */
int ofdm_radar_batch_used_graph(const ofdm_radar_batch* b);

void ofdm_radar_batch_destroy(ofdm_radar_batch* b);

/* ---- Learned proposal (the paper has no counterpart: its conclusion names
 * machine learning as future work).  A coarse range-Doppler map -- an M/4-
 * point Doppler DFT of the first M/4 symbols of the DFT-CE range profile,
 * max-pooled 4x over range rows, x = log(1 + C / mean C) -- feeds a 3-layer
 * CNN (3x3 convolutions 1->16->16->1 with ReLU, BF16 weights, FP32
 * accumulation).  Coarse cells whose logit exceeds a threshold are refined
 * exactly: the periodogram value of Eq. (17) on the 8 x 8 fine cells around
 * each, local maxima of the inner 6 x 6, strongest max_targets reported.
 * Frames with more candidates than the cap fall back to the full
 * periodogram and detection (status bit OFDM_STATUS_FALLBACK).
 * Requirements: M in {256, 512, 1024}, M' = M, L_cp + 2 < N (Hann/Hamming) or
 * L_cp < N (rect). */
enum { OFDM_STATUS_FALLBACK = 16u };

/* Allocate the learned path's workspace for max_frames (coarse maps, CNN
 * activations, logits).  Must precede the two calls below. */
int ofdm_radar_learned_prepare(ofdm_radar_plan* plan);

/* Coarse-map height and width for this plan. */
int ofdm_radar_coarse_shape(const ofdm_radar_plan* plan, int32_t* height, int32_t* width);

/* Steps a1-a5 and the coarse map: x_out [frames][height][width] float32
 * (the CNN input).  x_out may be NULL (kept in the workspace). */
int ofdm_radar_coarse_map(ofdm_radar_plan* plan, const ofdm_c32* Y, const ofdm_c32* X, int32_t frames,
                          float* x_out, void* stream);

/* The chain with the learned proposal in place of the full Doppler stage and
 * detection.  theta: DEVICE float32 network parameters in the order
 * w1[16][1][3][3], b1[16], w2[16][16][3][3], b2[16], w3[1][16][3][3], b3[1]
 * (ofdm_cnn_param_count() floats; weights rounded to BF16 when used, biases
 * FP32).  A coarse cell
 * is a candidate when its logit exceeds logit_threshold; more than
 * max_candidates (1..256) candidates send the frame to the fallback. */
int ofdm_radar_process_learned(ofdm_radar_plan* plan, const float* theta, const ofdm_c32* Y, const ofdm_c32* X,
                               int32_t frames, float logit_threshold, int32_t max_candidates,
                               ofdm_target* out_targets, int32_t* n_targets, uint32_t* status, void* stream);

/* The CNN's own kernels, on device buffers [B][C][H][W] (no plan needed).
 * bf16 != 0 rounds the weights (not the biases) to BF16 as they are used
 * (inference and training alike); accumulation is FP32. */
int ofdm_cnn_param_count(void);
int ofdm_cnn_forward(const float* theta, int32_t bf16, const float* x, int32_t B, int32_t H, int32_t W,
                     float* a1, float* a2, float* logits, void* stream);
/* Gradient of the loss w.r.t. theta (written to gtheta) given d loss / d logits;
 * ga1, ga2: [B][16][H][W] workspace. */
int ofdm_cnn_backward(const float* theta, int32_t bf16, const float* x, const float* a1, const float* a2,
                      const float* glogits, int32_t B, int32_t H, int32_t W, float* ga1, float* ga2,
                      float* gtheta, void* stream);
/* Mean binary cross-entropy with logits (positives weighted by pos_weight):
 * *loss (device float) and d loss / d logits. */
int ofdm_cnn_bce(const float* logits, const float* labels, int32_t n, float pos_weight, float* loss,
                 float* glogits, void* stream);
/* One Adam step (bias-corrected, step >= 1) on theta in place. */
int ofdm_cnn_adam(float* theta, const float* grad, float* m, float* v, int32_t n, int32_t step, float lr,
                  float beta1, float beta2, float eps, void* stream);

/* Transmit side of Sec. III-B: the PAPR (Eq. (25)) of each OFDM symbol's
 * time signal and the share of its power that the power amplifier pushes
 * out of the occupied band (adjacent-channel interference).
 *   S     [frames][M][N] complex64: the transmitted frequency-domain grid
 *         (X_p from ofdm_zc_precode, or the QAM grid without precoding)
 *   oversample  L in {1, 2, 4, 8}, L N <= 4096: subcarrier k sits at bin k
 *         (k < N/2) or k + (L-1) N of an L N-point grid; x = its inverse DFT
 *   q     amplifier state level: |y| = |x| / sqrt(1 + (|x| / (x_bar 10^(q/10)))^2),
 *         phase kept, x_bar the mean modulus of the symbol's samples (q = 2 in the paper)
 *   papr  [frames][M] float32, max |x|^2 / mean |x|^2 (linear); may be NULL
 *   aci   [frames][M] float32, power of DFT(y) outside the N occupied bins over
 *         its total power; may be NULL
 * The first call for a given L N builds that transform's twiddle table (a
 * small device allocation). */
int ofdm_tx_amplifier(ofdm_radar_plan* plan, const ofdm_c32* S, int32_t frames, int32_t oversample, float q,
                      float* papr, float* aci, void* stream);

/* Kernel launches made by the last successful call on this plan. */
int ofdm_radar_last_launch_count(const ofdm_radar_plan* plan);

/* Per-kernel timing for profiling.  enable = 1 makes every later call on
 * the plan record a CUDA event pair around each of its kernels on the
 * launching stream (up to 4096 launches, then recording stops); enable = 0
 * stops.  ofdm_radar_timing_read waits for the recorded events, writes up to
 * `n` entries of per-kernel-kind totals (milliseconds) and launch counts in
 * the order column, zero_rows, doppler, detect, zct, coarse, cnn, refine
 * (the last three from ofdm_radar_process_learned; cnn spans its three
 * layers, refine its select, candidate and merge kernels), and clears the
 * record.
 * Returns the number of kinds written. */
int ofdm_radar_timing_enable(ofdm_radar_plan* plan, int32_t enable);
int ofdm_radar_timing_read(ofdm_radar_plan* plan, float* total_ms, int32_t* launches, int32_t n);

/* No-allocation variant of ofdm_radar_process (the paper has no counterpart).
 * For callers that cannot allocate device memory -- code running under an
 * allocator it does not own, in a memory-capped process, or with all device
 * memory committed up front -- so cannot create a plan.  Takes the parameters
 * directly (max_frames is ignored) and keeps tables and workspace in one
 * fixed array compiled into the library (about 14.1 MB, held on every device
 * that loads the library until the process exits).  Same inputs, outputs,
 * layouts and results as ofdm_radar_process on device buffers.
 * Limits: frames <= 4096 and frames * support_rows * max(M, M') <= 2^20
 * (e.g. 31 frames of 1024 x 256 with L_cp = 128 and a Hann window); larger
 * requests return OFDM_ERR_UNSUPPORTED_SIZE before anything is launched.
 * The first call on a device looks up the array's address
 * (cudaGetSymbolAddress): make it before any stream capture.  Every call on
 * a device shares the array and leaves its contents behind; each call clears
 * the status words and work counters it uses on the caller's stream first,
 * and rebuilds the tables there when the parameters differ from the previous
 * call's.  Calls that overlap on the GPU race on the array.
 * Calls no cudaMalloc/cudaFree. */
int ofdm_radar_process_noalloc(const ofdm_radar_params* p, const ofdm_c32* Y, const ofdm_c32* X,
                               int32_t frames, float* out_map, ofdm_target* out_targets,
                               int32_t* n_targets, uint32_t* status, void* stream);

/* Memory-safety check for tests and debugging (no counterpart in the paper,
 * which has no software).  Every device buffer the library allocates -- plan
 * tables and workspace, the host path's staging buffers, batch offset tables
 * -- ends in a 256-byte canary of 0xFF bytes (a NaN for float data) that no
 * kernel writes.  Returns 1 if the canary of every live buffer on the current
 * device is intact, 0 if some launch wrote past the end of one, or a negative
 * OFDM_ERR_* code.  Waits for all work on the current device
 * (cudaDeviceSynchronize) and copies 256 bytes per buffer to the host: not for
 * the timed path.  Buffers on other devices are checked with that device
 * current. */
int ofdm_radar_workspace_intact(void);

/* Static description of an error code; for OFDM_ERR_CUDA the last CUDA
 * error string of the calling thread is appended. */
const char* ofdm_radar_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif /* OFDM_RADAR_H */
