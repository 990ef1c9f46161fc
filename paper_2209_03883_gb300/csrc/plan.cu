// plan.cu -- plan creation (parameter checks, FP64-derived tables,
// workspace), the C ABI entry points and the host-buffer pipeline.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <complex>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "fft.cuh"
#include "internal.h"
#include "refine.cuh"

using ofdm::ColumnArgs;
using ofdm::DetectArgs;
using ofdm::DopplerArgs;
using ofdm::ZctArgs;

constexpr int kHostChunks = 16;  // frame chunks of the host-buffer pipeline

struct ofdm_radar_plan {
  ofdm_radar_params p;
  int Np, Mp;
  int gen = 0;                 // M' not a power of two: two-factor Doppler DFT and general detection
  int rows, row0, full;        // DFT-CE support (Eqs. (17), (21))
  int z0, nz;                  // contiguous zero rows of the map
  int rinv;
  float c0, c1;
  float2* d_tables = nullptr;  // one allocation: pre, post, pre_conj, post_conj, twN, twM
  float2 *pre, *post, *pre_conj, *post_conj, *twN, *twM;
  float2* twG = nullptr;       // N >= 1024: twiddles for 16 points per thread (groups of N / 16 threads)
  float4* d_df = nullptr;      // double-float pre-chirp [N] and roots of unity [N]
  unsigned char* d_tc = nullptr;  // split-FP16 form: DFT-32 operand images (hi, lo) and inter-stage twiddles
  float2* d_fps = nullptr;        // FPS-SFT slice workspace (allocated by the first ofdm_fps_sft call)
  size_t fps_elems = 0;
  float2* d_twL = nullptr;        // ofdm_tx_amplifier: L N-point pass twiddles (first call per L N)
  int twL_n = 0;
  // range zero padding N' > N: kept taps [max_frames][L_cp][M], window over k and the two transforms' twiddles
  float2* d_taps = nullptr;
  float2* d_padtab = nullptr;
  float2 *twPN = nullptr, *twPP = nullptr;
  float* d_wk = nullptr;
  float* d_alpha = nullptr;       // CFAR: alpha(n) = n (P_fa^(-1/n) - 1), n = 0 .. 17^2
  float* d_wl = nullptr;
  float2* d_strip = nullptr;   // [max_frames][rows][M]
  float* d_pow = nullptr;      // [max_frames][rows][M']
  uint32_t* d_wstatus = nullptr;
  // detection workspace: per-band keys, per-frame tickets / counters / eta
  uint64_t* d_detkeys = nullptr;
  unsigned* d_dettick = nullptr;   // [2][max_frames]: tickets, counts
  float* d_eta = nullptr;
  int det_bands = 0;
  // Ticket counters of the dynamically scheduled column kernel: slot 0 for
  // calls on the caller's stream, slot 1 for the kernel stream of the host
  // pipeline (launches that may run concurrently need separate counters);
  // slots 2-4 are spare.
  unsigned long long* d_ctr = nullptr;
  unsigned long long ctr_base[1 + 4] = {0, 0, 0, 0, 0};
  int ctr_slot = 0;
  // host-buffer path (allocated on first use)
  float2* d_Y = nullptr;
  float2* d_X = nullptr;
  float* d_map = nullptr;
  ofdm_target* d_tg = nullptr;
  int32_t* d_nt = nullptr;
  uint32_t* d_st = nullptr;
  cudaStream_t hs[3] = {nullptr, nullptr, nullptr};   // uploads, kernels, downloads
  cudaEvent_t ev[2 + 2 * kHostChunks] = {};            // fork, join, per-chunk upload / kernel done
  int last_launches = 0;
  // learned proposal workspace (ofdm_radar_learned_prepare)
  int Hc = 0, Mc = 0;
  unsigned* d_cpow = nullptr;
  float *d_cx = nullptr, *d_a1 = nullptr, *d_a2 = nullptr, *d_logit = nullptr, *d_w4 = nullptr;
  float2* d_twMc = nullptr;
  float2* d_rootsM = nullptr;   // exp(-2 pi i m / M)
  int* d_mask = nullptr;
  int* d_cand = nullptr;        // [max_frames][256] candidate cells
  int* d_ncand = nullptr;       // [max_frames]
  uint64_t* d_keys = nullptr;   // [max_frames][256][36] local-maximum keys
  // per-kernel timing (ofdm_radar_timing_enable)
  int timing = 0;
  int nrec = 0;
  cudaEvent_t* tev = nullptr;  // 2 * kMaxTimed events
  int* tkind = nullptr;
};

namespace {

constexpr int kMaxTimed = 4096;
constexpr int kKinds = 8;  // column, zero_rows, doppler, detect, zct, coarse, cnn, refine
enum { K_COLUMN = 0, K_ZERO = 1, K_DOPPLER = 2, K_DETECT = 3, K_ZCT = 4, K_COARSE = 5, K_CNN = 6, K_REFINE = 7 };

// Records an event pair around one launch when timing is enabled.
struct ScopedTimer {
  ofdm_radar_plan* pl;
  cudaStream_t s;
  int idx = -1;
  ScopedTimer(ofdm_radar_plan* p, cudaStream_t st, int kind) : pl(p), s(st) {
    if (pl->timing && pl->nrec < kMaxTimed) {
      idx = pl->nrec++;
      pl->tkind[idx] = kind;
      cudaEventRecord(pl->tev[2 * idx], s);
    }
  }
  ~ScopedTimer() {
    if (idx >= 0) cudaEventRecord(pl->tev[2 * idx + 1], s);
  }
};
}  // namespace

namespace {

__global__ void mark_fallback_kernel(const int* mask, uint32_t* status, int frames) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f < frames && mask[f] && status) status[f] |= OFDM_STATUS_FALLBACK;
}

cudaError_t mark_fallback(const int* mask, uint32_t* status, int frames, cudaStream_t s) {
  if (!status) return cudaSuccess;
  mark_fallback_kernel<<<(frames + 255) / 256, 256, 0, s>>>(mask, status, frames);
  return cudaGetLastError();
}

thread_local char g_errbuf[512];

bool is_pow2(long v) { return v > 0 && (v & (v - 1)) == 0; }

int cuda_fail(cudaError_t e) {
  snprintf(g_errbuf, sizeof g_errbuf, "CUDA error: %s", cudaGetErrorString(e));
  return OFDM_ERR_CUDA;
}

// exp(i pi m / half) for an exact integer phase index m in [0, 2 half).
float2 unit_phase(long long m, long long half) {
  const double a = M_PI * (double)m / (double)half;
  return make_float2((float)cos(a), (float)sin(a));
}

long long mod_ll(long long a, long long m) {
  long long r = a % m;
  return r < 0 ? r + m : r;
}

// Pass twiddles of the Stockham schedule in fft.cuh, for DIR = +1.
void build_twiddles(std::vector<float2>& out, int n, int e) {
  out.assign((size_t)ofdm::tw_size(n, e) + 1, make_float2(1.f, 0.f));
  const int np = ofdm::num_passes(n, e);
  for (int p = 1; p < np; ++p) {
    const int R = ofdm::pass_radix(n, e, p), NS = ofdm::pass_ns(n, e, p), off = ofdm::tw_offset(n, e, p);
    const long long span = (long long)NS * R;
    for (int r = 0; r < R; ++r)
      for (int u = 0; u < NS; ++u) {
        const long long m = ((long long)u * r) % span;
        const double a = 2.0 * M_PI * (double)m / (double)span;
        out[(size_t)off + r * NS + u] = make_float2((float)cos(a), (float)sin(a));
      }
  }
}

int column_points_per_thread(int N) { return N <= 1024 ? N / 32 : 32; }

// Every device buffer the library allocates ends in a 256-byte canary of
// all-ones bytes (a NaN for float data), written at allocation and never by a
// kernel; ofdm_radar_workspace_intact() checks that no launch wrote past the
// end of its buffer.  The tail also covers reads of up to 16 bytes past it.
constexpr size_t kCanaryBytes = 256;
std::mutex g_canary_mu;
std::map<const char*, std::pair<size_t, int>> g_canary;   // allocation -> (bytes before its canary, device)

template <class T>
cudaError_t dalloc(T** p, size_t count) {
  const size_t bytes = count * sizeof(T);
  cudaError_t e = cudaMalloc((void**)p, bytes + kCanaryBytes);
  if (e != cudaSuccess) return e;
  e = cudaMemset(reinterpret_cast<char*>(*p) + bytes, 0xFF, kCanaryBytes);
  if (e != cudaSuccess) {
    cudaFree(*p);
    *p = nullptr;
    return e;
  }
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(g_canary_mu);
  g_canary[reinterpret_cast<const char*>(*p)] = std::make_pair(bytes, dev);
  return cudaSuccess;
}

// Frees a dalloc buffer (null: nothing).
void dfree(void* p) {
  if (!p) return;
  {
    std::lock_guard<std::mutex> lk(g_canary_mu);
    g_canary.erase(reinterpret_cast<const char*>(p));
  }
  cudaFree(p);
}

}  // namespace

extern "C" {

void ofdm_radar_default_params(ofdm_radar_params* p) {
  if (!p) return;
  memset(p, 0, sizeof *p);
  p->zc_root = 1;
  p->window = OFDM_WINDOW_HANN;
  p->detect_mode = OFDM_DETECT_TOPK;
  p->cfar_guard = 1;
  p->cfar_train = 4;
  p->max_targets = 8;
  p->max_frames = 1;
  p->precision = OFDM_PREC_FP32;
  p->pfa = 1e-2f;
  p->noise_var = -1.f;
  p->fc_hz = 77e9;
  p->df_hz = 240e3;
}

const char* ofdm_radar_strerror(int code) {
  switch (code) {
    case OFDM_OK: return "ok";
    case OFDM_ERR_INVALID_ARG: return "invalid argument";
    case OFDM_ERR_UNSUPPORTED_SIZE: return "unsupported size";
    case OFDM_ERR_CUDA: return g_errbuf[0] ? g_errbuf : "CUDA error";
    case OFDM_ERR_TIMEOUT: return "device wait timed out";
    case OFDM_ERR_NO_MEMORY: return "out of device memory";
    default: return "unknown error";
  }
}

int ofdm_radar_workspace_intact(void) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(e);
  std::lock_guard<std::mutex> lk(g_canary_mu);
  unsigned char tail[kCanaryBytes];
  for (const auto& a : g_canary) {
    if (a.second.second != dev) continue;   // other devices' work is not synchronised here
    e = cudaMemcpy(tail, a.first + a.second.first, kCanaryBytes, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e);
    for (size_t i = 0; i < kCanaryBytes; ++i)
      if (tail[i] != 0xFF) return 0;
  }
  return 1;
}

void ofdm_radar_plan_destroy(ofdm_radar_plan* plan) {
  if (!plan) return;
  dfree(plan->d_tables);
  dfree(plan->d_df);
  dfree(plan->d_tc);
  dfree(plan->d_fps);
  dfree(plan->d_twL);
  dfree(plan->d_taps);
  dfree(plan->d_padtab);
  dfree(plan->d_wk);
  dfree(plan->d_alpha);
  dfree(plan->d_wl);
  dfree(plan->d_strip);
  dfree(plan->d_pow);
  dfree(plan->d_wstatus);
  dfree(plan->d_ctr);
  dfree(plan->d_detkeys);
  dfree(plan->d_dettick);
  dfree(plan->d_eta);
  dfree(plan->d_cpow);
  dfree(plan->d_cx);
  dfree(plan->d_a1);
  dfree(plan->d_a2);
  dfree(plan->d_logit);
  dfree(plan->d_w4);
  dfree(plan->d_twMc);
  dfree(plan->d_rootsM);
  dfree(plan->d_mask);
  dfree(plan->d_cand);
  dfree(plan->d_ncand);
  dfree(plan->d_keys);
  dfree(plan->d_Y);
  dfree(plan->d_X);
  dfree(plan->d_map);
  dfree(plan->d_tg);
  dfree(plan->d_nt);
  dfree(plan->d_st);
  for (auto& s : plan->hs)
    if (s) cudaStreamDestroy(s);
  for (auto& e : plan->ev)
    if (e) cudaEventDestroy(e);
  if (plan->tev) {
    for (int i = 0; i < 2 * kMaxTimed; ++i) cudaEventDestroy(plan->tev[i]);
    delete[] plan->tev;
    delete[] plan->tkind;
  }
  delete plan;
}

int ofdm_radar_plan_create(const ofdm_radar_params* pin, ofdm_radar_plan** out) {
  ofdm::NvtxRange nvtx_range("ofdm_radar_plan_create");
  if (!pin || !out) return OFDM_ERR_INVALID_ARG;
  *out = nullptr;
  const ofdm_radar_params& p = *pin;
  const int N = p.N, M = p.M;
  const int Np = p.N_pad ? p.N_pad : N, Mp = p.M_pad ? p.M_pad : M;
  if (!is_pow2(N) || N < 64 || N > 4096) return OFDM_ERR_UNSUPPORTED_SIZE;
  // M: 16..1024, a multiple of 4 (Table I's 560 included); M' >= M likewise
  if (M < 16 || M > 1024 || M % 4) return OFDM_ERR_UNSUPPORTED_SIZE;
  // range zero padding: N' = 2N, 4N or 8N, at most 4096
  if (Np != N && (!is_pow2(Np) || Np < 2 * N || Np > 8 * N || Np > 4096)) return OFDM_ERR_UNSUPPORTED_SIZE;
  if (Mp < M || Mp > 1024 || Mp % 4) return OFDM_ERR_UNSUPPORTED_SIZE;
  if (p.L_cp < 1 || p.L_cp > N) return OFDM_ERR_INVALID_ARG;
  if (p.n_cp < 0) return OFDM_ERR_INVALID_ARG;
  if (p.zc_root < 0 || (p.zc_root > 0 && (p.zc_root % 2) == 0)) return OFDM_ERR_INVALID_ARG;
  if (p.window < OFDM_WINDOW_RECT || p.window > OFDM_WINDOW_HAMMING) return OFDM_ERR_INVALID_ARG;
  if (p.detect_mode != OFDM_DETECT_TOPK && p.detect_mode != OFDM_DETECT_THRESHOLD && p.detect_mode != OFDM_DETECT_CFAR)
    return OFDM_ERR_INVALID_ARG;
  if (p.detect_mode == OFDM_DETECT_CFAR &&
      (p.cfar_guard < 0 || p.cfar_train < 1 || p.cfar_guard + p.cfar_train > 8))
    return OFDM_ERR_INVALID_ARG;
  if (p.max_targets < 1 || p.max_targets > 32) return OFDM_ERR_INVALID_ARG;
  if (p.max_frames < 1) return OFDM_ERR_INVALID_ARG;
  if (p.precision != OFDM_PREC_FP32 && p.precision != OFDM_PREC_SPLIT_BF16 && p.precision != OFDM_PREC_SPLIT_FP16)
    return OFDM_ERR_INVALID_ARG;
  if (p.precision == OFDM_PREC_SPLIT_BF16) return OFDM_ERR_UNSUPPORTED_SIZE;   // not built
  if (p.precision == OFDM_PREC_SPLIT_FP16) {
    // the tensor-core column kernel: 1024 = 32 x 32, tiles of 4 symbols,
    // taps n < 256 from the last stage, and a support narrower than N
    // (rows up to L_cp itself with a Hann / Hamming window: L_cp <= 255)
    const int spread_tc = p.window == OFDM_WINDOW_RECT ? 0 : 1;
    if (N != 1024 || Np != N || M % 4 || p.L_cp + spread_tc > 256) return OFDM_ERR_UNSUPPORTED_SIZE;
  }
  if (!(p.pfa > 0.f && p.pfa < 1.f)) return OFDM_ERR_INVALID_ARG;
  if (!(p.fc_hz > 0.0 && p.df_hz > 0.0)) return OFDM_ERR_INVALID_ARG;

  ofdm_radar_plan* pl = new ofdm_radar_plan();
  pl->p = p;
  pl->Np = Np;
  pl->Mp = Mp;
  pl->gen = is_pow2(Mp) ? 0 : 1;
  // Support rows: taps n < L_cp (Eq. (21)); a periodic Hann/Hamming window
  // over k spreads each tap to r - 1 and r + 1 (circular).
  const int spread = p.window == OFDM_WINDOW_RECT ? 0 : 2;
  if (Np > N) {   // on a padded grid every range row carries signal (range_pad.cu)
    pl->rows = Np; pl->row0 = 0; pl->full = 1;
  } else if (p.L_cp + spread >= N) {
    pl->rows = N; pl->row0 = 0; pl->full = 1;
  } else {
    pl->rows = p.L_cp + spread; pl->row0 = spread ? N - 1 : 0; pl->full = 0;
  }
  pl->nz = Np - pl->rows;
  pl->z0 = (pl->row0 + pl->rows) % Np;
  if (p.window == OFDM_WINDOW_HANN) { pl->c0 = 0.5f; pl->c1 = -0.25f; }
  else if (p.window == OFDM_WINDOW_HAMMING) { pl->c0 = 0.54f; pl->c1 = -0.23f; }
  else { pl->c0 = 1.f; pl->c1 = 0.f; }

  // ZC tables (Sec. III-B, Eqs. (23)-(24)) with exact int64 phase indices:
  //   Z_m(i, j) = exp(i pi m / N^2),
  //   m = r' [ (i mod 2) N^2 + 2 N (i j mod N) + j^2 + 2 q' (i N + j) ]  mod 2 N^2
  // which factors into pre_j = exp(i pi r'(j^2 + 2q'j)/N^2), the DFT kernel
  // exp(2 pi i r' i j / N) and post_i = exp(i pi r'((i mod 2) N^2 + 2q' i N)/N^2).
  const long long NN = (long long)N * N, two = 2 * NN;
  const int r = p.zc_root ? p.zc_root : 1;
  const long long rr = mod_ll(r, two), qq = mod_ll(p.zc_q, two);
  std::vector<float2> pre(N), post(N), prec(N), postc(N);
  std::vector<float4> df(2 * (size_t)N);  // [0, N): pre-chirp, [N, 2N): exp(+2 pi i m / N)
  auto split = [](double v) {
    const float hi = (float)v;
    return make_float2(hi, (float)(v - (double)hi));
  };
  auto df_phase = [&](double a) {
    const float2 re = split(cos(a)), im = split(sin(a));
    return make_float4(re.x, re.y, im.x, im.y);
  };
  for (int m = 0; m < N; ++m) df[(size_t)N + m] = df_phase(2.0 * M_PI * (double)m / (double)N);
  for (int j = 0; j < N; ++j) {
    const long long base = mod_ll((long long)j * j + 2 * qq % two * j % two, two);
    const long long m = (rr * base) % two;
    pre[j] = unit_phase(m, NN);
    df[j] = df_phase(M_PI * (double)m / (double)NN);
    prec[j] = make_float2(pre[j].x, -pre[j].y);
  }
  for (int i = 0; i < N; ++i) {
    const long long base = mod_ll((long long)(i & 1) * NN + (2 * qq % two) * ((long long)i * N % two) % two, two);
    const long long m = (rr * base) % two;
    post[i] = unit_phase(m, NN);
    postc[i] = make_float2(post[i].x, -post[i].y);
  }
  // r'^{-1} mod N (r' odd, N a power of two)
  int rinv = 1;
  for (int c = 1; c < N; c += 2)
    if (((long long)c * r) % N == 1) { rinv = c; break; }
  pl->rinv = rinv;

  std::vector<float2> twN, twM, twG;
  build_twiddles(twN, N, column_points_per_thread(N));
  if (N >= 1024) build_twiddles(twG, N, 16);   // column kernel in groups of N / 16 threads
  if (!is_pow2(Mp)) {   // roots e^{-2 pi i m / M'} of the two-factor Doppler DFT
    twM.resize(Mp);
    for (int m = 0; m < Mp; ++m) {
      const double a = -2.0 * M_PI * m / Mp;
      twM[m] = make_float2((float)cos(a), (float)sin(a));
    }
  } else if (Mp <= 32) {
    twM.resize(Mp);
    for (int m = 0; m < Mp; ++m) {
      const double a = 2.0 * M_PI * m / Mp;
      twM[m] = make_float2((float)cos(a), (float)sin(a));
    }
  } else {
    build_twiddles(twM, Mp, Mp / 32);
  }
  std::vector<float2> twPN, twPP;
  std::vector<float> wk;
  if (Np > N) {
    const int T = ofdm::pad_threads(Np);
    build_twiddles(twPN, N, N / T);
    build_twiddles(twPP, Np, Np / T);
    wk.resize(N);
    for (int k = 0; k < N; ++k) {
      const double c = cos(2.0 * M_PI * k / N);
      wk[k] = p.window == OFDM_WINDOW_HANN ? (float)(0.5 - 0.5 * c)
            : p.window == OFDM_WINDOW_HAMMING ? (float)(0.54 - 0.46 * c) : 1.f;
    }
  }
  std::vector<float> wl(M);
  for (int l = 0; l < M; ++l) {
    const double c = cos(2.0 * M_PI * l / M);
    wl[l] = p.window == OFDM_WINDOW_HANN ? (float)(0.5 - 0.5 * c)
          : p.window == OFDM_WINDOW_HAMMING ? (float)(0.54 - 0.46 * c) : 1.f;
  }

  const size_t ntab = 4 * (size_t)N + twN.size() + twM.size() + twG.size();
  cudaError_t e = dalloc(&pl->d_tables, ntab);
  if (e == cudaSuccess) e = dalloc(&pl->d_df, 2 * (size_t)N);
  if (e == cudaSuccess) e = dalloc(&pl->d_wl, (size_t)M);
  if (e == cudaSuccess) e = dalloc(&pl->d_strip, (size_t)p.max_frames * pl->rows * M);
  if (e == cudaSuccess) e = dalloc(&pl->d_pow, (size_t)p.max_frames * pl->rows * Mp);
  if (e == cudaSuccess) e = dalloc(&pl->d_wstatus, (size_t)p.max_frames);
  if (e == cudaSuccess) e = dalloc(&pl->d_ctr, 5);
  {
    int br = 0;
    ofdm::detect_bands(pl->rows, Mp, &br, &pl->det_bands);
    if (!is_pow2(Mp)) pl->det_bands = ofdm::detect_general_blocks(pl->rows, Mp);
  }
  if (e == cudaSuccess) e = dalloc(&pl->d_detkeys, (size_t)p.max_frames * pl->det_bands * 32);
  if (e == cudaSuccess) e = dalloc(&pl->d_dettick, 2 * (size_t)p.max_frames);
  if (e == cudaSuccess) e = dalloc(&pl->d_eta, (size_t)p.max_frames);
  const size_t tc_bytes = 2 * ofdm::tc_table_bytes() + 1024 * sizeof(float2);
  if (e == cudaSuccess && p.precision == OFDM_PREC_SPLIT_FP16) e = dalloc(&pl->d_tc, tc_bytes);
  if (e == cudaSuccess && Np > N) e = dalloc(&pl->d_taps, (size_t)p.max_frames * p.L_cp * M);
  if (e == cudaSuccess && Np > N) e = dalloc(&pl->d_padtab, twPN.size() + twPP.size());
  if (e == cudaSuccess && Np > N) e = dalloc(&pl->d_wk, (size_t)N);
  constexpr int kAlphaN = 17 * 17 + 1;
  if (e == cudaSuccess && p.detect_mode == OFDM_DETECT_CFAR) e = dalloc(&pl->d_alpha, (size_t)kAlphaN);
  if (e != cudaSuccess) {
    ofdm_radar_plan_destroy(pl);
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? OFDM_ERR_NO_MEMORY : cuda_fail(e);
  }
  pl->pre = pl->d_tables;
  pl->post = pl->pre + N;
  pl->pre_conj = pl->post + N;
  pl->post_conj = pl->pre_conj + N;
  pl->twN = pl->post_conj + N;
  pl->twM = pl->twN + twN.size();
  pl->twG = twG.empty() ? nullptr : pl->twM + twM.size();
  std::vector<float2> host(ntab);
  memcpy(host.data(), pre.data(), N * sizeof(float2));
  memcpy(host.data() + N, post.data(), N * sizeof(float2));
  memcpy(host.data() + 2 * N, prec.data(), N * sizeof(float2));
  memcpy(host.data() + 3 * N, postc.data(), N * sizeof(float2));
  memcpy(host.data() + 4 * N, twN.data(), twN.size() * sizeof(float2));
  memcpy(host.data() + 4 * N + twN.size(), twM.data(), twM.size() * sizeof(float2));
  if (!twG.empty())
    memcpy(host.data() + 4 * N + twN.size() + twM.size(), twG.data(), twG.size() * sizeof(float2));
  e = cudaMemcpy(pl->d_tables, host.data(), ntab * sizeof(float2), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(pl->d_wl, wl.data(), M * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(pl->d_df, df.data(), df.size() * sizeof(float4), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(pl->d_wstatus, 0, (size_t)p.max_frames * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMemset(pl->d_ctr, 0, 5 * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemset(pl->d_dettick, 0, 2 * (size_t)p.max_frames * sizeof(unsigned));
  if (e == cudaSuccess && pl->d_alpha) {
    float alpha[kAlphaN];
    alpha[0] = 0.f;
    for (int n = 1; n < kAlphaN; ++n) alpha[n] = (float)(n * (pow((double)p.pfa, -1.0 / n) - 1.0));
    e = cudaMemcpy(pl->d_alpha, alpha, sizeof(alpha), cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess && pl->d_padtab) {
    pl->twPN = pl->d_padtab;
    pl->twPP = pl->d_padtab + twPN.size();
    e = cudaMemcpy(pl->twPN, twPN.data(), twPN.size() * sizeof(float2), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(pl->twPP, twPP.data(), twPP.size() * sizeof(float2), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(pl->d_wk, wk.data(), N * sizeof(float), cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess && pl->d_tc) {
    std::vector<unsigned char> tc(tc_bytes);
    ofdm::build_tc_tables(tc.data(), reinterpret_cast<float2*>(tc.data() + 2 * ofdm::tc_table_bytes()));
    e = cudaMemcpy(pl->d_tc, tc.data(), tc_bytes, cudaMemcpyHostToDevice);
  }
  if (e != cudaSuccess) {
    ofdm_radar_plan_destroy(pl);
    return cuda_fail(e);
  }
  *out = pl;
  return OFDM_OK;
}

int ofdm_radar_support_rows(const ofdm_radar_plan* plan, int32_t* rows) {
  if (!plan) return OFDM_ERR_INVALID_ARG;
  if (rows)
    for (int i = 0; i < plan->rows; ++i) rows[i] = (plan->row0 + i) % plan->Np;
  return plan->rows;
}

int ofdm_radar_last_launch_count(const ofdm_radar_plan* plan) {
  return plan ? plan->last_launches : OFDM_ERR_INVALID_ARG;
}

int ofdm_radar_timing_enable(ofdm_radar_plan* pl, int32_t enable) {
  if (!pl) return OFDM_ERR_INVALID_ARG;
  if (enable && !pl->tev) {
    pl->tev = new cudaEvent_t[2 * kMaxTimed]();
    pl->tkind = new int[kMaxTimed]();
    for (int i = 0; i < 2 * kMaxTimed; ++i) {
      cudaError_t e = cudaEventCreate(&pl->tev[i]);
      if (e != cudaSuccess) return cuda_fail(e);
    }
  }
  pl->timing = enable ? 1 : 0;
  return OFDM_OK;
}

int ofdm_radar_timing_read(ofdm_radar_plan* pl, float* total_ms, int32_t* launches, int32_t n) {
  if (!pl || n < 0) return OFDM_ERR_INVALID_ARG;
  float tot[kKinds] = {0};
  int cnt[kKinds] = {0};
  for (int i = 0; i < pl->nrec; ++i) {
    cudaError_t e = cudaEventSynchronize(pl->tev[2 * i + 1]);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, pl->tev[2 * i], pl->tev[2 * i + 1]);
    if (e != cudaSuccess) return cuda_fail(e);
    tot[pl->tkind[i]] += ms;
    cnt[pl->tkind[i]] += 1;
  }
  pl->nrec = 0;
  const int m = n < kKinds ? n : kKinds;
  for (int k = 0; k < m; ++k) {
    if (total_ms) total_ms[k] = tot[k];
    if (launches) launches[k] = cnt[k];
  }
  return m;
}

}  // extern "C"

namespace {

ColumnArgs column_args(const ofdm_radar_plan* pl, int frames) {
  ColumnArgs a;
  a.M = pl->p.M;
  a.L_cp = pl->p.L_cp;
  a.rows = pl->rows;
  a.row0 = pl->row0;
  a.full = pl->full;
  a.frames = frames;
  a.zc = (pl->p.zc_root > 0 && !pl->p.x_is_precoded) ? 1 : 0;
  a.rinv = pl->rinv;
  a.c0 = pl->c0;
  a.c1 = pl->c1;
  a.sqrtN = (float)sqrt((double)pl->p.N);
  a.pre = pl->pre;
  a.post_conj = pl->post_conj;
  a.tw = pl->twN;
  a.post_sign = (mod_ll(pl->p.zc_q, pl->p.N) == 0) ? 1 : 0;
  a.rprime = pl->p.zc_root > 0 ? pl->p.zc_root : 1;
  a.refine_tau = ofdm::kRefineTau;
  a.pre_df = pl->d_df;
  a.w_df = pl->d_df + pl->p.N;
  a.work_ctr = pl->d_ctr + pl->ctr_slot;
  a.work_base = pl->ctr_base[pl->ctr_slot];
  a.frame_off = nullptr;
  a.pipe_warps = pl->twG ? 2 : 0;   // N >= 1024: groups of N / 16 threads (measured faster), else the widest CTA
  a.tw_group = pl->twG;
  if (pl->Np > pl->p.N) {   // the kept taps N h[n] (rect stencil) for the padded range transform
    a.rows = pl->p.L_cp;
    a.row0 = 0;
    a.full = pl->p.L_cp >= pl->p.N ? 1 : 0;
    a.c0 = 1.f;
    a.c1 = 0.f;
  }
  if (pl->d_tc) {
    a.tc_b = reinterpret_cast<const uint4*>(pl->d_tc);
    a.tc_t12 = reinterpret_cast<const float2*>(pl->d_tc + 2 * ofdm::tc_table_bytes());
  }
  return a;
}

// Grids, maps and strips are moved in 16-byte pieces (row copies into shared
// memory, bulk copies of the split-FP16 kernel, float4 loads and stores), so
// every such device buffer must start on a 16-byte boundary.  Null pointers
// (optional outputs) pass.
bool misaligned16(const void* a, const void* b = nullptr, const void* c = nullptr) {
  return (((uintptr_t)a | (uintptr_t)b | (uintptr_t)c) & 15u) != 0;
}

DopplerArgs doppler_args(const ofdm_radar_plan* pl, int frames) {
  DopplerArgs a;
  a.N = pl->p.N;
  a.Np = pl->Np;
  a.M = pl->p.M;
  a.Mp = pl->Mp;
  a.rows = pl->rows;
  a.row0 = pl->row0;
  a.frames = frames;
  a.inv_nm = (float)(1.0 / ((double)pl->p.N * (double)pl->p.M));
  a.wl = pl->d_wl;
  a.tw = pl->twM;
  a.map_off = nullptr;
  a.frame_mask = nullptr;
  return a;
}

DetectArgs detect_args(const ofdm_radar_plan* pl, int frames, int compact) {
  const ofdm_radar_params& p = pl->p;
  DetectArgs a;
  a.Np = pl->Np;
  a.Mp = pl->Mp;
  a.logMp = 0;
  while ((1 << a.logMp) < pl->Mp) ++a.logMp;
  a.rows = pl->rows;
  a.row0 = pl->row0;
  a.full = pl->full;
  a.compact = compact;
  a.out_idx = nullptr;
  a.frame_mask = nullptr;
  a.part_keys = pl->d_detkeys;
  a.tickets = pl->d_dettick;
  a.counts = pl->d_dettick + pl->p.max_frames;
  a.eta = pl->d_eta;
  a.frame_stride = compact ? (long)pl->rows * pl->Mp : (long)pl->Np * pl->Mp;
  a.frames = frames;
  a.mode = p.detect_mode;
  a.K = p.max_targets;
  a.use_fixed_eta = p.noise_var > 0.f ? 1 : 0;
  // eta = sigma^2 (-ln P_fa) (Eq. (18), reading of the garbled sign), in FP32.
  const float lnp = (float)(-log((double)p.pfa));
  a.eta_fixed = p.noise_var * lnp;
  a.eta_factor = (float)(-log((double)p.pfa) / log(2.0));
  const double c = 3.0e8;
  const int ncp = p.n_cp ? p.n_cp : p.L_cp;
  const double Ts = (double)(p.N + ncp) / ((double)p.N * p.df_hz);
  a.dd = (float)(c / (2.0 * pl->Np * p.df_hz));
  a.dv = (float)(c / (2.0 * p.fc_hz * pl->Mp * Ts));
  a.cfar_guard = p.cfar_guard;
  a.cfar_train = p.cfar_train;
  a.cfar_alpha = pl->d_alpha;
  return a;
}

void set_zero_rows(const ofdm_radar_plan* pl, float* map, const long long* map_off, DetectArgs* a) {
  if (!map || pl->nz <= 0) return;
  a->zmap = map;
  a->zmap_off = map_off;
  a->zframe = (long)pl->Np * pl->Mp;
  a->z_off = (long)pl->z0 * pl->Mp;
  a->z_floats = (long)pl->nz * pl->Mp;
}

bool bad_frames(const ofdm_radar_plan* pl, int frames) { return frames < 1 || frames > pl->p.max_frames; }

int finish(ofdm_radar_plan* pl, int launches, cudaError_t e) {
  if (e != cudaSuccess) return cuda_fail(e);
  pl->last_launches = launches;
  return OFDM_OK;
}

// Steps a1-a5 into `strip` ([frames][rows][M]): the column kernel, followed
// on a padded range grid by the full N'-row range transform of the kept taps.
cudaError_t run_column(ofdm_radar_plan* pl, const float2* Y, const float2* X, int frames, float2* strip,
                       cudaStream_t s, int* launches) {
  unsigned long long tk = 0;
  const bool padded = pl->Np > pl->p.N;
  cudaError_t e = ofdm::launch_column(pl->p.N, Y, X, padded ? pl->d_taps : strip, pl->d_wstatus,
                                      column_args(pl, frames), s, launches, &tk);
  pl->ctr_base[pl->ctr_slot] += tk;
  if (e != cudaSuccess || !padded) return e;
  ofdm::PadArgs pa;
  pa.M = pl->p.M;
  pa.L_cp = pl->p.L_cp;
  pa.frames = frames;
  pa.wk = pl->d_wk;
  pa.twN = pl->twPN;
  pa.twP = pl->twPP;
  return ofdm::launch_range_pad(pl->p.N, pl->Np, pl->d_taps, strip, pa, s, launches);
}

// The chain on device buffers; shared by the device and host entry points.
cudaError_t run_chain(ofdm_radar_plan* pl, const float2* Y, const float2* X, int frames, float* map,
                      ofdm_target* tg, int32_t* nt, uint32_t* st, cudaStream_t s, int* launches) {
  cudaError_t e;
  {
    ScopedTimer tm(pl, s, K_COLUMN);
    e = run_column(pl, Y, X, frames, pl->d_strip, s, launches);
  }
  if (e != cudaSuccess) return e;
  DetectArgs ta = detect_args(pl, frames, 1);
  set_zero_rows(pl, map, nullptr, &ta);   // the detection launch zeroes the rows outside the support
  if (pl->gen) {   // M' not a power of two
    {
      ScopedTimer tm(pl, s, K_DOPPLER);
      e = ofdm::launch_doppler_general(pl->d_strip, map, pl->d_pow, doppler_args(pl, frames), pl->twM, s, launches);
    }
    if (e != cudaSuccess) return e;
    ScopedTimer tm(pl, s, K_DETECT);
    return ofdm::launch_detect_general(pl->d_pow, tg, nt, st, pl->d_wstatus, ta, s, launches);
  }
  if (ofdm::doppler_detect_fusable(ta, pl->Mp)) {
    ScopedTimer tm(pl, s, K_DETECT);      // Doppler stage included
    return ofdm::launch_doppler_detect(pl->Mp, pl->d_strip, map, tg, nt, st, pl->d_wstatus, ta,
                                       doppler_args(pl, frames), s, launches);
  }
  {
    ScopedTimer tm(pl, s, K_DOPPLER);
    e = ofdm::launch_doppler(pl->Mp, pl->d_strip, map, pl->d_pow, doppler_args(pl, frames), s, launches);
  }
  if (e != cudaSuccess) return e;
  ScopedTimer tm(pl, s, K_DETECT);
  return ofdm::launch_detect(pl->d_pow, tg, nt, st, pl->d_wstatus, ta, s, launches);
}

}  // namespace

extern "C" {

int ofdm_radar_process(ofdm_radar_plan* pl, const ofdm_c32* Y, const ofdm_c32* X, int32_t frames,
                       float* out_map, ofdm_target* out_targets, int32_t* n_targets, uint32_t* status,
                       void* stream) {
  ofdm::NvtxRange nvtx_range("ofdm_radar_process");
  if (!pl || !Y || !X || bad_frames(pl, frames) || misaligned16(Y, X, out_map)) return OFDM_ERR_INVALID_ARG;
  int launches = 0;
  cudaError_t e = run_chain(pl, (const float2*)Y, (const float2*)X, frames, out_map, out_targets, n_targets,
                            status, (cudaStream_t)stream, &launches);
  return finish(pl, launches, e);
}

int ofdm_zc_precode(ofdm_radar_plan* pl, const ofdm_c32* in, ofdm_c32* out, int32_t frames, int32_t inverse,
                    void* stream) {
  ofdm::NvtxRange nvtx_range("ofdm_zc_precode");
  if (!pl || !in || !out || in == out || bad_frames(pl, frames) || misaligned16(in, out)) return OFDM_ERR_INVALID_ARG;
  if (pl->p.zc_root <= 0) return OFDM_ERR_INVALID_ARG;
  ZctArgs a;
  a.frames = frames;
  a.M = pl->p.M;
  a.rinv = pl->rinv;
  a.dir = inverse ? -1 : +1;
  a.scale = (float)(1.0 / sqrt((double)pl->p.N));
  a.in_tab = inverse ? pl->post_conj : pl->pre;
  a.out_tab = inverse ? pl->pre_conj : pl->post;
  a.tw = pl->twN;
  int launches = 0;
  cudaError_t e;
  {
    ScopedTimer tm(pl, (cudaStream_t)stream, K_ZCT);
    e = ofdm::launch_zct(pl->p.N, (const float2*)in, (float2*)out, a, (cudaStream_t)stream, &launches);
  }
  return finish(pl, launches, e);
}

int ofdm_radar_range_profile(ofdm_radar_plan* pl, const ofdm_c32* Y, const ofdm_c32* X, int32_t frames,
                             ofdm_c32* strip, void* stream) {
  ofdm::NvtxRange nvtx_range("ofdm_radar_range_profile");
  if (!pl || !Y || !X || !strip || bad_frames(pl, frames) || misaligned16(Y, X, strip)) return OFDM_ERR_INVALID_ARG;
  int launches = 0;
  cudaError_t e = run_column(pl, (const float2*)Y, (const float2*)X, frames, (float2*)strip, (cudaStream_t)stream,
                             &launches);
  // the status words of this call are not reported; clear them
  if (e == cudaSuccess)
    e = cudaMemsetAsync(pl->d_wstatus, 0, (size_t)frames * sizeof(uint32_t), (cudaStream_t)stream);
  return finish(pl, launches, e);
}

int ofdm_radar_doppler(ofdm_radar_plan* pl, const ofdm_c32* strip, int32_t frames, float* out_map,
                       void* stream) {
  ofdm::NvtxRange nvtx_range("ofdm_radar_doppler");
  if (!pl || !strip || !out_map || bad_frames(pl, frames) || misaligned16(strip, out_map)) return OFDM_ERR_INVALID_ARG;
  int launches = 0;
  cudaError_t e = ofdm::launch_zero_rows(out_map, frames, pl->Np, pl->Mp, pl->z0, pl->nz, (cudaStream_t)stream,
                                         &launches);
  if (e == cudaSuccess && pl->gen)
    e = ofdm::launch_doppler_general((const float2*)strip, out_map, nullptr, doppler_args(pl, frames), pl->twM,
                                     (cudaStream_t)stream, &launches);
  else if (e == cudaSuccess)
    e = ofdm::launch_doppler(pl->Mp, (const float2*)strip, out_map, pl->d_pow, doppler_args(pl, frames),
                             (cudaStream_t)stream, &launches);
  return finish(pl, launches, e);
}

int ofdm_radar_detect(ofdm_radar_plan* pl, const float* map, int32_t frames, ofdm_target* out_targets,
                      int32_t* n_targets, uint32_t* status, void* stream) {
  ofdm::NvtxRange nvtx_range("ofdm_radar_detect");
  if (!pl || !map || bad_frames(pl, frames) || misaligned16(map)) return OFDM_ERR_INVALID_ARG;
  int launches = 0;
  cudaError_t e = pl->gen ? ofdm::launch_detect_general(map, out_targets, n_targets, status, nullptr,
                                                        detect_args(pl, frames, 0), (cudaStream_t)stream, &launches)
                          : ofdm::launch_detect(map, out_targets, n_targets, status, nullptr,
                                                detect_args(pl, frames, 0), (cudaStream_t)stream, &launches);
  return finish(pl, launches, e);
}

int ofdm_radar_process_host(ofdm_radar_plan* pl, const ofdm_c32* Yh, const ofdm_c32* Xh, int32_t frames,
                            float* map_h, ofdm_target* tg_h, int32_t* nt_h, uint32_t* st_h, void* stream) {
  ofdm::NvtxRange nvtx_range("ofdm_radar_process_host");
  if (!pl || !Yh || !Xh || bad_frames(pl, frames)) return OFDM_ERR_INVALID_ARG;
  const ofdm_radar_params& p = pl->p;
  const size_t grid = (size_t)p.N * p.M, mapn = (size_t)pl->Np * pl->Mp;
  cudaError_t e = cudaSuccess;
  if (!pl->d_Y) {
    e = dalloc(&pl->d_Y, grid * p.max_frames);
    if (e == cudaSuccess) e = dalloc(&pl->d_X, grid * p.max_frames);
    if (e == cudaSuccess) e = dalloc(&pl->d_map, mapn * p.max_frames);
    if (e == cudaSuccess) e = dalloc(&pl->d_tg, (size_t)p.max_targets * p.max_frames);
    if (e == cudaSuccess) e = dalloc(&pl->d_nt, (size_t)p.max_frames);
    if (e == cudaSuccess) e = dalloc(&pl->d_st, (size_t)p.max_frames);
    for (int i = 0; i < 3 && e == cudaSuccess; ++i) e = cudaStreamCreateWithFlags(&pl->hs[i], cudaStreamNonBlocking);
    for (int i = 0; i < 2 + 2 * kHostChunks && e == cudaSuccess; ++i)
      e = cudaEventCreateWithFlags(&pl->ev[i], cudaEventDisableTiming);
    if (e != cudaSuccess) {
      dfree(pl->d_Y); pl->d_Y = nullptr;
      cudaGetLastError();
      return e == cudaErrorMemoryAllocation ? OFDM_ERR_NO_MEMORY : cuda_fail(e);
    }
  }
  // Three-stage pipeline over chunks of frames.  All uploads run back to back
  // on one stream (the host link is the bottleneck); chunk k's kernels start
  // when its upload is done, and its results go back on a third stream while
  // later chunks are still uploading or computing.
  cudaStream_t s0 = (cudaStream_t)stream, up = pl->hs[0], comp = pl->hs[1], down = pl->hs[2];
  cudaEvent_t* up_done = pl->ev + 2;
  cudaEvent_t* comp_done = pl->ev + 2 + kHostChunks;
  const int chunk = (frames + kHostChunks - 1) / kHostChunks;
  e = cudaEventRecord(pl->ev[0], s0);
  for (int i = 0; i < 3 && e == cudaSuccess; ++i) e = cudaStreamWaitEvent(pl->hs[i], pl->ev[0], 0);
  int launches = 0, k = 0;
  for (int f0 = 0; f0 < frames && e == cudaSuccess; f0 += chunk, ++k) {
    const int nf = frames - f0 < chunk ? frames - f0 : chunk;
    const size_t g0 = grid * f0, gn = grid * nf;
    e = cudaMemcpyAsync(pl->d_Y + g0, Yh + g0, gn * sizeof(float2), cudaMemcpyHostToDevice, up);
    if (e == cudaSuccess) e = cudaMemcpyAsync(pl->d_X + g0, Xh + g0, gn * sizeof(float2), cudaMemcpyHostToDevice, up);
    if (e == cudaSuccess) e = cudaEventRecord(up_done[k], up);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(comp, up_done[k], 0);
    if (e != cudaSuccess) break;
    // The chunk uses its own slice of the workspace (frame offset f0).
    ofdm_radar_plan view = *pl;
    view.ctr_slot = 1;
    view.d_strip = pl->d_strip + (size_t)f0 * pl->rows * p.M;
    view.d_pow = pl->d_pow + (size_t)f0 * pl->rows * pl->Mp;
    view.d_wstatus = pl->d_wstatus + f0;
    view.d_detkeys = pl->d_detkeys + (size_t)f0 * pl->det_bands * 32;
    view.d_dettick = pl->d_dettick + f0;  // tickets[f0..]; counts stay max_frames further on
    view.d_eta = pl->d_eta + f0;
    e = run_chain(&view, pl->d_Y + g0, pl->d_X + g0, nf, map_h ? pl->d_map + mapn * f0 : nullptr,
                  pl->d_tg + (size_t)p.max_targets * f0, pl->d_nt + f0, pl->d_st + f0, comp, &launches);
    pl->ctr_base[1] = view.ctr_base[1];
    if (e == cudaSuccess) e = cudaEventRecord(comp_done[k], comp);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(down, comp_done[k], 0);
    if (e != cudaSuccess) break;
    if (map_h)
      e = cudaMemcpyAsync(map_h + mapn * f0, pl->d_map + mapn * f0, mapn * nf * sizeof(float),
                          cudaMemcpyDeviceToHost, down);
    if (e == cudaSuccess && tg_h)
      e = cudaMemcpyAsync(tg_h + (size_t)p.max_targets * f0, pl->d_tg + (size_t)p.max_targets * f0,
                          (size_t)p.max_targets * nf * sizeof(ofdm_target), cudaMemcpyDeviceToHost, down);
    if (e == cudaSuccess && nt_h)
      e = cudaMemcpyAsync(nt_h + f0, pl->d_nt + f0, nf * sizeof(int32_t), cudaMemcpyDeviceToHost, down);
    if (e == cudaSuccess && st_h)
      e = cudaMemcpyAsync(st_h + f0, pl->d_st + f0, nf * sizeof(uint32_t), cudaMemcpyDeviceToHost, down);
  }
  // the downloads come last in every chunk's chain: joining them joins all three streams
  if (e == cudaSuccess) e = cudaEventRecord(pl->ev[1], down);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s0, pl->ev[1], 0);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s0);
  return finish(pl, launches, e);
}

}  // extern "C"

extern "C" {

void ofdm_fps_default_params(ofdm_fps_params* fp) {
  if (!fp) return;
  fp->iterations = 4;
  fp->offsets = 8;
  fp->max_recover = 32;
  fp->bin_pfa = 1e-6f;
  fp->coherence_min = 0.95f;
  fp->dynamic_range = 1e-10f;
}

int ofdm_fps_sft(ofdm_radar_plan* pl, const ofdm_c32* Y, const ofdm_c32* X, int32_t frames,
                 const ofdm_fps_params* fp, const int32_t* slices, ofdm_target* out_targets,
                 int32_t* n_targets, void* stream) {
  ofdm::NvtxRange nvtx_range("ofdm_fps_sft");
  if (!pl || !Y || !X || !fp || !slices || bad_frames(pl, frames) || misaligned16(Y, X))
    return OFDM_ERR_INVALID_ARG;
  const ofdm_radar_params& p = pl->p;
  const int N = p.N, M = p.M, Q = N > M ? N : M;
  if (Q > 1024 || pl->Mp != M || pl->Np != N || !is_pow2(M)) return OFDM_ERR_UNSUPPORTED_SIZE;
  if (fp->iterations < 1 || fp->iterations > 16 || fp->offsets < 3 || fp->offsets > 8 ||
      fp->max_recover < 1 || fp->max_recover > 64 || !(fp->bin_pfa > 0.f && fp->bin_pfa < 1.f) ||
      !(fp->coherence_min >= 0.f && fp->coherence_min <= 1.f) || !(fp->dynamic_range >= 0.f))
    return OFDM_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  // Slice workspace for max_frames frames of this (iterations, offsets).
  const size_t need = ofdm::fps_workspace_elems(p.max_frames, fp->iterations, fp->offsets, Q);
  if (need > pl->fps_elems) {
    cudaError_t ea = cudaStreamSynchronize(s);   // the old workspace may still be in use
    if (ea != cudaSuccess) return cuda_fail(ea);
    dfree(pl->d_fps);
    pl->d_fps = nullptr;
    pl->fps_elems = 0;
    ea = dalloc(&pl->d_fps, need);
    if (ea != cudaSuccess) {
      cudaGetLastError();
      return ea == cudaErrorMemoryAllocation ? OFDM_ERR_NO_MEMORY : cuda_fail(ea);
    }
    pl->fps_elems = need;
  }
  // F is cell-local when there is no precoding to undo and DFT-CE keeps every
  // tap (plain LS estimation): the samples then read only the sampled cells.
  const bool direct = (p.zc_root == 0 || p.x_is_precoded) && p.L_cp >= N;
  int launches = 0;
  cudaError_t e = cudaSuccess;
  if (direct) {
    e = cudaMemsetAsync(pl->d_wstatus, 0, (size_t)frames * sizeof(uint32_t), s);
  } else {
    // Column pass with a rect stencil: the strip then holds the kept taps N h[n].
    ColumnArgs ca = column_args(pl, frames);
    ca.rows = p.L_cp;
    ca.row0 = 0;
    ca.full = p.L_cp >= N ? 1 : 0;
    ca.c0 = 1.f;
    ca.c1 = 0.f;
    unsigned long long tk = 0;
    e = ofdm::launch_column(N, (const float2*)Y, (const float2*)X, pl->d_strip, pl->d_wstatus, ca, s, &launches,
                            &tk);
    pl->ctr_base[pl->ctr_slot] += tk;
  }
  if (e != cudaSuccess) return finish(pl, launches, e);
  ofdm::FpsArgs a;
  a.N = N; a.M = M; a.Q = Q; a.T = fp->offsets; a.rows = p.L_cp; a.iterations = fp->iterations; a.frames = frames;
  a.K = p.max_targets; a.max_recover = fp->max_recover;
  a.direct = direct ? 1 : 0;
  a.invN = (float)(1.0 / N);
  a.invNM = (float)(1.0 / ((double)N * M));
  a.NMoverQ = (float)((double)N * M / Q);
  a.median_factor = (float)(-log((double)fp->bin_pfa) / log(2.0));
  a.dynamic_range = fp->dynamic_range;
  a.coherence_min = fp->coherence_min;
  const DetectArgs d = detect_args(pl, frames, 1);
  a.dd = d.dd;
  a.dv = d.dv;
  a.w_df = pl->d_df + N;
  a.twQ = (Q == N) ? pl->twN : pl->twM;
  e = ofdm::launch_fps(Q, pl->d_strip, (const float2*)Y, (const float2*)X, slices, pl->d_fps, out_targets, n_targets,
                       pl->d_wstatus, a, s, &launches);
  return finish(pl, launches, e);
}

int ofdm_tx_amplifier(ofdm_radar_plan* pl, const ofdm_c32* S, int32_t frames, int32_t oversample, float q,
                      float* papr, float* aci, void* stream) {
  ofdm::NvtxRange nvtx_range("ofdm_tx_amplifier");
  if (!pl || !S || bad_frames(pl, frames) || !(q > -100.f && q < 100.f) || misaligned16(S)) return OFDM_ERR_INVALID_ARG;
  const int N = pl->p.N, LN = N * oversample;
  if (oversample < 1 || oversample > 8 || (oversample & (oversample - 1)) || LN > 4096)
    return OFDM_ERR_UNSUPPORTED_SIZE;
  cudaStream_t s = (cudaStream_t)stream;
  if (pl->twL_n != LN) {   // twiddles of the L N-point transforms, built once per size
    std::vector<float2> tw;
    build_twiddles(tw, LN, ofdm::tx_points_per_thread(LN));
    cudaError_t e = cudaStreamSynchronize(s);   // the previous table may still be in use
    if (e == cudaSuccess) {
      dfree(pl->d_twL);
      pl->d_twL = nullptr;
      pl->twL_n = 0;
      e = dalloc(&pl->d_twL, tw.size());
    }
    if (e == cudaSuccess) e = cudaMemcpy(pl->d_twL, tw.data(), tw.size() * sizeof(float2), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return e == cudaErrorMemoryAllocation ? OFDM_ERR_NO_MEMORY : cuda_fail(e);
    }
    pl->twL_n = LN;
  }
  ofdm::TxArgs a;
  a.N = N;
  a.M = pl->p.M;
  a.frames = frames;
  a.sat_factor = (float)pow(10.0, (double)q / 10.0);
  a.tw = pl->d_twL;
  int launches = 0;
  cudaError_t e = ofdm::launch_tx(LN, (const float2*)S, papr, aci, a, s, &launches);
  return finish(pl, launches, e);
}

}  // extern "C"

// ---------------------------------------------------------------- batches of uneven frames

namespace {

struct BatchGroup {
  ofdm_radar_plan* plan = nullptr;
  int N = 0, M = 0, L_cp = 0, n = 0;
  long long* d_frame_off = nullptr;  // Y / X offsets of the group's frames
  long long* d_map_off = nullptr;    // map offsets
  int* d_idx = nullptr;              // position of each frame in the caller's desc array
  int pipe_warps = -1;               // tuned column-kernel variant (-1: not tuned)
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
};

// Process-wide tuning results: (N, M, L_cp) -> column-kernel variant.
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int>, int> g_tune;

}  // namespace

struct ofdm_radar_batch {
  ofdm_radar_params base;
  int nframes = 0;
  uint32_t flags = 0;
  std::vector<BatchGroup> groups;
  cudaEvent_t fork = nullptr;
  bool tuned = false;
  bool have_graph = false;
  bool used_graph = false;
  cudaGraphExec_t exec = nullptr;
  const void* key[7] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
};

namespace {

// One group's chain on `s`.  Inside a graph the ticket counter is reset by a
// memset node (a replay reuses the captured kernel arguments).
cudaError_t run_group(BatchGroup& g, const float2* Y, const float2* X, float* map, ofdm_target* tg, int32_t* nt,
                      uint32_t* st, cudaStream_t s, int pipe_warps, int* launches) {
  ofdm_radar_plan* pl = g.plan;
  cudaError_t e = cudaMemsetAsync(pl->d_ctr, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  ColumnArgs ca = column_args(pl, g.n);
  ca.work_base = 0;
  ca.frame_off = g.d_frame_off;
  if (pipe_warps >= 0) ca.pipe_warps = pipe_warps;   // else the plan's default
  unsigned long long tk = 0;
  e = ofdm::launch_column(g.N, Y, X, pl->d_strip, pl->d_wstatus, ca, s, launches, &tk);
  if (e != cudaSuccess) return e;
  DopplerArgs da = doppler_args(pl, g.n);
  da.map_off = g.d_map_off;
  DetectArgs ta = detect_args(pl, g.n, 1);
  ta.out_idx = g.d_idx;
  set_zero_rows(pl, map, g.d_map_off, &ta);
  if (ofdm::doppler_detect_fusable(ta, pl->Mp))
    return ofdm::launch_doppler_detect(pl->Mp, pl->d_strip, map, tg, nt, st, pl->d_wstatus, ta, da, s, launches);
  e = ofdm::launch_doppler(pl->Mp, pl->d_strip, map, pl->d_pow, da, s, launches);
  if (e != cudaSuccess) return e;
  return ofdm::launch_detect(pl->d_pow, tg, nt, st, pl->d_wstatus, ta, s, launches);
}

// Time the column kernel variants of one group on the caller's inputs.
cudaError_t tune_group(BatchGroup& g, const float2* Y, const float2* X, cudaStream_t s) {
  const auto key = std::make_tuple(g.N, g.M, g.L_cp);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) { g.pipe_warps = it->second; return cudaSuccess; }
  }
  // N <= 1024: the widest one-warp CTA, 4-warp CTAs, or (N = 1024) groups of
  // N / 16 threads; N >= 2048: groups of N / 16 threads with 16 points each
  // or of N / 32 threads with 32 points each (points per thread, and with
  // them the FFT's pass radices, exchanges and registers).
  const int small_variants[3] = {0, 4, 2}, big_variants[2] = {2, 0};
  const bool big = g.N > 1024;
  const int* variants = big ? big_variants : small_variants;
  const int nvar = big ? 2 : (g.plan->twG ? 3 : 2);
  float best = 1e30f;
  int pick = 0;
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  for (int v = 0; v < nvar && e == cudaSuccess; ++v) {
    float ms = 0.f;
    for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
      int launches = 0;
      unsigned long long tk = 0;
      ColumnArgs ca = column_args(g.plan, g.n);
      ca.frame_off = g.d_frame_off;
      ca.pipe_warps = variants[v];
      e = cudaEventRecord(e0, s);
      if (e == cudaSuccess) e = ofdm::launch_column(g.N, Y, X, g.plan->d_strip, g.plan->d_wstatus, ca, s, &launches, &tk);
      g.plan->ctr_base[0] += tk;
      if (e == cudaSuccess) e = cudaEventRecord(e1, s);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      if (e == cudaSuccess && rep > 0) {  // the first run warms up
        float t = 0.f;
        e = cudaEventElapsedTime(&t, e0, e1);
        ms += t;
      }
    }
    if (e == cudaSuccess && ms < best) { best = ms; pick = variants[v]; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  // the tuning runs' status words are not reported
  if (e == cudaSuccess) e = cudaMemsetAsync(g.plan->d_wstatus, 0, (size_t)g.n * sizeof(uint32_t), s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return e;
  g.pipe_warps = pick;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune[key] = pick;
  return cudaSuccess;
}

bool valid_shape(int N, int M, int L) {
  return is_pow2(N) && N >= 64 && N <= 4096 && is_pow2(M) && M >= 16 && M <= 1024 && L >= 1 && L <= N;
}

}  // namespace

extern "C" {

void ofdm_radar_batch_destroy(ofdm_radar_batch* b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  for (auto& g : b->groups) {
    ofdm_radar_plan_destroy(g.plan);
    dfree(g.d_frame_off);
    dfree(g.d_map_off);
    dfree(g.d_idx);
    if (g.stream) cudaStreamDestroy(g.stream);
    if (g.done) cudaEventDestroy(g.done);
  }
  if (b->fork) cudaEventDestroy(b->fork);
  delete b;
}

int ofdm_radar_batch_create(const ofdm_radar_params* base, const ofdm_frame_desc* desc, int32_t nframes,
                            uint32_t flags, ofdm_radar_batch** out) {
  if (!base || !desc || !out || nframes < 1) return OFDM_ERR_INVALID_ARG;
  *out = nullptr;
  for (int f = 0; f < nframes; ++f) {
    if (!valid_shape(desc[f].N, desc[f].M, desc[f].L_cp)) return OFDM_ERR_UNSUPPORTED_SIZE;
    if (desc[f].yx_offset < 0 || (desc[f].yx_offset & 1) || desc[f].map_offset < 0 || (desc[f].map_offset & 3))
      return OFDM_ERR_INVALID_ARG;
  }
  ofdm_radar_batch* b = new ofdm_radar_batch();
  b->base = *base;
  b->nframes = nframes;
  b->flags = flags;
  std::vector<std::vector<int>> members;
  for (int f = 0; f < nframes; ++f) {
    size_t gi = 0;
    while (gi < b->groups.size() && !(b->groups[gi].N == desc[f].N && b->groups[gi].M == desc[f].M &&
                                      b->groups[gi].L_cp == desc[f].L_cp))
      ++gi;
    if (gi == b->groups.size()) {
      BatchGroup g;
      g.N = desc[f].N; g.M = desc[f].M; g.L_cp = desc[f].L_cp;
      b->groups.push_back(g);
      members.emplace_back();
    }
    members[gi].push_back(f);
  }
  int rc = OFDM_OK;
  cudaError_t e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
  for (size_t gi = 0; gi < b->groups.size() && rc == OFDM_OK && e == cudaSuccess; ++gi) {
    BatchGroup& g = b->groups[gi];
    g.n = (int)members[gi].size();
    ofdm_radar_params p = *base;
    p.N = g.N; p.M = g.M; p.L_cp = g.L_cp; p.N_pad = 0; p.M_pad = 0; p.max_frames = g.n;
    rc = ofdm_radar_plan_create(&p, &g.plan);
    if (rc != OFDM_OK) break;
    std::vector<long long> fo(g.n), mo(g.n);
    std::vector<int> idx(g.n);
    for (int i = 0; i < g.n; ++i) {
      const ofdm_frame_desc& d = desc[members[gi][i]];
      fo[i] = d.yx_offset;
      mo[i] = d.map_offset;
      idx[i] = members[gi][i];
    }
    e = dalloc(&g.d_frame_off, (size_t)g.n);
    if (e == cudaSuccess) e = dalloc(&g.d_map_off, (size_t)g.n);
    if (e == cudaSuccess) e = dalloc(&g.d_idx, (size_t)g.n);
    if (e == cudaSuccess) e = cudaMemcpy(g.d_frame_off, fo.data(), g.n * sizeof(long long), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(g.d_map_off, mo.data(), g.n * sizeof(long long), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(g.d_idx, idx.data(), g.n * sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&g.stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g.done, cudaEventDisableTiming);
  }
  if (rc == OFDM_OK && e != cudaSuccess) rc = e == cudaErrorMemoryAllocation ? OFDM_ERR_NO_MEMORY : cuda_fail(e);
  if (rc != OFDM_OK) {
    ofdm_radar_batch_destroy(b);
    cudaGetLastError();
    return rc;
  }
  *out = b;
  return OFDM_OK;
}

int ofdm_radar_batch_groups(const ofdm_radar_batch* b, int32_t* shapes) {
  if (!b) return OFDM_ERR_INVALID_ARG;
  if (shapes)
    for (size_t i = 0; i < b->groups.size(); ++i) {
      const BatchGroup& g = b->groups[i];
      const int32_t row[5] = {g.N, g.M, g.L_cp, g.n, g.pipe_warps};
      for (int k = 0; k < 5; ++k) shapes[5 * i + k] = row[k];
    }
  return (int)b->groups.size();
}

int ofdm_radar_batch_used_graph(const ofdm_radar_batch* b) { return b ? (b->used_graph ? 1 : 0) : OFDM_ERR_INVALID_ARG; }

int ofdm_radar_batch_process(ofdm_radar_batch* b, const ofdm_c32* Yc, const ofdm_c32* Xc, float* map,
                             ofdm_target* tg, int32_t* nt, uint32_t* st, void* stream) {
  ofdm::NvtxRange nvtx_range("ofdm_radar_batch_process");
  if (!b || !Yc || !Xc || misaligned16(Yc, Xc, map)) return OFDM_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const float2* Y = (const float2*)Yc;
  const float2* X = (const float2*)Xc;
  cudaError_t e = cudaSuccess;
  if (!b->tuned) {
    for (auto& g : b->groups) {
      if (b->flags & OFDM_BATCH_NO_TUNE) { g.pipe_warps = -1; continue; }
      e = tune_group(g, Y, X, s);
      if (e != cudaSuccess) return cuda_fail(e);
    }
    b->tuned = true;
  }
  int launches = 0;
  auto launch_all = [&](cudaStream_t main) -> cudaError_t {
    cudaError_t r = cudaEventRecord(b->fork, main);
    for (auto& g : b->groups) {
      if (r == cudaSuccess) r = cudaStreamWaitEvent(g.stream, b->fork, 0);
      if (r == cudaSuccess) r = run_group(g, Y, X, map, tg, nt, st, g.stream, g.pipe_warps, &launches);
      if (r == cudaSuccess) r = cudaEventRecord(g.done, g.stream);
      if (r == cudaSuccess) r = cudaStreamWaitEvent(main, g.done, 0);
    }
    return r;
  };
  const void* key[7] = {Y, X, map, tg, nt, st, stream};
  const bool graph_ok = !(b->flags & OFDM_BATCH_NO_GRAPH) && s != nullptr;
  if (graph_ok && b->have_graph && memcmp(key, b->key, sizeof key) == 0) {
    e = cudaGraphLaunch(b->exec, s);
    b->used_graph = true;
    return e == cudaSuccess ? OFDM_OK : cuda_fail(e);
  }
  if (graph_ok) {
    cudaGraph_t graph = nullptr;
    e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaError_t r = launch_all(s);
      e = cudaStreamEndCapture(s, &graph);
      if (r != cudaSuccess) e = r;
    }
    if (e == cudaSuccess) {
      if (b->exec) cudaGraphExecDestroy(b->exec);
      b->exec = nullptr;
      e = cudaGraphInstantiate(&b->exec, graph, 0);
    }
    if (graph) cudaGraphDestroy(graph);
    if (e == cudaSuccess) {
      memcpy(b->key, key, sizeof key);
      b->have_graph = true;
      e = cudaGraphLaunch(b->exec, s);
      b->used_graph = true;
      return e == cudaSuccess ? OFDM_OK : cuda_fail(e);
    }
    cudaGetLastError();  // capture failed: launch directly below
    b->have_graph = false;
  }
  b->used_graph = false;
  e = launch_all(s);
  return e == cudaSuccess ? OFDM_OK : cuda_fail(e);
}

}  // extern "C"

// ---------------------------------------------------------------- learned proposal
extern "C" {

int ofdm_radar_learned_prepare(ofdm_radar_plan* pl) {
  if (!pl) return OFDM_ERR_INVALID_ARG;
  const ofdm_radar_params& p = pl->p;
  if (!(p.M == 256 || p.M == 512 || p.M == 1024) || pl->Mp != p.M || pl->full) return OFDM_ERR_UNSUPPORTED_SIZE;
  if (pl->d_cpow) return OFDM_OK;
  pl->Mc = p.M / 4;
  pl->Hc = (pl->rows + 3) / 4;
  const size_t cells = (size_t)p.max_frames * pl->Hc * pl->Mc;
  std::vector<float2> tw;
  build_twiddles(tw, pl->Mc, pl->Mc / 32);
  std::vector<float> w4(pl->Mc);
  for (int l = 0; l < pl->Mc; ++l) {
    const double c = cos(2.0 * M_PI * l / pl->Mc);
    w4[l] = p.window == OFDM_WINDOW_HANN ? (float)(0.5 - 0.5 * c)
          : p.window == OFDM_WINDOW_HAMMING ? (float)(0.54 - 0.46 * c) : 1.f;
  }
  cudaError_t e = dalloc(&pl->d_cpow, cells);
  if (e == cudaSuccess) e = dalloc(&pl->d_cx, cells);
  if (e == cudaSuccess) e = dalloc(&pl->d_a1, 16 * cells);
  if (e == cudaSuccess) e = dalloc(&pl->d_a2, 16 * cells);
  if (e == cudaSuccess) e = dalloc(&pl->d_logit, cells);
  if (e == cudaSuccess) e = dalloc(&pl->d_w4, (size_t)pl->Mc);
  if (e == cudaSuccess) e = dalloc(&pl->d_twMc, tw.size());
  if (e == cudaSuccess) e = dalloc(&pl->d_mask, (size_t)p.max_frames);
  if (e == cudaSuccess) e = dalloc(&pl->d_cand, (size_t)p.max_frames * 256);
  if (e == cudaSuccess) e = dalloc(&pl->d_ncand, (size_t)p.max_frames);
  if (e == cudaSuccess) e = dalloc(&pl->d_keys, (size_t)p.max_frames * 256 * 36);
  if (e == cudaSuccess) e = cudaMemcpy(pl->d_w4, w4.data(), w4.size() * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(pl->d_twMc, tw.data(), tw.size() * sizeof(float2), cudaMemcpyHostToDevice);
  std::vector<float2> roots(p.M);
  for (int m = 0; m < p.M; ++m) {
    const double a = 2.0 * M_PI * m / p.M;
    roots[m] = make_float2((float)cos(a), (float)-sin(a));
  }
  if (e == cudaSuccess) e = dalloc(&pl->d_rootsM, (size_t)p.M);
  if (e == cudaSuccess) e = cudaMemcpy(pl->d_rootsM, roots.data(), roots.size() * sizeof(float2), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? OFDM_ERR_NO_MEMORY : cuda_fail(e);
  }
  return OFDM_OK;
}

int ofdm_radar_coarse_shape(const ofdm_radar_plan* pl, int32_t* h, int32_t* w) {
  if (!pl || !pl->d_cpow) return OFDM_ERR_INVALID_ARG;
  if (h) *h = pl->Hc;
  if (w) *w = pl->Mc;
  return OFDM_OK;
}

int ofdm_radar_coarse_map(ofdm_radar_plan* pl, const ofdm_c32* Y, const ofdm_c32* X, int32_t frames, float* x_out,
                          void* stream) {
  ofdm::NvtxRange nvtx_range("ofdm_radar_coarse_map");
  if (!pl || !Y || !X || !pl->d_cpow || bad_frames(pl, frames) || misaligned16(Y, X)) return OFDM_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  int launches = 0;
  unsigned long long tk = 0;
  cudaError_t e = ofdm::launch_column(pl->p.N, (const float2*)Y, (const float2*)X, pl->d_strip, pl->d_wstatus,
                                      column_args(pl, frames), s, &launches, &tk);
  pl->ctr_base[pl->ctr_slot] += tk;
  if (e == cudaSuccess)
    e = ofdm::launch_coarse(pl->d_strip, pl->d_cpow, x_out ? x_out : pl->d_cx, pl->rows, pl->p.M, frames, pl->d_w4,
                            pl->d_twMc, s, &launches);
  // status words of this call are not reported
  if (e == cudaSuccess) e = cudaMemsetAsync(pl->d_wstatus, 0, (size_t)frames * sizeof(uint32_t), s);
  return finish(pl, launches, e);
}

int ofdm_radar_process_learned(ofdm_radar_plan* pl, const float* theta, const ofdm_c32* Y, const ofdm_c32* X,
                               int32_t frames, float zthr, int32_t cap, ofdm_target* out, int32_t* nt,
                               uint32_t* st, void* stream) {
  ofdm::NvtxRange nvtx_range("ofdm_radar_process_learned");
  if (!pl || !theta || !Y || !X || !pl->d_cpow || bad_frames(pl, frames) || cap < 1 || cap > 256 ||
      misaligned16(Y, X))
    return OFDM_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  int launches = 0;
  unsigned long long tk = 0;
  cudaError_t e;
  {
    ScopedTimer tm(pl, s, K_COLUMN);
    e = ofdm::launch_column(pl->p.N, (const float2*)Y, (const float2*)X, pl->d_strip, pl->d_wstatus,
                            column_args(pl, frames), s, &launches, &tk);
    pl->ctr_base[pl->ctr_slot] += tk;
  }
  if (e == cudaSuccess) {
    ScopedTimer tm(pl, s, K_COARSE);
    e = ofdm::launch_coarse(pl->d_strip, pl->d_cpow, pl->d_cx, pl->rows, pl->p.M, frames, pl->d_w4, pl->d_twMc, s,
                            &launches);
  }
  if (e == cudaSuccess) {
    ScopedTimer tm(pl, s, K_CNN);
    e = ofdm::cnn_forward(theta, 1, pl->d_cx, frames, pl->Hc, pl->Mc, pl->d_a1, pl->d_a2, pl->d_logit, s);
    launches += 3;
  }
  if (e != cudaSuccess) return finish(pl, launches, e);
  ofdm::RefineArgs ra;
  const DetectArgs da = detect_args(pl, frames, 1);
  ra.N = pl->p.N; ra.M = pl->p.M; ra.rows = pl->rows; ra.row0 = pl->row0; ra.Hc = pl->Hc; ra.Mc = pl->Mc;
  ra.frames = frames; ra.K = pl->p.max_targets; ra.cap = cap; ra.zthr = zthr;
  ra.inv_nm = (float)(1.0 / ((double)pl->p.N * pl->p.M));
  ra.dd = da.dd; ra.dv = da.dv; ra.wl = pl->d_wl; ra.rootsM = pl->d_rootsM;
  {
    ScopedTimer tm(pl, s, K_REFINE);
    e = ofdm::launch_refine(pl->d_strip, pl->d_logit, out, nt, st, pl->d_wstatus, pl->d_mask, pl->d_cand,
                            pl->d_ncand, pl->d_keys, ra, s, &launches);
  }
  // fallback: the full Doppler stage and detection on the flagged frames only,
  // through the same kernels as ofdm_radar_process (so the outputs are equal)
  DopplerArgs dop = doppler_args(pl, frames);
  dop.frame_mask = pl->d_mask;
  DetectArgs det = detect_args(pl, frames, 1);
  det.frame_mask = pl->d_mask;
  if (e == cudaSuccess && ofdm::doppler_detect_fusable(det, pl->Mp)) {
    ScopedTimer tm(pl, s, K_DETECT);
    e = ofdm::launch_doppler_detect(pl->Mp, pl->d_strip, nullptr, out, nt, st, pl->d_wstatus, det, dop, s,
                                    &launches);
  } else {
    if (e == cudaSuccess) {
      ScopedTimer tm(pl, s, K_DOPPLER);
      e = ofdm::launch_doppler(pl->Mp, pl->d_strip, nullptr, pl->d_pow, dop, s, &launches);
    }
    if (e == cudaSuccess) {
      ScopedTimer tm(pl, s, K_DETECT);
      e = ofdm::launch_detect(pl->d_pow, out, nt, st, pl->d_wstatus, det, s, &launches);
    }
  }
  if (e == cudaSuccess) e = mark_fallback(pl->d_mask, st, frames, s);
  return finish(pl, launches, e);
}

}  // extern "C"
