// noalloc.cu -- ofdm_radar_process_noalloc: the whole receive chain without
// any device allocation, for callers that cannot call cudaMalloc (for
// example code running under an allocator owned by someone else, inside a
// memory-capped sandbox, or in a process whose device memory is fully
// committed up front).  Tables and workspace live in one file-scope
// __device__ array of fixed size, loaded with the library; the caller still
// passes every input and output buffer.
//
// The array is shared by every call on a device and keeps the last call's
// contents: the per-frame status words, the column kernel's ticket counter
// and the detection's per-frame tickets and counts are cleared on the
// caller's stream at the start of each call, so no call depends on what an
// earlier one left behind, and the tables are regenerated (by a kernel on the
// caller's stream) whenever the parameters differ from the previous call's on
// that device.
// Calls that overlap on the GPU -- on two streams, or from two host threads
// -- race on the array.  The first call on a device looks up the array's
// device address with cudaGetSymbolAddress; make that first call before any
// stream capture.
#include <math.h>
#include <string.h>

#include <mutex>

#include "fft.cuh"
#include "internal.h"

namespace ofdm {
namespace {

constexpr int kNoallocMaxCells = 1 << 20;    // frames * support rows * M' (and * M)
constexpr int kNoallocMaxFrames = 4096;
constexpr int kMaxN = 4096, kMaxM = 1024;
constexpr float kNoallocRefineTau = 5e-5f;   // same threshold as the plan path

// Byte layout of the scratch array (every region 256-byte aligned).
constexpr size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }
constexpr size_t kOffPre = 0;                                          // float2[N] x 4 tables
constexpr size_t kOffDf = align256(kOffPre + 4 * kMaxN * sizeof(float2));   // float4[2N]
constexpr size_t kOffTwN = align256(kOffDf + 2 * kMaxN * sizeof(float4));   // float2[tw_size(N)+1]
constexpr size_t kOffTwM = align256(kOffTwN + 2 * kMaxN * sizeof(float2));  // float2[tw_size(M')+1]
constexpr size_t kOffWl = align256(kOffTwM + 2 * kMaxM * sizeof(float2));   // float[M]
constexpr size_t kOffStatus = align256(kOffWl + kMaxM * sizeof(float));     // uint32[frames]
constexpr size_t kOffStrip = align256(kOffStatus + kNoallocMaxFrames * sizeof(uint32_t));
constexpr size_t kOffPow = align256(kOffStrip + (size_t)kNoallocMaxCells * sizeof(float2));
constexpr size_t kOffCtr = align256(kOffPow + (size_t)kNoallocMaxCells * sizeof(float));  // ticket counter
// detection workspace: frames * bands <= 2^20 / kDetBandCells + frames (see detect_bands)
constexpr size_t kMaxBandSlots = (kNoallocMaxCells / kDetBandCells) + kNoallocMaxFrames;
constexpr size_t kOffDetKeys = align256(kOffCtr + sizeof(unsigned long long));
constexpr size_t kOffDetTick = align256(kOffDetKeys + kMaxBandSlots * 32 * sizeof(uint64_t));
constexpr size_t kOffEta = align256(kOffDetTick + 2 * kNoallocMaxFrames * sizeof(unsigned));
constexpr size_t kScratchBytes = align256(kOffEta + kNoallocMaxFrames * sizeof(float));

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

struct TableArgs {
  int N, M, Mp, eN, window;
  long long zc_root, zc_q;
};

// exp(i pi m / half) in double from an exact integer phase index.
__device__ void unit_phase_d(long long m, long long half, double* c, double* s) { sincospi((double)m / (double)half, s, c); }

__device__ float4 df_pair(double c, double s) {
  const float ch = (float)c, sh = (float)s;
  return make_float4(ch, (float)(c - (double)ch), sh, (float)(s - (double)sh));
}

// One thread per table entry: the same FP64 definitions as the plan's host
// tables (ZC chirps from exact int64 phases, Stockham pass twiddles, roots of
// unity, the window over l), rounded once to float.
__global__ void noalloc_tables_kernel(unsigned char* base, TableArgs t) {
  const int N = t.N;
  const long long NN = (long long)N * N, two = 2 * NN;
  float2* pre = reinterpret_cast<float2*>(base + kOffPre);
  float2* post = pre + N;
  float2* prec = post + N;
  float2* postc = prec + N;
  float4* df = reinterpret_cast<float4*>(base + kOffDf);
  float2* twN = reinterpret_cast<float2*>(base + kOffTwN);
  float2* twM = reinterpret_cast<float2*>(base + kOffTwM);
  float* wl = reinterpret_cast<float*>(base + kOffWl);
  const long long rr = ((t.zc_root % two) + two) % two, qq = ((t.zc_q % two) + two) % two;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double c, s;
  if (i < N) {
    const long long j = i;
    const long long b = ((j * j) % two + ((2 * qq) % two) * j % two) % two;
    unit_phase_d((rr * b) % two, NN, &c, &s);
    pre[i] = make_float2((float)c, (float)s);
    prec[i] = make_float2((float)c, -(float)s);
    df[i] = df_pair(c, s);
    const long long bp = ((long long)(i & 1) * NN + ((2 * qq) % two) * ((j * N) % two) % two) % two;
    unit_phase_d((rr * bp) % two, NN, &c, &s);
    post[i] = make_float2((float)c, (float)s);
    postc[i] = make_float2((float)c, -(float)s);
    unit_phase_d(2 * j, N, &c, &s);  // exp(+2 pi i j / N)
    df[N + i] = df_pair(c, s);
  }
  // Stockham pass twiddles: tab[off(p) + r Ns + u] = exp(+2 pi i u r / (Ns R)).
  auto pass_tw = [&](float2* tab, int n, int e, int idx) {
    const int np = num_passes(n, e);
    if (idx >= tw_size(n, e) + 1) return;
    float2 v = make_float2(1.f, 0.f);
    for (int p = 1; p < np; ++p) {
      const int R = pass_radix(n, e, p), NS = pass_ns(n, e, p), off = tw_offset(n, e, p);
      if (idx >= off && idx < off + NS * R) {
        const int r = (idx - off) / NS, u = (idx - off) % NS;
        const long long span = (long long)NS * R;
        double cc, ss;
        sincospi(2.0 * (double)(((long long)u * r) % span) / (double)span, &ss, &cc);
        v = make_float2((float)cc, (float)ss);
      }
    }
    tab[idx] = v;
  };
  pass_tw(twN, N, t.eN, i);
  if (t.Mp <= 32) {
    if (i < t.Mp) {
      sincospi(2.0 * i / t.Mp, &s, &c);
      twM[i] = make_float2((float)c, (float)s);
    }
  } else {
    pass_tw(twM, t.Mp, t.Mp / 32, i);
  }
  if (i < t.M) {
    const double cw = cospi(2.0 * i / t.M);
    wl[i] = t.window == OFDM_WINDOW_HANN ? (float)(0.5 - 0.5 * cw)
          : t.window == OFDM_WINDOW_HAMMING ? (float)(0.54 - 0.46 * cw) : 1.f;
  }
}

bool is_pow2(long v) { return v > 0 && (v & (v - 1)) == 0; }

int validate(const ofdm_radar_params& p) {
  const int N = p.N, M = p.M, Np = p.N_pad ? p.N_pad : N, Mp = p.M_pad ? p.M_pad : M;
  if (!is_pow2(N) || N < 64 || N > kMaxN) return OFDM_ERR_UNSUPPORTED_SIZE;
  if (!is_pow2(M) || M < 16 || M > kMaxM) return OFDM_ERR_UNSUPPORTED_SIZE;
  if (Np != N) return OFDM_ERR_UNSUPPORTED_SIZE;
  if (!is_pow2(Mp) || Mp < M || Mp > kMaxM) return OFDM_ERR_UNSUPPORTED_SIZE;
  if (p.L_cp < 1 || p.L_cp > N || p.n_cp < 0) return OFDM_ERR_INVALID_ARG;
  if (p.zc_root < 0 || (p.zc_root > 0 && (p.zc_root % 2) == 0)) return OFDM_ERR_INVALID_ARG;
  if (p.window < OFDM_WINDOW_RECT || p.window > OFDM_WINDOW_HAMMING) return OFDM_ERR_INVALID_ARG;
  if (p.detect_mode == OFDM_DETECT_CFAR) return OFDM_ERR_UNSUPPORTED_SIZE;   // no alpha table in the array
  if (p.detect_mode != OFDM_DETECT_TOPK && p.detect_mode != OFDM_DETECT_THRESHOLD) return OFDM_ERR_INVALID_ARG;
  if (p.max_targets < 1 || p.max_targets > 32) return OFDM_ERR_INVALID_ARG;
  if (p.precision != OFDM_PREC_FP32) return OFDM_ERR_UNSUPPORTED_SIZE;
  if (!(p.pfa > 0.f && p.pfa < 1.f) || !(p.fc_hz > 0.0 && p.df_hz > 0.0)) return OFDM_ERR_INVALID_ARG;
  return OFDM_OK;
}

}  // namespace
}  // namespace ofdm

namespace ofdm {
namespace {

struct DeviceState {
  bool ready = false;
  unsigned char* base = nullptr;  // device address of g_noalloc_scratch
  bool have_tables = false;
  ofdm_radar_params tables_for;   // parameters the tables in the array were built for
};
constexpr int kMaxDevices = 64;
DeviceState g_dev[kMaxDevices];
std::mutex g_mu;

bool same_tables(const ofdm_radar_params& a, const ofdm_radar_params& b) {
  return a.N == b.N && a.M == b.M && a.M_pad == b.M_pad && a.zc_root == b.zc_root && a.zc_q == b.zc_q &&
         a.window == b.window;
}

}  // namespace
}  // namespace ofdm

extern "C" int ofdm_radar_process_noalloc(const ofdm_radar_params* pin, const ofdm_c32* Y, const ofdm_c32* X,
                                          int32_t frames, float* out_map, ofdm_target* out_targets,
                                          int32_t* n_targets, uint32_t* status, void* stream) {
  using namespace ofdm;
  if (!pin || !Y || !X || (((uintptr_t)Y | (uintptr_t)X | (uintptr_t)out_map) & 15u)) return OFDM_ERR_INVALID_ARG;
  const ofdm_radar_params& p = *pin;
  int rc = validate(p);
  if (rc != OFDM_OK) return rc;
  const int N = p.N, M = p.M, Mp = p.M_pad ? p.M_pad : M;
  const int spread = p.window == OFDM_WINDOW_RECT ? 0 : 2;
  const int full = (p.L_cp + spread >= N) ? 1 : 0;
  const int rows = full ? N : p.L_cp + spread;
  const int row0 = (full || !spread) ? 0 : N - 1;
  if (frames < 1) return OFDM_ERR_INVALID_ARG;
  if (frames > kNoallocMaxFrames) return OFDM_ERR_UNSUPPORTED_SIZE;  // beyond the fixed scratch array
  const long cells = (long)frames * rows * (Mp > M ? Mp : M);
  if (cells > kNoallocMaxCells) return OFDM_ERR_UNSUPPORTED_SIZE;  // beyond the fixed scratch array

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return OFDM_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return OFDM_ERR_UNSUPPORTED_SIZE;
  cudaStream_t s = (cudaStream_t)stream;
  std::lock_guard<std::mutex> lock(g_mu);
  DeviceState& st = g_dev[dev];
  if (!st.ready) {
    // One-time set-up on this device (the current one): the array's device
    // address.  Host code must not pass g_noalloc_scratch itself to a kernel.
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess || ptr == nullptr) return OFDM_ERR_CUDA;
    st.base = static_cast<unsigned char*>(ptr);
    st.ready = true;
  }
  int launches = 0;
  if (!st.have_tables || !same_tables(st.tables_for, p)) {
    TableArgs t;
    t.N = N; t.M = M; t.Mp = Mp; t.eN = N <= 1024 ? N / 32 : 32; t.window = p.window;
    t.zc_root = p.zc_root > 0 ? p.zc_root : 1;
    t.zc_q = p.zc_q;
    const int span = 2 * kMaxN + 1;
    noalloc_tables_kernel<<<(span + 255) / 256, 256, 0, s>>>(st.base, t);
    if ((e = cudaGetLastError()) != cudaSuccess) return OFDM_ERR_CUDA;
    ++launches;
    st.tables_for = p;
    st.have_tables = true;
  }
  unsigned char* b = st.base;
  uint32_t* wstatus = reinterpret_cast<uint32_t*>(b + kOffStatus);
  // Everything a kernel of this call counts or accumulates starts at zero:
  // status words, the column kernel's symbol tickets, and the detection's
  // per-frame tickets and candidate counts.
  e = cudaMemsetAsync(wstatus, 0, (size_t)frames * sizeof(uint32_t), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(b + kOffCtr, 0, sizeof(unsigned long long), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(b + kOffDetTick, 0, (size_t)frames * sizeof(unsigned), s);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(b + kOffDetTick + kNoallocMaxFrames * sizeof(unsigned), 0, (size_t)frames * sizeof(unsigned), s);
  if (e != cudaSuccess) return OFDM_ERR_CUDA;
  float2* strip = reinterpret_cast<float2*>(b + kOffStrip);
  float* pow = reinterpret_cast<float*>(b + kOffPow);
  float2* pre = reinterpret_cast<float2*>(b + kOffPre);

  ColumnArgs ca;
  ca.M = M; ca.L_cp = p.L_cp; ca.rows = rows; ca.row0 = row0; ca.full = full; ca.frames = frames;
  ca.zc = (p.zc_root > 0 && !p.x_is_precoded) ? 1 : 0;
  int rinv = 1;
  const int r = p.zc_root > 0 ? p.zc_root : 1;
  for (int c = 1; c < N; c += 2)
    if (((long long)c * r) % N == 1) { rinv = c; break; }
  ca.rinv = rinv;
  ca.c0 = p.window == OFDM_WINDOW_HANN ? 0.5f : p.window == OFDM_WINDOW_HAMMING ? 0.54f : 1.f;
  ca.c1 = p.window == OFDM_WINDOW_HANN ? -0.25f : p.window == OFDM_WINDOW_HAMMING ? -0.23f : 0.f;
  ca.sqrtN = (float)sqrt((double)N);
  ca.pre = pre;
  ca.post_conj = pre + 3 * N;
  ca.tw = reinterpret_cast<float2*>(b + kOffTwN);
  ca.post_sign = ((p.zc_q % N) == 0) ? 1 : 0;
  ca.rprime = r;
  ca.refine_tau = kNoallocRefineTau;
  ca.pre_df = reinterpret_cast<float4*>(b + kOffDf);
  ca.w_df = ca.pre_df + N;
  ca.work_ctr = reinterpret_cast<unsigned long long*>(b + kOffCtr);
  ca.work_base = 0;                  // the counter was cleared above
  ca.frame_off = nullptr;
  ca.pipe_warps = 0;

  DopplerArgs da;
  da.N = N; da.Np = N; da.M = M; da.Mp = Mp; da.rows = rows; da.row0 = row0; da.frames = frames;
  da.inv_nm = (float)(1.0 / ((double)N * (double)M));
  da.wl = reinterpret_cast<float*>(b + kOffWl);
  da.tw = reinterpret_cast<float2*>(b + kOffTwM);
  da.map_off = nullptr;
  da.frame_mask = nullptr;

  DetectArgs ta;
  ta.Np = N; ta.Mp = Mp; ta.logMp = 0;
  while ((1 << ta.logMp) < Mp) ++ta.logMp;
  ta.rows = rows; ta.row0 = row0; ta.full = full; ta.compact = 1;
  ta.out_idx = nullptr;
  ta.frame_mask = nullptr;
  ta.part_keys = reinterpret_cast<uint64_t*>(b + kOffDetKeys);
  ta.tickets = reinterpret_cast<unsigned*>(b + kOffDetTick);   // cleared above for this call's frames
  ta.counts = ta.tickets + kNoallocMaxFrames;
  ta.eta = reinterpret_cast<float*>(b + kOffEta);
  ta.frame_stride = (long)rows * Mp; ta.frames = frames; ta.mode = p.detect_mode; ta.K = p.max_targets;
  ta.use_fixed_eta = p.noise_var > 0.f ? 1 : 0;
  ta.eta_fixed = p.noise_var * (float)(-log((double)p.pfa));
  ta.eta_factor = (float)(-log((double)p.pfa) / log(2.0));
  const int ncp = p.n_cp ? p.n_cp : p.L_cp;
  const double Ts = (double)(N + ncp) / ((double)N * p.df_hz);
  ta.dd = (float)(3.0e8 / (2.0 * N * p.df_hz));
  ta.dv = (float)(3.0e8 / (2.0 * p.fc_hz * Mp * Ts));

  unsigned long long tk = 0;
  e = launch_column(N, reinterpret_cast<const float2*>(Y), reinterpret_cast<const float2*>(X), strip, wstatus, ca,
                    s, &launches, &tk);
  if (out_map && rows < N) {  // the detection launch zeroes the rows outside the support
    ta.zmap = out_map;
    ta.zframe = (long)N * Mp;
    ta.z_off = (long)((row0 + rows) % N) * Mp;
    ta.z_floats = (long)(N - rows) * Mp;
  }
  if (e == cudaSuccess) e = launch_doppler(Mp, strip, out_map, pow, da, s, &launches);
  if (e == cudaSuccess) e = launch_detect(pow, out_targets, n_targets, status, wstatus, ta, s, &launches);
  return e == cudaSuccess ? OFDM_OK : OFDM_ERR_CUDA;
}
