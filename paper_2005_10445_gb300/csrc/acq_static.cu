// acq_static.cu -- atlas_acq_run_static: the search for one code without a
// context and without any device allocation.
//
// Some callers cannot call cudaMalloc at the point where they need a search:
// code running under a framework whose caching allocator owns all device
// memory and forbids raw allocations, callbacks and plug-ins that must not
// change the process's memory footprint, or a real-time loop where an
// allocation (which may synchronise the device) is not acceptable.  This
// entry point serves them: the caller passes the samples, the chips and the
// output buffers; every intermediate array of the search (twiddle tables,
// phase increments, the code spectrum, one window's spectra and the
// per-phase partial results) lives in one file-scope static device array,
// g_scratch, of kStaticBytes = 4,342,016 bytes (about 4.14 MiB).  A GPU holds
// it from the moment the library's device code is loaded there (with CUDA's
// lazy module loading, the first call on that device) until the process exits.
//
// Limits: one code, N = fft_len <= 16384, at most 32 frequency bins,
// samples_per_chip a power of two <= 16, N / samples_per_chip >= 1024, and the
// stream bound of atlas_acq_run (n_samples <= 8 * INT32_MAX).  Larger sizes
// return ATLAS_ERR_UNSUPPORTED (ATLAS_ERR_INVALID_ARG for the stream length)
// before any device work.  The chips are device memory and are not checked:
// values other than +1 / -1 give scores that do not match atlas_acq_run.
//
// The twiddle tables and phase increments are computed on the host by the
// same functions as the context path's and handed to the set-up kernel as a
// parameter, so the records equal atlas_acq_run's bit for bit.
//
// Every call uses the same array and leaves its contents behind; a call
// rewrites every region it reads before reading it.  Calls whose device work
// overlaps (two host threads, or two streams without ordering between them)
// race on the array: order them on one stream.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <mutex>

#include "acq_internal.h"
#include "atlas_acq.h"
#include "host_util.h"

namespace atlas {
namespace {

constexpr int kStaticMaxN = 16384;
constexpr int kStaticMaxBins = 32;
constexpr int kStaticMaxDevices = 64;

// byte offsets of the regions of g_scratch (each a multiple of 256)
constexpr size_t kOffTw = 0;                                   // twiddle tables, <= 256 float2
constexpr size_t kOffInc = 4096;                               // [kStaticMaxBins] uint64
constexpr size_t kOffMeta = kOffInc + 4096;                    // chip offset, chip count, hop, code id
constexpr size_t kOffPart = kOffMeta + 256;                    // [K][sps] float4
constexpr size_t kOffD = kOffPart + (size_t)kStaticMaxBins * kMaxSps * 16;  // [M] float2
constexpr size_t kOffG = kOffD + (size_t)kStaticMaxN * 8;      // [K][N] float2, one window
constexpr size_t kStaticBytes = kOffG + (size_t)kStaticMaxBins * kStaticMaxN * 8;

struct StaticMeta {
  int64_t chip_off;
  int n_chips;
  int hop;
  int code;
};

constexpr int kStaticMaxTw = 256;  // table entries for M <= 2^14: 2^7 + 2^7

struct StaticSetup {
  uint64_t inc[kStaticMaxBins];
  float2 tw[kStaticMaxTw];
  int K, n_tw, n_chips, hop;
};
static_assert(sizeof(StaticSetup) <= 4096, "kernel parameter block");

}  // namespace

static __device__ __align__(256) unsigned char g_scratch[kStaticBytes];

namespace {

// Writes the small per-call tables into g_scratch: phase increments, the
// code's bookkeeping for the refinement kernel, and the W_M^t twiddle tables
// (high table then low table) that the host computed.
__global__ void k_static_setup(StaticSetup s) {
  uint64_t* inc = reinterpret_cast<uint64_t*>(g_scratch + kOffInc);
  StaticMeta* meta = reinterpret_cast<StaticMeta*>(g_scratch + kOffMeta);
  float2* tw = reinterpret_cast<float2*>(g_scratch + kOffTw);
  for (int k = threadIdx.x; k < s.K; k += blockDim.x) inc[k] = s.inc[k];
  if (threadIdx.x == 0) {
    meta->chip_off = 0;
    meta->n_chips = s.n_chips;
    meta->hop = s.hop;
    meta->code = 0;
  }
  for (int i = threadIdx.x; i < s.n_tw; i += blockDim.x) tw[i] = s.tw[i];
}

std::mutex g_mutex;
void* g_addr[kStaticMaxDevices] = {};

bool is_pow2(int64_t v) { return v > 0 && (v & (v - 1)) == 0; }
int ilog2(int64_t v) {
  int r = 0;
  while ((1ll << r) < v) ++r;
  return r;
}

// Device address of g_scratch on the current device, looked up once per device.
cudaError_t scratch_address(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kStaticMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return e;
    e = prepare_kernels();
    if (e != cudaSuccess) return e;
    g_addr[dev] = p;
  }
  *out = static_cast<unsigned char*>(g_addr[dev]);
  return cudaSuccess;
}

}  // namespace
}  // namespace atlas

extern "C" int atlas_acq_run_static(void* stream, const float* d_iq, int64_t n_samples, const int8_t* d_chips,
                                    int32_t n_chips, int32_t samples_per_chip, double fs_hz,
                                    const double* freq_offsets_hz, int32_t n_freq, int32_t fft_len,
                                    float threshold, atlas_detection* d_out, int32_t capacity,
                                    int32_t* d_count) {
  using namespace atlas;
  if (!d_iq || !d_chips || !d_count || !freq_offsets_hz || n_chips <= 0 || samples_per_chip <= 0 ||
      !(fs_hz > 0.0) || n_freq <= 0 || capacity < 0 || (capacity > 0 && !d_out) || !(threshold >= 0.f) ||
      fft_len < 0)
    return ATLAS_ERR_INVALID_ARG;
  for (int k = 0; k < n_freq; ++k)
    if (!isfinite(freq_offsets_hz[k])) return ATLAS_ERR_INVALID_ARG;
  const int sps = samples_per_chip;
  const int64_t L = (int64_t)n_chips * sps;
  if (n_samples < L) return ATLAS_ERR_INVALID_ARG;
  const int64_t N = fft_len ? fft_len : 2 * (1ll << ilog2(L));
  if (!is_pow2(sps) || sps > kMaxSps || n_freq > kStaticMaxBins || !is_pow2(N) || N > kStaticMaxN || N <= L ||
      N / sps < (1 << kMinLogM))
    return ATLAS_ERR_UNSUPPORTED;
  const int M = (int)(N / sps);
  const int logM = ilog2(M);
  const int hop = (int)(N - L);
  if (n_samples > (int64_t)INT32_MAX * 8) return ATLAS_ERR_INVALID_ARG;  // atlas_acq_run's stream bound
  const int64_t W64 = n_samples <= N ? 1 : (n_samples - N + hop - 1) / hop + 1;
  if (W64 > INT32_MAX) return ATLAS_ERR_UNSUPPORTED;
  const int W = (int)W64;

  unsigned char* base = nullptr;
  if (scratch_address(&base) != cudaSuccess) return ATLAS_ERR_CUDA;
  cudaStream_t st = (cudaStream_t)stream;
  float2* tw = reinterpret_cast<float2*>(base + kOffTw);
  uint64_t* inc = reinterpret_cast<uint64_t*>(base + kOffInc);
  StaticMeta* meta = reinterpret_cast<StaticMeta*>(base + kOffMeta);
  float4* part = reinterpret_cast<float4*>(base + kOffPart);
  float2* D = reinterpret_cast<float2*>(base + kOffD);
  float2* G = reinterpret_cast<float2*>(base + kOffG);
  const float2* x = reinterpret_cast<const float2*>(d_iq);

  StaticSetup su;
  for (int k = 0; k < kStaticMaxBins; ++k) su.inc[k] = k < n_freq ? phase_increment(freq_offsets_hz[k], fs_hz) : 0;
  const std::vector<float2> tables = twiddle_tables(logM);
  if (tables.size() > (size_t)kStaticMaxTw) return ATLAS_ERR_UNSUPPORTED;
  for (int i = 0; i < kStaticMaxTw; ++i) su.tw[i] = i < (int)tables.size() ? tables[i] : make_float2(0.f, 0.f);
  su.n_tw = (int)tables.size();
  su.K = n_freq;
  su.n_chips = n_chips;
  su.hop = hop;
  k_static_setup<<<1, 256, 0, st>>>(su);
  if (cudaGetLastError() != cudaSuccess) return ATLAS_ERR_CUDA;

  CodeBankParams cb;
  cb.chips = d_chips;
  cb.chip_off = &meta->chip_off;
  cb.n_chips = &meta->n_chips;
  cb.tw = tw;
  cb.D = D;
  cb.M = M;
  cb.scale = 1.0f / (float)M;
  if (launch_code_bank(logM, cb, 1, st) != cudaSuccess) return ATLAS_ERR_CUDA;
  if (cudaMemsetAsync(d_count, 0, sizeof(int32_t), st) != cudaSuccess) return ATLAS_ERR_CUDA;

  for (int w = 0; w < W; ++w) {
    MixParams m;
    m.x = x;
    m.S = n_samples;
    m.N = (int)N;
    m.M = M;
    m.sps = sps;
    m.hop = hop;
    m.w0 = w;
    m.nw = 1;
    m.K = n_freq;
    m.inc = inc;
    m.B = G;
    if (launch_mix(m, st) != cudaSuccess) return ATLAS_ERR_CUDA;
    WindowFftParams a;
    a.M = M;
    a.sps = sps;
    a.K = n_freq;
    a.nw = 1;
    a.tw = tw;
    a.G = G;
    if (launch_window_fft(logM, 5, false, a, st) != cudaSuccess) return ATLAS_ERR_CUDA;
    CorrParams b;
    b.G = G;
    b.D = D;
    b.tw = tw;
    b.tw2 = nullptr;
    b.part = part;
    b.S = n_samples;
    b.N = (int)N;
    b.M = M;
    b.sps = sps;
    b.hop = hop;
    b.W = W;
    b.L = (int)L;
    b.w0 = w;
    b.nw = 1;
    b.K = n_freq;
    b.Cg = 1;
    b.status = nullptr;
    if (launch_corr(logM, 5, false, b, st) != cudaSuccess) return ATLAS_ERR_CUDA;
    SelectParams c;
    c.part = part;
    c.codes = &meta->code;
    c.Cg = 1;
    c.C = 1;
    c.K = n_freq;
    c.sps = sps;
    c.N = (int)N;
    c.W = W;
    c.w0 = w;
    c.nw = 1;
    c.threshold = threshold;
    c.out = d_out;
    c.capacity = capacity;
    c.count = d_count;
    c.cells = nullptr;
    if (launch_select(c, st) != cudaSuccess) return ATLAS_ERR_CUDA;
  }
  if (capacity > 0) {
    RefineParams r;
    r.x = x;
    r.S = n_samples;
    r.chips = d_chips;
    r.chip_off = &meta->chip_off;
    r.chips_per_code = &meta->n_chips;
    r.hop = &meta->hop;
    r.inc = inc;
    r.sps = sps;
    r.out = d_out;
    r.capacity = capacity;
    r.count = d_count;
    if (launch_refine(r, capacity < 1024 ? capacity : 1024, st) != cudaSuccess) return ATLAS_ERR_CUDA;
  }
  return ATLAS_OK;
}
