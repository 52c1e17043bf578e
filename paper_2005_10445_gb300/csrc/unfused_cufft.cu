// unfused_cufft.cu -- the comparison pipeline of include/atlas_unfused.h: the
// coherent search organised like the paper's GPU implementation (Section 4.4:
// cuFFT for every transform, separate element-wise kernels, every
// intermediate -- mixed windows, their spectra, the products and the whole
// correlation surface -- in device memory).  cuFFT is used as a library;
// selection and refinement are the fused search's kernels, so the two
// pipelines report the same detections.  Measurement baseline only.
#include <cuda_runtime.h>
#include <cufft.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "acq_common.cuh"
#include "acq_internal.h"
#include "atlas_unfused.h"
#include "host_util.h"

namespace atlas {
namespace {

// y[(wl K + k) N + m] = x[(w0 + wl) hop + m] exp(-j 2 pi f_k m / fs), zero past the stream
__global__ void k_uf_mix(const float2* x, int64_t S, int N, int hop, int w0, int nw, int K, const uint64_t* inc,
                         float2* y) {
  const int64_t total = (int64_t)nw * K * N;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int m = (int)(e % N);
    const int64_t r = e / N;
    const int k = (int)(r % K), wl = (int)(r / K);
    const int64_t i = (int64_t)(w0 + wl) * hop + m;
    const float2 v = i < S ? x[i] : make_float2(0.f, 0.f);
    y[e] = cmul(v, expi_neg((uint64_t)m * inc[k]));
  }
}

// Z[((wl C + c) K + k) N + i] = Y[(wl K + k) N + i] * D[c N + i]
__global__ void k_uf_mul(const float2* Y, const float2* D, int N, int nw, int C, int K, float2* Z) {
  const int64_t total = (int64_t)nw * C * K * N;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % N);
    const int64_t r = e / N;
    const int k = (int)(r % K);
    const int64_t r2 = r / K;
    const int c = (int)(r2 % C), wl = (int)(r2 / C);
    Z[e] = cmul(Y[((int64_t)wl * K + k) * N + i], D[(int64_t)c * N + i]);
  }
}

// one block per (window, code, bin) transform: floor sum, max and argmax over the valid lags
constexpr int kUfPowerThreads = 512;
__global__ void __launch_bounds__(kUfPowerThreads) k_uf_power(const float2* Z, int N, int C, int K, int w0,
                                                             int hop, int W, int L, int64_t S, float4* part) {
  __shared__ float4 red[32];
  const int64_t t = blockIdx.x;  // ((wl C + c) K + k)
  const int wl = (int)(t / ((int64_t)C * K));
  const int w = w0 + wl;
  int nvalid = hop;
  if (w == W - 1) {
    const int64_t lim = S - L - (int64_t)w * hop;
    nvalid = (int)(lim < hop ? lim : hop) + 1;
  }
  const float2* z = Z + t * N;
  float sum = 0.f, best = -1.f;
  int bt = 0x7fffffff;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    const float2 v = z[i];
    const float P = fmaf(v.x, v.x, v.y * v.y);
    sum += P;
    if (i < nvalid && P > best) {  // increasing i: the first maximum is the smallest lag
      best = P;
      bt = i;
    }
  }
  block_reduce_stats(sum, best, bt, red);
  if (threadIdx.x == 0) part[t] = make_float4(sum, best, __int_as_float(bt), 0.f);
}

__global__ void k_uf_replica(const int8_t* chips, int n_chips, int sps, int N, int C, float2* r) {
  const int64_t total = (int64_t)C * N;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int n = (int)(e % N), c = (int)(e / N);
    r[e] = make_float2(n < n_chips * sps ? (float)chips[(int64_t)c * n_chips + n / sps] : 0.f, 0.f);
  }
}

__global__ void k_uf_conj_scale(float2* D, int64_t n, float s) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const float2 v = D[e];
    D[e] = make_float2(v.x * s, -v.y * s);
  }
}

int grid_for(int64_t n) { return (int)std::min<int64_t>((n + 255) / 256, 152 * 16); }

}  // namespace
}  // namespace atlas

struct atlas_unfused {
  int C = 0, K = 0, sps = 0, n_chips = 0, L = 0, N = 0, hop = 0, wc = 1;
  float threshold = 25.f;
  int8_t* d_chips = nullptr;
  int64_t* d_chip_off = nullptr;
  int* d_n_chips = nullptr;
  int* d_hop = nullptr;
  int* d_codes = nullptr;
  uint64_t* d_inc = nullptr;
  float2* d_D = nullptr;   // [C][N] conj(FFT_N(r_c)) / N
  float2* d_Y = nullptr;   // [wc][K][N]
  float2* d_Z = nullptr;   // [wc][C][K][N]
  float4* d_part = nullptr;
  cufftHandle plan_fwd = 0, plan_inv = 0;
  bool has_fwd = false, has_inv = false;
  std::string last_error;
};

namespace {

void free_uf(atlas_unfused* u) {
  if (!u) return;
  if (u->has_fwd) cufftDestroy(u->plan_fwd);
  if (u->has_inv) cufftDestroy(u->plan_inv);
  cudaFree(u->d_chips);
  cudaFree(u->d_chip_off);
  cudaFree(u->d_n_chips);
  cudaFree(u->d_hop);
  cudaFree(u->d_codes);
  cudaFree(u->d_inc);
  cudaFree(u->d_D);
  cudaFree(u->d_Y);
  cudaFree(u->d_Z);
  cudaFree(u->d_part);
  delete u;
}

int fail(atlas_unfused* u, const char* what) {
  u->last_error = what;
  return ATLAS_ERR_CUDA;
}

#define UCK(call)                                                   \
  do {                                                              \
    cudaError_t e_ = (call);                                        \
    if (e_ != cudaSuccess) return fail(u, cudaGetErrorString(e_));  \
  } while (0)
#define FCK(call)                                       \
  do {                                                  \
    if ((call) != CUFFT_SUCCESS) return fail(u, #call); \
  } while (0)

template <class T>
cudaError_t upload(T** d, const T* h, size_t n) {
  cudaError_t e = cudaMalloc((void**)d, sizeof(T) * (n ? n : 1));
  if (e == cudaSuccess && n) e = cudaMemcpy(*d, h, sizeof(T) * n, cudaMemcpyHostToDevice);
  return e;
}

int create_impl(atlas_unfused* u, const int8_t* chips, const int32_t* cpc, int32_t n_codes, int32_t sps,
                double fs, const double* freqs, int32_t n_freq, int32_t fft_len, int32_t wpl) {
  u->C = n_codes;
  u->K = n_freq;
  u->sps = sps;
  u->n_chips = cpc[0];
  u->L = cpc[0] * sps;
  int lg = 0;
  while ((1 << lg) < u->L) ++lg;
  u->N = fft_len ? fft_len : 2 << lg;
  if ((u->N & (u->N - 1)) != 0 || u->N <= u->L || u->N > (1 << 24)) return ATLAS_ERR_UNSUPPORTED;
  u->hop = u->N - u->L;
  // 16 windows by default (an 8 GiB surface for 16 codes x 31 bins at N = 2^17):
  // larger cuFFT batches measured faster (78.7, 79.5, 79.9 Msamples/s at 4, 8, 16)
  u->wc = wpl > 0 ? wpl : 16;
  const int C = u->C, K = u->K, N = u->N;
  std::vector<int64_t> off(C);
  std::vector<int> nch(C, u->n_chips), hop(C, u->hop), codes(C);
  for (int c = 0; c < C; ++c) {
    off[c] = (int64_t)c * u->n_chips;
    codes[c] = c;
  }
  std::vector<uint64_t> inc(K);
  for (int k = 0; k < K; ++k) inc[k] = atlas::phase_increment(freqs[k], fs);
  UCK(upload(&u->d_chips, chips, (size_t)C * u->n_chips));
  UCK(upload(&u->d_chip_off, off.data(), off.size()));
  UCK(upload(&u->d_n_chips, nch.data(), nch.size()));
  UCK(upload(&u->d_hop, hop.data(), hop.size()));
  UCK(upload(&u->d_codes, codes.data(), codes.size()));
  UCK(upload(&u->d_inc, inc.data(), inc.size()));
  if (cudaMalloc((void**)&u->d_D, sizeof(float2) * (size_t)C * N) != cudaSuccess ||
      cudaMalloc((void**)&u->d_Y, sizeof(float2) * (size_t)u->wc * K * N) != cudaSuccess ||
      cudaMalloc((void**)&u->d_Z, sizeof(float2) * (size_t)u->wc * C * K * N) != cudaSuccess ||
      cudaMalloc((void**)&u->d_part, sizeof(float4) * (size_t)u->wc * C * K) != cudaSuccess)
    return ATLAS_ERR_NO_MEMORY;
  // code spectra: replica -> cuFFT forward -> conj / N
  cufftHandle pc;
  FCK(cufftPlan1d(&pc, N, CUFFT_C2C, C));
  atlas::k_uf_replica<<<atlas::grid_for((int64_t)C * N), 256>>>(u->d_chips, u->n_chips, sps, N, C, u->d_D);
  const cufftResult r = cufftExecC2C(pc, (cufftComplex*)u->d_D, (cufftComplex*)u->d_D, CUFFT_FORWARD);
  cufftDestroy(pc);
  if (r != CUFFT_SUCCESS) return fail(u, "cufftExecC2C (code spectra)");
  atlas::k_uf_conj_scale<<<atlas::grid_for((int64_t)C * N), 256>>>(u->d_D, (int64_t)C * N, 1.0f / (float)N);
  UCK(cudaDeviceSynchronize());
  FCK(cufftPlan1d(&u->plan_fwd, N, CUFFT_C2C, u->wc * K));
  u->has_fwd = true;
  FCK(cufftPlan1d(&u->plan_inv, N, CUFFT_C2C, u->wc * C * K));
  u->has_inv = true;
  return ATLAS_OK;
}

}  // namespace

extern "C" {

int atlas_unfused_create(atlas_unfused_t* out, const int8_t* chips, const int32_t* chips_per_code,
                         int32_t n_codes, int32_t samples_per_chip, double fs_hz, const double* freq_offsets_hz,
                         int32_t n_freq, int32_t fft_len, float threshold, int32_t windows_per_launch) {
  if (!out) return ATLAS_ERR_INVALID_ARG;
  *out = nullptr;
  if (!chips || !chips_per_code || n_codes <= 0 || samples_per_chip <= 0 || !(fs_hz > 0.0) || !freq_offsets_hz ||
      n_freq <= 0 || !(threshold >= 0.f) || windows_per_launch < 0 || fft_len < 0)
    return ATLAS_ERR_INVALID_ARG;
  for (int c = 0; c < n_codes; ++c)
    if (chips_per_code[c] != chips_per_code[0] || chips_per_code[c] <= 0) return ATLAS_ERR_UNSUPPORTED;
  for (int64_t i = 0; i < (int64_t)n_codes * chips_per_code[0]; ++i)
    if (chips[i] != 1 && chips[i] != -1) return ATLAS_ERR_INVALID_ARG;
  atlas_unfused* u = new (std::nothrow) atlas_unfused();
  if (!u) return ATLAS_ERR_NO_MEMORY;
  u->threshold = threshold;
  const int st = create_impl(u, chips, chips_per_code, n_codes, samples_per_chip, fs_hz, freq_offsets_hz, n_freq,
                             fft_len, windows_per_launch);
  if (st != ATLAS_OK) {
    free_uf(u);
    return st;
  }
  *out = u;
  return ATLAS_OK;
}

int atlas_unfused_run(atlas_unfused_t u, void* stream, const float* d_iq, int64_t n_samples,
                      atlas_detection* d_out, int32_t capacity, int32_t* d_count) {
  if (!u || !d_iq || !d_count || capacity < 0 || (capacity > 0 && !d_out) || n_samples < u->L)
    return ATLAS_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const float2* x = reinterpret_cast<const float2*>(d_iq);
  const int C = u->C, K = u->K, N = u->N;
  const int W = n_samples <= N ? 1 : (int)((n_samples - N + u->hop - 1) / u->hop) + 1;
  FCK(cufftSetStream(u->plan_fwd, st));
  FCK(cufftSetStream(u->plan_inv, st));
  UCK(cudaMemsetAsync(d_count, 0, sizeof(int), st));
  for (int w0 = 0; w0 < W; w0 += u->wc) {
    const int nw = std::min(u->wc, W - w0);
    atlas::k_uf_mix<<<atlas::grid_for((int64_t)nw * K * N), 256, 0, st>>>(x, n_samples, N, u->hop, w0, nw, K,
                                                                         u->d_inc, u->d_Y);
    UCK(cudaGetLastError());
    // the plans are sized for full groups: in a short last group the rows past
    // its windows hold stale values, which are transformed but never read
    FCK(cufftExecC2C(u->plan_fwd, (cufftComplex*)u->d_Y, (cufftComplex*)u->d_Y, CUFFT_FORWARD));
    atlas::k_uf_mul<<<atlas::grid_for((int64_t)nw * C * K * N), 256, 0, st>>>(u->d_Y, u->d_D, N, nw, C, K,
                                                                             u->d_Z);
    UCK(cudaGetLastError());
    FCK(cufftExecC2C(u->plan_inv, (cufftComplex*)u->d_Z, (cufftComplex*)u->d_Z, CUFFT_INVERSE));
    atlas::k_uf_power<<<nw * C * K, atlas::kUfPowerThreads, 0, st>>>(u->d_Z, N, C, K, w0, u->hop, W, u->L,
                                                                     n_samples, u->d_part);
    UCK(cudaGetLastError());
    atlas::SelectParams sp;
    sp.part = u->d_part;
    sp.codes = u->d_codes;
    sp.Cg = C;
    sp.C = C;
    sp.K = K;
    sp.sps = 1;
    sp.N = N;
    sp.W = W;
    sp.w0 = w0;
    sp.nw = nw;
    sp.threshold = u->threshold;
    sp.out = d_out;
    sp.capacity = capacity;
    sp.count = d_count;
    sp.cells = nullptr;
    UCK(atlas::launch_select(sp, st));
  }
  if (capacity > 0) {
    atlas::RefineParams r;
    r.x = x;
    r.S = n_samples;
    r.chips = u->d_chips;
    r.chip_off = u->d_chip_off;
    r.chips_per_code = u->d_n_chips;
    r.hop = u->d_hop;
    r.inc = u->d_inc;
    r.sps = u->sps;
    r.out = d_out;
    r.capacity = capacity;
    r.count = d_count;
    UCK(atlas::launch_refine(r, std::min(capacity, 1024), st));
  }
  return ATLAS_OK;
}

const char* atlas_unfused_last_error(atlas_unfused_t u) { return u ? u->last_error.c_str() : ""; }

void atlas_unfused_destroy(atlas_unfused_t u) { free_uf(u); }

}  // extern "C"
