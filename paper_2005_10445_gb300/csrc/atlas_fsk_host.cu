// atlas_fsk_host.cu -- host side of the FSK front end's C ABI (include/atlas_fsk.h):
// filter composition and transformation in FP64, the code bank (replicas,
// d_c, stored spectra), workspaces, and the stream-ordered launch sequence
// of a search.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <complex>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "acq_internal.h"
#include "atlas_fsk.h"
#include "fsk_internal.h"
#include "host_util.h"

namespace {

// Codes of one length share the window plan (n_c = L + T - 1, hop = N - n_c).
struct FskGroup {
  int n_chips = 0, L = 0, n_c = 0, N = 0, logN = 0, logM = 0, R = 1, hop = 0;
  std::vector<int> codes;
  int* d_codes = nullptr;      // [Cg] global code ids
  float2* d_spec = nullptr;    // [Cg][N] conj(DFT_N(d_c)) / N, permuted
  const float2* d_tw = nullptr;   // tables of the block transform (M = N / R)
  const float2* d_twN = nullptr;  // tables of N
  int windows(int64_t S) const {
    if (S <= N) return 1;
    return (int)((S - N + hop - 1) / hop) + 1;
  }
};

}  // namespace

struct atlas_fsk_ctx {
  int device = 0;
  int C = 0, sps = 0, T = 0;
  double fs = 0, f1 = 0, f0 = 0, f_lo = 0;
  float threshold = 49.f;
  int max_nc = 0;
  int wc = 16;  // windows per launch group
  std::vector<FskGroup> groups;
  std::vector<int> code_group;
  uint64_t lo_inc = 0;
  std::map<int, float2*> d_tw;
  float2* d_G1 = nullptr;
  float2* d_G0 = nullptr;
  float* d_dc = nullptr;  // [C][max_nc]
  // workspaces of one launch group
  float* d_dbuf = nullptr;
  float* d_ubuf = nullptr;
  int64_t buf_len = 0;
  float2* d_X = nullptr;
  float4* d_part = nullptr;
  atlas_detection* d_cand = nullptr;
  int cand_cap = 0;
  int* d_ncand = nullptr;
  double* d_stats_part = nullptr;
  // two-pass exchange of the cluster-sized transforms
  int exchange = 0;               // 1: cluster, 2: two passes
  float2* d_scratch = nullptr;
  size_t scratch_elems = 0;
  // code selection of atlas_fsk_run_codes: per group, the group-local indices
  // then the global ids of the searched codes (pinned host staging, device copy)
  int* h_sel = nullptr;
  int* d_sel = nullptr;
  cudaEvent_t ev_sel = nullptr;
  bool sel_pending = false;
  // host-buffer path
  int16_t* d_stage = nullptr;
  int64_t stage_samples = 0;
  atlas_fsk_detection* d_stage_out = nullptr;
  int stage_cap = 0;
  int* d_stage_count = nullptr;
  // pinned read-back of the count and the first records (one synchronisation
  // when they are all)
  static constexpr int kEager = 64;
  int* h_eager_count = nullptr;
  atlas_fsk_detection* h_eager = nullptr;
  // the input goes to d_stage in kCopyChunks copies on copy_st, so that the
  // demodulation of the first chunks overlaps the copy of the rest; while
  // host_chunks is set, run_impl demodulates d_stage chunk by chunk
  static constexpr int kCopyChunks = 4;
  cudaStream_t copy_st = nullptr;
  cudaEvent_t ev_main = nullptr;
  cudaEvent_t ev_copy[kCopyChunks] = {};
  int64_t copy_end[kCopyChunks] = {};
  int n_copy = 0;
  bool host_chunks = false;
  std::string last_error;
  // profiling (atlas_fsk_profile_begin / _end): event pairs per timed launch
  bool profiling = false;
  std::vector<cudaEvent_t> ev_corr, ev_demod;
  int corr_used = 0, demod_used = 0;
  atlas_fsk_profile prof = {};
};

namespace {

int fail_cuda(atlas_fsk_ctx* ctx, cudaError_t e) {
  if (ctx) ctx->last_error = cudaGetErrorString(e);
  return ATLAS_ERR_CUDA;
}

#define CK(call)                                      \
  do {                                                \
    cudaError_t e_ = (call);                          \
    if (e_ != cudaSuccess) return fail_cuda(ctx, e_); \
  } while (0)

int ilog2_ceil(int64_t v) {
  int r = 0;
  while ((1ll << r) < v) ++r;
  return r;
}

void free_ctx(atlas_fsk_ctx* ctx) {
  if (!ctx) return;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(ctx->device);
  for (auto& g : ctx->groups) {
    cudaFree(g.d_codes);
    cudaFree(g.d_spec);
  }
  for (auto& kv : ctx->d_tw) cudaFree(kv.second);
  cudaFree(ctx->d_G1);
  cudaFree(ctx->d_G0);
  cudaFree(ctx->d_dc);
  cudaFree(ctx->d_dbuf);
  cudaFree(ctx->d_ubuf);
  cudaFree(ctx->d_X);
  cudaFree(ctx->d_part);
  cudaFree(ctx->d_cand);
  cudaFree(ctx->d_ncand);
  cudaFree(ctx->d_stats_part);
  cudaFree(ctx->d_scratch);
  cudaFreeHost(ctx->h_sel);
  cudaFree(ctx->d_sel);
  if (ctx->ev_sel) cudaEventDestroy(ctx->ev_sel);
  cudaFree(ctx->d_stage);
  cudaFree(ctx->d_stage_out);
  cudaFree(ctx->d_stage_count);
  cudaFreeHost(ctx->h_eager_count);
  cudaFreeHost(ctx->h_eager);
  for (auto e : ctx->ev_copy)
    if (e) cudaEventDestroy(e);
  if (ctx->ev_main) cudaEventDestroy(ctx->ev_main);
  if (ctx->copy_st) cudaStreamDestroy(ctx->copy_st);
  for (auto e : ctx->ev_corr) cudaEventDestroy(e);
  for (auto e : ctx->ev_demod) cudaEventDestroy(e);
  cudaSetDevice(prev);
  delete ctx;
}

template <class T>
cudaError_t upload(T** dptr, const T* h, size_t n) {
  cudaError_t e = cudaMalloc((void**)dptr, sizeof(T) * (n ? n : 1));
  if (e != cudaSuccess) return e;
  if (n) e = cudaMemcpy(*dptr, h, sizeof(T) * n, cudaMemcpyHostToDevice);
  return e;
}

using cd = std::complex<double>;

// exp(-2 pi i num / den) with the argument reduced exactly (num mod den)
cd unit(int64_t num, int64_t den) {
  const double a = -6.283185307179586476925286766559 * (double)(((num % den) + den) % den) / (double)den;
  return cd(cos(a), sin(a));
}

// g_b = h_bp * m_b, m_b[t] = exp(-j 2 pi f_b (sps-1-t) / fs) (Section 4.1 composition), FP64
std::vector<cd> compose(const std::vector<cd>& h, double f_hz, int sps, double fs_hz) {
  std::vector<cd> m(sps);
  for (int t = 0; t < sps; ++t) {
    const double a = -6.283185307179586476925286766559 * (f_hz / fs_hz) * (double)(sps - 1 - t);
    m[t] = cd(cos(a), sin(a));
  }
  std::vector<cd> g(h.size() + sps - 1, cd(0.0, 0.0));
  for (size_t s = 0; s < h.size(); ++s)
    for (int t = 0; t < sps; ++t) g[s + t] += h[s] * m[t];
  return g;
}

// FFT_B(g zero padded)[k] / B, FP64 then rounded
std::vector<float2> filter_spectrum(const std::vector<cd>& g, int B) {
  std::vector<float2> out(B);
  for (int k = 0; k < B; ++k) {
    cd acc(0.0, 0.0);
    for (size_t t = 0; t < g.size(); ++t) acc += g[t] * unit((int64_t)t * k, B);
    acc /= (double)B;
    out[k] = make_float2((float)acc.real(), (float)acc.imag());
  }
  return out;
}

// (pair, code) items per pass of the two-pass exchange: a whole launch group,
// up to 1 GiB of scratch.  Larger passes measured faster than passes sized to
// stay in L2 (more blocks in flight outweighs the DRAM round trip of the
// scratch): 8 MiB 0.95 ms, 64 MiB 0.385 ms, 512 MiB 0.306 ms per launch group of
// 64 windows x 16 codes at N = 2^17.
int fsk_chunk_items(const atlas_fsk_ctx* ctx, const FskGroup& g) {
  const int64_t per = (int64_t)g.N * (int64_t)sizeof(float2);
  const int64_t by_size = std::max<int64_t>(1, (1ll << 30) / per);
  const int64_t group = (int64_t)((ctx->wc + 1) / 2) * (int64_t)g.codes.size();
  return (int)std::min(by_size, group);
}

int create_impl(atlas_fsk_ctx* ctx, const int8_t* chips, const int32_t* chips_per_code, int32_t n_codes,
                int32_t sps, double fs_hz, double f1_hz, double f0_hz, double f_lo_hz, const double* h_bp,
                int32_t n_bp, const atlas_fsk_opts& o) {
  ctx->C = n_codes;
  ctx->sps = sps;
  ctx->fs = fs_hz;
  ctx->f1 = f1_hz;
  ctx->f0 = f0_hz;
  ctx->f_lo = f_lo_hz;
  ctx->T = n_bp + sps - 1;
  ctx->threshold = o.threshold;
  if (ctx->T > atlas::kFskMaxTaps) return ATLAS_ERR_UNSUPPORTED;
  if (o.windows_per_launch < 0 || o.exchange < 0 || o.exchange > 2 ||
      (o.block_log2 != 0 && o.block_log2 != 13 && o.block_log2 != 14))
    return ATLAS_ERR_INVALID_ARG;
  ctx->exchange = o.exchange == 0 ? 2 : o.exchange;
  if (o.fft_len != 0 && (o.fft_len < (1 << atlas::kFskMinLogN) || o.fft_len > (1 << atlas::kFskMaxLogN) ||
                         (o.fft_len & (o.fft_len - 1)) != 0))
    return ATLAS_ERR_UNSUPPORTED;

  // groups by code length
  std::map<int, int> by_len;
  std::vector<int64_t> off(n_codes);
  int64_t total = 0;
  ctx->code_group.resize(n_codes);
  for (int c = 0; c < n_codes; ++c) {
    off[c] = total;
    total += chips_per_code[c];
    const int nch = chips_per_code[c];
    auto it = by_len.find(nch);
    if (it == by_len.end()) {
      FskGroup g;
      g.n_chips = nch;
      g.L = nch * sps;
      g.n_c = g.L + ctx->T - 1;
      g.N = o.fft_len ? o.fft_len : 2 * (int)(1ll << ilog2_ceil(g.L));
      g.logN = ilog2_ceil(g.N);
      if (g.logN < atlas::kFskMinLogN || g.logN > atlas::kFskMaxLogN || g.N <= g.n_c) return ATLAS_ERR_UNSUPPORTED;
      g.logM = g.logN > atlas::kFskLogMBlock && o.block_log2 ? o.block_log2 : atlas::fsk_default_log_m(g.logN);
      if (!atlas::fsk_plan_supported(g.logN, g.logM)) return ATLAS_ERR_UNSUPPORTED;
      g.R = 1 << (g.logN - g.logM);
      if (ctx->exchange != 2 && !atlas::fsk_plan_has_cluster_form(g.logN, g.logM)) return ATLAS_ERR_UNSUPPORTED;
      g.hop = g.N - g.n_c;
      by_len[nch] = (int)ctx->groups.size();
      ctx->groups.push_back(g);
      it = by_len.find(nch);
    }
    ctx->code_group[c] = it->second;
    ctx->groups[it->second].codes.push_back(c);
    ctx->max_nc = std::max(ctx->max_nc, nch * sps + ctx->T - 1);
  }
  for (int64_t i = 0; i < total; ++i)
    if (chips[i] != 1 && chips[i] != -1) return ATLAS_ERR_INVALID_ARG;

  CK(cudaGetDevice(&ctx->device));
  CK(atlas::fsk_prepare());

  // composed filters and their 4096-point spectra (FP64 on the host)
  std::vector<cd> h(n_bp);
  for (int i = 0; i < n_bp; ++i) h[i] = cd(h_bp[2 * i], h_bp[2 * i + 1]);
  const int B = 1 << atlas::kFskLogB;
  std::vector<float2> G1 = filter_spectrum(compose(h, f1_hz, sps, fs_hz), B);
  std::vector<float2> G0 = filter_spectrum(compose(h, f0_hz, sps, fs_hz), B);
  CK(upload(&ctx->d_G1, G1.data(), G1.size()));
  CK(upload(&ctx->d_G0, G0.data(), G0.size()));
  ctx->lo_inc = atlas::phase_increment(f_lo_hz, fs_hz);

  auto tables = [&](int lm, const float2** dst) -> int {
    if (!ctx->d_tw.count(lm)) {
      std::vector<float2> t = atlas::twiddle_tables(lm);
      float2* d = nullptr;
      CK(upload(&d, t.data(), t.size()));
      ctx->d_tw[lm] = d;
    }
    *dst = ctx->d_tw[lm];
    return ATLAS_OK;
  };
  const float2* twB = nullptr;
  int st = tables(atlas::kFskLogB, &twB);
  if (st != ATLAS_OK) return st;

  // windows per launch group, an even count: windows are transformed in the
  // pairs (2k, 2k + 1) of the whole stream whatever the grouping, so results
  // do not depend on it
  // 128 by default: a 1-s stream at 8 MS/s in one group at N = 2^17 (122
  // windows), 10,220 against 9,311 Msamples/s with groups of 64
  const int wpl = o.windows_per_launch > 0 ? o.windows_per_launch : 128;
  ctx->wc = std::min((wpl + 1) / 2 * 2, 256);
  // scratch of one pass of the two-pass transforms (also used by the code
  // bank's forward transforms below)
  if (ctx->exchange == 2) {
    for (auto& g : ctx->groups)
      if (g.R > 1)
        ctx->scratch_elems = std::max(ctx->scratch_elems, (size_t)fsk_chunk_items(ctx, g) * g.N);
    if (ctx->scratch_elems &&
        cudaMalloc((void**)&ctx->d_scratch, sizeof(float2) * ctx->scratch_elems) != cudaSuccess)
      return ATLAS_ERR_NO_MEMORY;
  }

  // code bank: replica -> d_c -> conj(DFT_N(d_c)) / N (Section 3 step 6, kept: Section 4.2)
  int8_t* d_chips = nullptr;
  int64_t* d_off = nullptr;
  int64_t* d_ones = nullptr;
  std::vector<int64_t> ones(total);
  for (int c = 0; c < n_codes; ++c) {
    int64_t k = 0;
    for (int i = 0; i < chips_per_code[c]; ++i) {
      ones[off[c] + i] = k;
      k += chips[off[c] + i] > 0;
    }
  }
  cudaError_t e = upload(&d_chips, chips, (size_t)total);
  if (e == cudaSuccess) e = upload(&d_off, off.data(), off.size());
  if (e == cudaSuccess) e = upload(&d_ones, ones.data(), ones.size());
  if (e == cudaSuccess) e = cudaMalloc((void**)&ctx->d_dc, sizeof(float) * (size_t)n_codes * ctx->max_nc);
  float2* d_rep = nullptr;
  int maxL = 0;
  for (auto& g : ctx->groups) maxL = std::max(maxL, g.L);
  if (e == cudaSuccess) e = cudaMalloc((void**)&d_rep, sizeof(float2) * (size_t)maxL);
  std::vector<int64_t> one_off(1);
  int64_t* d_one_off = nullptr;
  if (e == cudaSuccess) e = cudaMalloc((void**)&d_one_off, sizeof(int64_t));
  for (auto& g : ctx->groups) {
    if (e != cudaSuccess) break;
    const float2* tw = nullptr;
    if ((st = tables(g.logN - (g.R > 1 ? ilog2_ceil(g.R) : 0), &tw)) != ATLAS_OK) return st;
    g.d_tw = tw;
    if ((st = tables(g.logN, &g.d_twN)) != ATLAS_OK) return st;
    e = upload(&g.d_codes, g.codes.data(), g.codes.size());
    if (e == cudaSuccess) e = cudaMalloc((void**)&g.d_spec, sizeof(float2) * (size_t)g.N * g.codes.size());
    for (size_t i = 0; i < g.codes.size() && e == cudaSuccess; ++i) {
      const int c = g.codes[i];
      e = cudaMemcpy(d_one_off, &off[c], sizeof(int64_t), cudaMemcpyHostToDevice);
      atlas::FskReplicaParams rp;
      rp.chips = d_chips;
      rp.chip_off = d_one_off;
      rp.ones_before = d_ones;
      rp.n_chips = g.n_chips;
      rp.sps = sps;
      rp.inc1 = atlas::phase_increment(f1_hz, fs_hz);
      rp.inc0 = atlas::phase_increment(f0_hz, fs_hz);
      rp.r = d_rep;
      if (e == cudaSuccess) e = atlas::launch_fsk_replica(rp, 1, g.L, 0);
      atlas::FskDemodParams dp;
      dp.xf = d_rep;
      dp.S = g.L;
      dp.S_out = g.n_c;
      dp.start = 0;
      dp.count = g.n_c;
      dp.T = ctx->T;
      dp.lo_inc = 0;
      dp.G1 = ctx->d_G1;
      dp.G0 = ctx->d_G0;
      dp.tw = twB;
      dp.d = ctx->d_dc + (int64_t)c * ctx->max_nc;
      dp.u = nullptr;
      if (e == cudaSuccess) e = atlas::launch_fsk_demod(dp, 0);
      atlas::FskFwdParams fp;
      fp.rows = ctx->d_dc + (int64_t)c * ctx->max_nc;
      fp.ld = ctx->max_nc;
      fp.n_valid = g.n_c;
      fp.n_items = 1;
      fp.tw = g.d_tw;
      fp.twN = g.d_twN;
      fp.X = g.d_spec + (int64_t)i * g.N;
      fp.scale = 1.0f / (float)g.N;
      fp.conj_out = 1;
      fp.d = nullptr;
      fp.base = 0;
      fp.len = 0;
      fp.hop = 0;
      fp.w0 = 0;
      fp.nw = 0;
      if (ctx->exchange == 2 && g.R > 1) {
        fp.scratch = ctx->d_scratch;
        fp.chunk_items = (int)(ctx->scratch_elems / (size_t)g.N);
      }
      if (e == cudaSuccess) e = atlas::launch_fsk_fwd(g.logN, g.logM, fp, 0);
      if (e == cudaSuccess) e = cudaDeviceSynchronize();
    }
  }
  cudaFree(d_chips);
  cudaFree(d_off);
  cudaFree(d_ones);
  cudaFree(d_rep);
  cudaFree(d_one_off);
  if (e != cudaSuccess) return fail_cuda(ctx, e);

  // workspaces of one launch group: demodulated range, pair spectra, partial
  // results, candidates
  const int wc = ctx->wc;
  int64_t buf = 0;
  size_t X_elems = 0, part_elems = 0;
  int cand = 0;
  for (auto& g : ctx->groups) {
    buf = std::max<int64_t>(buf, (int64_t)(wc - 1) * g.hop + g.N + 2);
    X_elems = std::max(X_elems, (size_t)((wc + 1) / 2) * g.N);
    part_elems = std::max(part_elems, (size_t)wc * g.codes.size() * g.R);
    cand = std::max(cand, wc * (int)g.codes.size());
  }
  ctx->buf_len = buf;
  ctx->cand_cap = cand;
  if (cudaMalloc((void**)&ctx->d_dbuf, sizeof(float) * buf) != cudaSuccess ||
      cudaMalloc((void**)&ctx->d_ubuf, sizeof(float) * buf) != cudaSuccess ||
      cudaMalloc((void**)&ctx->d_X, sizeof(float2) * X_elems) != cudaSuccess ||
      cudaMalloc((void**)&ctx->d_part, sizeof(float4) * part_elems) != cudaSuccess ||
      cudaMalloc((void**)&ctx->d_cand, sizeof(atlas_detection) * cand) != cudaSuccess ||
      cudaMalloc((void**)&ctx->d_ncand, sizeof(int)) != cudaSuccess ||
      cudaMalloc((void**)&ctx->d_stats_part, sizeof(double) * 5 * atlas::kFskStatsSlices * (size_t)cand) !=
          cudaSuccess)
    return ATLAS_ERR_NO_MEMORY;
  if (cudaMallocHost((void**)&ctx->h_sel, sizeof(int) * 2 * (size_t)n_codes) != cudaSuccess ||
      cudaMalloc((void**)&ctx->d_sel, sizeof(int) * 2 * (size_t)n_codes) != cudaSuccess)
    return ATLAS_ERR_NO_MEMORY;
  CK(cudaEventCreateWithFlags(&ctx->ev_sel, cudaEventDisableTiming));
  return ATLAS_OK;
}

// Where a launch group's raw samples come from: a linear device stream whose
// sample 0 is absolute index first_sample, or a cyclic buffer read at the
// device-side block start *ring_start.
struct SampleSource {
  const int16_t* iq = nullptr;
  int64_t first_sample = 0;
  const int16_t* ring = nullptr;
  int64_t ring_cap = 0;
  const int64_t* ring_start = nullptr;
  // linear input that arrives in chunks: samples [0, chunk_end[k]) are in
  // place once chunk_ev[k] has completed (chunk_end ascending, the last = S)
  int n_chunks = 0;
  const int64_t* chunk_end = nullptr;
  const cudaEvent_t* chunk_ev = nullptr;
};

// One launch group of one code-length group: windows [w0, w0 + nw) of a block
// of S samples, Cg codes (device lists of their group-local indices and global
// ids), records appended to d_out / d_count.  timed: CUDA events may be recorded
// (not while a graph is being captured).
int enqueue_group(atlas_fsk_ctx* ctx, cudaStream_t st, const FskGroup& g, int W, int w0, int nw, int64_t S,
                  const SampleSource& src, int Cg, const int* d_sel_local, const int* d_sel_global,
                  atlas_fsk_detection* d_out, int capacity, int* d_count, bool timed) {
  // demodulated range of the group's windows, one sample of margin on each
  // side for the neighbours of the interpolation
  const int64_t base = (int64_t)w0 * g.hop - 1;
  const int64_t len = (int64_t)(nw - 1) * g.hop + g.N + 2;
  atlas::FskDemodParams dp;
  dp.iq = src.iq;
  dp.ring = src.ring;
  dp.ring_cap = src.ring_cap;
  dp.ring_start = src.ring_start;
  dp.S = S;
  dp.S_out = S;
  dp.start = base;
  dp.count = len;
  dp.T = ctx->T;
  dp.lo_inc = ctx->lo_inc;
  dp.lo_first = src.first_sample;
  dp.G1 = ctx->d_G1;
  dp.G0 = ctx->d_G0;
  dp.tw = ctx->d_tw.at(atlas::kFskLogB);
  dp.d = ctx->d_dbuf;
  dp.u = ctx->d_ubuf;
  const bool td = timed && ctx->profiling && 2 * ctx->demod_used + 1 < (int)ctx->ev_demod.size();
  if (td) CK(cudaEventRecord(ctx->ev_demod[2 * ctx->demod_used], st));
  int demod_launches = 1;
  if (src.n_chunks > 0) {
    // one launch per input chunk as it arrives.  The demodulation blocks sit
    // on a grid of multiples of `per` outputs and the chunk ends are on it, so
    // a launch that ends at a chunk end reads only inputs below it, and every
    // output is computed by the same block as in one launch.
    const int64_t per = atlas::fsk_demod_outputs_per_block(ctx->T);
    const int64_t end = base + len;
    demod_launches = 0;
    int k = 0;
    for (int64_t a = base; a < end;) {
      while (k < src.n_chunks - 1 && src.chunk_end[k] <= a) ++k;
      const int64_t e = k < src.n_chunks - 1 ? std::min(end, src.chunk_end[k]) : end;
      const int64_t need = std::min(S, (std::max<int64_t>(e, 0) + per - 1) / per * per);  // inputs read: [0, need)
      int kk = 0;
      while (kk < src.n_chunks - 1 && src.chunk_end[kk] < need) ++kk;
      CK(cudaStreamWaitEvent(st, src.chunk_ev[kk], 0));
      atlas::FskDemodParams sub = dp;
      sub.start = a;
      sub.count = e - a;
      sub.d = dp.d + (a - base);
      sub.u = dp.u + (a - base);
      CK(atlas::launch_fsk_demod(sub, st));
      ++demod_launches;
      a = e;
    }
  } else {
    CK(atlas::launch_fsk_demod(dp, st));
  }
  if (td) CK(cudaEventRecord(ctx->ev_demod[2 * ctx->demod_used++ + 1], st));
  atlas::FskFwdParams fp;
  fp.d = ctx->d_dbuf;
  fp.base = base;
  fp.len = len;
  fp.hop = g.hop;
  fp.w0 = w0;
  fp.nw = nw;
  fp.n_items = (nw + 1) / 2;
  fp.tw = g.d_tw;
  fp.twN = g.d_twN;
  fp.X = ctx->d_X;
  fp.scale = 1.0f;
  fp.conj_out = 0;
  const bool two_pass = ctx->exchange == 2 && g.R > 1;
  if (two_pass) {
    fp.scratch = ctx->d_scratch;
    fp.chunk_items = (int)(ctx->scratch_elems / (size_t)g.N);
  }
  CK(atlas::launch_fsk_fwd(g.logN, g.logM, fp, st));
  atlas::FskCorrParams cp;
  cp.X = ctx->d_X;
  cp.C = g.d_spec;
  cp.tw = g.d_tw;
  cp.twN = g.d_twN;
  cp.part = ctx->d_part;
  cp.S = S;
  cp.N = g.N;
  cp.hop = g.hop;
  cp.W = W;
  cp.n_c = g.n_c;
  cp.w0 = w0;
  cp.nw = nw;
  cp.Cg = Cg;
  cp.sel = d_sel_local;
  if (two_pass) {
    cp.scratch = ctx->d_scratch;
    cp.chunk_items = fsk_chunk_items(ctx, g);
  }
  const bool tc = timed && ctx->profiling && 2 * ctx->corr_used + 1 < (int)ctx->ev_corr.size();
  if (tc) CK(cudaEventRecord(ctx->ev_corr[2 * ctx->corr_used], st));
  CK(atlas::launch_fsk_corr(g.logN, g.logM, cp, st));
  if (tc) CK(cudaEventRecord(ctx->ev_corr[2 * ctx->corr_used++ + 1], st));
  if (timed && ctx->profiling) {
    // demod, select, two stats kernels, advance; the forward and the correlation
    // transforms: one launch each, or two per pass of the two-pass form
    const int fwd_items = fp.n_items, corr_items = ((nw + 1) / 2) * Cg;
    auto passes = [](int items, int per) { return (items + per - 1) / per; };
    // select and the two peak-sum stages, and the count's advance unless the
    // final stage does it (small groups)
    ctx->prof.launches += 3 + (nw * Cg > atlas::kFskStatsFinalOneBlock ? 1 : 0) + demod_launches +
                          (two_pass ? 2 * passes(fwd_items, fp.chunk_items) : 1) +
                          (two_pass ? 2 * passes(corr_items, cp.chunk_items) : 1);
    ctx->prof.corr_launches += 1;
    ctx->prof.corr_units += (int64_t)nw * Cg;
    ctx->prof.demod_launches += 1;
    ctx->prof.demod_samples += len;
  }
  atlas::SelectParams sp;  // writes the group's candidate count (the list starts empty)
  sp.part = ctx->d_part;
  sp.codes = d_sel_global;
  sp.Cg = Cg;
  sp.C = ctx->C;
  sp.K = 1;
  sp.sps = g.R;
  sp.N = g.N;
  sp.W = W;
  sp.w0 = w0;
  sp.nw = nw;
  sp.threshold = ctx->threshold;
  sp.out = ctx->d_cand;
  sp.capacity = nw * Cg;
  sp.count = ctx->d_ncand;
  sp.cells = nullptr;
  CK(atlas::launch_fsk_select(sp, st));
  atlas::FskStatsParams tp;
  tp.cand = ctx->d_cand;
  tp.n_cand = ctx->d_ncand;
  tp.d = ctx->d_dbuf;
  tp.u = ctx->d_ubuf;
  tp.base = base;
  tp.len = len;
  tp.dc = ctx->d_dc;
  tp.ld = ctx->max_nc;
  tp.n_c = g.n_c;
  tp.hop = g.hop;
  tp.S = S;
  tp.out = d_out;
  tp.capacity = capacity;
  tp.count = d_count;
  tp.part = ctx->d_stats_part;
  CK(atlas::launch_fsk_stats(tp, nw * Cg, st));
  return ATLAS_OK;
}

// sel: host list of the searched codes (n_sel of them), or null for every code.
int run_impl(atlas_fsk_ctx* ctx, cudaStream_t st, const int16_t* d_iq, int64_t S, int64_t first_sample,
             const int32_t* sel, int n_sel, atlas_fsk_detection* d_out, int capacity, int* d_count) {
  // per group: offset of its lists in h_sel / d_sel and its number of searched codes
  std::vector<int> sel_off(ctx->groups.size(), 0), sel_n(ctx->groups.size(), 0);
  if (sel) {
    std::vector<char> on(ctx->C, 0);
    for (int i = 0; i < n_sel; ++i) {
      if (sel[i] < 0 || sel[i] >= ctx->C || on[sel[i]]) return ATLAS_ERR_INVALID_ARG;
      on[sel[i]] = 1;
    }
    if (ctx->sel_pending) CK(cudaEventSynchronize(ctx->ev_sel));  // the previous list has been copied
    int off = 0;
    for (size_t gi = 0; gi < ctx->groups.size(); ++gi) {
      const FskGroup& g = ctx->groups[gi];
      sel_off[gi] = off;
      int n = 0;
      for (size_t i = 0; i < g.codes.size(); ++i)
        if (on[g.codes[i]]) ctx->h_sel[off + n++] = (int)i;  // ascending: (window, code) order is kept
      for (int i = 0; i < n; ++i) ctx->h_sel[off + n + i] = g.codes[ctx->h_sel[off + i]];
      sel_n[gi] = n;
      off += 2 * n;
    }
    if (off > 0) {
      CK(cudaMemcpyAsync(ctx->d_sel, ctx->h_sel, sizeof(int) * off, cudaMemcpyHostToDevice, st));
      CK(cudaEventRecord(ctx->ev_sel, st));
      ctx->sel_pending = true;
    }
  }
  CK(cudaMemsetAsync(d_count, 0, sizeof(int), st));
  SampleSource src;
  src.iq = d_iq;
  src.first_sample = first_sample;
  if (ctx->host_chunks && d_iq == ctx->d_stage) {
    src.n_chunks = ctx->n_copy;
    src.chunk_end = ctx->copy_end;
    src.chunk_ev = ctx->ev_copy;
  }
  for (size_t gi = 0; gi < ctx->groups.size(); ++gi) {
    const FskGroup& g = ctx->groups[gi];
    const int W = g.windows(S);
    const int Cg = sel ? sel_n[gi] : (int)g.codes.size();
    if (Cg == 0) continue;
    const int* d_sel_local = sel ? ctx->d_sel + sel_off[gi] : nullptr;
    const int* d_sel_global = sel ? ctx->d_sel + sel_off[gi] + Cg : g.d_codes;
    for (int w0 = 0; w0 < W; w0 += ctx->wc) {
      const int r = enqueue_group(ctx, st, g, W, w0, std::min(ctx->wc, W - w0), S, src, Cg, d_sel_local,
                                  d_sel_global, d_out, capacity, d_count, true);
      if (r != ATLAS_OK) return r;
    }
  }
  return ATLAS_OK;
}

}  // namespace

struct atlas_fsk_tracker {
  atlas_fsk_ctx* ctx = nullptr;
  int gi = 0;         // code-length group
  int64_t len = 0;    // block samples
  int W = 0;          // windows of a block
  struct Desc {       // read by the graph's kernels
    int64_t start;    // absolute index of the block's first sample
    int32_t local;    // the code's index within its group
    int32_t global;   // the code
  };
  // One block of device memory, mirrored by one pinned host block:
  //   [0, 16)   Desc
  //   [16, 32)  the record count (int32, then padding)
  //   [32, ..)  W records
  // The graph's first node copies [0, 32) in (the descriptor and a zero
  // count) and its last node copies [16, ..) out (the count and the records).
  static constexpr size_t kCount = 16, kRecords = 32;
  char* d_blk = nullptr;
  char* h_blk = nullptr;
  Desc* d_desc = nullptr;                // views into d_blk / h_blk
  Desc* h_desc = nullptr;
  int* d_count = nullptr;
  int* h_count = nullptr;
  atlas_fsk_detection* d_out = nullptr;
  atlas_fsk_detection* h_out = nullptr;
  size_t blk_bytes() const { return kRecords + sizeof(atlas_fsk_detection) * (size_t)W; }
  cudaStream_t cs = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int kernels = 0;  // kernel nodes of the graph
};

namespace {

void free_tracker(atlas_fsk_tracker* t) {
  if (!t) return;
  if (t->exec) cudaGraphExecDestroy(t->exec);
  if (t->graph) cudaGraphDestroy(t->graph);
  if (t->cs) cudaStreamDestroy(t->cs);
  cudaFreeHost(t->h_blk);
  cudaFree(t->d_blk);
  delete t;
}

int capture_tracker(atlas_fsk_tracker* t, const int16_t* d_ring, int64_t ring_samples) {
  atlas_fsk_ctx* ctx = t->ctx;
  const FskGroup& g = ctx->groups[t->gi];
  cudaStream_t cs = t->cs;
  CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  SampleSource src;
  src.ring = d_ring;
  src.ring_cap = ring_samples;
  src.ring_start = &t->d_desc->start;
  int r = ATLAS_OK;
  // the descriptor and a zero count in one copy
  cudaError_t e = cudaMemcpyAsync(t->d_blk, t->h_blk, atlas_fsk_tracker::kRecords, cudaMemcpyHostToDevice, cs);
  for (int w0 = 0; e == cudaSuccess && r == ATLAS_OK && w0 < t->W; w0 += ctx->wc)
    r = enqueue_group(ctx, cs, g, t->W, w0, std::min(ctx->wc, t->W - w0), t->len, src, 1, &t->d_desc->local,
                      &t->d_desc->global, t->d_out, t->W, t->d_count, false);
  if (e == cudaSuccess && r == ATLAS_OK)  // the count and the records in one copy
    e = cudaMemcpyAsync(t->h_blk + atlas_fsk_tracker::kCount, t->d_blk + atlas_fsk_tracker::kCount,
                        t->blk_bytes() - atlas_fsk_tracker::kCount, cudaMemcpyDeviceToHost, cs);
  const cudaError_t e_end = cudaStreamEndCapture(cs, &t->graph);  // always leaves capture mode
  if (r != ATLAS_OK) return r;
  if (e != cudaSuccess) return fail_cuda(ctx, e);
  if (e_end != cudaSuccess) return fail_cuda(ctx, e_end);
  CK(cudaGraphInstantiate(&t->exec, t->graph, 0));
  size_t n_nodes = 0;
  CK(cudaGraphGetNodes(t->graph, nullptr, &n_nodes));
  std::vector<cudaGraphNode_t> nodes(n_nodes);
  if (n_nodes) CK(cudaGraphGetNodes(t->graph, nodes.data(), &n_nodes));
  t->kernels = 0;
  for (cudaGraphNode_t nd : nodes) {
    cudaGraphNodeType ty;
    CK(cudaGraphNodeGetType(nd, &ty));
    t->kernels += ty == cudaGraphNodeTypeKernel;
  }
  return ATLAS_OK;
}

}  // namespace

extern "C" {

int atlas_fsk_tracker_create(atlas_fsk_tracker_t* out, atlas_fsk_t ctx, int32_t code, int64_t n_samples,
                             const int16_t* d_ring, int64_t ring_samples) {
  if (!out) return ATLAS_ERR_INVALID_ARG;
  *out = nullptr;
  if (!ctx || code < 0 || code >= ctx->C || !d_ring || ring_samples < n_samples) return ATLAS_ERR_INVALID_ARG;
  const int gi = ctx->code_group[code];
  const FskGroup& g = ctx->groups[gi];
  if (n_samples < g.n_c || n_samples > ((int64_t)1 << 31)) return ATLAS_ERR_INVALID_ARG;
  atlas_fsk_tracker* t = new (std::nothrow) atlas_fsk_tracker();
  if (!t) return ATLAS_ERR_NO_MEMORY;
  t->ctx = ctx;
  t->gi = gi;
  t->len = n_samples;
  t->W = g.windows(n_samples);
  static_assert(sizeof(atlas_fsk_tracker::Desc) <= atlas_fsk_tracker::kCount, "descriptor fits its slot");
  if (cudaMallocHost((void**)&t->h_blk, t->blk_bytes()) != cudaSuccess ||
      cudaMalloc((void**)&t->d_blk, t->blk_bytes()) != cudaSuccess) {
    free_tracker(t);
    return ATLAS_ERR_NO_MEMORY;
  }
  memset(t->h_blk, 0, t->blk_bytes());
  t->d_desc = reinterpret_cast<atlas_fsk_tracker::Desc*>(t->d_blk);
  t->h_desc = reinterpret_cast<atlas_fsk_tracker::Desc*>(t->h_blk);
  t->d_count = reinterpret_cast<int*>(t->d_blk + atlas_fsk_tracker::kCount);
  t->h_count = reinterpret_cast<int*>(t->h_blk + atlas_fsk_tracker::kCount);
  t->d_out = reinterpret_cast<atlas_fsk_detection*>(t->d_blk + atlas_fsk_tracker::kRecords);
  t->h_out = reinterpret_cast<atlas_fsk_detection*>(t->h_blk + atlas_fsk_tracker::kRecords);
  memset(t->h_desc, 0, sizeof(atlas_fsk_tracker::Desc));
  int r = ATLAS_OK;
  if (cudaStreamCreateWithFlags(&t->cs, cudaStreamNonBlocking) != cudaSuccess) r = ATLAS_ERR_CUDA;
  if (r == ATLAS_OK) r = capture_tracker(t, d_ring, ring_samples);
  if (r != ATLAS_OK) {
    free_tracker(t);
    return r;
  }
  *out = t;
  return ATLAS_OK;
}

int atlas_fsk_tracker_run(atlas_fsk_tracker_t t, void* stream, int32_t code, int64_t block_start,
                          atlas_fsk_detection* h_out, int32_t capacity, int32_t* h_count) {
  if (!t || !h_count || capacity < 0 || (capacity > 0 && !h_out) || block_start < 0) return ATLAS_ERR_INVALID_ARG;
  atlas_fsk_ctx* ctx = t->ctx;
  if (code < 0 || code >= ctx->C || ctx->code_group[code] != t->gi) return ATLAS_ERR_INVALID_ARG;
  const FskGroup& g = ctx->groups[t->gi];
  int local = 0;
  while (g.codes[local] != code) ++local;
  t->h_desc->start = block_start;
  t->h_desc->local = local;
  t->h_desc->global = code;
  *t->h_count = 0;  // copied in with the descriptor
  cudaStream_t st = (cudaStream_t)stream;
  CK(cudaGraphLaunch(t->exec, st));
  CK(cudaStreamSynchronize(st));  // the descriptor has been read, the results are in
  const int n = std::min(*t->h_count, std::min(capacity, t->W));
  if (n > 0) memcpy(h_out, t->h_out, sizeof(atlas_fsk_detection) * (size_t)n);
  *h_count = *t->h_count;
  return ATLAS_OK;
}

int32_t atlas_fsk_tracker_kernels(atlas_fsk_tracker_t t) { return t ? t->kernels : -1; }

void atlas_fsk_tracker_destroy(atlas_fsk_tracker_t t) { free_tracker(t); }

void atlas_fsk_default_opts(atlas_fsk_opts* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->threshold = 49.f;
}

int atlas_fsk_create(atlas_fsk_t* out, const int8_t* chips, const int32_t* chips_per_code, int32_t n_codes,
                     int32_t samples_per_chip, double fs_hz, double f1_hz, double f0_hz, double f_lo_hz,
                     const double* h_bp, int32_t n_bp, const atlas_fsk_opts* opts) {
  if (!out) return ATLAS_ERR_INVALID_ARG;
  *out = nullptr;
  if (!chips || !chips_per_code || n_codes <= 0 || samples_per_chip <= 0 || !(fs_hz > 0.0) || !h_bp || n_bp < 1 ||
      !isfinite(f1_hz) || !isfinite(f0_hz) || !isfinite(f_lo_hz))
    return ATLAS_ERR_INVALID_ARG;
  for (int c = 0; c < n_codes; ++c)
    if (chips_per_code[c] <= 0) return ATLAS_ERR_INVALID_ARG;
  for (int i = 0; i < 2 * n_bp; ++i)
    if (!isfinite(h_bp[i])) return ATLAS_ERR_INVALID_ARG;
  atlas_fsk_opts o;
  atlas_fsk_default_opts(&o);
  if (opts) o = *opts;
  if (!(o.threshold >= 0.f)) return ATLAS_ERR_INVALID_ARG;
  atlas_fsk_ctx* ctx = new (std::nothrow) atlas_fsk_ctx();
  if (!ctx) return ATLAS_ERR_NO_MEMORY;
  const int st = create_impl(ctx, chips, chips_per_code, n_codes, samples_per_chip, fs_hz, f1_hz, f0_hz, f_lo_hz,
                             h_bp, n_bp, o);
  if (st != ATLAS_OK) {
    free_ctx(ctx);
    return st;
  }
  *out = ctx;
  return ATLAS_OK;
}

int atlas_fsk_windows(atlas_fsk_t ctx, int32_t code, int64_t n_samples, int32_t* n_windows, int32_t* hop,
                      int32_t* fft_len, int32_t* support) {
  if (!ctx || code < 0 || code >= ctx->C || n_samples <= 0) return ATLAS_ERR_INVALID_ARG;
  const FskGroup& g = ctx->groups[ctx->code_group[code]];
  if (n_windows) *n_windows = g.windows(n_samples);
  if (hop) *hop = g.hop;
  if (fft_len) *fft_len = g.N;
  if (support) *support = g.n_c;
  return ATLAS_OK;
}

int atlas_fsk_run_codes(atlas_fsk_t ctx, void* stream, const int16_t* d_iq, int64_t n_samples,
                        int64_t first_sample, const int32_t* h_codes, int32_t n_sel, atlas_fsk_detection* d_out,
                        int32_t capacity, int32_t* d_count) {
  if (!ctx || !d_iq || !d_count || capacity < 0 || (capacity > 0 && !d_out)) return ATLAS_ERR_INVALID_ARG;
  if (n_sel < 0 || (n_sel > 0 && !h_codes) || first_sample < 0) return ATLAS_ERR_INVALID_ARG;
  if (n_samples > ((int64_t)1 << 40) || first_sample > ((int64_t)1 << 62)) return ATLAS_ERR_INVALID_ARG;
  int max_nc = 0;
  if (h_codes) {
    for (int i = 0; i < n_sel; ++i)
      if (h_codes[i] >= 0 && h_codes[i] < ctx->C)
        max_nc = std::max(max_nc, ctx->groups[ctx->code_group[h_codes[i]]].n_c);
  } else {
    max_nc = ctx->max_nc;
  }
  if (n_samples < max_nc) return ATLAS_ERR_INVALID_ARG;
  for (const FskGroup& g : ctx->groups)
    if ((int64_t)g.windows(n_samples) * g.hop + g.N > ((int64_t)1 << 31) - 2) return ATLAS_ERR_UNSUPPORTED;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != ctx->device) return ATLAS_ERR_INVALID_ARG;
  if (h_codes && n_sel == 0) {  // nothing to search
    CK(cudaMemsetAsync(d_count, 0, sizeof(int), (cudaStream_t)stream));
    return ATLAS_OK;
  }
  return run_impl(ctx, (cudaStream_t)stream, d_iq, n_samples, first_sample, h_codes, n_sel, d_out, capacity,
                  d_count);
}

int atlas_fsk_run(atlas_fsk_t ctx, void* stream, const int16_t* d_iq, int64_t n_samples,
                  atlas_fsk_detection* d_out, int32_t capacity, int32_t* d_count) {
  return atlas_fsk_run_codes(ctx, stream, d_iq, n_samples, 0, nullptr, 0, d_out, capacity, d_count);
}

int atlas_fsk_run_host(atlas_fsk_t ctx, void* stream, const int16_t* h_iq, int64_t n_samples,
                       atlas_fsk_detection* h_out, int32_t capacity, int32_t* h_count) {
  if (!ctx || !h_iq || !h_count || capacity < 0 || (capacity > 0 && !h_out)) return ATLAS_ERR_INVALID_ARG;
  if (n_samples < ctx->max_nc || n_samples > ((int64_t)1 << 40)) return ATLAS_ERR_INVALID_ARG;
  int dev = 0;  // the staging buffers and the copy stream live on the context's device
  if (cudaGetDevice(&dev) != cudaSuccess || dev != ctx->device) return ATLAS_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  if (ctx->stage_samples < n_samples) {
    cudaFree(ctx->d_stage);
    ctx->d_stage = nullptr;
    ctx->stage_samples = 0;
    if (cudaMalloc((void**)&ctx->d_stage, sizeof(int16_t) * 2 * (size_t)n_samples) != cudaSuccess)
      return ATLAS_ERR_NO_MEMORY;
    ctx->stage_samples = n_samples;
  }
  if (ctx->stage_cap < std::max(capacity, 1) || !ctx->d_stage_count) {
    cudaFree(ctx->d_stage_out);
    ctx->d_stage_out = nullptr;
    ctx->stage_cap = 0;
    if (cudaMalloc((void**)&ctx->d_stage_out, sizeof(atlas_fsk_detection) * (size_t)std::max(capacity, 1)) !=
        cudaSuccess)
      return ATLAS_ERR_NO_MEMORY;
    ctx->stage_cap = std::max(capacity, 1);
    if (!ctx->d_stage_count && cudaMalloc((void**)&ctx->d_stage_count, sizeof(int)) != cudaSuccess)
      return ATLAS_ERR_NO_MEMORY;
  }
  if (!ctx->h_eager &&
      (cudaMallocHost((void**)&ctx->h_eager_count, sizeof(int)) != cudaSuccess ||
       cudaMallocHost((void**)&ctx->h_eager, sizeof(atlas_fsk_detection) * atlas_fsk_ctx::kEager) != cudaSuccess)) {
    cudaFreeHost(ctx->h_eager_count);
    ctx->h_eager_count = nullptr;
    return ATLAS_ERR_NO_MEMORY;
  }
  if (!ctx->copy_st) {
    CK(cudaStreamCreateWithFlags(&ctx->copy_st, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&ctx->ev_main, cudaEventDisableTiming));
    for (auto& e : ctx->ev_copy) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  }
  // chunks end on the demodulation block grid (multiples of `per` samples)
  const int64_t per = atlas::fsk_demod_outputs_per_block(ctx->T);
  CK(cudaEventRecord(ctx->ev_main, st));  // earlier work on the stream is done with d_stage
  CK(cudaStreamWaitEvent(ctx->copy_st, ctx->ev_main, 0));
  ctx->n_copy = 0;
  int64_t c0 = 0;
  for (int k = 0; k < atlas_fsk_ctx::kCopyChunks; ++k) {
    const int64_t c1 = k == atlas_fsk_ctx::kCopyChunks - 1
                           ? n_samples
                           : std::min(n_samples, ((k + 1) * n_samples / atlas_fsk_ctx::kCopyChunks + per - 1) / per * per);
    if (c1 <= c0) continue;  // short streams: fewer, whole-block chunks
    const int j = ctx->n_copy++;
    CK(cudaMemcpyAsync(ctx->d_stage + 2 * c0, h_iq + 2 * c0, sizeof(int16_t) * 2 * (size_t)(c1 - c0),
                       cudaMemcpyHostToDevice, ctx->copy_st));
    CK(cudaEventRecord(ctx->ev_copy[j], ctx->copy_st));
    ctx->copy_end[j] = c1;
    c0 = c1;
  }
  ctx->host_chunks = true;
  int r = atlas_fsk_run(ctx, stream, ctx->d_stage, n_samples, ctx->d_stage_out, capacity, ctx->d_stage_count);
  ctx->host_chunks = false;
  if (r != ATLAS_OK) {
    cudaStreamSynchronize(ctx->copy_st);  // the copies read the caller's buffer
    return r;
  }
  // the count and up to kEager records in one round trip; the rest after it
  const int eager = std::min(capacity, atlas_fsk_ctx::kEager);
  CK(cudaMemcpyAsync(ctx->h_eager_count, ctx->d_stage_count, sizeof(int), cudaMemcpyDeviceToHost, st));
  if (eager > 0)
    CK(cudaMemcpyAsync(ctx->h_eager, ctx->d_stage_out, sizeof(atlas_fsk_detection) * (size_t)eager,
                       cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  *h_count = *ctx->h_eager_count;
  const int n = std::min(*h_count, capacity);
  if (n > 0) memcpy(h_out, ctx->h_eager, sizeof(atlas_fsk_detection) * (size_t)std::min(n, eager));
  if (n > eager) {
    CK(cudaMemcpyAsync(h_out + eager, ctx->d_stage_out + eager, sizeof(atlas_fsk_detection) * (size_t)(n - eager),
                       cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
  }
  return ATLAS_OK;
}

int atlas_fsk_demod(atlas_fsk_t ctx, void* stream, const int16_t* d_iq, int64_t n_samples, int64_t start,
                    int64_t count, float* d_d, float* d_u) {
  if (!ctx || !d_iq || !d_d || n_samples <= 0 || count < 0) return ATLAS_ERR_INVALID_ARG;
  atlas::FskDemodParams dp;
  dp.iq = d_iq;
  dp.S = n_samples;
  dp.S_out = n_samples;
  dp.start = start;
  dp.count = count;
  dp.T = ctx->T;
  dp.lo_inc = ctx->lo_inc;
  dp.G1 = ctx->d_G1;
  dp.G0 = ctx->d_G0;
  dp.tw = ctx->d_tw.at(atlas::kFskLogB);
  dp.d = d_d;
  dp.u = d_u;
  CK(atlas::launch_fsk_demod(dp, (cudaStream_t)stream));
  return ATLAS_OK;
}

int atlas_fsk_code_demod(atlas_fsk_t ctx, int32_t code, float* h_dc, int32_t cap, int32_t* n) {
  if (!ctx || code < 0 || code >= ctx->C || !n) return ATLAS_ERR_INVALID_ARG;
  const FskGroup& g = ctx->groups[ctx->code_group[code]];
  *n = g.n_c;
  if (!h_dc || cap < g.n_c) return cap < g.n_c && h_dc ? ATLAS_ERR_INVALID_ARG : ATLAS_OK;
  CK(cudaMemcpy(h_dc, ctx->d_dc + (int64_t)code * ctx->max_nc, sizeof(float) * g.n_c, cudaMemcpyDeviceToHost));
  return ATLAS_OK;
}

int atlas_fsk_profile_begin(atlas_fsk_t ctx, int32_t max_timed) {
  if (!ctx || max_timed < 0) return ATLAS_ERR_INVALID_ARG;
  for (auto* v : {&ctx->ev_corr, &ctx->ev_demod}) {
    while ((int)v->size() < 2 * max_timed) {
      cudaEvent_t e;
      CK(cudaEventCreate(&e));
      v->push_back(e);
    }
  }
  ctx->profiling = true;
  ctx->corr_used = ctx->demod_used = 0;
  ctx->prof = atlas_fsk_profile{};
  return ATLAS_OK;
}

int atlas_fsk_profile_end(atlas_fsk_t ctx, atlas_fsk_profile* out) {
  if (!ctx || !out || !ctx->profiling) return ATLAS_ERR_INVALID_ARG;
  ctx->profiling = false;
  atlas_fsk_profile p = ctx->prof;
  for (int i = 0; i < ctx->corr_used; ++i) {
    float ms = 0.f;
    CK(cudaEventSynchronize(ctx->ev_corr[2 * i + 1]));
    CK(cudaEventElapsedTime(&ms, ctx->ev_corr[2 * i], ctx->ev_corr[2 * i + 1]));
    p.corr_ms += ms;
  }
  for (int i = 0; i < ctx->demod_used; ++i) {
    float ms = 0.f;
    CK(cudaEventSynchronize(ctx->ev_demod[2 * i + 1]));
    CK(cudaEventElapsedTime(&ms, ctx->ev_demod[2 * i], ctx->ev_demod[2 * i + 1]));
    p.demod_ms += ms;
  }
  p.corr_timed = ctx->corr_used;
  p.demod_timed = ctx->demod_used;
  *out = p;
  return ATLAS_OK;
}

const char* atlas_fsk_last_error(atlas_fsk_t ctx) { return ctx ? ctx->last_error.c_str() : ""; }

void atlas_fsk_destroy(atlas_fsk_t ctx) { free_ctx(ctx); }

}  // extern "C"
