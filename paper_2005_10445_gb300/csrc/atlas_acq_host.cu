// atlas_acq_host.cu -- host side of the C ABI declared in include/atlas_acq.h:
// context creation (code bank, workspaces, twiddle tables), argument
// validation, and the stream-ordered launch sequence of a search.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <fstream>
#include <map>
#include <sstream>
#include <new>
#include <string>
#include <vector>

#include "acq_internal.h"
#include "host_util.h"
#include "atlas_acq.h"
#include "prop_internal.h"

using atlas::CodeBankParams;
using atlas::CorrParams;
using atlas::RefineParams;
using atlas::SelectParams;
using atlas::WindowFftParams;

namespace atlas {

// turns * 2^64 of f/fs, reduced to [-1/2, 1/2) turns, as two's complement.
uint64_t phase_increment(double f_hz, double fs_hz) {
  double t = f_hz / fs_hz;
  t -= nearbyint(t);
  if (t >= 0.5) t -= 1.0;
  const double scaled = ldexp(t, 64);
  return (uint64_t)(int64_t)llrint(scaled);
}

// W_M^t = exp(-2 pi i t / M): HI[i] = W^{i << LB}, LO[i] = W^i, FP64 then rounded.
std::vector<float2> twiddle_tables(int logM) {
  const int LB = logM / 2, HB = logM - LB;
  const int nlo = 1 << LB, nhi = 1 << HB;
  const double M = (double)(1 << logM);
  std::vector<float2> t(nlo + nhi);
  const double two_pi = 6.283185307179586476925286766559;
  for (int i = 0; i < nhi; ++i) {
    const double a = -two_pi * (double)((int64_t)i << LB) / M;
    t[i] = make_float2((float)cos(a), (float)sin(a));
  }
  for (int i = 0; i < nlo; ++i) {
    const double a = -two_pi * (double)i / M;
    t[nhi + i] = make_float2((float)cos(a), (float)sin(a));
  }
  return t;
}

}  // namespace atlas

namespace {

// Codes of one length share windows (hop = N - L) and therefore the window
// spectra; each such group is searched by one launch sequence.
struct Group {
  int n_chips = 0, L = 0, N = 0, M = 0, logM = 0, hop = 0;
  bool split = false;          // two-block transforms (always for M = 2^15, optional for 2^14)
  int loge = 5;                // log2 of complex values per thread in the transform kernels
  int wc = 0;                  // windows per launch group (0 = the context default)
  std::vector<int> codes;      // global code ids
  int* d_codes = nullptr;      // [Cg]
  float2* d_spec = nullptr;    // [Cg][M] conj(FFT_M(chips)) / M
  float2* d_spec3 = nullptr;   // M = 2^15: [Cg][3][M/2] tables of the split correlation
  const float2* d_tw_full = nullptr;  // tables of M
  const float2* d_tw_half = nullptr;  // tables of M / 2
  const float2* tw() const { return split ? d_tw_half : d_tw_full; }  // tables of the block transform
  int parts() const { return split ? 2 : 1; }  // partial results per (cell, rho)
  int windows(int64_t S) const {
    if (S <= N) return 1;
    return (int)((S - N + hop - 1) / hop) + 1;
  }
};

}  // namespace

struct atlas_acq_ctx {
  int device = 0;
  int C = 0, K = 0, sps = 0;
  double fs = 0.0;
  float threshold = 25.f;
  int max_L = 0;
  int windows_per_launch = 0;
  int precision = 0;  // 0 FP32; 1 / 2: FP16 / BF16 tensor-core inverse transforms (M = 2^14)
  std::vector<int> n_chips;
  std::vector<double> freqs;
  std::vector<Group> groups;
  std::vector<int> code_group;  // code -> group index
  // device resources
  int8_t* d_chips = nullptr;
  int64_t* d_chip_off = nullptr;
  int* d_n_chips = nullptr;
  int* d_hop = nullptr;
  uint64_t* d_inc = nullptr;
  std::map<int, float2*> d_tw;  // logM -> twiddle tables
  float2* d_G = nullptr;
  size_t G_elems = 0;
  float4* d_part = nullptr;
  size_t part_elems = 0;
  // per-pair selection results of one launch group (the many-block selection)
  int* d_sel_flags = nullptr;
  atlas_detection* d_sel_recs = nullptr;
  int* d_status = nullptr;
  // the selection of a launch group runs on a side stream, overlapping the next
  // group's mix and window transforms (its partial results are read before the
  // next correlation overwrites them: ev_sel orders the two)
  cudaStream_t aux = nullptr;
  cudaEvent_t ev_corr = nullptr, ev_sel = nullptr;
  int wc_max = 1;  // windows per launch group (sizes the workspaces)
  // host-buffer path (allocated on first use per size, kept)
  float2* d_stage = nullptr;
  int64_t stage_samples = 0;
  cudaStream_t copy_st = nullptr;  // the second part of the host-to-device copy
  cudaEvent_t ev_copy_in = nullptr, ev_copy_done = nullptr;
  atlas_detection* d_stage_out = nullptr;
  int stage_cap = 0;
  int* d_stage_count = nullptr;
  std::string last_error;
  // proposal-search workspace (grown on first use, kept)
  int2* d_items = nullptr;
  int4* d_pairs = nullptr;
  float4* d_pair_stats = nullptr;
  int list_cap = 0;
  atlas_detection* d_fb_out = nullptr;
  int fb_cap = 0;
  int* d_fb_count = nullptr;
  // profiling (atlas_acq_profile_begin / _end)
  bool profiling = false;
  std::vector<cudaEvent_t> ev;  // pairs
  int ev_used = 0;
  int64_t prof_launches = 0, prof_corr_launches = 0, prof_corr_units = 0;
};

namespace {

int fail_cuda(atlas_acq_ctx* ctx, cudaError_t e) {
  if (ctx) ctx->last_error = cudaGetErrorString(e);
  return ATLAS_ERR_CUDA;
}

#define CK(call)                                   \
  do {                                             \
    cudaError_t e_ = (call);                       \
    if (e_ != cudaSuccess) return fail_cuda(ctx, e_); \
  } while (0)

bool is_pow2(int64_t v) { return v > 0 && (v & (v - 1)) == 0; }

int __float_as_int_host(float f) {
  int i;
  memcpy(&i, &f, sizeof(i));
  return i;
}
int ilog2(int64_t v) {
  int r = 0;
  while ((1ll << r) < v) ++r;
  return r;
}

using atlas::phase_increment;
using atlas::twiddle_tables;

void free_ctx(atlas_acq_ctx* ctx) {
  if (!ctx) return;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(ctx->device);
  for (auto& g : ctx->groups) {
    cudaFree(g.d_codes);
    cudaFree(g.d_spec);
    cudaFree(g.d_spec3);
  }
  for (auto& kv : ctx->d_tw) cudaFree(kv.second);
  cudaFree(ctx->d_chips);
  cudaFree(ctx->d_chip_off);
  cudaFree(ctx->d_n_chips);
  cudaFree(ctx->d_hop);
  cudaFree(ctx->d_inc);
  cudaFree(ctx->d_G);
  cudaFree(ctx->d_part);
  cudaFree(ctx->d_sel_flags);
  cudaFree(ctx->d_sel_recs);
  cudaFree(ctx->d_status);
  cudaFree(ctx->d_stage);
  cudaFree(ctx->d_stage_out);
  cudaFree(ctx->d_stage_count);
  if (ctx->ev_corr) cudaEventDestroy(ctx->ev_corr);
  if (ctx->ev_sel) cudaEventDestroy(ctx->ev_sel);
  if (ctx->aux) cudaStreamDestroy(ctx->aux);
  if (ctx->ev_copy_in) cudaEventDestroy(ctx->ev_copy_in);
  if (ctx->ev_copy_done) cudaEventDestroy(ctx->ev_copy_done);
  if (ctx->copy_st) cudaStreamDestroy(ctx->copy_st);
  cudaFree(ctx->d_items);
  cudaFree(ctx->d_pairs);
  cudaFree(ctx->d_pair_stats);
  cudaFree(ctx->d_fb_out);
  cudaFree(ctx->d_fb_count);
  for (auto e : ctx->ev) cudaEventDestroy(e);
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

int create_impl(atlas_acq_ctx* ctx, const int8_t* chips, const int32_t* chips_per_code, int32_t n_codes,
                int32_t sps, double fs_hz, const double* freqs, int32_t n_freq, const atlas_acq_opts& o) {
  ctx->C = n_codes;
  ctx->K = n_freq;
  ctx->sps = sps;
  ctx->fs = fs_hz;
  ctx->threshold = o.threshold;
  ctx->windows_per_launch = o.windows_per_launch;
  ctx->precision = o.precision;
  ctx->freqs.assign(freqs, freqs + n_freq);
  ctx->n_chips.assign(chips_per_code, chips_per_code + n_codes);

  // groups by code length
  std::map<int, int> by_len;
  std::vector<int64_t> off(n_codes);
  int64_t total = 0;
  ctx->code_group.resize(n_codes);
  for (int c = 0; c < n_codes; ++c) {
    off[c] = total;
    total += chips_per_code[c];
    const int nc = chips_per_code[c];
    auto it = by_len.find(nc);
    if (it == by_len.end()) {
      Group g;
      g.n_chips = nc;
      g.L = nc * sps;
      g.N = o.fft_len ? o.fft_len : 2 * (int)(1ll << ilog2(g.L));
      if (!is_pow2(g.N) || g.N <= g.L) return o.fft_len ? ATLAS_ERR_UNSUPPORTED : ATLAS_ERR_INVALID_ARG;
      g.M = g.N / sps;
      g.logM = ilog2(g.M);
      if (g.logM < atlas::kMinLogM || g.logM > atlas::kMaxLogM) return ATLAS_ERR_UNSUPPORTED;
      g.hop = g.N - g.L;
      g.split = (g.logM == 15) || (g.logM == 14 && o.split == 1);
      if (o.tile_log2 == 4 || o.tile_log2 == 5) g.loge = o.tile_log2;
      else if (o.tile_log2 != 0) return ATLAS_ERR_INVALID_ARG;
      if (o.split != 0 && o.split != 1) return ATLAS_ERR_INVALID_ARG;
      by_len[nc] = (int)ctx->groups.size();
      ctx->groups.push_back(g);
      it = by_len.find(nc);
    }
    ctx->code_group[c] = it->second;
    ctx->groups[it->second].codes.push_back(c);
    ctx->max_L = std::max(ctx->max_L, nc * sps);
  }
  for (int64_t i = 0; i < total; ++i)
    if (chips[i] != 1 && chips[i] != -1) return ATLAS_ERR_INVALID_ARG;

  CK(cudaGetDevice(&ctx->device));
  CK(atlas::prepare_kernels());
  CK(upload(&ctx->d_chips, chips, (size_t)total));
  CK(upload(&ctx->d_chip_off, off.data(), off.size()));
  CK(upload(&ctx->d_n_chips, chips_per_code, (size_t)n_codes));
  std::vector<int> hops(n_codes);
  for (int c = 0; c < n_codes; ++c) hops[c] = ctx->groups[ctx->code_group[c]].hop;
  CK(upload(&ctx->d_hop, hops.data(), hops.size()));
  std::vector<uint64_t> inc(n_freq);
  for (int k = 0; k < n_freq; ++k) inc[k] = phase_increment(freqs[k], fs_hz);
  CK(upload(&ctx->d_inc, inc.data(), inc.size()));
  CK(cudaMalloc((void**)&ctx->d_status, sizeof(int)));
  CK(cudaMemset(ctx->d_status, 0, sizeof(int)));
  CK(cudaStreamCreateWithFlags(&ctx->aux, cudaStreamNonBlocking));
  CK(cudaEventCreateWithFlags(&ctx->ev_corr, cudaEventDisableTiming));
  CK(cudaEventCreateWithFlags(&ctx->ev_sel, cudaEventDisableTiming));

  // windows per launch group: as many as a 2 GiB workspace of window spectra
  // holds (at most 64).  The correlation takes the codes of one window before
  // the next window, so one window's spectra (31 MiB for 31 bins at N = 2^17)
  // are what must stay in L2; larger groups only cut launches and tails
  // (realistic stream: 4 windows 29.03 ms, 16 windows 28.41, 64 windows 28.05)
  const size_t budget = 2048ull << 20;
  size_t max_win_bytes = 0;
  size_t max_part_per_win = 0;
  size_t max_codes = 0;
  for (auto& g : ctx->groups) {
    max_win_bytes = std::max(max_win_bytes, (size_t)n_freq * g.N * sizeof(float2));
    max_part_per_win = std::max(max_part_per_win, (size_t)g.codes.size() * n_freq * sps * 2);
    max_codes = std::max(max_codes, g.codes.size());
  }
  int wc = o.windows_per_launch > 0 ? o.windows_per_launch : (int)std::max<size_t>(1, budget / max_win_bytes);
  wc = std::min(wc, 64);
  ctx->wc_max = wc;
  ctx->G_elems = (size_t)wc * max_win_bytes / sizeof(float2);
  ctx->part_elems = (size_t)wc * max_part_per_win;
  if (cudaMalloc((void**)&ctx->d_G, ctx->G_elems * sizeof(float2)) != cudaSuccess) return ATLAS_ERR_NO_MEMORY;
  if (cudaMalloc((void**)&ctx->d_part, ctx->part_elems * sizeof(float4)) != cudaSuccess) return ATLAS_ERR_NO_MEMORY;
  const size_t sel_pairs = (size_t)wc * max_codes;
  if (cudaMalloc((void**)&ctx->d_sel_flags, sel_pairs * sizeof(int)) != cudaSuccess ||
      cudaMalloc((void**)&ctx->d_sel_recs, sel_pairs * sizeof(atlas_detection)) != cudaSuccess)
    return ATLAS_ERR_NO_MEMORY;

  // twiddle tables and code banks
  auto tables = [&](int lm, const float2** dst) -> int {
    if (!ctx->d_tw.count(lm)) {
      std::vector<float2> t = twiddle_tables(lm);
      float2* d = nullptr;
      CK(upload(&d, t.data(), t.size()));
      ctx->d_tw[lm] = d;
    }
    *dst = ctx->d_tw[lm];
    return ATLAS_OK;
  };
  for (auto& g : ctx->groups) {
    int st = tables(g.logM, &g.d_tw_full);
    if (st != ATLAS_OK) return st;
    if (g.logM > atlas::kMinLogM && (st = tables(g.logM - 1, &g.d_tw_half)) != ATLAS_OK) return st;
    CK(upload(&g.d_codes, g.codes.data(), g.codes.size()));
    if (cudaMalloc((void**)&g.d_spec, sizeof(float2) * (size_t)g.M * g.codes.size()) != cudaSuccess)
      return ATLAS_ERR_NO_MEMORY;
    if (g.logM == 15 &&
        cudaMalloc((void**)&g.d_spec3, sizeof(float2) * (size_t)3 * (g.M / 2) * g.codes.size()) != cudaSuccess)
      return ATLAS_ERR_NO_MEMORY;
    std::vector<int64_t> goff(g.codes.size());
    std::vector<int> gn(g.codes.size());
    for (size_t i = 0; i < g.codes.size(); ++i) {
      goff[i] = off[g.codes[i]];
      gn[i] = chips_per_code[g.codes[i]];
    }
    int64_t* d_goff = nullptr;
    int* d_gn = nullptr;
    CK(upload(&d_goff, goff.data(), goff.size()));
    CK(upload(&d_gn, gn.data(), gn.size()));
    CodeBankParams p;
    p.chips = ctx->d_chips;
    p.chip_off = d_goff;
    p.n_chips = d_gn;
    p.tw = g.logM == 15 ? g.d_tw_half : g.d_tw_full;
    p.D = g.d_spec;
    p.D3 = g.d_spec3;
    p.M = g.M;
    p.scale = 1.0f / (float)g.M;
    cudaError_t e = atlas::launch_code_bank(g.logM, p, (int)g.codes.size(), 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    cudaFree(d_goff);
    cudaFree(d_gn);
    if (e != cudaSuccess) return fail_cuda(ctx, e);
  }
  return ATLAS_OK;
}

// One launch group: windows [w0, w0 + nw) of group g (mix, window transforms,
// per-code correlation, selection appending to out / d_count).
// sel_pending: a selection of this run is in flight on the side stream (its
// completion must be awaited before the partial results are rewritten).
int launch_chunk(atlas_acq_ctx* ctx, const Group& g, cudaStream_t st, const float2* x, int64_t S, int W, int w0,
                 int nw, atlas_cell* cells, atlas_detection* out, int capacity, int* d_count, bool profiling,
                 bool& sel_pending) {
  const int Cg = (int)g.codes.size();
  atlas::MixParams m;
  m.x = x;
  m.S = S;
  m.N = g.N;
  m.M = g.M;
  m.sps = ctx->sps;
  m.hop = g.hop;
  m.w0 = w0;
  m.nw = nw;
  m.K = ctx->K;
  m.inc = ctx->d_inc;
  m.B = ctx->d_G;
  CK(atlas::launch_mix(m, st));
  WindowFftParams a;
  a.M = g.M;
  a.sps = ctx->sps;
  a.K = ctx->K;
  a.nw = nw;
  a.tw = g.tw();
  a.G = ctx->d_G;
  CK(atlas::launch_window_fft(g.logM, g.loge, g.split, a, st));
  if (profiling) ctx->prof_launches += 2;
  CorrParams b;
  b.G = ctx->d_G;
  b.D = g.d_spec;
  b.D3 = g.d_spec3;
  b.tw = g.tw();
  b.tw2 = g.d_tw_full;
  b.part = ctx->d_part;
  b.S = S;
  b.N = g.N;
  b.M = g.M;
  b.sps = ctx->sps;
  b.hop = g.hop;
  b.W = W;
  b.L = g.L;
  b.w0 = w0;
  b.nw = nw;
  b.K = ctx->K;
  b.Cg = Cg;
  b.status = ctx->d_status;
  const bool timed = profiling && 2 * ctx->ev_used + 1 < (int)ctx->ev.size();
  if (timed) CK(cudaEventRecord(ctx->ev[2 * ctx->ev_used], st));
  if (sel_pending) CK(cudaStreamWaitEvent(st, ctx->ev_sel, 0));  // previous selection has read the partials
  if (ctx->precision != 0 && g.logM == 14 && !g.split) CK(atlas::launch_corr_tc5(ctx->precision, b, st));
  else CK(atlas::launch_corr(g.logM, g.loge, g.split, b, st));
  if (timed) {
    CK(cudaEventRecord(ctx->ev[2 * ctx->ev_used + 1], st));
    ctx->ev_used += 1;
  }
  if (profiling) {
    ctx->prof_launches += 1;
    ctx->prof_corr_launches += 1;
    ctx->prof_corr_units += (int64_t)nw * Cg * ctx->K;
  }
  SelectParams c;
  c.part = ctx->d_part;
  c.codes = g.d_codes;
  c.Cg = Cg;
  c.C = ctx->C;
  c.K = ctx->K;
  c.sps = ctx->sps * g.parts();
  c.N = g.N;
  c.W = W;
  c.w0 = w0;
  c.nw = nw;
  c.threshold = ctx->threshold;
  c.out = out;
  c.capacity = capacity;
  c.count = d_count;
  c.cells = cells;
  c.tmp_flags = ctx->d_sel_flags;  // the selections of a context run in order on its side stream
  c.tmp_recs = ctx->d_sel_recs;
  CK(cudaEventRecord(ctx->ev_corr, st));
  CK(cudaStreamWaitEvent(ctx->aux, ctx->ev_corr, 0));
  CK(atlas::launch_select(c, ctx->aux));
  CK(cudaEventRecord(ctx->ev_sel, ctx->aux));
  sel_pending = true;
  if (profiling) ctx->prof_launches += atlas::select_launches(c);
  return ATLAS_OK;
}

int launch_refine_all(atlas_acq_ctx* ctx, cudaStream_t st, const float2* x, int64_t S, atlas_detection* out,
                      int capacity, const int* d_count) {
  if (capacity <= 0) return ATLAS_OK;
  RefineParams r;
  r.x = x;
  r.S = S;
  r.chips = ctx->d_chips;
  r.chip_off = ctx->d_chip_off;
  r.chips_per_code = ctx->d_n_chips;
  r.hop = ctx->d_hop;
  r.inc = ctx->d_inc;
  r.sps = ctx->sps;
  r.out = out;
  r.capacity = capacity;
  r.count = d_count;
  CK(atlas::launch_refine(r, std::min(capacity, 1024), st));
  return ATLAS_OK;
}

// only_group >= 0 restricts the search to one code-length group (autotuning).
int run_impl(atlas_acq_ctx* ctx, cudaStream_t st, const float2* x, int64_t S, atlas_cell* cells,
             atlas_detection* out, int capacity, int* d_count, int only_group = -1,
             cudaEvent_t rest_ready = nullptr) {
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  CK(cudaStreamIsCapturing(st, &cap));
  const bool profiling = ctx->profiling && cap == cudaStreamCaptureStatusNone;
  CK(cudaMemsetAsync(d_count, 0, sizeof(int), st));
  if (cells) {
    int wmax = 0;
    for (auto& g : ctx->groups) wmax = std::max(wmax, g.windows(S));
    CK(cudaMemsetAsync(cells, 0, sizeof(atlas_cell) * (size_t)wmax * ctx->C * ctx->K, st));
  }
  bool sel_pending = false;
  for (int gi = 0; gi < (int)ctx->groups.size(); ++gi) {
    if (only_group >= 0 && gi != only_group) continue;
    const Group& g = ctx->groups[gi];
    const int W = g.windows(S);
    int wc = std::max(1, std::min<int>(ctx->wc_max, (int)(ctx->G_elems / ((size_t)ctx->K * g.N))));
    if (g.wc > 0) wc = std::min(wc, g.wc);
    for (int w0 = 0; w0 < W; w0 += wc) {
      // rest_ready: only the samples of the first launch group are known to be on the device
      if (rest_ready && !(gi == 0 && w0 == 0)) {
        CK(cudaStreamWaitEvent(st, rest_ready, 0));
        rest_ready = nullptr;
      }
      const int r = launch_chunk(ctx, g, st, x, S, W, w0, std::min(wc, W - w0), cells, out, capacity, d_count,
                                 profiling, sel_pending);
      if (r != ATLAS_OK) return r;
    }
  }
  if (rest_ready) CK(cudaStreamWaitEvent(st, rest_ready, 0));  // the refinement reads the whole stream
  if (sel_pending) CK(cudaStreamWaitEvent(st, ctx->ev_sel, 0));  // every selection joins the caller's stream
  const int r = launch_refine_all(ctx, st, x, S, out, capacity, d_count);
  if (r == ATLAS_OK && profiling && capacity > 0) ctx->prof_launches += 1;
  return r;
}

int check_run_args(atlas_acq_ctx* ctx, const void* x, int64_t S, const void* out, int capacity,
                   const void* count) {
  if (!ctx || !x || !count || capacity < 0 || (capacity > 0 && !out)) return ATLAS_ERR_INVALID_ARG;
  if (S < ctx->max_L || S > (int64_t)INT32_MAX * 8) return ATLAS_ERR_INVALID_ARG;
  int dev = 0;  // the workspaces live on the context's device
  if (cudaGetDevice(&dev) != cudaSuccess || dev != ctx->device) return ATLAS_ERR_INVALID_ARG;
  return ATLAS_OK;
}

}  // namespace

extern "C" {

void atlas_acq_default_opts(atlas_acq_opts* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->threshold = 25.f;
  o->fft_len = 0;
  o->windows_per_launch = 0;
  o->tile_log2 = 0;
}

int atlas_acq_create(atlas_acq_t* out, const int8_t* chips, const int32_t* chips_per_code, int32_t n_codes,
                     int32_t samples_per_chip, double fs_hz, const double* freq_offsets_hz, int32_t n_freq,
                     const atlas_acq_opts* opts) {
  if (!out) return ATLAS_ERR_INVALID_ARG;
  *out = nullptr;
  if (!chips || !chips_per_code || n_codes <= 0 || samples_per_chip <= 0 || !(fs_hz > 0.0) ||
      !freq_offsets_hz || n_freq <= 0)
    return ATLAS_ERR_INVALID_ARG;
  if (!is_pow2(samples_per_chip) || samples_per_chip > atlas::kMaxSps) return ATLAS_ERR_UNSUPPORTED;
  for (int c = 0; c < n_codes; ++c)
    if (chips_per_code[c] <= 0) return ATLAS_ERR_INVALID_ARG;
  for (int k = 0; k < n_freq; ++k)
    if (!isfinite(freq_offsets_hz[k])) return ATLAS_ERR_INVALID_ARG;
  atlas_acq_opts o;
  atlas_acq_default_opts(&o);
  if (opts) o = *opts;
  if (!(o.threshold >= 0.f) || o.fft_len < 0 || o.windows_per_launch < 0 || o.precision < 0 || o.precision > 2)
    return ATLAS_ERR_INVALID_ARG;
  atlas_acq_ctx* ctx = new (std::nothrow) atlas_acq_ctx();
  if (!ctx) return ATLAS_ERR_NO_MEMORY;
  const int st = create_impl(ctx, chips, chips_per_code, n_codes, samples_per_chip, fs_hz, freq_offsets_hz,
                             n_freq, o);
  if (st != ATLAS_OK) {
    free_ctx(ctx);
    return st;
  }
  *out = ctx;
  return ATLAS_OK;
}

int atlas_acq_windows(atlas_acq_t ctx, int32_t code, int64_t n_samples, int32_t* n_windows, int32_t* hop,
                      int32_t* fft_len) {
  if (!ctx || code < 0 || code >= ctx->C || n_samples < ctx->max_L) return ATLAS_ERR_INVALID_ARG;
  const Group& g = ctx->groups[ctx->code_group[code]];
  if (n_windows) *n_windows = g.windows(n_samples);
  if (hop) *hop = g.hop;
  if (fft_len) *fft_len = g.N;
  return ATLAS_OK;
}

int atlas_acq_run(atlas_acq_t ctx, void* stream, const float* d_iq, int64_t n_samples, atlas_detection* d_out,
                  int32_t capacity, int32_t* d_count) {
  const int a = check_run_args(ctx, d_iq, n_samples, d_out, capacity, d_count);
  if (a != ATLAS_OK) return a;
  return run_impl(ctx, (cudaStream_t)stream, reinterpret_cast<const float2*>(d_iq), n_samples, nullptr, d_out,
                  capacity, d_count);
}

int atlas_acq_run_cells(atlas_acq_t ctx, void* stream, const float* d_iq, int64_t n_samples, atlas_cell* d_cells,
                        atlas_detection* d_out, int32_t capacity, int32_t* d_count) {
  const int a = check_run_args(ctx, d_iq, n_samples, d_out, capacity, d_count);
  if (a != ATLAS_OK) return a;
  if (!d_cells) return ATLAS_ERR_INVALID_ARG;
  return run_impl(ctx, (cudaStream_t)stream, reinterpret_cast<const float2*>(d_iq), n_samples, d_cells, d_out,
                  capacity, d_count);
}

int atlas_acq_run_host(atlas_acq_t ctx, void* stream, const float* h_iq, int64_t n_samples, atlas_detection* h_out,
                       int32_t capacity, int32_t* h_count) {
  const int a = check_run_args(ctx, h_iq, n_samples, h_out, capacity, h_count);
  if (a != ATLAS_OK) return a;
  cudaStream_t st = (cudaStream_t)stream;
  if (ctx->stage_samples < n_samples) {
    CK(cudaFree(ctx->d_stage));
    ctx->d_stage = nullptr;
    ctx->stage_samples = 0;
    if (cudaMalloc((void**)&ctx->d_stage, sizeof(float2) * (size_t)n_samples) != cudaSuccess)
      return ATLAS_ERR_NO_MEMORY;
    ctx->stage_samples = n_samples;
  }
  if (ctx->stage_cap < std::max(capacity, 1)) {
    CK(cudaFree(ctx->d_stage_out));
    ctx->d_stage_out = nullptr;
    ctx->stage_cap = 0;
    if (cudaMalloc((void**)&ctx->d_stage_out, sizeof(atlas_detection) * (size_t)std::max(capacity, 1)) !=
        cudaSuccess)
      return ATLAS_ERR_NO_MEMORY;
    ctx->stage_cap = std::max(capacity, 1);
  }
  if (!ctx->d_stage_count) {
    if (cudaMalloc((void**)&ctx->d_stage_count, sizeof(int)) != cudaSuccess) return ATLAS_ERR_NO_MEMORY;
  }
  // The first launch group's samples go on the caller's stream; the rest on a
  // copy stream, overlapping that group's transforms (its later groups and the
  // refinement wait for the copy).  The copy stream first waits for the
  // caller's earlier work, which may still read the staging buffer.
  const Group& g0 = ctx->groups[0];
  int wc0 = std::max(1, std::min<int>(ctx->wc_max, (int)(ctx->G_elems / ((size_t)ctx->K * g0.N))));
  if (g0.wc > 0) wc0 = std::min(wc0, g0.wc);
  const int64_t head = std::min<int64_t>(n_samples, (int64_t)(std::min(wc0, g0.windows(n_samples)) - 1) * g0.hop + g0.N);
  const float2* h2 = reinterpret_cast<const float2*>(h_iq);
  cudaEvent_t rest = nullptr;
  if (head < n_samples) {
    if (!ctx->copy_st) {
      CK(cudaStreamCreateWithFlags(&ctx->copy_st, cudaStreamNonBlocking));
      CK(cudaEventCreateWithFlags(&ctx->ev_copy_in, cudaEventDisableTiming));
      CK(cudaEventCreateWithFlags(&ctx->ev_copy_done, cudaEventDisableTiming));
    }
    CK(cudaEventRecord(ctx->ev_copy_in, st));
    CK(cudaStreamWaitEvent(ctx->copy_st, ctx->ev_copy_in, 0));
    CK(cudaMemcpyAsync(ctx->d_stage, h2, sizeof(float2) * (size_t)head, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(ctx->d_stage + head, h2 + head, sizeof(float2) * (size_t)(n_samples - head),
                       cudaMemcpyHostToDevice, ctx->copy_st));
    CK(cudaEventRecord(ctx->ev_copy_done, ctx->copy_st));
    rest = ctx->ev_copy_done;
  } else {
    CK(cudaMemcpyAsync(ctx->d_stage, h_iq, sizeof(float2) * (size_t)n_samples, cudaMemcpyHostToDevice, st));
  }
  const int r = run_impl(ctx, st, ctx->d_stage, n_samples, nullptr, ctx->d_stage_out, capacity, ctx->d_stage_count,
                         -1, rest);
  if (r != ATLAS_OK) return r;
  CK(cudaMemcpyAsync(h_count, ctx->d_stage_count, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  const int n = std::min(*h_count, capacity);
  if (n > 0) {
    CK(cudaMemcpyAsync(h_out, ctx->d_stage_out, sizeof(atlas_detection) * (size_t)n, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
  }
  return ATLAS_OK;
}

int atlas_acq_autotune(atlas_acq_t ctx, void* stream, const float* d_iq, int64_t n_samples,
                       const char* cache_path) {
  const int a = check_run_args(ctx, d_iq, n_samples, nullptr, 0, d_iq);
  if (a != ATLAS_OK) return a;
  cudaStream_t st = (cudaStream_t)stream;
  cudaDeviceProp prop;
  CK(cudaGetDeviceProperties(&prop, ctx->device));
  // cache: one JSON object per line
  // {"key": "...", "tile_log2": t, "windows_per_launch": w, "split": s, "ms": m}
  struct Choice {
    int t, w, s;
  };
  std::map<std::string, Choice> cache;
  if (cache_path) {
    std::ifstream in(cache_path);
    std::string line;
    while (std::getline(in, line)) {
      char key[512];
      int t = 0, w = 0, sp = 0;
      double ms = 0.0;
      if (sscanf(line.c_str(),
                 "{\"key\": \"%511[^\"]\", \"tile_log2\": %d, \"windows_per_launch\": %d, \"split\": %d, "
                 "\"ms\": %lf}",
                 key, &t, &w, &sp, &ms) == 5 &&
          (t == 4 || t == 5) && w >= 1 && (sp == 0 || sp == 1))
        cache[key] = Choice{t, w, sp};
    }
  }
  atlas_detection* d_out = nullptr;
  int* d_count = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int status = ATLAS_OK;
  auto fail = [&](cudaError_t e) {
    ctx->last_error = cudaGetErrorString(e);
    status = ATLAS_ERR_CUDA;
  };
  cudaError_t e;
  if ((e = cudaMalloc((void**)&d_out, sizeof(atlas_detection) * 64)) != cudaSuccess ||
      (e = cudaMalloc((void**)&d_count, sizeof(int))) != cudaSuccess || (e = cudaEventCreate(&e0)) != cudaSuccess ||
      (e = cudaEventCreate(&e1)) != cudaSuccess)
    fail(e);
  std::ofstream outf;
  if (status == ATLAS_OK && cache_path) outf.open(cache_path, std::ios::app);
  const bool was_profiling = ctx->profiling;
  ctx->profiling = false;
  for (int gi = 0; status == ATLAS_OK && gi < (int)ctx->groups.size(); ++gi) {
    Group& g = ctx->groups[gi];
    std::ostringstream ks;
    ks << prop.name << "|N=" << g.N << "|M=" << g.M << "|sps=" << ctx->sps << "|K=" << ctx->K
       << "|codes=" << g.codes.size();
    const std::string key = ks.str();
    auto it = cache.find(key);
    if (it != cache.end()) {
      g.loge = it->second.t;
      g.wc = it->second.w;
      g.split = g.logM == 15 || (g.logM == 14 && it->second.s == 1);
      continue;
    }
    // time on (at most) the first 64 windows of the group
    const int64_t S_tune = std::min<int64_t>(n_samples, (int64_t)g.N + 63ll * g.hop);
    const int W = g.windows(S_tune);
    const int fit = std::max(1, (int)(ctx->G_elems / ((size_t)ctx->K * g.N)));
    int best_t = g.loge, best_w = g.wc;
    bool best_s = g.split;
    double best_ms = 1e30;
    std::vector<bool> splits;
    if (g.logM == 15) splits = {true};
    else if (g.logM == 14) splits = {false, true};
    else splits = {false};
    for (bool sp : splits)
    for (int t : {5, 4}) {
      for (int w : {1, 2, 4, 8, 16, 32, 64}) {
        if (w > std::min(fit, ctx->wc_max) || (w > 1 && w >= 2 * W)) continue;
        g.loge = t;
        g.wc = w;
        g.split = sp;
        int r = run_impl(ctx, st, reinterpret_cast<const float2*>(d_iq), S_tune, nullptr, d_out, 64, d_count, gi);
        if (r != ATLAS_OK) {
          status = r;
          break;
        }
        if ((e = cudaEventRecord(e0, st)) != cudaSuccess) { fail(e); break; }
        for (int rep = 0; rep < 2 && status == ATLAS_OK; ++rep)
          status = run_impl(ctx, st, reinterpret_cast<const float2*>(d_iq), S_tune, nullptr, d_out, 64, d_count, gi);
        if (status != ATLAS_OK) break;
        float ms = 0.f;
        if ((e = cudaEventRecord(e1, st)) != cudaSuccess || (e = cudaEventSynchronize(e1)) != cudaSuccess ||
            (e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) {
          fail(e);
          break;
        }
        if (ms / 2 < best_ms) {
          best_ms = ms / 2;
          best_t = t;
          best_w = w;
          best_s = sp;
        }
      }
      if (status != ATLAS_OK) break;
    }
    g.loge = best_t;
    g.wc = best_w;
    g.split = best_s;
    if (status == ATLAS_OK && outf.is_open())
      outf << "{\"key\": \"" << key << "\", \"tile_log2\": " << best_t << ", \"windows_per_launch\": " << best_w
           << ", \"split\": " << (best_s ? 1 : 0) << ", \"ms\": " << best_ms << "}\n";
  }
  ctx->profiling = was_profiling;
  cudaFree(d_out);
  cudaFree(d_count);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  return status;
}

int atlas_acq_tuning(atlas_acq_t ctx, int32_t code, int32_t* tile_log2, int32_t* windows_per_launch,
                     int32_t* split) {
  if (!ctx || code < 0 || code >= ctx->C) return ATLAS_ERR_INVALID_ARG;
  const Group& g = ctx->groups[ctx->code_group[code]];
  if (tile_log2) *tile_log2 = g.loge;
  if (split) *split = g.split ? 1 : 0;
  if (windows_per_launch) {
    const int fit = std::max(1, std::min<int>(ctx->wc_max, (int)(ctx->G_elems / ((size_t)ctx->K * g.N))));
    *windows_per_launch = g.wc > 0 ? std::min(g.wc, fit) : fit;
  }
  return ATLAS_OK;
}

int atlas_acq_profile_begin(atlas_acq_t ctx, int32_t max_timed) {
  if (!ctx || max_timed < 0) return ATLAS_ERR_INVALID_ARG;
  for (auto e : ctx->ev) cudaEventDestroy(e);
  ctx->ev.assign(2 * (size_t)max_timed, nullptr);
  for (auto& e : ctx->ev) CK(cudaEventCreate(&e));
  ctx->ev_used = 0;
  ctx->prof_launches = ctx->prof_corr_launches = ctx->prof_corr_units = 0;
  ctx->profiling = true;
  return ATLAS_OK;
}

int atlas_acq_profile_end(atlas_acq_t ctx, atlas_acq_profile* out) {
  if (!ctx || !out) return ATLAS_ERR_INVALID_ARG;
  CK(cudaDeviceSynchronize());
  double ms = 0.0;
  for (int i = 0; i < ctx->ev_used; ++i) {
    float t = 0.f;
    CK(cudaEventElapsedTime(&t, ctx->ev[2 * i], ctx->ev[2 * i + 1]));
    ms += t;
  }
  out->launches = ctx->prof_launches;
  out->corr_launches = ctx->prof_corr_launches;
  out->corr_ms = ms;
  out->corr_units = ctx->prof_corr_units;
  out->timed_launches = ctx->ev_used;
  for (auto e : ctx->ev) cudaEventDestroy(e);
  ctx->ev.clear();
  ctx->ev_used = 0;
  ctx->profiling = false;
  return ATLAS_OK;
}

}  // extern "C"

namespace {

// The proposal search: n_sel (code, bin) pairs per window (bins_mode false) or
// every code in n_sel bins per window (bins_mode true).
int run_proposed_impl(atlas_acq_t ctx, atlas_prop_t prop, void* stream, const float* d_iq, int64_t n_samples,
                      int32_t n_sel, bool bins_mode, float tau_fb, atlas_detection* d_out, int32_t capacity,
                      int32_t* d_count, int32_t* h_n_fallback) {
  const int a = check_run_args(ctx, d_iq, n_samples, d_out, capacity, d_count);
  if (a != ATLAS_OK) return a;
  if (!prop || n_sel < 1 || n_sel > 32 || !(tau_fb >= 0.f)) return ATLAS_ERR_INVALID_ARG;
  if (prop->lay.C != ctx->C || prop->lay.K != ctx->K || (bins_mode && n_sel > ctx->K)) return ATLAS_ERR_INVALID_ARG;
  if (ctx->groups.size() != 1 || ctx->groups[0].logM > 14 || ctx->groups[0].N % 4096) return ATLAS_ERR_UNSUPPORTED;
  cudaStream_t st = (cudaStream_t)stream;
  const Group& g = ctx->groups[0];
  const int W = g.windows(n_samples);
  const int K = ctx->K, C = ctx->C, sps = ctx->sps;
  const float2* x = reinterpret_cast<const float2*>(d_iq);
  const int per_window = bins_mode ? n_sel * C : n_sel;  // listed cells per window at most
  // workspaces
  if (prop->ws_windows < W) {
    cudaFree(prop->feat);
    cudaFree(prop->cand);
    cudaFree(prop->conf);
    prop->feat = nullptr;
    prop->cand = nullptr;
    prop->conf = nullptr;
    prop->ws_windows = 0;
    if (cudaMalloc((void**)&prop->feat, (size_t)W * atlas_prop_feature_len(prop) * 4) != cudaSuccess ||
        cudaMalloc((void**)&prop->cand, (size_t)W * 32 * 2 * 4) != cudaSuccess ||
        cudaMalloc((void**)&prop->conf, (size_t)W * 2 * 4) != cudaSuccess)
      return ATLAS_ERR_NO_MEMORY;
    prop->ws_windows = W;
  }
  if (ctx->list_cap < W * per_window) {
    cudaFree(ctx->d_items);
    cudaFree(ctx->d_pairs);
    cudaFree(ctx->d_pair_stats);
    ctx->d_items = nullptr;
    ctx->d_pairs = nullptr;
    ctx->d_pair_stats = nullptr;
    ctx->list_cap = 0;
    if (cudaMalloc((void**)&ctx->d_items, sizeof(int2) * (size_t)W * per_window) != cudaSuccess ||
        cudaMalloc((void**)&ctx->d_pairs, sizeof(int4) * (size_t)W * per_window) != cudaSuccess ||
        cudaMalloc((void**)&ctx->d_pair_stats, sizeof(float4) * (size_t)W * per_window) != cudaSuccess)
      return ATLAS_ERR_NO_MEMORY;
    ctx->list_cap = W * per_window;
  }
  if (!ctx->d_fb_count && cudaMalloc((void**)&ctx->d_fb_count, sizeof(int)) != cudaSuccess) return ATLAS_ERR_NO_MEMORY;
  // 1-2: features (spectrum and carrier lines of the context's grid) and candidates
  int r = atlas_prop_set_grid(prop, ctx->fs, ctx->freqs.data(), K);
  if (r != ATLAS_OK) return r;
  r = atlas_prop_features(prop, st, d_iq, n_samples, 0, g.hop, g.N, W, prop->feat);
  if (r != ATLAS_OK) return r;
  r = bins_mode ? atlas_prop_bin_candidates(prop, st, prop->feat, W, n_sel, prop->cand, prop->conf)
                : atlas_prop_candidates(prop, st, prop->feat, W, n_sel, prop->cand, prop->conf);
  if (r != ATLAS_OK) return r;
  const int topk = n_sel;
  std::vector<int> cand((size_t)W * topk * (bins_mode ? 1 : 2));
  std::vector<float> conf((size_t)W * 2);
  CK(cudaMemcpyAsync(cand.data(), prop->cand, cand.size() * 4, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(conf.data(), prop->conf, conf.size() * 4, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  // 3: work lists, per window: its distinct candidate bins (items) and its
  // (item, code) cells (pairs); item indices are local to the window
  std::vector<int> fallback;
  std::vector<int> win;                       // windows searched over candidates
  std::vector<std::vector<int2>> win_items;   // (window, bin)
  std::vector<std::vector<int4>> win_pairs;   // (local item, code, window, bin)
  for (int w = 0; w < W; ++w) {
    // confident -- pairs: sure of a (code, bin) pair, or sure the window holds no
    // transmission; bins: the proposed bins hold probability mass >= tau_fb (a
    // window without a visible carrier line is never skipped: a weak tag and an
    // empty window look alike to the features)
    const float c_w = bins_mode ? conf[2 * w] : std::max(conf[2 * w], 1.f - conf[2 * w + 1]);
    if (!(c_w >= tau_fb)) {
      fallback.push_back(w);
      continue;
    }
    std::vector<int2> it;
    std::vector<int4> pr;
    if (bins_mode) {  // every code in each proposed bin
      for (int i = 0; i < topk; ++i) {
        const int k = cand[(size_t)w * topk + i];
        if (k < 0 || k >= K) return ATLAS_ERR_DEVICE;
        it.push_back(make_int2(w, k));
        for (int c = 0; c < C; ++c) pr.push_back(make_int4(i, c, w, k));
      }
    } else {
      for (int i = 0; i < topk; ++i) {
        const int c = cand[((size_t)w * topk + i) * 2], k = cand[((size_t)w * topk + i) * 2 + 1];
        if (c < 0 || c >= C || k < 0 || k >= K) return ATLAS_ERR_DEVICE;
        int item = -1;
        for (int j = 0; j < (int)it.size(); ++j)
          if (it[j].y == k) item = j;
        if (item < 0) {
          item = (int)it.size();
          it.push_back(make_int2(w, k));
        }
        pr.push_back(make_int4(item, c, w, k));
      }
    }
    win.push_back(w);
    win_items.push_back(it);
    win_pairs.push_back(pr);
  }
  // 4: listed cells, in chunks of whole windows that fit the window-spectrum
  // and partial-result workspaces
  std::vector<int4> pairs;   // every listed cell, in chunk order (x = global item index)
  std::vector<float4> stats;
  const int items_per_chunk = std::max<int>(1, (int)(ctx->G_elems / (size_t)g.N));
  const int pairs_per_chunk = std::max<int>(1, (int)(ctx->part_elems / (size_t)sps));
  for (size_t v0 = 0; v0 < win.size();) {
    std::vector<int2> ci;
    std::vector<int4> cp;
    size_t v1 = v0;
    while (v1 < win.size() && (v1 == v0 || ((int)(ci.size() + win_items[v1].size()) <= items_per_chunk &&
                                            (int)(cp.size() + win_pairs[v1].size()) <= pairs_per_chunk))) {
      const int base = (int)ci.size();
      for (auto& q : win_pairs[v1]) cp.push_back(make_int4(q.x + base, q.y, q.z, q.w));
      ci.insert(ci.end(), win_items[v1].begin(), win_items[v1].end());
      ++v1;
    }
    if ((int)ci.size() > items_per_chunk || (int)cp.size() > pairs_per_chunk || (int)cp.size() > ctx->list_cap)
      return ATLAS_ERR_UNSUPPORTED;  // a single window's candidates exceed the workspaces
    for (auto& q : cp)
      if (q.x < 0 || q.x >= (int)ci.size()) return ATLAS_ERR_DEVICE;
    CK(cudaMemcpyAsync(ctx->d_items, ci.data(), ci.size() * sizeof(int2), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(ctx->d_pairs, cp.data(), cp.size() * sizeof(int4), cudaMemcpyHostToDevice, st));
    atlas::MixParams m;
    m.x = x;
    m.S = n_samples;
    m.N = g.N;
    m.M = g.M;
    m.sps = sps;
    m.hop = g.hop;
    m.w0 = 0;
    m.nw = 0;
    m.K = K;
    m.inc = ctx->d_inc;
    m.B = ctx->d_G;
    m.items = ctx->d_items;
    m.n_items = (int)ci.size();
    CK(atlas::launch_mix(m, st));
    WindowFftParams wf;
    wf.M = g.M;
    wf.sps = sps;
    wf.K = 1;
    wf.nw = (int)ci.size();
    wf.tw = g.d_tw_full;
    wf.G = ctx->d_G;
    CK(atlas::launch_window_fft(g.logM, g.loge, false, wf, st));
    CorrParams b;
    b.G = ctx->d_G;
    b.D = g.d_spec;
    b.tw = g.d_tw_full;
    b.part = ctx->d_part;
    b.S = n_samples;
    b.N = g.N;
    b.M = g.M;
    b.sps = sps;
    b.hop = g.hop;
    b.W = W;
    b.L = g.L;
    b.w0 = 0;
    b.nw = 0;
    b.K = K;
    b.Cg = C;
    b.status = ctx->d_status;
    b.pairs = ctx->d_pairs;
    b.n_pairs = (int)cp.size();
    CK(atlas::launch_corr(g.logM, g.loge, false, b, st));
    atlas::PairStatsParams ps;
    ps.part = ctx->d_part;
    ps.n = (int)cp.size();
    ps.sps = sps;
    ps.N = g.N;
    ps.out = ctx->d_pair_stats;
    CK(atlas::launch_pair_stats(ps, st));
    const size_t off = stats.size();
    stats.resize(off + cp.size());
    CK(cudaMemcpyAsync(stats.data() + off, ctx->d_pair_stats, cp.size() * sizeof(float4), cudaMemcpyDeviceToHost,
                       st));
    CK(cudaStreamSynchronize(st));
    pairs.insert(pairs.end(), cp.begin(), cp.end());
    v0 = v1;
  }
  // 5: exhaustive search of the fallback windows (ordered by window, then code)
  int n_fb = 0;
  std::vector<atlas_detection> fb;
  if (!fallback.empty()) {
    const int cap_fb = (int)fallback.size() * C;
    if (ctx->fb_cap < cap_fb) {
      cudaFree(ctx->d_fb_out);
      ctx->d_fb_out = nullptr;
      ctx->fb_cap = 0;
      if (cudaMalloc((void**)&ctx->d_fb_out, sizeof(atlas_detection) * (size_t)cap_fb) != cudaSuccess)
        return ATLAS_ERR_NO_MEMORY;
      ctx->fb_cap = cap_fb;
    }
    CK(cudaMemsetAsync(ctx->d_fb_count, 0, sizeof(int), st));
    bool sel_pending = false;
    for (size_t i = 0; i < fallback.size();) {  // runs of consecutive windows share a launch group
      size_t j = i + 1;
      const int wc = std::max(1, std::min<int>(ctx->wc_max, (int)(ctx->G_elems / ((size_t)K * g.N))));
      while (j < fallback.size() && fallback[j] == fallback[j - 1] + 1 && (int)(j - i) < wc) ++j;
      r = launch_chunk(ctx, g, st, x, n_samples, W, fallback[i], (int)(j - i), nullptr, ctx->d_fb_out, cap_fb,
                       ctx->d_fb_count, false, sel_pending);
      if (r != ATLAS_OK) return r;
      i = j;
    }
    if (sel_pending) CK(cudaStreamWaitEvent(st, ctx->ev_sel, 0));
    CK(cudaMemcpyAsync(&n_fb, ctx->d_fb_count, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    fb.resize(std::min(n_fb, cap_fb));
    if (!fb.empty())
      CK(cudaMemcpy(fb.data(), ctx->d_fb_out, fb.size() * sizeof(atlas_detection), cudaMemcpyDeviceToHost));
  }
  // 6: per (window, code) of the listed cells, the best candidate bin (smallest on ties)
  std::vector<atlas_detection> dets(fb.begin(), fb.end());
  {
    std::map<std::pair<int, int>, size_t> best;  // (window, code) -> pair index
    for (size_t q = 0; q < pairs.size(); ++q) {
      const auto key = std::make_pair(pairs[q].z, pairs[q].y);
      auto it = best.find(key);
      if (it == best.end()) {
        best[key] = q;
      } else {
        const float4 a0 = stats[it->second], a1 = stats[q];
        if (a1.x > a0.x || (a1.x == a0.x && pairs[q].w < pairs[it->second].w)) it->second = q;
      }
    }
    for (auto& kv : best) {
      const float4 v = stats[kv.second];
      if (!(v.x >= ctx->threshold)) continue;
      atlas_detection d;
      d.code = kv.first.second;
      d.window = kv.first.first;
      d.lag = __float_as_int_host(v.z);
      d.freq_bin = pairs[kv.second].w;
      d.score = v.x;
      d.peak_power = v.y;
      d.toa = 0.0;
      dets.push_back(d);
    }
  }
  std::stable_sort(dets.begin(), dets.end(), [](const atlas_detection& u, const atlas_detection& v) {
    return u.window != v.window ? u.window < v.window : u.code < v.code;
  });
  const int n_total = (int)dets.size();
  const int n_write = std::min(n_total, capacity);
  if (n_write > 0)
    CK(cudaMemcpyAsync(d_out, dets.data(), sizeof(atlas_detection) * (size_t)n_write, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(d_count, &n_total, sizeof(int), cudaMemcpyHostToDevice, st));
  r = launch_refine_all(ctx, st, x, n_samples, d_out, capacity, d_count);
  if (r != ATLAS_OK) return r;
  CK(cudaStreamSynchronize(st));
  if (h_n_fallback) *h_n_fallback = (int)fallback.size();
  return ATLAS_OK;
}

}  // namespace

extern "C" {

int atlas_acq_run_proposed(atlas_acq_t ctx, atlas_prop_t prop, void* stream, const float* d_iq,
                           int64_t n_samples, int32_t topk, float tau_fb, atlas_detection* d_out, int32_t capacity,
                           int32_t* d_count, int32_t* h_n_fallback) {
  return run_proposed_impl(ctx, prop, stream, d_iq, n_samples, topk, false, tau_fb, d_out, capacity, d_count,
                           h_n_fallback);
}

int atlas_acq_run_proposed_bins(atlas_acq_t ctx, atlas_prop_t prop, void* stream, const float* d_iq,
                                int64_t n_samples, int32_t n_top, float tau_fb, atlas_detection* d_out,
                                int32_t capacity, int32_t* d_count, int32_t* h_n_fallback) {
  return run_proposed_impl(ctx, prop, stream, d_iq, n_samples, n_top, true, tau_fb, d_out, capacity, d_count,
                           h_n_fallback);
}

int atlas_acq_last_device_status(atlas_acq_t ctx) {
  if (!ctx) return ATLAS_ERR_INVALID_ARG;
  int v = 0;
  CK(cudaDeviceSynchronize());
  CK(cudaMemcpy(&v, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost));
  return v;
}

const char* atlas_acq_last_error(atlas_acq_t ctx) { return ctx ? ctx->last_error.c_str() : ""; }

void atlas_acq_destroy(atlas_acq_t ctx) { free_ctx(ctx); }

const char* atlas_acq_strerror(int status) {
  switch (status) {
    case ATLAS_OK: return "ok";
    case ATLAS_ERR_INVALID_ARG: return "invalid argument";
    case ATLAS_ERR_CUDA: return "CUDA runtime error";
    case ATLAS_ERR_NO_MEMORY: return "out of memory";
    case ATLAS_ERR_UNSUPPORTED: return "unsupported size";
    case ATLAS_ERR_TIMEOUT: return "device wait timed out";
    case ATLAS_ERR_DEVICE: return "device-side check failed";
    default: return "unknown status";
  }
}

}  // extern "C"

// ---------------------------------------------------------------------------
// batched search: many receiver streams, one CUDA graph
// ---------------------------------------------------------------------------

struct atlas_acq_batch {
  int device = 0;
  std::vector<cudaStream_t> streams;
  cudaStream_t origin = nullptr;
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> joins;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int64_t kernel_nodes = 0;
};

namespace {
void free_batch(atlas_acq_batch* b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (auto e : b->joins) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  for (auto s : b->streams) cudaStreamDestroy(s);
  if (b->origin) cudaStreamDestroy(b->origin);
  delete b;
}
}  // namespace

extern "C" {

int atlas_acq_batch_create(atlas_acq_batch_t* out, const atlas_acq_t* ctxs, int32_t n_streams,
                           const float* const* d_iq, const int64_t* n_samples, atlas_detection* d_out,
                           int32_t capacity, int32_t* d_count) {
  if (!out) return ATLAS_ERR_INVALID_ARG;
  *out = nullptr;
  if (!ctxs || n_streams <= 0 || !d_iq || !n_samples || !d_count || capacity < 0 || (capacity > 0 && !d_out))
    return ATLAS_ERR_INVALID_ARG;
  for (int i = 0; i < n_streams; ++i) {
    if (!ctxs[i] || !d_iq[i] || n_samples[i] < ctxs[i]->max_L) return ATLAS_ERR_INVALID_ARG;
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == ctxs[i]) return ATLAS_ERR_INVALID_ARG;  // each stream needs its own workspace
  }
  atlas_acq_batch* b = new (std::nothrow) atlas_acq_batch();
  if (!b) return ATLAS_ERR_NO_MEMORY;
  atlas_acq_ctx* ctx = ctxs[0];
  int status = ATLAS_OK;
  bool capturing = false;
  cudaError_t e = cudaGetDevice(&b->device);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
  for (int i = 0; e == cudaSuccess && i < n_streams; ++i) {
    cudaStream_t s = nullptr;
    cudaEvent_t j = nullptr;
    e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) b->streams.push_back(s);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&j, cudaEventDisableTiming);
    if (e == cudaSuccess) b->joins.push_back(j);
  }
  if (e == cudaSuccess) e = cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    capturing = true;
    e = cudaEventRecord(b->fork, b->origin);
  }
  for (int i = 0; e == cudaSuccess && status == ATLAS_OK && i < n_streams; ++i) {
    e = cudaStreamWaitEvent(b->streams[i], b->fork, 0);
    if (e != cudaSuccess) break;
    status = run_impl(ctxs[i], b->streams[i], reinterpret_cast<const float2*>(d_iq[i]), n_samples[i], nullptr,
                      d_out ? d_out + (size_t)i * capacity : nullptr, capacity, d_count + i);
    if (status != ATLAS_OK) {
      ctx = ctxs[i];
      break;
    }
    e = cudaEventRecord(b->joins[i], b->streams[i]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->origin, b->joins[i], 0);
  }
  if (capturing) {
    cudaGraph_t g = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(b->origin, &g);
    b->graph = g;
    if (e == cudaSuccess) e = e2;
  }
  if (e == cudaSuccess && status == ATLAS_OK) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
  if (e == cudaSuccess && status == ATLAS_OK) {
    size_t n = 0;
    e = cudaGraphGetNodes(b->graph, nullptr, &n);
    std::vector<cudaGraphNode_t> nodes(n);
    if (e == cudaSuccess && n) e = cudaGraphGetNodes(b->graph, nodes.data(), &n);
    for (size_t k = 0; e == cudaSuccess && k < n; ++k) {
      cudaGraphNodeType t;
      e = cudaGraphNodeGetType(nodes[k], &t);
      if (e == cudaSuccess && t == cudaGraphNodeTypeKernel) b->kernel_nodes += 1;
    }
  }
  if (e != cudaSuccess) status = fail_cuda(ctx, e);
  if (status != ATLAS_OK) {
    free_batch(b);
    return status;
  }
  *out = b;
  return ATLAS_OK;
}

int atlas_acq_batch_run(atlas_acq_batch_t b, void* stream) {
  if (!b || !b->exec) return ATLAS_ERR_INVALID_ARG;
  return cudaGraphLaunch(b->exec, (cudaStream_t)stream) == cudaSuccess ? ATLAS_OK : ATLAS_ERR_CUDA;
}

int64_t atlas_acq_batch_kernels(atlas_acq_batch_t b) { return b ? b->kernel_nodes : -1; }

void atlas_acq_batch_destroy(atlas_acq_batch_t b) { free_batch(b); }

}  // extern "C"
