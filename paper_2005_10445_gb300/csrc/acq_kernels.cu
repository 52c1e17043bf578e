// acq_kernels.cu -- the CUDA kernels of the acquisition search.
//
// Polyphase form of the correlation.  The replica is piecewise constant:
// r[n] = chip[n / sps] (Section 3 step 6), so with tau = sps*q + rho and
// B[t] = sum_{s<sps} y[(t + s) mod N] (a box sum of the mixed window),
//
//   corr[sps*q + rho] = sum_i chip[i] * B_rho[(q + i) mod M],  B_rho[q] = B[sps*q + rho],
//
// a circular correlation of length M = N / sps.  By the identity of
// Section 4.1 it equals IFFT_M(FFT_M(B_rho) * conj(FFT_M(chip))) / M.  This is
// the same N-point correlation, with the first stage of the N-point inverse
// transform (the sps-point DFT across stride-M elements) hoisted out of the
// per-code loop because the code spectrum factors into
// (chip spectrum periodised) x (box spectrum).  Per (window, bin) there are
// sps forward transforms of M points; per (window, code, bin) there are sps
// inverse transforms of M points, each of which fits in one block's shared
// memory for M <= 2^14.
//
// Kernels, in launch order per group of windows:
//   k_code_bank   (create time) D_c = conj(FFT_M(chip_c)) / M; for M = 2^15 also
//                 k_code_split_tables, the three half-length tables of the split form
//   k_mix         per (tile, bins, w): read the window once, mix it for each bin
//                 (one LO mix per bin, Section 3 step 2), box sum and decimate
//                 by sps -> B[w][k][rho]
//   k_window_fft  per (rho, k, w): G = FFT_M(B), in place
//   k_corr_dif    per (rho, k, w, c): G * D_c -> IFFT_M -> |.|^2 -> sum and
//                 argmax over the window's valid lags (Section 3 steps 7-8);
//                 the correlation never leaves the chip (k_corr / k_corr_split:
//                 the block-FFT forms for other sizes and tile shapes;
//                 acq_fft_kernels.cuh)
//   k_select      per (w, c): combine the sps partial results of each bin,
//                 score = P_max / floor, best bin, threshold, ordered compaction
//                 (one block; or k_select_pairs over many blocks into a
//                 workspace, then k_select_compact in one)
//   k_refine      per detection: direct |corr|^2 at a-1, a, a+1 (exact fixed-point
//                 phase, FP32 rotation, FP32 within a chip and FP64 across
//                 chips) and the parabola vertex in FP64 (Section 3 step 8,
//                 "interpolated")
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "acq_common.cuh"
#include "acq_fft_kernels.cuh"
#include "acq_internal.h"
#include "fft_block.cuh"

namespace atlas {

// ---------------------------------------------------------------------------
// code bank (create time)
// ---------------------------------------------------------------------------

template <int LOGM>
__global__ void __launch_bounds__((1 << LOGM) >> kLogE) k_code_bank(CodeBankParams p) {
  using FFT = BlockFFT<LOGM, kLogE, -1>;
  extern __shared__ float4 smem_raw[];
  float2* sm = reinterpret_cast<float2*>(smem_raw);
  float2* sm_tw = sm + FFT::SMEM_ELEMS;
  load_tables<LOGM>(sm_tw, p.tw);
  __syncthreads();
  const int c = blockIdx.x;
  const int8_t* ch = p.chips + p.chip_off[c];
  const int nc = p.n_chips[c];
  float2* D = p.D + (int64_t)c * FFT::M;
  auto load = [&](int i) { return make_float2(i < nc ? (float)ch[i] : 0.f, 0.f); };
  const float sc = p.scale;
  auto emit = [&](int k, float2 v) { D[k] = make_float2(v.x * sc, -v.y * sc); };
  FFT::run(sm, sm_tw, load, emit);
}

// 2^15-point code spectra: block h transforms the even (h = 0) or odd chips
// into its half of D (decimation in time), then k_code_bank_combine forms
// D[k] = conj(E[k] + W^k O[k]) / M and D[k + M/2] = conj(E[k] - W^k O[k]) / M.
template <int LOGH>
__global__ void __launch_bounds__((1 << LOGH) >> kLogE) k_code_bank_half(CodeBankParams p) {
  using FFT = BlockFFT<LOGH, kLogE, -1>;
  constexpr int H = 1 << LOGH;
  extern __shared__ float4 smem_raw[];
  float2* sm = reinterpret_cast<float2*>(smem_raw);
  float2* sm_tw = sm + FFT::SMEM_ELEMS;
  load_tables<LOGH>(sm_tw, p.tw);
  __syncthreads();
  const int c = blockIdx.x, h = blockIdx.y;
  const int8_t* ch = p.chips + p.chip_off[c];
  const int nc = p.n_chips[c];
  float2* D = p.D + (int64_t)c * (2 * H) + h * H;
  auto load = [&](int i) { return make_float2(2 * i + h < nc ? (float)ch[2 * i + h] : 0.f, 0.f); };
  auto emit = [&](int k, float2 v) { D[k] = v; };
  FFT::run(sm, sm_tw, load, emit);
}

__global__ void k_code_bank_combine(float2* D, int H, int n_codes, float scale) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)H * n_codes) return;
  const int c = (int)(i / H), k = (int)(i % H);
  float2* Dc = D + (int64_t)c * (2 * H);
  double sn, cs;
  sincospi(-(double)k / (double)H, &sn, &cs);  // W^k, W = exp(-2 pi i / 2H)
  const float2 w = make_float2((float)cs, (float)sn);
  const float2 e = Dc[k];
  const float2 o = cmul(w, Dc[k + H]);
  Dc[k] = make_float2((e.x + o.x) * scale, -(e.y + o.y) * scale);
  Dc[k + H] = make_float2((e.x - o.x) * scale, -(e.y - o.y) * scale);
}

// The split correlation of 2^15 points takes the lags q = 2k + h as two
// half-length inverse transforms of Y_h (radix-2 decimation in frequency).
// With G[i] = E[i] + W^i O[i], G[i + H] = E[i] - W^i O[i] and Z = G D:
//   Y_0[i] = Z[i] + Z[i + H]          = E[i] Dp[i] + O[i] W^i Dm[i]
//   Y_1[i] = (Z[i] - Z[i + H]) W^-i   = E[i] W^-i Dm[i] + O[i] Dp[i]
// (Dp = D[i] + D[i + H], Dm = D[i] - D[i + H], W = exp(-2 pi i / 2H)), so the
// three code tables below make each output a sum of two products.
__global__ void k_code_split_tables(const float2* D, float2* D3, int H, int n_codes) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)H * n_codes) return;
  const int c = (int)(i / H), k = (int)(i % H);
  const float2* Dc = D + (int64_t)c * (2 * H);
  float2* T = D3 + (int64_t)c * (3 * H);
  double sn, cs;
  sincospi(-(double)k / (double)H, &sn, &cs);  // W^k
  const double px = (double)Dc[k].x + Dc[k + H].x, py = (double)Dc[k].y + Dc[k + H].y;
  const double mx = (double)Dc[k].x - Dc[k + H].x, my = (double)Dc[k].y - Dc[k + H].y;
  T[k] = make_float2((float)px, (float)py);
  T[H + k] = make_float2((float)(cs * mx - sn * my), (float)(cs * my + sn * mx));
  T[2 * H + k] = make_float2((float)(cs * mx + sn * my), (float)(cs * my - sn * mx));
}

// ---------------------------------------------------------------------------
// mix + box sum + decimation (one read of each window for all bins)
// ---------------------------------------------------------------------------

constexpr int kMixQ = 256;   // q values per block (one per thread)
constexpr int kMixKG = 8;    // bins per block
constexpr int kMixRow = kMixQ + 2;  // row pitch of the de-interleaved tile (== 2 mod 16: no bank conflicts)

// B_rho[q] = sum_{s<sps} y[(sps q + rho + s) mod N] with y[m] = x_w[m] exp(-2 pi i f m / fs)
//          = exp(-2 pi i f sps q / fs) * sum_s x_w[sps q + rho + s] exp(-2 pi i f (rho + s) / fs),
// the index rho + s >= sps reaching into column q + 1; column M (past the window end)
// wraps to the window start, whose phase is that of m - N: one extra factor exp(+2 pi i f N / fs).
template <int SPS>
__global__ void __launch_bounds__(kMixQ) k_mix(MixParams p) {
  __shared__ float2 X[SPS * kMixRow];
  __shared__ float2 inner[kMixKG][2 * SPS];
  const int q0 = blockIdx.x * kMixQ;
  const int wl = blockIdx.z;
  int k0, nk, w;
  if (p.items) {  // one listed (window, bin) per block row
    w = p.items[wl].x;
    k0 = p.items[wl].y;
    nk = 1;
  } else {
    w = p.w0 + wl;
    k0 = blockIdx.y * kMixKG;
    nk = min(kMixKG, p.K - k0);
  }
  const int64_t base = (int64_t)w * p.hop;
  const int N = p.N;
  for (int i = threadIdx.x; i < SPS * (kMixQ + 1); i += kMixQ) {
    int t = SPS * q0 + i;
    if (t >= N) t -= N;
    const int64_t idx = base + t;
    X[(i % SPS) * kMixRow + i / SPS] = idx < p.S ? p.x[idx] : make_float2(0.f, 0.f);
  }
  for (int i = threadIdx.x; i < nk * 2 * SPS; i += kMixQ) {
    const int kk = i / (2 * SPS), j = i % (2 * SPS);
    const uint64_t inc = p.inc[k0 + kk];
    inner[kk][j] = j < 2 * SPS - 1 ? expi_neg(inc * (uint64_t)j) : expi_neg((uint64_t)0 - inc * (uint64_t)N);
  }
  __syncthreads();
  const int ql = threadIdx.x;
  const int q = q0 + ql;
  float2 xa[SPS], xb[SPS];
#pragma unroll
  for (int r = 0; r < SPS; ++r) {
    xa[r] = X[r * kMixRow + ql];
    xb[r] = X[r * kMixRow + ql + 1];
  }
  const bool last = (q == p.M - 1);
  for (int kk = 0; kk < nk; ++kk) {
    const int k = k0 + kk;
    const float2 outer = expi_neg(p.inc[k] * (uint64_t)SPS * (uint64_t)q);
    float2* Bk = p.B + (p.items ? (int64_t)wl * SPS : ((int64_t)wl * p.K + k) * SPS) * p.M + q;
    // y[j] = x_w[sps q + j] exp(-2 pi i f j / fs) for j < 2 sps - 1, each
    // product formed once; for the last column the samples j >= sps (past the
    // window end) carry the wrap phase
    float2 y[2 * SPS - 1];
#pragma unroll
    for (int j = 0; j < SPS; ++j) y[j] = cmul(xa[j], inner[kk][j]);
#pragma unroll
    for (int j = SPS; j < 2 * SPS - 1; ++j) y[j] = cmul(xb[j - SPS], inner[kk][j]);
    if (last) {
      const float2 wrap = inner[kk][2 * SPS - 1];
#pragma unroll
      for (int j = SPS; j < 2 * SPS - 1; ++j) y[j] = cmul(y[j], wrap);
    }
    // the sps box sums B_rho = sum_{s < sps} y[rho + s] by doubling: after the
    // pass of width v, y[i] = sum_{s < 2 v} y[i + s] for i < 2 sps - 2 v
    // (34 complex additions at sps = 8 instead of 56, and 15 products instead of 64)
#pragma unroll
    for (int l = 0; (1 << l) < SPS; ++l) {
      const int v = 1 << l;
#pragma unroll
      for (int i = 0; i < 2 * SPS - 2 * v; ++i) y[i] = cadd(y[i], y[i + v]);
    }
#pragma unroll
    for (int rho = 0; rho < SPS; ++rho) Bk[(int64_t)rho * p.M] = cmul(y[rho], outer);
  }
}

// ---------------------------------------------------------------------------
// selection and ordered compaction (one block per launch group)
// ---------------------------------------------------------------------------

constexpr int kSelectThreads = 512;  // one warp per (window, code) pair

// One (window, code) pair by one warp: the best bin by score (ties keep the
// smaller bin), its lag and peak; the per-cell statistics when asked.  The
// result is valid in lane 0.
__device__ __forceinline__ void select_pair(const SelectParams& p, int pi, int lane, int& flag,
                                            atlas_detection& d) {
  const int wl = pi / p.Cg, c = pi % p.Cg;
  const int w = p.w0 + wl;
  float bscore = -1.f, bpmax = 0.f;
  int bk = 0x7fffffff, btau = 0;
  for (int k = lane; k < p.K; k += 32) {
    const float4* pr = p.part + (((int64_t)wl * p.Cg + c) * p.K + k) * p.sps;
    float sum = 0.f, best = -1.f;
    int bt = 0x7fffffff;
    for (int r = 0; r < p.sps; ++r) {
      const float4 v = pr[r];
      sum += v.x;
      better(best, bt, v.y, __float_as_int(v.z));
    }
    const float floor_ = sum / (float)p.N;
    const float score = floor_ > 0.f ? best / floor_ : 0.f;
    if (p.cells) {
      atlas_cell cell;
      cell.p_max = best;
      cell.floor = floor_;
      cell.lag = bt;
      cell.valid = 1;
      p.cells[((int64_t)w * p.C + p.codes[c]) * p.K + k] = cell;
    }
    if (score > bscore) {  // k increases along the loop: ties keep the smaller bin
      bscore = score;
      bk = k;
      btau = bt;
      bpmax = best;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float s2 = __shfl_down_sync(0xffffffffu, bscore, o);
    const int k2 = __shfl_down_sync(0xffffffffu, bk, o);
    const int t2 = __shfl_down_sync(0xffffffffu, btau, o);
    const float p2 = __shfl_down_sync(0xffffffffu, bpmax, o);
    if (s2 > bscore || (s2 == bscore && k2 < bk)) {
      bscore = s2;
      bk = k2;
      btau = t2;
      bpmax = p2;
    }
  }
  flag = bscore >= p.threshold ? 1 : 0;
  d.code = p.codes[c];
  d.window = w;
  d.lag = btau;
  d.freq_bin = bk;
  d.score = bscore;
  d.peak_power = bpmax;
  d.toa = 0.0;
}

// Single block: rounds of one pair per warp, compacted in order by thread 0.
__global__ void __launch_bounds__(kSelectThreads) k_select(SelectParams p) {
  __shared__ int flags[kSelectThreads / 32];
  __shared__ atlas_detection recs[kSelectThreads / 32];
  __shared__ int base_sh;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) base_sh = *p.count;
  const int n_pairs = p.nw * p.Cg;
  for (int p0 = 0; p0 < n_pairs; p0 += kSelectThreads / 32) {
    const int pi = p0 + warp;
    int flag = 0;
    if (pi < n_pairs) {
      atlas_detection d;
      select_pair(p, pi, lane, flag, d);
      if (lane == 0) recs[warp] = d;
    }
    if (lane == 0) flags[warp] = flag;
    __syncthreads();
    if (threadIdx.x == 0) {  // ordered compaction of this round's pairs
      int n = base_sh;
      for (int i = 0; i < kSelectThreads / 32; ++i) {
        if (flags[i]) {
          if (n < p.capacity) p.out[n] = recs[i];
          ++n;
        }
      }
      base_sh = n;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) *p.count = base_sh;
}

// Many blocks: one pair per warp into the workspace.
__global__ void __launch_bounds__(kSelectThreads) k_select_pairs(SelectParams p) {
  const int lane = threadIdx.x & 31;
  const int pi = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (pi >= p.nw * p.Cg) return;  // whole warps leave together
  int flag = 0;
  atlas_detection d;
  select_pair(p, pi, lane, flag, d);
  if (lane == 0) {
    p.tmp_flags[pi] = flag;
    p.tmp_recs[pi] = d;
  }
}

// One block: the flagged pairs appended in pair order after the running
// count, by a block-wide exclusive prefix sum per round of kCompactThreads.
constexpr int kCompactThreads = 1024;

__global__ void __launch_bounds__(kCompactThreads) k_select_compact(SelectParams p) {
  __shared__ int warp_tot[kCompactThreads / 32];
  __shared__ int base_sh;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) base_sh = *p.count;
  const int n_pairs = p.nw * p.Cg;
  for (int p0 = 0; p0 < n_pairs; p0 += kCompactThreads) {
    const int pi = p0 + threadIdx.x;
    const int flag = pi < n_pairs ? p.tmp_flags[pi] : 0;
    const unsigned m = __ballot_sync(0xffffffffu, flag);
    const int in_warp = __popc(m & ((1u << lane) - 1u));
    if (lane == 0) warp_tot[warp] = __popc(m);
    __syncthreads();
    if (warp == 0) {
      const int v = warp_tot[lane];
      int x = v;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
      }
      warp_tot[lane] = x - v;  // exclusive
    }
    __syncthreads();
    const int base = base_sh;
    if (flag) {
      const int idx = base + warp_tot[warp] + in_warp;
      if (idx < p.capacity) p.out[idx] = p.tmp_recs[pi];
    }
    __syncthreads();  // every thread has read base_sh and warp_tot
    if (threadIdx.x == kCompactThreads - 1) base_sh = base + warp_tot[warp] + in_warp + flag;
    __syncthreads();
  }
  if (threadIdx.x == 0) *p.count = base_sh;
}

__global__ void k_pair_stats(PairStatsParams p) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= p.n) return;
  float sum = 0.f, best = -1.f;
  int bt = 0x7fffffff;
  for (int r = 0; r < p.sps; ++r) {
    const float4 v = p.part[(int64_t)i * p.sps + r];
    sum += v.x;
    better(best, bt, v.y, __float_as_int(v.z));
  }
  const float floor_ = sum / (float)p.N;
  p.out[i] = make_float4(floor_ > 0.f ? best / floor_ : 0.f, best, __int_as_float(bt), floor_);
}

// ---------------------------------------------------------------------------
// FP64 refinement
// ---------------------------------------------------------------------------

constexpr int kRefineThreads = 256;

__device__ __forceinline__ void dadd_shfl(double& v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
}

__global__ void __launch_bounds__(kRefineThreads) k_refine(RefineParams p) {
  __shared__ double red[6][kRefineThreads / 32];
  const int n = min(*p.count, p.capacity);
  for (int di = blockIdx.x; di < n; di += gridDim.x) {
    atlas_detection det = p.out[di];
    const int c = det.code;
    const int sps = p.sps;
    const int L = p.chips_per_code[c] * sps;
    const int8_t* ch = p.chips + p.chip_off[c];
    const int64_t a = (int64_t)det.window * p.hop[c] + det.lag;
    const uint64_t inc = p.inc[det.freq_bin];
    // y[m] = x[m] exp(-2 pi i f m / fs) for m in [a-1, a+L]: the phase is the exact
    // 64-bit fixed-point product m * inc, the rotation FP32; the three direct
    // correlations sum_n y[a+d+n] r[n] (d = -1, 0, +1).
    double acc[6] = {0, 0, 0, 0, 0, 0};
    if (sps >= 2) {
      // r is constant over a chip, so a thread takes runs of sps samples
      // m = a - 1 + k sps + s: for lag d = j - 1 (j <= 2 <= sps) the samples
      // s < j belong to chip k - 1 and the others to chip k.  Each chip's
      // samples are summed in FP32 (at most sps terms), the run's two chip
      // sums combined with their signs in FP32, and the runs accumulate in
      // FP64: one FP64 addition per run and component, not one per sample.
      const int n_chips = L / sps;
      for (int64_t k = threadIdx.x; k <= n_chips; k += kRefineThreads) {
        const int64_t m0 = a - 1 + k * sps;
        float2 lo[3] = {}, hi[3] = {};
        for (int s = 0; s < sps; ++s) {
          const int64_t m = m0 + s;
          if (m > a + L) break;
          if (m < 0 || m >= p.S) continue;
          const float2 y = cmul(p.x[m], expi_neg(inc * (uint64_t)m));
#pragma unroll
          for (int j = 0; j < 3; ++j) {
            float2& t = s < j ? lo[j] : hi[j];
            t.x += y.x;
            t.y += y.y;
          }
        }
        const float sk = k < n_chips ? (ch[k] < 0 ? -1.f : 1.f) : 0.f;   // chip k
        const float sk1 = k >= 1 ? (ch[k - 1] < 0 ? -1.f : 1.f) : 0.f;   // chip k - 1
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          acc[2 * j] += (double)fmaf(sk, hi[j].x, sk1 * lo[j].x);
          acc[2 * j + 1] += (double)fmaf(sk, hi[j].y, sk1 * lo[j].y);
        }
      }
    } else {
      // one sample per chip: every term accumulates in FP64
      for (int64_t m = a - 1 + threadIdx.x; m <= a + L; m += kRefineThreads) {
        if (m < 0 || m >= p.S) continue;
        const float2 y = cmul(p.x[m], expi_neg(inc * (uint64_t)m));
#pragma unroll
        for (int d = -1; d <= 1; ++d) {
          const int64_t nn = m - a - d;
          if (nn >= 0 && nn < L) {
            const bool neg = ch[nn] < 0;
            acc[2 * (d + 1)] += neg ? -(double)y.x : (double)y.x;
            acc[2 * (d + 1) + 1] += neg ? -(double)y.y : (double)y.y;
          }
        }
      }
    }
#pragma unroll
    for (int j = 0; j < 6; ++j) dadd_shfl(acc[j]);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
#pragma unroll
      for (int j = 0; j < 6; ++j) red[j][warp] = acc[j];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double s[6];
      for (int j = 0; j < 6; ++j) {
        double v = 0.0;
        for (int q = 0; q < kRefineThreads / 32; ++q) v += red[j][q];
        s[j] = v;
      }
      const double pm = s[0] * s[0] + s[1] * s[1];
      const double p0 = s[2] * s[2] + s[3] * s[3];
      const double pp = s[4] * s[4] + s[5] * s[5];
      double delta = 0.0;
      if (a - 1 >= 0 && a + 1 <= p.S - L) {
        const double den = pm - 2.0 * p0 + pp;
        if (den < 0.0) {
          delta = 0.5 * (pm - pp) / den;
          delta = delta > 0.5 ? 0.5 : (delta < -0.5 ? -0.5 : delta);
        }
      }
      p.out[di].toa = (double)a + delta;
      p.out[di].peak_power = (float)p0;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// launch wrappers
// ---------------------------------------------------------------------------

template <int LOGM>
static cudaError_t prepare_code_bank() {
  return cudaFuncSetAttribute(k_code_bank<LOGM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)fft_smem<LOGM>());
}

cudaError_t prepare_kernels() {
  cudaError_t e;
  if ((e = prepare_code_bank<10>()) != cudaSuccess) return e;
  if ((e = prepare_code_bank<11>()) != cudaSuccess) return e;
  if ((e = prepare_code_bank<12>()) != cudaSuccess) return e;
  if ((e = prepare_code_bank<13>()) != cudaSuccess) return e;
  if ((e = prepare_code_bank<14>()) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k_code_bank_half<14>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)fft_smem<14>())) != cudaSuccess)
    return e;
  if ((e = prepare_fft_e4()) != cudaSuccess) return e;
  if ((e = prepare_tc5()) != cudaSuccess) return e;
  return prepare_fft_e5();
}

cudaError_t launch_code_bank(int logM, const CodeBankParams& p, int n_codes, cudaStream_t s) {
  switch (logM) {
    case 10: k_code_bank<10><<<n_codes, fft_threads<10, kLogE>(), fft_smem<10>(), s>>>(p); break;
    case 11: k_code_bank<11><<<n_codes, fft_threads<11, kLogE>(), fft_smem<11>(), s>>>(p); break;
    case 12: k_code_bank<12><<<n_codes, fft_threads<12, kLogE>(), fft_smem<12>(), s>>>(p); break;
    case 13: k_code_bank<13><<<n_codes, fft_threads<13, kLogE>(), fft_smem<13>(), s>>>(p); break;
    case 14: k_code_bank<14><<<n_codes, fft_threads<14, kLogE>(), fft_smem<14>(), s>>>(p); break;
    case 15: {
      k_code_bank_half<14><<<dim3(n_codes, 2), fft_threads<14, kLogE>(), fft_smem<14>(), s>>>(p);
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return e;
      const int H = 1 << 14;
      const int64_t n = (int64_t)H * n_codes;
      k_code_bank_combine<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(p.D, H, n_codes, p.scale);
      if (p.D3) {
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        k_code_split_tables<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(p.D, p.D3, H, n_codes);
      }
      break;
    }
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_mix(const MixParams& p, cudaStream_t s) {
  dim3 grid(p.M / kMixQ, p.items ? 1 : (p.K + kMixKG - 1) / kMixKG, p.items ? p.n_items : p.nw);
  switch (p.sps) {
    case 1: k_mix<1><<<grid, kMixQ, 0, s>>>(p); break;
    case 2: k_mix<2><<<grid, kMixQ, 0, s>>>(p); break;
    case 4: k_mix<4><<<grid, kMixQ, 0, s>>>(p); break;
    case 8: k_mix<8><<<grid, kMixQ, 0, s>>>(p); break;
    case 16: k_mix<16><<<grid, kMixQ, 0, s>>>(p); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_window_fft(int logM, int loge, bool split, const WindowFftParams& p, cudaStream_t s) {
  return loge == 4 ? launch_window_fft_e4(logM, split, p, s) : launch_window_fft_e5(logM, split, p, s);
}

cudaError_t launch_corr(int logM, int loge, bool split, const CorrParams& p, cudaStream_t s) {
  return loge == 4 ? launch_corr_e4(logM, split, p, s) : launch_corr_e5(logM, split, p, s);
}

cudaError_t launch_select(const SelectParams& p, cudaStream_t s) {
  const int n_pairs = p.nw * p.Cg;
  constexpr int warps = kSelectThreads / 32;
  if (p.tmp_flags && p.tmp_recs && n_pairs > warps) {
    k_select_pairs<<<(n_pairs + warps - 1) / warps, kSelectThreads, 0, s>>>(p);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_select_compact<<<1, kCompactThreads, 0, s>>>(p);
    return cudaGetLastError();
  }
  k_select<<<1, kSelectThreads, 0, s>>>(p);
  return cudaGetLastError();
}

int select_launches(const SelectParams& p) {
  return (p.tmp_flags && p.tmp_recs && p.nw * p.Cg > kSelectThreads / 32) ? 2 : 1;
}

cudaError_t launch_pair_stats(const PairStatsParams& p, cudaStream_t s) {
  k_pair_stats<<<(p.n + 127) / 128, 128, 0, s>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_refine(const RefineParams& p, int grid, cudaStream_t s) {
  k_refine<<<grid, kRefineThreads, 0, s>>>(p);
  return cudaGetLastError();
}

}  // namespace atlas
