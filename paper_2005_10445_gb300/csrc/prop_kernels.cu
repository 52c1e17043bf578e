// prop_kernels.cu -- the learned (code, bin) proposal: Welch log-power-spectrum
// features, a small conv1d + MLP network (forward, backward, Adam), and the
// top-k candidate selection; C ABI atlas_prop_*.
//
// The paper has no learned component.  The proposal prunes the exhaustive
// search (every code correlated in every block, Sections 2.1 and 3): the
// network ranks (code, bin) candidates from a window's power spectrum, the
// exhaustive search produces its training labels and stays as the fallback.
//
// Features per window (one row of 4096 + K floats): the Welch log power
// spectrum f[4096], then K carrier-line values L[k] (for +/-1 chips the squared
// transmission is a pure tone at twice the carrier offset; L[k] = log10 of the
// squared window's |DFT|^2 at 2 f_k over sum |x|^4, plus 1).
// Network: f -> conv1d (8 channels, kernel 16, stride 8) + ReLU -> dense 4096
// -> 48 + ReLU -> heads: code logits [C], bin logits [K] (+ a L[k]), presence
// logit (+ c max_k L[k]).  Loss per window: BCE(presence) + present *
// (CE(code) + CE(bin)), averaged over the batch.  Parameters are one FP32
// array in the order conv_w [8][16], conv_b [8], w1 [4096][48], b1 [48],
// wc [48][C], bc [C], wb [48][K], bb [K], wp [48], bp [1], wl [2] = (a, c);
// inference can run on an FP16 copy of the weights (FP32 accumulation).
// Every reduction has a fixed order, so results are bit-reproducible.
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdio.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <new>
#include <string>
#include <vector>

#include "acq_common.cuh"
#include "atlas_acq.h"
#include "host_util.h"
#include "prop_internal.h"

namespace atlas {
namespace prop {

constexpr int kSeg = 4096;
constexpr int kCh = 8, kKw = 16, kSt = 8, kHid = 48;
constexpr int kP = kSeg / kSt;   // conv positions
constexpr int kX1 = kCh * kP;    // flattened conv outputs
constexpr int kTile = 16;

Layout make_layout(int C, int K) {
  Layout l;
  l.C = C;
  l.K = K;
  size_t o = 0;
  l.conv_w = o; o += kCh * kKw;
  l.conv_b = o; o += kCh;
  l.w1 = o; o += (size_t)kX1 * kHid;
  l.b1 = o; o += kHid;
  l.wc = o; o += (size_t)kHid * C;
  l.bc = o; o += C;
  l.wb = o; o += (size_t)kHid * K;
  l.bb = o; o += K;
  l.wp = o; o += kHid;
  l.bp = o; o += 1;
  l.wl = o; o += 2;
  l.total = o;
  return l;
}

int feature_len(int K) { return kSeg + K; }

__device__ __forceinline__ float to_f(float v) { return v; }
__device__ __forceinline__ float to_f(__half v) { return __half2float(v); }

// ---------------------------------------------------------------------------
// features: Welch log power spectrum (segments of 4096, periodic Hann taper)
// ---------------------------------------------------------------------------

constexpr int kPsdThreads = kSeg / 32;  // 128 threads x 32 values

__global__ void __launch_bounds__(kPsdThreads) k_psd(const float2* x, int64_t S, int64_t first, int64_t stride,
                                                      int n_seg, const float2* tw, float* feat, int row_len) {
  using FFT = BlockFFT<12, 5, -1>;
  __shared__ float2 sm[FFT::SMEM_ELEMS];
  __shared__ float2 sm_tw[TwTables<12>::N];
  __shared__ float red[kPsdThreads / 32];
  load_tables<12>(sm_tw, tw);
  __syncthreads();
  const int64_t base = first + (int64_t)blockIdx.x * stride;
  const int t = threadIdx.x;
  float acc[32];
#pragma unroll
  for (int i = 0; i < 32; ++i) acc[i] = 0.f;
  for (int s = 0; s < n_seg; ++s) {
    const int64_t seg0 = base + (int64_t)s * kSeg;
    auto load = [&](int i) {
      const int64_t idx = seg0 + i;
      const float2 v = (idx >= 0 && idx < S) ? x[idx] : make_float2(0.f, 0.f);
      const float h = 0.5f - 0.5f * cospif((float)i * (1.0f / 2048.0f));
      return make_float2(v.x * h, v.y * h);
    };
    // the last pass has read every value before it emits, so the outputs can
    // be parked in the same shared buffer
    auto emit = [&](int k, float2 v) { sm[spad(k)] = make_float2(fmaf(v.x, v.x, v.y * v.y), 0.f); };
    FFT::run(sm, sm_tw, load, emit);
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 32; ++i) acc[i] += sm[spad(t + kPsdThreads * i)].x;
    __syncthreads();
  }
  float sum = 0.f;
  const float inv = 1.0f / (float)n_seg;
#pragma unroll
  for (int i = 0; i < 32; ++i) {
    acc[i] = log10f(fmaf(acc[i], inv, 1.0f));
    sum += acc[i];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) sum += __shfl_down_sync(0xffffffffu, sum, o);
  if ((t & 31) == 0) red[t >> 5] = sum;
  __syncthreads();
  float tot = 0.f;
  for (int i = 0; i < kPsdThreads / 32; ++i) tot += red[i];
  const float mean = tot * (1.0f / kSeg);
  float* out = feat + (int64_t)blockIdx.x * row_len;
#pragma unroll
  for (int i = 0; i < 32; ++i) out[t + kPsdThreads * i] = acc[i] - mean;
}

// ---------------------------------------------------------------------------
// carrier-line features: L[k] = log10(|sum_m x[m]^2 e^{-2 pi i 2 f_k m / fs}|^2
// / sum_m |x[m]|^4 + 1) over one window (m window-relative).  One block per
// window; the window goes through shared memory in chunks of kLineChunk
// samples (squared on the way in); thread (r, k) accumulates bin k over the
// r-th eighth of each chunk with a phasor that starts exactly (64-bit
// fixed-point phase of 2 f_k) and advances by one complex product per sample.
// ---------------------------------------------------------------------------

constexpr int kLineThreads = 512;
constexpr int kLineChunk = 4096;
constexpr int kLineSub = 8;                      // sub-ranges per chunk
constexpr int kLineBinsPerPass = kLineThreads / kLineSub;  // 64

__global__ void __launch_bounds__(kLineThreads) k_line(const float2* x, int64_t S, int64_t first, int64_t stride,
                                                       int N, const uint64_t* inc2, int K, float* feat,
                                                       int row_len) {
  __shared__ float2 x2[kLineChunk];
  __shared__ float2 part[kLineSub][kLineBinsPerPass];
  __shared__ float red[kLineThreads / 32];
  const int t = threadIdx.x, r = t / kLineBinsPerPass, kk = t % kLineBinsPerPass;
  const int64_t base = first + (int64_t)blockIdx.x * stride;
  constexpr int kPasses = 4;  // up to 256 bins
  float2 acc[kPasses];
#pragma unroll
  for (int g = 0; g < kPasses; ++g) acc[g] = make_float2(0.f, 0.f);
  float e4 = 0.f;
  for (int c0 = 0; c0 < N; c0 += kLineChunk) {
    __syncthreads();  // the previous chunk is consumed
    for (int i = t; i < kLineChunk; i += kLineThreads) {
      const int64_t idx = base + c0 + i;
      const float2 v = (c0 + i < N && idx >= 0 && idx < S) ? x[idx] : make_float2(0.f, 0.f);
      const float2 v2 = make_float2(fmaf(v.x, v.x, -v.y * v.y), 2.f * v.x * v.y);
      x2[i] = v2;
      e4 = fmaf(v2.x, v2.x, fmaf(v2.y, v2.y, e4));
    }
    __syncthreads();
#pragma unroll
    for (int g = 0; g < kPasses; ++g) {
      const int k = kk + g * kLineBinsPerPass;
      if (k >= K) break;
      const int m0 = c0 + r * (kLineChunk / kLineSub);
      float2 ph = expi_neg(inc2[k] * (uint64_t)m0);
      const float2 step = expi_neg(inc2[k]);
      float2 a = acc[g];
      const float2* src = x2 + r * (kLineChunk / kLineSub);
      for (int i = 0; i < kLineChunk / kLineSub; ++i) {
        const float2 v = src[i];
        a.x = fmaf(v.x, ph.x, fmaf(-v.y, ph.y, a.x));
        a.y = fmaf(v.x, ph.y, fmaf(v.y, ph.x, a.y));
        ph = cmul(ph, step);
      }
      acc[g] = a;
    }
  }
  // total |x|^4 (fixed order)
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) e4 += __shfl_down_sync(0xffffffffu, e4, o);
  if ((t & 31) == 0) red[t >> 5] = e4;
  __syncthreads();
  float tot = 0.f;
  for (int i = 0; i < kLineThreads / 32; ++i) tot += red[i];
  float* out = feat + (int64_t)blockIdx.x * row_len + kSeg;
  for (int g = 0; g < kPasses; ++g) {
    if (g * kLineBinsPerPass >= K) break;
    __syncthreads();
    part[r][kk] = acc[g];
    __syncthreads();
    const int k = kk + g * kLineBinsPerPass;
    if (r == 0 && k < K) {
      float2 s2 = part[0][kk];
      for (int q = 1; q < kLineSub; ++q) s2 = make_float2(s2.x + part[q][kk].x, s2.y + part[q][kk].y);
      const float p2 = fmaf(s2.x, s2.x, s2.y * s2.y);
      out[k] = tot > 0.f ? log10f(p2 / tot + 1.f) : 0.f;
    }
  }
}

// bin logit k += a L[k]; presence logit += c max_k L[k]  (one thread per window)
template <typename TW>
__global__ void k_line_heads(const float* f, int row_len, int K, const TW* wl, int B, float* zb, float* zp) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  const float a = to_f(wl[0]), c = to_f(wl[1]);
  const float* L = f + (int64_t)b * row_len + kSeg;
  float mx = -INFINITY;
  for (int k = 0; k < K; ++k) {
    zb[(int64_t)b * K + k] = fmaf(a, L[k], zb[(int64_t)b * K + k]);
    mx = fmaxf(mx, L[k]);
  }
  zp[b] = fmaf(c, mx, zp[b]);
}

// g_a = sum_b sum_k dzb[b][k] L[b][k], g_c = sum_b dzp[b] max_k L[b][k]  (one block, fixed order)
__global__ void __launch_bounds__(256) k_line_grad(const float* f, int row_len, int K, int B, const float* dzb,
                                                   const float* dzp, float* g) {
  __shared__ float red[2][8];
  float ga = 0.f, gc = 0.f;
  for (int b = threadIdx.x; b < B; b += 256) {
    const float* L = f + (int64_t)b * row_len + kSeg;
    float mx = -INFINITY;
    for (int k = 0; k < K; ++k) {
      ga = fmaf(dzb[(int64_t)b * K + k], L[k], ga);
      mx = fmaxf(mx, L[k]);
    }
    gc = fmaf(dzp[b], mx, gc);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    ga += __shfl_down_sync(0xffffffffu, ga, o);
    gc += __shfl_down_sync(0xffffffffu, gc, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = ga;
    red[1][threadIdx.x >> 5] = gc;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    float a = 0.f, c = 0.f;
    for (int i = 0; i < 8; ++i) {
      a += red[0][i];
      c += red[1][i];
    }
    g[0] = a;
    g[1] = c;
  }
}

// ---------------------------------------------------------------------------
// dense layers: C = beta C + op(A) op(B) (+ bias) (+ ReLU), 16 x 16 tiles
// ---------------------------------------------------------------------------

template <bool TA, bool TB, typename TW>
__global__ void __launch_bounds__(kTile* kTile)
    k_gemm(int M, int N, int K, const float* A, int lda, const TW* B, int ldb, float* C, int ldc, const TW* bias,
           int relu, float beta) {
  __shared__ float As[kTile][kTile + 1];
  __shared__ float Bs[kTile][kTile + 1];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int m = blockIdx.y * kTile + ty, n = blockIdx.x * kTile + tx;
  float acc = 0.f;
  for (int k0 = 0; k0 < K; k0 += kTile) {
    {
      const int am = blockIdx.y * kTile + ty, ak = k0 + tx;
      As[ty][tx] = (am < M && ak < K) ? (TA ? A[(int64_t)ak * lda + am] : A[(int64_t)am * lda + ak]) : 0.f;
      const int bk = k0 + ty, bn = blockIdx.x * kTile + tx;
      Bs[ty][tx] = (bk < K && bn < N) ? to_f(TB ? B[(int64_t)bn * ldb + bk] : B[(int64_t)bk * ldb + bn]) : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kTile; ++k) acc = fmaf(As[ty][k], Bs[k][tx], acc);
    __syncthreads();
  }
  if (m < M && n < N) {
    float v = acc;
    if (bias) v += to_f(bias[n]);
    if (beta != 0.f) v += beta * C[(int64_t)m * ldc + n];
    if (relu) v = fmaxf(v, 0.f);
    C[(int64_t)m * ldc + n] = v;
  }
}

template <bool TA, bool TB, typename TW>
static void gemm(cudaStream_t s, int M, int N, int K, const float* A, int lda, const TW* B, int ldb, float* C,
                 int ldc, const TW* bias, int relu, float beta) {
  dim3 grid((N + kTile - 1) / kTile, (M + kTile - 1) / kTile);
  k_gemm<TA, TB, TW><<<grid, dim3(kTile, kTile), 0, s>>>(M, N, K, A, lda, B, ldb, C, ldc, bias, relu, beta);
}

// ---------------------------------------------------------------------------
// conv1d forward / weight gradient
// ---------------------------------------------------------------------------

template <typename TW>
__global__ void __launch_bounds__(kP) k_conv_fwd(const float* f, int row_len, const TW* w, const TW* b, float* a1p,
                                                 float* x1) {
  __shared__ float fs[kSeg + kKw];
  const float* fb = f + (int64_t)blockIdx.x * row_len;
  for (int i = threadIdx.x; i < kSeg + kKw; i += kP) fs[i] = i < kSeg ? fb[i] : 0.f;
  __syncthreads();
  const int p = threadIdx.x;
#pragma unroll
  for (int o = 0; o < kCh; ++o) {
    float acc = to_f(b[o]);
#pragma unroll
    for (int t = 0; t < kKw; ++t) acc = fmaf(to_f(w[o * kKw + t]), fs[kSt * p + t], acc);
    const int64_t idx = (int64_t)blockIdx.x * kX1 + o * kP + p;
    if (a1p) a1p[idx] = acc;
    x1[idx] = fmaxf(acc, 0.f);
  }
}

// g[o][t] = sum_b sum_p da1p[b][o][p] f[b][8p + t]  (blocks 0 .. 127), g_b[o] = sum da1p (blocks 128 .. 135)
__global__ void __launch_bounds__(256) k_conv_bwd(const float* f, int row_len, const float* da1p, int B, float* gw,
                                                  float* gb) {
  __shared__ float red[8];
  const int id = blockIdx.x;
  const bool bias = id >= kCh * kKw;
  const int o = bias ? id - kCh * kKw : id / kKw, t = bias ? 0 : id % kKw;
  float acc = 0.f;
  const int n = B * kP;
  for (int i = threadIdx.x; i < n; i += 256) {
    const int b = i / kP, p = i % kP;
    const float d = da1p[(int64_t)b * kX1 + o * kP + p];
    if (bias) {
      acc += d;
    } else {
      const int j = kSt * p + t;
      acc = fmaf(d, j < kSeg ? f[(int64_t)b * row_len + j] : 0.f, acc);
    }
  }
#pragma unroll
  for (int s = 16; s > 0; s >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    float v = 0.f;
    for (int i = 0; i < 8; ++i) v += red[i];
    if (bias) gb[o] = v;
    else gw[o * kKw + t] = v;
  }
}

// ---------------------------------------------------------------------------
// heads: softmax cross-entropies, presence BCE, and their gradients
// ---------------------------------------------------------------------------

// one warp per window
__global__ void k_heads_loss(const float* zc, const float* zb, const float* zp, const int* code, const int* bin,
                             int B, int C, int K, float* dzc, float* dzb, float* dzp, float* loss) {
  const int b = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (b >= B) return;
  const bool present = code[b] >= 0;
  const float invB = 1.0f / (float)B;
  float l = 0.f;
  // code head and bin head
  for (int head = 0; head < 2; ++head) {
    const float* z = head == 0 ? zc + (int64_t)b * C : zb + (int64_t)b * K;
    float* dz = head == 0 ? dzc + (int64_t)b * C : dzb + (int64_t)b * K;
    const int n = head == 0 ? C : K;
    const int lab = head == 0 ? code[b] : bin[b];
    float mx = -INFINITY;
    for (int i = lane; i < n; i += 32) mx = fmaxf(mx, z[i]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    float se = 0.f;
    for (int i = lane; i < n; i += 32) se += expf(z[i] - mx);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) se += __shfl_xor_sync(0xffffffffu, se, o);
    const float lse = mx + logf(se);
    for (int i = lane; i < n; i += 32) {
      const float pr = expf(z[i] - lse);
      dz[i] = present ? (pr - (i == lab ? 1.f : 0.f)) * invB : 0.f;
    }
    if (present) l += lse - z[lab];
  }
  if (lane == 0) {
    const float zv = zp[b];
    const float y = present ? 1.f : 0.f;
    l += fmaxf(zv, 0.f) - zv * y + log1pf(expf(-fabsf(zv)));
    dzp[b] = (1.f / (1.f + expf(-zv)) - y) * invB;
    loss[b] = l;
  }
}

__global__ void k_mask_relu(float* d, const float* pre, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && !(pre[i] > 0.f)) d[i] = 0.f;
}

// g[n] = sum_b dZ[b][n] (fixed order)
__global__ void k_colsum(const float* dz, int B, int N, float* g) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  float acc = 0.f;
  for (int b = 0; b < B; ++b) acc += dz[(int64_t)b * N + n];
  g[n] = acc;
}

__global__ void k_mean(const float* v, int n, float* out) {
  __shared__ float red[32];
  float acc = 0.f;
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc += v[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    float s = 0.f;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
    *out = s / (float)n;
  }
}

__global__ void k_adam(float* p, const float* g, float* m, float* v, int64_t n, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
}

__global__ void k_to_half(const float* a, __half* h, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) h[i] = __float2half_rn(a[i]);
}

// ---------------------------------------------------------------------------
// candidates: top-k (code, bin) pairs by log p(code) + log p(bin), per window
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(256) k_candidates(const float* zc, const float* zb, const float* zp, int C, int K,
                                                    int topk, int* cand, float* conf) {
  __shared__ float lc[256], lb[256];
  __shared__ float bv[8];
  __shared__ int bi[8];
  __shared__ int chosen[32];
  const int w = blockIdx.x;
  const int t = threadIdx.x;
  // log-softmax of both heads (C, K <= 256)
  for (int head = 0; head < 2; ++head) {
    const float* z = head == 0 ? zc + (int64_t)w * C : zb + (int64_t)w * K;
    const int n = head == 0 ? C : K;
    float* l = head == 0 ? lc : lb;
    if (t < 32) {
      float mx = -INFINITY;
      for (int i = t; i < n; i += 32) mx = fmaxf(mx, z[i]);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      float se = 0.f;
      for (int i = t; i < n; i += 32) se += expf(z[i] - mx);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) se += __shfl_xor_sync(0xffffffffu, se, o);
      const float lse = mx + logf(se);
      for (int i = t; i < n; i += 32) l[i] = z[i] - lse;
    }
    __syncthreads();
  }
  const int n = C * K;
  for (int r = 0; r < topk; ++r) {
    float best = -INFINITY;
    int besti = 0x7fffffff;
    for (int i = t; i < n; i += 256) {
      bool taken = false;
      for (int q = 0; q < r; ++q) taken |= (chosen[q] == i);
      if (taken) continue;
      const float s = lc[i / K] + lb[i % K];
      if (s > best || (s == best && i < besti)) {
        best = s;
        besti = i;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float s2 = __shfl_down_sync(0xffffffffu, best, o);
      const int i2 = __shfl_down_sync(0xffffffffu, besti, o);
      if (s2 > best || (s2 == best && i2 < besti)) {
        best = s2;
        besti = i2;
      }
    }
    if ((t & 31) == 0) {
      bv[t >> 5] = best;
      bi[t >> 5] = besti;
    }
    __syncthreads();
    if (t == 0) {
      float b0 = bv[0];
      int i0 = bi[0];
      for (int q = 1; q < 8; ++q)
        if (bv[q] > b0 || (bv[q] == b0 && bi[q] < i0)) {
          b0 = bv[q];
          i0 = bi[q];
        }
      chosen[r] = i0;
      cand[((int64_t)w * topk + r) * 2 + 0] = i0 / K;
      cand[((int64_t)w * topk + r) * 2 + 1] = i0 % K;
      if (r == 0) {
        conf[2 * w + 0] = expf(b0);
        conf[2 * w + 1] = 1.f / (1.f + expf(-zp[w]));
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// bin candidates: the top-nb bins by the bin head (ties to the smaller bin),
// every code searched in them; conf = {probability mass of the chosen bins,
// presence probability}
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(32) k_bin_candidates(const float* zb, const float* zp, int K, int nb, int* bins,
                                                       float* conf) {
  __shared__ float lb[256];
  const int w = blockIdx.x, t = threadIdx.x;
  const float* z = zb + (int64_t)w * K;
  float mx = -INFINITY;
  for (int i = t; i < K; i += 32) mx = fmaxf(mx, z[i]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  float se = 0.f;
  for (int i = t; i < K; i += 32) se += expf(z[i] - mx);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) se += __shfl_xor_sync(0xffffffffu, se, o);
  const float lse = mx + logf(se);
  for (int i = t; i < K; i += 32) lb[i] = z[i] - lse;
  __syncwarp();
  if (t == 0) {
    uint64_t taken[4] = {0, 0, 0, 0};
    float mass = 0.f;
    for (int r = 0; r < nb; ++r) {
      int bi = -1;
      for (int k = 0; k < K; ++k)
        if (!((taken[k >> 6] >> (k & 63)) & 1) && (bi < 0 || lb[k] > lb[bi])) bi = k;
      taken[bi >> 6] |= 1ull << (bi & 63);
      bins[(int64_t)w * nb + r] = bi;
      mass += expf(lb[bi]);
    }
    conf[2 * w + 0] = mass;
    conf[2 * w + 1] = 1.f / (1.f + expf(-zp[w]));
  }
}

}  // namespace prop
}  // namespace atlas

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------

using namespace atlas::prop;

namespace {

int fail(atlas_prop* p, cudaError_t e) {
  if (p) p->last_error = cudaGetErrorString(e);
  return ATLAS_ERR_CUDA;
}

#define PCK(call)                                \
  do {                                           \
    cudaError_t e_ = (call);                     \
    if (e_ != cudaSuccess) return fail(p, e_);   \
  } while (0)

void free_prop(atlas_prop* p) {
  if (!p) return;
  for (void* ptr : {(void*)p->params, (void*)p->half, (void*)p->grad, (void*)p->m, (void*)p->v, (void*)p->a1p,
                    (void*)p->x1, (void*)p->dx1, (void*)p->hp, (void*)p->h, (void*)p->zc, (void*)p->zb, (void*)p->zp,
                    (void*)p->dzc, (void*)p->dzb, (void*)p->dzp, (void*)p->dh, (void*)p->loss, (void*)p->tw,
                    (void*)p->feat, (void*)p->cand, (void*)p->conf, (void*)p->inc2})
    cudaFree(ptr);
  delete p;
}

uint64_t splitmix(uint64_t& s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

int ensure_batch(atlas_prop* p, int B) {
  if (B <= p->max_batch) return ATLAS_OK;
  for (float** q : {&p->a1p, &p->x1, &p->dx1, &p->hp, &p->h, &p->zc, &p->zb, &p->zp, &p->dzc, &p->dzb, &p->dzp,
                    &p->dh, &p->loss}) {
    cudaFree(*q);
    *q = nullptr;
  }
  p->max_batch = 0;
  const int C = p->lay.C, K = p->lay.K;
  const size_t x1 = (size_t)B * kX1 * sizeof(float);
  if (cudaMalloc((void**)&p->a1p, x1) != cudaSuccess || cudaMalloc((void**)&p->x1, x1) != cudaSuccess ||
      cudaMalloc((void**)&p->dx1, x1) != cudaSuccess ||
      cudaMalloc((void**)&p->hp, (size_t)B * kHid * 4) != cudaSuccess ||
      cudaMalloc((void**)&p->h, (size_t)B * kHid * 4) != cudaSuccess ||
      cudaMalloc((void**)&p->dh, (size_t)B * kHid * 4) != cudaSuccess ||
      cudaMalloc((void**)&p->zc, (size_t)B * C * 4) != cudaSuccess ||
      cudaMalloc((void**)&p->dzc, (size_t)B * C * 4) != cudaSuccess ||
      cudaMalloc((void**)&p->zb, (size_t)B * K * 4) != cudaSuccess ||
      cudaMalloc((void**)&p->dzb, (size_t)B * K * 4) != cudaSuccess ||
      cudaMalloc((void**)&p->zp, (size_t)B * 4) != cudaSuccess ||
      cudaMalloc((void**)&p->dzp, (size_t)B * 4) != cudaSuccess ||
      cudaMalloc((void**)&p->loss, (size_t)B * 4) != cudaSuccess)
    return ATLAS_ERR_NO_MEMORY;
  p->max_batch = B;
  return ATLAS_OK;
}

// forward pass on batch B; with half weights when `half` (inference) else FP32 (training)
int forward(atlas_prop* p, cudaStream_t s, const float* f, int B, bool half) {
  const Layout& L = p->lay;
  const int C = L.C, K = L.K, R = feature_len(K);
  if (half) {
    const __half* w = p->half;
    k_conv_fwd<__half><<<B, kP, 0, s>>>(f, R, w + L.conv_w, w + L.conv_b, nullptr, p->x1);
    gemm<false, false, __half>(s, B, kHid, kX1, p->x1, kX1, w + L.w1, kHid, p->h, kHid, w + L.b1, 1, 0.f);
    gemm<false, false, __half>(s, B, C, kHid, p->h, kHid, w + L.wc, C, p->zc, C, w + L.bc, 0, 0.f);
    gemm<false, false, __half>(s, B, K, kHid, p->h, kHid, w + L.wb, K, p->zb, K, w + L.bb, 0, 0.f);
    gemm<false, false, __half>(s, B, 1, kHid, p->h, kHid, w + L.wp, 1, p->zp, 1, w + L.bp, 0, 0.f);
    k_line_heads<__half><<<(B + 127) / 128, 128, 0, s>>>(f, R, K, w + L.wl, B, p->zb, p->zp);
  } else {
    const float* w = p->params;
    k_conv_fwd<float><<<B, kP, 0, s>>>(f, R, w + L.conv_w, w + L.conv_b, p->a1p, p->x1);
    gemm<false, false, float>(s, B, kHid, kX1, p->x1, kX1, w + L.w1, kHid, p->hp, kHid, w + L.b1, 0, 0.f);
    cudaMemcpyAsync(p->h, p->hp, (size_t)B * kHid * 4, cudaMemcpyDeviceToDevice, s);
    k_mask_relu<<<(B * kHid + 255) / 256, 256, 0, s>>>(p->h, p->hp, (int64_t)B * kHid);
    gemm<false, false, float>(s, B, C, kHid, p->h, kHid, w + L.wc, C, p->zc, C, w + L.bc, 0, 0.f);
    gemm<false, false, float>(s, B, K, kHid, p->h, kHid, w + L.wb, K, p->zb, K, w + L.bb, 0, 0.f);
    gemm<false, false, float>(s, B, 1, kHid, p->h, kHid, w + L.wp, 1, p->zp, 1, w + L.bp, 0, 0.f);
    k_line_heads<float><<<(B + 127) / 128, 128, 0, s>>>(f, R, K, w + L.wl, B, p->zb, p->zp);
  }
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? ATLAS_OK : fail(p, e);
}

}  // namespace

extern "C" {

int atlas_prop_create(atlas_prop_t* out, int32_t n_codes, int32_t n_bins, uint64_t seed) {
  if (!out) return ATLAS_ERR_INVALID_ARG;
  *out = nullptr;
  if (n_codes <= 0 || n_bins <= 0 || n_codes > 256 || n_bins > 256) return ATLAS_ERR_INVALID_ARG;
  atlas_prop* p = new (std::nothrow) atlas_prop();
  if (!p) return ATLAS_ERR_NO_MEMORY;
  p->lay = make_layout(n_codes, n_bins);
  const size_t n = p->lay.total;
  if (cudaMalloc((void**)&p->params, n * 4) != cudaSuccess || cudaMalloc((void**)&p->half, n * 2) != cudaSuccess ||
      cudaMalloc((void**)&p->grad, n * 4) != cudaSuccess || cudaMalloc((void**)&p->m, n * 4) != cudaSuccess ||
      cudaMalloc((void**)&p->v, n * 4) != cudaSuccess) {
    free_prop(p);
    return ATLAS_ERR_NO_MEMORY;
  }
  // He-style uniform initialisation from splitmix64; zero biases and Adam state
  std::vector<float> h(n, 0.f);
  uint64_t st = seed;
  const Layout& L = p->lay;
  auto fill = [&](size_t off, size_t cnt, int fan_in) {
    const double lim = sqrt(6.0 / fan_in);
    for (size_t i = 0; i < cnt; ++i) {
      const double u = (double)(splitmix(st) >> 11) * (1.0 / 9007199254740992.0);
      h[off + i] = (float)((2.0 * u - 1.0) * lim);
    }
  };
  fill(L.conv_w, kCh * kKw, kKw);
  fill(L.w1, (size_t)kX1 * kHid, kX1);
  fill(L.wc, (size_t)kHid * L.C, kHid);
  fill(L.wb, (size_t)kHid * L.K, kHid);
  fill(L.wp, kHid, kHid);
  // the carrier-line weights start from a prior: a line raises its bin's logit
  // (a = 4 per log10 unit) and the presence logit (c = 1); training adjusts both
  h[L.wl] = 4.f;
  h[L.wl + 1] = 1.f;
  int st2 = ATLAS_OK;
  cudaError_t e = cudaMemcpy(p->params, h.data(), n * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(p->m, 0, n * 4);
  if (e == cudaSuccess) e = cudaMemset(p->v, 0, n * 4);
  if (e == cudaSuccess) {
    std::vector<float2> t(atlas::TwTables<12>::N);
    for (int i = 0; i < atlas::TwTables<12>::NHI; ++i) {
      const double a = -6.283185307179586476925 * (double)(i << atlas::TwTables<12>::LB) / 4096.0;
      t[i] = make_float2((float)cos(a), (float)sin(a));
    }
    for (int i = 0; i < atlas::TwTables<12>::NLO; ++i) {
      const double a = -6.283185307179586476925 * (double)i / 4096.0;
      t[atlas::TwTables<12>::NHI + i] = make_float2((float)cos(a), (float)sin(a));
    }
    e = cudaMalloc((void**)&p->tw, t.size() * sizeof(float2));
    if (e == cudaSuccess) e = cudaMemcpy(p->tw, t.data(), t.size() * sizeof(float2), cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess) {
    k_to_half<<<(unsigned)((n + 255) / 256), 256>>>(p->params, p->half, (int64_t)n);
    e = cudaDeviceSynchronize();
  }
  if (e != cudaSuccess) st2 = ATLAS_ERR_CUDA;
  if (st2 != ATLAS_OK) {
    free_prop(p);
    return st2;
  }
  *out = p;
  return ATLAS_OK;
}

int64_t atlas_prop_num_params(atlas_prop_t p) { return p ? (int64_t)p->lay.total : -1; }

int atlas_prop_get_params(atlas_prop_t p, float* h) {
  if (!p || !h) return ATLAS_ERR_INVALID_ARG;
  PCK(cudaMemcpy(h, p->params, p->lay.total * 4, cudaMemcpyDeviceToHost));
  return ATLAS_OK;
}

int atlas_prop_set_params(atlas_prop_t p, const float* h) {
  if (!p || !h) return ATLAS_ERR_INVALID_ARG;
  const size_t n = p->lay.total;
  PCK(cudaMemcpy(p->params, h, n * 4, cudaMemcpyHostToDevice));
  PCK(cudaMemset(p->m, 0, n * 4));
  PCK(cudaMemset(p->v, 0, n * 4));
  p->step = 0;
  k_to_half<<<(unsigned)((n + 255) / 256), 256>>>(p->params, p->half, (int64_t)n);
  PCK(cudaDeviceSynchronize());
  return ATLAS_OK;
}

// CRC-32 of the IEEE 802.3 polynomial in its reflected form (0xEDB88320),
// initial value and final xor 0xFFFFFFFF, bit by bit.
static uint32_t crc32_update(uint32_t crc, const unsigned char* d, size_t n) {
  for (size_t i = 0; i < n; ++i) {
    crc ^= d[i];
    for (int b = 0; b < 8; ++b) crc = (crc >> 1) ^ (0xEDB88320u & (0u - (crc & 1u)));
  }
  return crc;
}

namespace {
constexpr char kCkptMagic[8] = {'A', 'T', 'L', 'P', 'R', 'O', 'P', '1'};
constexpr uint32_t kCkptVersion = 2;  // 2: the carrier-line head weights wl follow bp
struct CkptHeader {  // 40 bytes, little-endian
  char magic[8];
  uint32_t version;
  int32_t n_codes, n_bins;
  uint32_t crc;      // of the payload: params, m, v (float32, n_params each)
  int64_t n_params;
  int64_t step;      // Adam steps taken
};
static_assert(sizeof(CkptHeader) == 40, "checkpoint header layout");
}  // namespace

int atlas_prop_save(atlas_prop_t p, const char* path) {
  if (!p || !path) return ATLAS_ERR_INVALID_ARG;
  const size_t n = p->lay.total;
  std::vector<float> buf(3 * n);
  PCK(cudaMemcpy(buf.data(), p->params, n * 4, cudaMemcpyDeviceToHost));
  PCK(cudaMemcpy(buf.data() + n, p->m, n * 4, cudaMemcpyDeviceToHost));
  PCK(cudaMemcpy(buf.data() + 2 * n, p->v, n * 4, cudaMemcpyDeviceToHost));
  CkptHeader h;
  memcpy(h.magic, kCkptMagic, 8);
  h.version = kCkptVersion;
  h.n_codes = p->lay.C;
  h.n_bins = p->lay.K;
  h.n_params = (int64_t)n;
  h.step = p->step;
  h.crc = crc32_update(0xFFFFFFFFu, reinterpret_cast<const unsigned char*>(buf.data()), buf.size() * 4) ^ 0xFFFFFFFFu;
  FILE* f = fopen(path, "wb");
  if (!f) return ATLAS_ERR_INVALID_ARG;
  const bool ok = fwrite(&h, sizeof(h), 1, f) == 1 && fwrite(buf.data(), 4, buf.size(), f) == buf.size();
  const bool closed = fclose(f) == 0;
  return ok && closed ? ATLAS_OK : ATLAS_ERR_INVALID_ARG;
}

int atlas_prop_load(atlas_prop_t p, const char* path) {
  if (!p || !path) return ATLAS_ERR_INVALID_ARG;
  FILE* f = fopen(path, "rb");
  if (!f) return ATLAS_ERR_INVALID_ARG;
  CkptHeader h;
  const size_t n = p->lay.total;
  std::vector<float> buf(3 * n);
  bool ok = fread(&h, sizeof(h), 1, f) == 1 && memcmp(h.magic, kCkptMagic, 8) == 0 && h.version == kCkptVersion &&
            h.n_codes == p->lay.C && h.n_bins == p->lay.K && h.n_params == (int64_t)n && h.step >= 0 &&
            fread(buf.data(), 4, buf.size(), f) == buf.size();
  unsigned char extra;
  ok = ok && fread(&extra, 1, 1, f) == 0;  // nothing after the payload
  fclose(f);
  if (!ok) return ATLAS_ERR_INVALID_ARG;
  const uint32_t crc =
      crc32_update(0xFFFFFFFFu, reinterpret_cast<const unsigned char*>(buf.data()), buf.size() * 4) ^ 0xFFFFFFFFu;
  if (crc != h.crc) return ATLAS_ERR_INVALID_ARG;
  PCK(cudaMemcpy(p->params, buf.data(), n * 4, cudaMemcpyHostToDevice));
  PCK(cudaMemcpy(p->m, buf.data() + n, n * 4, cudaMemcpyHostToDevice));
  PCK(cudaMemcpy(p->v, buf.data() + 2 * n, n * 4, cudaMemcpyHostToDevice));
  p->step = h.step;
  k_to_half<<<(unsigned)((n + 255) / 256), 256>>>(p->params, p->half, (int64_t)n);
  PCK(cudaDeviceSynchronize());
  return ATLAS_OK;
}

int atlas_prop_features(atlas_prop_t p, void* stream, const float* d_iq, int64_t n_samples, int64_t first_sample,
                        int64_t stride, int32_t window_len, int32_t n_windows, float* d_feat) {
  if (!p || !d_iq || !d_feat || n_samples <= 0 || n_windows <= 0 || window_len < kSeg || stride <= 0)
    return ATLAS_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const int R = feature_len(p->lay.K);
  k_psd<<<n_windows, kPsdThreads, 0, s>>>(reinterpret_cast<const float2*>(d_iq), n_samples, first_sample, stride,
                                          window_len / kSeg, p->tw, d_feat, R);
  if (p->inc2) {
    k_line<<<n_windows, kLineThreads, 0, s>>>(reinterpret_cast<const float2*>(d_iq), n_samples, first_sample, stride,
                                              window_len, p->inc2, p->lay.K, d_feat, R);
  } else {
    PCK(cudaMemset2DAsync(d_feat + kSeg, (size_t)R * 4, 0, (size_t)p->lay.K * 4, n_windows, s));
  }
  PCK(cudaGetLastError());
  return ATLAS_OK;
}

int32_t atlas_prop_feature_len(atlas_prop_t p) { return p ? feature_len(p->lay.K) : -1; }

int atlas_prop_set_grid(atlas_prop_t p, double fs_hz, const double* freq_offsets_hz, int32_t n_freq) {
  if (!p || !freq_offsets_hz || !(fs_hz > 0.0) || n_freq != p->lay.K) return ATLAS_ERR_INVALID_ARG;
  std::vector<uint64_t> inc2(n_freq);
  for (int k = 0; k < n_freq; ++k) {
    if (!isfinite(freq_offsets_hz[k])) return ATLAS_ERR_INVALID_ARG;
    inc2[k] = 2ull * atlas::phase_increment(freq_offsets_hz[k], fs_hz);  // 2 f_k, modulo one turn
  }
  if (!p->inc2) PCK(cudaMalloc((void**)&p->inc2, sizeof(uint64_t) * n_freq));
  PCK(cudaMemcpy(p->inc2, inc2.data(), sizeof(uint64_t) * n_freq, cudaMemcpyHostToDevice));
  return ATLAS_OK;
}

int atlas_prop_loss_grad(atlas_prop_t p, void* stream, const float* d_feat, const int32_t* d_code,
                         const int32_t* d_bin, int32_t batch, float* d_loss, float* d_grad) {
  if (!p || !d_feat || !d_code || !d_bin || batch <= 0 || !d_loss) return ATLAS_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  int st = ensure_batch(p, batch);
  if (st != ATLAS_OK) return st;
  if ((st = forward(p, s, d_feat, batch, false)) != ATLAS_OK) return st;
  const Layout& L = p->lay;
  const int B = batch, C = L.C, K = L.K;
  float* g = d_grad ? d_grad : p->grad;
  const float* w = p->params;
  k_heads_loss<<<(B + 7) / 8, 256, 0, s>>>(p->zc, p->zb, p->zp, d_code, d_bin, B, C, K, p->dzc, p->dzb, p->dzp,
                                           p->loss);
  k_mean<<<1, 256, 0, s>>>(p->loss, B, d_loss);
  k_line_grad<<<1, 256, 0, s>>>(d_feat, feature_len(K), K, B, p->dzb, p->dzp, g + L.wl);
  // head weight and bias gradients
  gemm<true, false, float>(s, kHid, C, B, p->h, kHid, p->dzc, C, g + L.wc, C, nullptr, 0, 0.f);
  gemm<true, false, float>(s, kHid, K, B, p->h, kHid, p->dzb, K, g + L.wb, K, nullptr, 0, 0.f);
  gemm<true, false, float>(s, kHid, 1, B, p->h, kHid, p->dzp, 1, g + L.wp, 1, nullptr, 0, 0.f);
  k_colsum<<<(C + 127) / 128, 128, 0, s>>>(p->dzc, B, C, g + L.bc);
  k_colsum<<<(K + 127) / 128, 128, 0, s>>>(p->dzb, B, K, g + L.bb);
  k_colsum<<<1, 128, 0, s>>>(p->dzp, B, 1, g + L.bp);
  // dh = dzc wc^T + dzb wb^T + dzp wp^T, masked by ReLU
  gemm<false, true, float>(s, B, kHid, C, p->dzc, C, w + L.wc, C, p->dh, kHid, nullptr, 0, 0.f);
  gemm<false, true, float>(s, B, kHid, K, p->dzb, K, w + L.wb, K, p->dh, kHid, nullptr, 0, 1.f);
  gemm<false, true, float>(s, B, kHid, 1, p->dzp, 1, w + L.wp, 1, p->dh, kHid, nullptr, 0, 1.f);
  k_mask_relu<<<(B * kHid + 255) / 256, 256, 0, s>>>(p->dh, p->hp, (int64_t)B * kHid);
  gemm<true, false, float>(s, kX1, kHid, B, p->x1, kX1, p->dh, kHid, g + L.w1, kHid, nullptr, 0, 0.f);
  k_colsum<<<1, 128, 0, s>>>(p->dh, B, kHid, g + L.b1);
  // dx1 = dh w1^T, masked by ReLU of the conv outputs
  gemm<false, true, float>(s, B, kX1, kHid, p->dh, kHid, w + L.w1, kHid, p->dx1, kX1, nullptr, 0, 0.f);
  k_mask_relu<<<(unsigned)(((int64_t)B * kX1 + 255) / 256), 256, 0, s>>>(p->dx1, p->a1p, (int64_t)B * kX1);
  k_conv_bwd<<<kCh * kKw + kCh, 256, 0, s>>>(d_feat, feature_len(K), p->dx1, B, g + L.conv_w, g + L.conv_b);
  PCK(cudaGetLastError());
  return ATLAS_OK;
}

int atlas_prop_adam(atlas_prop_t p, void* stream, const float* d_grad, float lr) {
  if (!p || !(lr > 0.f)) return ATLAS_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const float b1 = 0.9f, b2 = 0.999f;
  p->step += 1;
  const float c1 = 1.f / (1.f - powf(b1, (float)p->step));
  const float c2 = 1.f / (1.f - powf(b2, (float)p->step));
  const int64_t n = (int64_t)p->lay.total;
  k_adam<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(p->params, d_grad ? d_grad : p->grad, p->m, p->v, n, lr, b1,
                                                     b2, 1e-8f, c1, c2);
  k_to_half<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(p->params, p->half, n);
  PCK(cudaGetLastError());
  return ATLAS_OK;
}

int atlas_prop_logits(atlas_prop_t p, void* stream, const float* d_feat, int32_t batch, int32_t half_weights,
                      float* d_zc, float* d_zb, float* d_zp) {
  if (!p || !d_feat || batch <= 0) return ATLAS_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  int st = ensure_batch(p, batch);
  if (st != ATLAS_OK) return st;
  if ((st = forward(p, s, d_feat, batch, half_weights != 0)) != ATLAS_OK) return st;
  if (d_zc) PCK(cudaMemcpyAsync(d_zc, p->zc, (size_t)batch * p->lay.C * 4, cudaMemcpyDeviceToDevice, s));
  if (d_zb) PCK(cudaMemcpyAsync(d_zb, p->zb, (size_t)batch * p->lay.K * 4, cudaMemcpyDeviceToDevice, s));
  if (d_zp) PCK(cudaMemcpyAsync(d_zp, p->zp, (size_t)batch * 4, cudaMemcpyDeviceToDevice, s));
  return ATLAS_OK;
}

int atlas_prop_candidates(atlas_prop_t p, void* stream, const float* d_feat, int32_t n_windows, int32_t topk,
                          int32_t* d_cand, float* d_conf) {
  if (!p || !d_feat || n_windows <= 0 || topk <= 0 || topk > 32 || topk > p->lay.C * p->lay.K || !d_cand ||
      !d_conf)
    return ATLAS_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  int st = ensure_batch(p, n_windows);
  if (st != ATLAS_OK) return st;
  if ((st = forward(p, s, d_feat, n_windows, true)) != ATLAS_OK) return st;
  k_candidates<<<n_windows, 256, 0, s>>>(p->zc, p->zb, p->zp, p->lay.C, p->lay.K, topk, d_cand, d_conf);
  PCK(cudaGetLastError());
  return ATLAS_OK;
}

int atlas_prop_bin_candidates(atlas_prop_t p, void* stream, const float* d_feat, int32_t n_windows, int32_t n_top,
                              int32_t* d_bins, float* d_conf) {
  if (!p || !d_feat || n_windows <= 0 || n_top <= 0 || n_top > 32 || n_top > p->lay.K || !d_bins || !d_conf)
    return ATLAS_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  int st = ensure_batch(p, n_windows);
  if (st != ATLAS_OK) return st;
  if ((st = forward(p, s, d_feat, n_windows, true)) != ATLAS_OK) return st;
  k_bin_candidates<<<n_windows, 32, 0, s>>>(p->zb, p->zp, p->lay.K, n_top, d_bins, d_conf);
  PCK(cudaGetLastError());
  return ATLAS_OK;
}

const char* atlas_prop_last_error(atlas_prop_t p) { return p ? p->last_error.c_str() : ""; }

void atlas_prop_destroy(atlas_prop_t p) { free_prop(p); }

}  // extern "C"
