// fsk_fft.cu -- the N-point transforms of the FSK cross-correlation (Section 3
// step 7, computed with FFTs as in Section 4.1).  N = R * M: M points live in
// one block's shared memory (all of N up to 2^14 in one block; 2^13 or 2^14 per
// block beyond) and R in {4, 8, 16} blocks exchange either through the
// distributed shared memory of a thread-block cluster (M = 2^13, N up to 2^17:
// 75 KB per block, three blocks per SM, clusters of up to 16 blocks spread
// over every SM) or through a scratch buffer in global memory between two
// passes (every plan, N up to 2^18).
//
// Index maps (n = m + M n2, k = R k2 + r with m, k2 < M and n2, r < R):
//   forward   X[R k2 + r] = sum_m W_M^{m k2} ( W_N^{m r} sum_n2 x[m + M n2] W_R^{n2 r} )
//     Block rho of the cluster takes the m of its range [rho M/R, (rho+1) M/R),
//     forms the R-point DFT of the values M apart, multiplies value r by
//     W_N^{m r} and stores it at position m of block r's shared memory.  After
//     a cluster barrier block r runs the M-point block FFT and writes the run
//     X_perm[r M + k2] = X[R k2 + r] (the "permuted" spectrum: each block
//     writes one contiguous run).
//   inverse   z[m + M n2] = sum_r W_R^{-n2 r} ( W_N^{-m r} sum_k2 Z[R k2 + r] W_M^{-m k2} )
//     Block r inverse-transforms its run Z_perm[r M + .] with the block FFT,
//     multiplies by W_N^{-m r} and keeps the values in its shared memory.
//     After a cluster barrier block rho reads, for each m of its range, the
//     R values at m from the R blocks and takes the R-point DFT across them:
//     the lags m + M n2.
// Window and code spectra share the permuted layout, so the pointwise product
// of the correlation needs no reordering.
//
// Real inputs are packed two per transform: the forward transform takes
// x = d_w + j d_{w+1} (two windows of the real demodulated stream); with the
// code spectra conj(DFT(d_c)) / N, the inverse transform of X * C gives
// corr_w + j corr_{w+1}.
#include <cooperative_groups.h>
#include <algorithm>
#include <limits.h>

#include "acq_common.cuh"
#include "acq_fft_kernels.cuh"
#include "fsk_internal.h"

namespace atlas {
namespace cg = cooperative_groups;

template <int LOGM>
constexpr int fsk_fft_threads() { return (1 << LOGM) >> kLogE; }

// The tables of N sit in shared memory up to N = 2^17; beyond, blocks of 2^13
// points read them through L1 so that three blocks still fit on an SM.
template <int LOGN>
constexpr bool fsk_twN_shared() { return LOGN <= 17; }

// padded transform buffer, tables of M and of N, reduction scratch (2 x 32)
template <int LOGM, int LOGN>
constexpr size_t fsk_fft_smem() {
  return sizeof(float2) * (BlockFFT<LOGM, kLogE, -1>::SMEM_ELEMS + TwTables<LOGM>::N +
                           (fsk_twN_shared<LOGN>() ? TwTables<LOGN>::N : 0)) +
         64 * sizeof(float4);
}

// clusters hold at most 16 blocks
template <int LOGM, int R>
constexpr bool fsk_cluster_form() { return R == 1 || (LOGM <= 13 && R <= 16); }

// The passes of a block FFT whose input is already in shared memory (natural
// index i at spad(i)).
template <class FFT, int LOGM, int D, class Emit>
__device__ __forceinline__ void passes_from_shared(float2* sm, const float2* tw, Emit& emit) {
  constexpr int RB = (LOGM - D) < kLogE ? (LOGM - D) : kLogE;
  constexpr bool LAST = (D + RB == LOGM);
  auto none = [](int) { return make_float2(0.f, 0.f); };
  FFT::template pass<D, RB, false, LAST>(sm, tw, none, emit);
  if constexpr (!LAST) passes_from_shared<FFT, LOGM, D + RB>(sm, tw, emit);
}

// value n of item `item`'s real sequence `which` (0: real part, 1: imaginary)
__device__ __forceinline__ float fsk_fwd_value(const FskFwdParams& p, int item, int which, int n) {
  if (p.rows) {
    if (which) return 0.f;
    return n < p.n_valid ? p.rows[(int64_t)item * p.ld + n] : 0.f;
  }
  const int wl = 2 * item + which;
  if (wl >= p.nw) return 0.f;
  const int64_t i = (int64_t)(p.w0 + wl) * p.hop + n - p.base;
  return (i >= 0 && i < p.len) ? p.d[i] : 0.f;
}

// blocks per SM the multi-block kernels are compiled for (register budget):
// three of 2^13 points, one of 2^14
template <int LOGM, int R>
constexpr int fsk_min_blocks() { return (R > 1 && LOGM <= 13) ? 3 : 1; }

template <int LOGM, int R>
__global__ void __launch_bounds__(fsk_fft_threads<LOGM>(), fsk_min_blocks<LOGM, R>()) k_fsk_fwd(FskFwdParams p) {
  using FFT = BlockFFT<LOGM, kLogE, -1>;
  constexpr int M = 1 << LOGM;
  constexpr int N = M * R;
  constexpr int LOGN = LOGM + ct_log2(R);
  extern __shared__ float4 smem_raw[];
  float2* sm = reinterpret_cast<float2*>(smem_raw);
  float2* sm_tw = sm + FFT::SMEM_ELEMS;
  float2* sm_twN = sm_tw + TwTables<LOGM>::N;
  load_tables<LOGM>(sm_tw, p.tw);
  if constexpr (R > 1) load_tables<LOGN>(sm_twN, p.twN);
  const int item = blockIdx.x / R;
  const int rank = blockIdx.x % R;  // the block's rank in its cluster of R
  float2* X = p.X + (int64_t)item * N + (int64_t)rank * M;
  const float sc = p.scale;
  const float sy = p.conj_out ? -sc : sc;
  auto emit = [&](int k, float2 v) { X[k] = make_float2(v.x * sc, v.y * sy); };
  __syncthreads();  // tables
  if constexpr (R == 1) {
    auto load = [&](int n) { return make_float2(fsk_fwd_value(p, item, 0, n), fsk_fwd_value(p, item, 1, n)); };
    FFT::run(sm, sm_tw, load, emit);
  } else {
    cg::cluster_group cluster = cg::this_cluster();
    cluster.sync();  // every block of the cluster runs before the first remote store
    constexpr int MR = M / R;
    float2* dst[R];
#pragma unroll
    for (int r = 0; r < R; ++r) dst[r] = cluster.map_shared_rank(sm, r);
    for (int j = threadIdx.x; j < MR; j += blockDim.x) {
      const int m = rank * MR + j;
      float2 v[R];
#pragma unroll
      for (int n2 = 0; n2 < R; ++n2)
        v[n2] = make_float2(fsk_fwd_value(p, item, 0, m + M * n2), fsk_fwd_value(p, item, 1, m + M * n2));
      dft_reg<R, -1>(v);
      dst[0][spad(m)] = v[0];
#pragma unroll
      for (int r = 1; r < R; ++r) dst[r][spad(m)] = cmul(v[r], twiddle<LOGN, -1>(sm_twN, m * r));
    }
    cluster.sync();  // every block's M values are in place
    passes_from_shared<FFT, LOGM, 0>(sm, sm_tw, emit);
  }
}

// The scratch of the two-pass forms is written and read once each with
// streaming (evict-first) accesses, so that it does not push the window and
// code spectra, which every block reads, out of L2.
//
// Two-pass form of k_fsk_fwd for R > 1: the same index maps and arithmetic,
// with the exchange through a scratch buffer in global memory instead of
// distributed shared memory, so no block waits on another and a block may hold
// 2^14 points (one per SM, more than a cluster of 16 can place at once).
//   pass A: block (item, rho) takes the m of its range, forms the R-point DFT
//           of the values x[m + M n2] and writes value r times W_N^{m r} to
//           scratch[(item - item0) R + r][m]
//   pass B: block (item, r) transforms scratch row r with the block FFT and
//           writes the run X_perm[r M + .]
// The first pass of the block FFT reads the same values the cluster form
// reads from shared memory, so the results are bit-identical.
template <int LOGM, int R>
__global__ void __launch_bounds__(256) k_fsk_fwd_a(FskFwdParams p, int item0) {
  constexpr int M = 1 << LOGM;
  constexpr int N = M * R;
  constexpr int LOGN = LOGM + ct_log2(R);
  constexpr int MR = M / R;
  __shared__ float2 sm_twN[TwTables<LOGN>::N];
  load_tables<LOGN>(sm_twN, p.twN);
  __syncthreads();
  const int local = blockIdx.x / R;
  const int rank = blockIdx.x % R;
  const int item = item0 + local;
  float2* dst = p.scratch + (int64_t)local * N;
  for (int j = threadIdx.x; j < MR; j += blockDim.x) {
    const int m = rank * MR + j;
    float2 v[R];
#pragma unroll
    for (int n2 = 0; n2 < R; ++n2)
      v[n2] = make_float2(fsk_fwd_value(p, item, 0, m + M * n2), fsk_fwd_value(p, item, 1, m + M * n2));
    dft_reg<R, -1>(v);
    __stcs(dst + m, v[0]);
#pragma unroll
    for (int r = 1; r < R; ++r) __stcs(dst + (int64_t)r * M + m, cmul(v[r], twiddle<LOGN, -1>(sm_twN, m * r)));
  }
}

template <int LOGM, int R>
__global__ void __launch_bounds__(fsk_fft_threads<LOGM>(), fsk_min_blocks<LOGM, R>()) k_fsk_fwd_b(FskFwdParams p,
                                                                                                 int item0) {
  using FFT = BlockFFT<LOGM, kLogE, -1>;
  constexpr int M = 1 << LOGM;
  constexpr int N = M * R;
  extern __shared__ float4 smem_raw[];
  float2* sm = reinterpret_cast<float2*>(smem_raw);
  float2* sm_tw = sm + FFT::SMEM_ELEMS;
  load_tables<LOGM>(sm_tw, p.tw);
  const int local = blockIdx.x / R;
  const int rank = blockIdx.x % R;
  const float2* src = p.scratch + ((int64_t)local * R + rank) * M;
  float2* X = p.X + (int64_t)(item0 + local) * N + (int64_t)rank * M;
  const float sc = p.scale;
  const float sy = p.conj_out ? -sc : sc;
  auto load = [&](int i) { return __ldcs(src + i); };
  auto emit = [&](int k, float2 v) { X[k] = make_float2(v.x * sc, v.y * sy); };
  __syncthreads();  // tables
  FFT::run(sm, sm_tw, load, emit);
}

// valid lags of window w (the overlap rule with the support n_c)
__device__ __forceinline__ int fsk_valid_lags(const FskCorrParams& p, int w) {
  if (w < p.W - 1) return p.hop;
  const int64_t lim = p.S - p.n_c - (int64_t)w * p.hop;
  return (int)(lim < p.hop ? lim : p.hop) + 1;
}

template <int LOGM, int R>
__global__ void __launch_bounds__(fsk_fft_threads<LOGM>(), fsk_min_blocks<LOGM, R>()) k_fsk_corr(FskCorrParams p) {
  using FFT = BlockFFT<LOGM, kLogE, +1>;
  constexpr int M = 1 << LOGM;
  constexpr int N = M * R;
  constexpr int LOGN = LOGM + ct_log2(R);
  extern __shared__ float4 smem_raw[];
  float2* sm = reinterpret_cast<float2*>(smem_raw);
  float2* sm_tw = sm + FFT::SMEM_ELEMS;
  float2* sm_twN = sm_tw + TwTables<LOGM>::N;
  float4* red = reinterpret_cast<float4*>(sm_twN + TwTables<LOGN>::N);
  load_tables<LOGM>(sm_tw, p.tw);
  if constexpr (R > 1) load_tables<LOGN>(sm_twN, p.twN);
  const int item = blockIdx.x / R;
  const int rank = blockIdx.x % R;
  const int pr = item / p.Cg, c = item % p.Cg;
  const int wl0 = 2 * pr, wl1 = 2 * pr + 1;
  const bool has1 = wl1 < p.nw;
  const int nv0 = fsk_valid_lags(p, p.w0 + wl0);
  const int nv1 = has1 ? fsk_valid_lags(p, p.w0 + wl1) : 0;
  const float2* X = p.X + (int64_t)pr * N + (int64_t)rank * M;
  const float2* C = p.C + (int64_t)(p.sel ? p.sel[c] : c) * N + (int64_t)rank * M;
  auto load = [&](int k) { return cmul(X[k], C[k]); };
  float s0 = 0.f, b0 = -1.f, s1 = 0.f, b1 = -1.f;
  int t0 = INT_MAX, t1 = INT_MAX;
  auto take = [&](int tau, float2 z) {
    const float P0 = z.x * z.x, P1 = z.y * z.y;
    s0 += P0;
    s1 += P1;
    if (tau < nv0) better(b0, t0, P0, tau);
    if (tau < nv1) better(b1, t1, P1, tau);
  };
  __syncthreads();  // tables
  if constexpr (R == 1) {
    auto emit = [&](int m, float2 v) { take(m, v); };
    FFT::run(sm, sm_tw, load, emit);
  } else {
    // the last pass has read all of its inputs (block barrier) before it
    // emits, so the outputs can go back into the same buffer
    auto emit = [&](int m, float2 v) { sm[spad(m)] = cmul(v, twiddle<LOGN, +1>(sm_twN, m * rank)); };
    FFT::run(sm, sm_tw, load, emit);
    cg::cluster_group cluster = cg::this_cluster();
    cluster.sync();  // every block's inverse transform is in its shared memory
    constexpr int MR = M / R;
    const float2* src[R];
#pragma unroll
    for (int r = 0; r < R; ++r) src[r] = cluster.map_shared_rank(sm, r);
    for (int j = threadIdx.x; j < MR; j += blockDim.x) {
      const int m = rank * MR + j;
      float2 v[R];
#pragma unroll
      for (int r = 0; r < R; ++r) v[r] = src[r][spad(m)];
      dft_reg<R, +1>(v);
#pragma unroll
      for (int n2 = 0; n2 < R; ++n2) take(m + M * n2, v[n2]);
    }
    cluster.sync();  // no block leaves while another still reads its shared memory
  }
  block_reduce_stats(s0, b0, t0, red);
  block_reduce_stats(s1, b1, t1, red + 32);
  if (threadIdx.x == 0) {
    p.part[((int64_t)wl0 * p.Cg + c) * R + rank] = make_float4(s0, b0, __int_as_float(t0), 0.f);
    if (has1) p.part[((int64_t)wl1 * p.Cg + c) * R + rank] = make_float4(s1, b1, __int_as_float(t1), 0.f);
  }
}

// Two-pass form of k_fsk_corr for R > 1: the same index maps with the
// exchange through a scratch buffer in global memory instead of distributed
// shared memory, so no block waits on another.
//   pass A: block (item, r) inverse-transforms its run Z_perm[r M + .] and
//           writes W_N^{-m r} Y_r[m] to scratch[(item - item0) R + r][m]
//   pass B: block (item, rho) reads, for each m of its range, the R values
//           scratch[.. r][m], takes the R-point DFT and the epilogue; its
//           partial results are those of cluster block rho.
// The values are the cluster form's, so the results are bit-identical.
template <int LOGM, int R>
__global__ void __launch_bounds__(fsk_fft_threads<LOGM>(), fsk_min_blocks<LOGM, R>()) k_fsk_corr_a(FskCorrParams p,
                                                                                           int item0) {
  using FFT = BlockFFT<LOGM, kLogE, +1>;
  constexpr int M = 1 << LOGM;
  constexpr int N = M * R;
  constexpr int LOGN = LOGM + ct_log2(R);
  extern __shared__ float4 smem_raw[];
  float2* sm = reinterpret_cast<float2*>(smem_raw);
  float2* sm_tw = sm + FFT::SMEM_ELEMS;
  float2* sm_twN = sm_tw + TwTables<LOGM>::N;
  load_tables<LOGM>(sm_tw, p.tw);
  if constexpr (fsk_twN_shared<LOGN>()) load_tables<LOGN>(sm_twN, p.twN);
  const float2* twN = fsk_twN_shared<LOGN>() ? sm_twN : p.twN;
  const int local = blockIdx.x / R;
  const int rank = blockIdx.x % R;
  const int item = item0 + local;
  const int pr = item / p.Cg, c = item % p.Cg;
  const float2* X = p.X + (int64_t)pr * N + (int64_t)rank * M;
  const float2* C = p.C + (int64_t)(p.sel ? p.sel[c] : c) * N + (int64_t)rank * M;
  float2* out = p.scratch + ((int64_t)local * R + rank) * M;
  auto load = [&](int k) { return cmul(X[k], C[k]); };
  auto emit = [&](int m, float2 v) { __stcs(out + m, cmul(v, twiddle<LOGN, +1>(twN, m * rank))); };
  __syncthreads();  // tables
  FFT::run(sm, sm_tw, load, emit);
}

// Pass A for M = 2^14, R = 16 with the warp-private inverse transform of
// k_corr_dif (decimation in frequency, 16 chunks of 1024 points; see
// acq_fft_kernels.cuh): persistent over the units (local item, rank).  Step A
// (whole block) takes the 16-point DFTs of the columns j = t and t + 512 and
// the twiddles W_M^{j m'}; step B (warp m' alone) transforms chunk m' with two
// radix-32 passes.  Output m = m' + 16 k gets W_N^{m r} = W_N^{(m' + 16 lane) r}
// W_512^{(r' r) mod 512} (k = lane + 32 r') and goes to scratch position
// m' 1024 + k, one contiguous run per warp: the chunk order that
// k_fsk_corr_b<14, 16, true> reads.
constexpr size_t fsk_dif_smem() {
  return sizeof(float2) * ((size_t)16 * kDifChunkPad + TwTables<14>::N + 32 * kDifTwPitch + 512);
}

__global__ void __launch_bounds__(512, 1) k_fsk_corr_a_dif(FskCorrParams p, int item0, int n_units) {
  constexpr int LOGM = 14, M = 1 << LOGM, R = 16, N = M * R, LOGN = 18;
  extern __shared__ float4 smem_raw[];
  float2* sm = reinterpret_cast<float2*>(smem_raw);
  float2* sm_tw = sm + 16 * kDifChunkPad;
  const float2* trow = sm_tw + TwTables<LOGM>::N + kDifTwPitch * (threadIdx.x & 31);  // W_1024^{lane r}
  float2* t512 = sm_tw + TwTables<LOGM>::N + 32 * kDifTwPitch;  // W_N^{512 i} = W_512^i
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  load_tables<LOGM>(sm_tw, p.tw);
  __syncthreads();
  build_dif_tw<LOGM>(sm_tw);
  for (int i = t; i < 512; i += blockDim.x) t512[i] = twiddle<LOGN, +1>(p.twN, i << 9);
  for (int u = blockIdx.x; u < n_units; u += gridDim.x) {
    const int local = u >> 4, rank = u & 15;
    const int item = item0 + local;
    const int pr = item / p.Cg, c = item % p.Cg;
    const float2* X = p.X + (int64_t)pr * N + (int64_t)rank * M;
    const float2* C = p.C + (int64_t)(p.sel ? p.sel[c] : c) * N + (int64_t)rank * M;
    float2 a[16], b[16];
#pragma unroll
    for (int m = 0; m < 16; ++m) {
      a[m] = cmul(X[t + 1024 * m], C[t + 1024 * m]);
      b[m] = cmul(X[t + 512 + 1024 * m], C[t + 512 + 1024 * m]);
    }
    dft_reg<16, +1>(a);
    dft_reg<16, +1>(b);
    {  // W_M^{t m'} and W_M^{(t + 512) m'} = W_M^{t m'} W_32^{m'}; W_M^{t m'} by
       // repeated multiplication with W_M^t (a table read of W_M^{8 t} would be
       // an 8-way bank conflict)
      const float2 wt1 = twiddle<LOGM, +1>(sm_tw, t);
      float2 wt = wt1;
#define ATLAS_FSK_TW(M_)                                                               \
  if (M_ > 1) wt = cmul(wt, wt1);                                                      \
  a[M_] = cmul(a[M_], wt);                                                             \
  b[M_] = cmul(b[M_], cmul(wt, make_float2(Tw<M_, 32, +1>::re, Tw<M_, 32, +1>::im)));
      ATLAS_FSK_TW(1) ATLAS_FSK_TW(2) ATLAS_FSK_TW(3) ATLAS_FSK_TW(4) ATLAS_FSK_TW(5) ATLAS_FSK_TW(6)
      ATLAS_FSK_TW(7) ATLAS_FSK_TW(8) ATLAS_FSK_TW(9) ATLAS_FSK_TW(10) ATLAS_FSK_TW(11) ATLAS_FSK_TW(12)
      ATLAS_FSK_TW(13) ATLAS_FSK_TW(14) ATLAS_FSK_TW(15)
#undef ATLAS_FSK_TW
    }
    __syncthreads();  // (1) the previous unit's chunks are read (and the tables are ready)
#pragma unroll
    for (int m = 0; m < 16; ++m) {
      sm[m * kDifChunkPad + dif_pos(t)] = a[m];
      sm[m * kDifChunkPad + dif_pos(t + 512)] = b[m];
    }
    __syncthreads();  // (2) every chunk is complete
    float2* ch = sm + warp * kDifChunkPad;
    float2 x[32];
#pragma unroll
    for (int r = 0; r < 32; ++r) x[r] = ch[dif_pos(lane + 32 * r)];
    __syncwarp();
    dft_reg<32, +1>(x);
    float4* rowp = reinterpret_cast<float4*>(ch + dif_pos(32 * lane));
#pragma unroll
    for (int r = 0; r < 32; r += 2) rowp[r / 2] = make_float4(x[r].x, x[r].y, x[r + 1].x, x[r + 1].y);
    __syncwarp();
    const float4* tw2 = reinterpret_cast<const float4*>(trow);
#pragma unroll
    for (int r = 0; r < 32; r += 2) {
      const float4 w = tw2[r / 2];  // W_1024^{lane r}, W_1024^{lane (r + 1)} (forward: conjugated here)
      x[r] = ch[dif_pos(lane + 32 * r)];
      x[r + 1] = ch[dif_pos(lane + 32 * (r + 1))];
      if (r > 0) x[r] = cmul_conj(x[r], make_float2(w.x, w.y));
      x[r + 1] = cmul_conj(x[r + 1], make_float2(w.z, w.w));
    }
    dft_reg<32, +1>(x);
    // m = warp + 16 (lane + 32 r): twiddle W_N^{m rank}, chunk-ordered store
    const float2 base = twiddle<LOGN, +1>(p.twN, (warp + 16 * lane) * rank);
    float2* out = p.scratch + ((int64_t)local * R + rank) * M + warp * 1024 + lane;
#pragma unroll
    for (int r = 0; r < 32; ++r) __stcs(out + 32 * r, cmul(x[r], cmul(base, t512[(r * rank) & 511])));
  }
}

// CHUNKED: pass A wrote the scratch in the chunk order of the warp-private
// transform (M = 2^14, R = 16: position m' 1024 + k holds m = m' + 16 k), so
// block rho's positions [rho 1024, rho 1024 + 1024) are the m = 16 j + rho.
template <int LOGM, int R, bool CHUNKED = false>
__global__ void __launch_bounds__(256) k_fsk_corr_b(FskCorrParams p, int item0) {
  constexpr int M = 1 << LOGM;
  constexpr int MR = M / R;
  static_assert(!CHUNKED || (LOGM == 14 && R == 16), "chunk order of 16 x 1024 points");
  __shared__ float4 red[64];
  const int local = blockIdx.x / R;
  const int rank = blockIdx.x % R;
  const int item = item0 + local;
  const int pr = item / p.Cg, c = item % p.Cg;
  const int wl0 = 2 * pr, wl1 = 2 * pr + 1;
  const bool has1 = wl1 < p.nw;
  const int nv0 = fsk_valid_lags(p, p.w0 + wl0);
  const int nv1 = has1 ? fsk_valid_lags(p, p.w0 + wl1) : 0;
  const float2* src = p.scratch + (int64_t)local * R * M;
  float s0 = 0.f, b0 = -1.f, s1 = 0.f, b1 = -1.f;
  int t0 = INT_MAX, t1 = INT_MAX;
  for (int j = threadIdx.x; j < MR; j += blockDim.x) {
    const int pos = rank * MR + j;
    const int m = CHUNKED ? 16 * j + rank : pos;
    float2 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = __ldcs(src + (int64_t)r * M + pos);
    dft_reg<R, +1>(v);
#pragma unroll
    for (int n2 = 0; n2 < R; ++n2) {
      const int tau = m + M * n2;
      const float P0 = v[n2].x * v[n2].x, P1 = v[n2].y * v[n2].y;
      s0 += P0;
      s1 += P1;
      if (tau < nv0) better(b0, t0, P0, tau);
      if (tau < nv1) better(b1, t1, P1, tau);
    }
  }
  block_reduce_stats(s0, b0, t0, red);
  block_reduce_stats(s1, b1, t1, red + 32);
  if (threadIdx.x == 0) {
    p.part[((int64_t)wl0 * p.Cg + c) * R + rank] = make_float4(s0, b0, __int_as_float(t0), 0.f);
    if (has1) p.part[((int64_t)wl1 * p.Cg + c) * R + rank] = make_float4(s1, b1, __int_as_float(t1), 0.f);
  }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------

namespace {

template <int LOGM, int R>
cudaError_t prepare_one() {
  constexpr int LOGN = LOGM + ct_log2(R);
  constexpr int smem = (int)fsk_fft_smem<LOGM, LOGN>();
  cudaError_t e;
  if constexpr (fsk_cluster_form<LOGM, R>()) {  // the single-block and cluster forms
    if ((e = cudaFuncSetAttribute(k_fsk_fwd<LOGM, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) !=
        cudaSuccess)
      return e;
    if ((e = cudaFuncSetAttribute(k_fsk_corr<LOGM, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) !=
        cudaSuccess)
      return e;
    if constexpr (R > 8) {  // clusters of 16 blocks are beyond the portable size
      if ((e = cudaFuncSetAttribute(k_fsk_fwd<LOGM, R>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1)) !=
          cudaSuccess)
        return e;
      if ((e = cudaFuncSetAttribute(k_fsk_corr<LOGM, R>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1)) !=
          cudaSuccess)
        return e;
    }
  }
  if constexpr (R > 1) {  // the two-pass forms
    if ((e = cudaFuncSetAttribute(k_fsk_fwd_b<LOGM, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) !=
        cudaSuccess)
      return e;
    if ((e = cudaFuncSetAttribute(k_fsk_corr_a<LOGM, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) !=
        cudaSuccess)
      return e;
    if constexpr (LOGM == 14 && R == 16) {
      if ((e = cudaFuncSetAttribute(k_fsk_corr_a_dif, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)fsk_dif_smem())) != cudaSuccess)
        return e;
    }
  }
  return cudaSuccess;
}

template <class P>
cudaError_t launch_clustered(void (*kern)(P), int R, int blocks, int threads, size_t smem, const P& p,
                             cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(blocks, 1, 1);
  cfg.blockDim = dim3(threads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = R;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = R > 1 ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kern, p);
}

template <int LOGM, int R>
cudaError_t fwd_one(const FskFwdParams& p, cudaStream_t s) {
  constexpr int LOGN = LOGM + ct_log2(R);
  if constexpr (R > 1) {
    if (p.scratch) {
      if (p.chunk_items < 1) return cudaErrorInvalidValue;
      for (int i0 = 0; i0 < p.n_items; i0 += p.chunk_items) {
        const int n = std::min(p.chunk_items, p.n_items - i0);
        k_fsk_fwd_a<LOGM, R><<<n * R, 256, 0, s>>>(p, i0);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        k_fsk_fwd_b<LOGM, R><<<n * R, fsk_fft_threads<LOGM>(), fsk_fft_smem<LOGM, LOGN>(), s>>>(p, i0);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
      }
      return cudaSuccess;
    }
  }
  if constexpr (!fsk_cluster_form<LOGM, R>()) {
    return cudaErrorInvalidValue;  // two-pass form only
  } else {
    return launch_clustered(k_fsk_fwd<LOGM, R>, R, p.n_items * R, fsk_fft_threads<LOGM>(),
                            fsk_fft_smem<LOGM, LOGN>(), p, s);
  }
}

template <int LOGM, int R>
cudaError_t corr_one(const FskCorrParams& p, cudaStream_t s) {
  constexpr int LOGN = LOGM + ct_log2(R);
  const int items = ((p.nw + 1) / 2) * p.Cg;
  if constexpr (R > 1) {
    if (p.scratch) {
      if (p.chunk_items < 1) return cudaErrorInvalidValue;
      for (int i0 = 0; i0 < items; i0 += p.chunk_items) {
        const int n = std::min(p.chunk_items, items - i0);
        cudaError_t e;
        if constexpr (LOGM == 14 && R == 16) {
          static int resident = 0;  // blocks of k_fsk_corr_a_dif resident on the device
          if (resident == 0) {
            int dev = 0, sms = 0, per_sm = 0;
            if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
                (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess ||
                (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fsk_corr_a_dif, 512, fsk_dif_smem())) !=
                    cudaSuccess)
              return e;
            resident = std::max(1, per_sm) * sms;
          }
          k_fsk_corr_a_dif<<<std::min(n * R, resident), 512, fsk_dif_smem(), s>>>(p, i0, n * R);
          if ((e = cudaGetLastError()) != cudaSuccess) return e;
          k_fsk_corr_b<LOGM, R, true><<<n * R, 256, 0, s>>>(p, i0);
        } else {
          k_fsk_corr_a<LOGM, R><<<n * R, fsk_fft_threads<LOGM>(), fsk_fft_smem<LOGM, LOGN>(), s>>>(p, i0);
          if ((e = cudaGetLastError()) != cudaSuccess) return e;
          k_fsk_corr_b<LOGM, R><<<n * R, 256, 0, s>>>(p, i0);
        }
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
      }
      return cudaSuccess;
    }
  }
  if constexpr (!fsk_cluster_form<LOGM, R>()) {
    return cudaErrorInvalidValue;  // two-pass form only
  } else {
    return launch_clustered(k_fsk_corr<LOGM, R>, R, items * R, fsk_fft_threads<LOGM>(),
                            fsk_fft_smem<LOGM, LOGN>(), p, s);
  }
}

}  // namespace

cudaError_t fsk_prepare_fft() {
  cudaError_t e;
  if ((e = prepare_one<10, 1>()) != cudaSuccess) return e;
  if ((e = prepare_one<11, 1>()) != cudaSuccess) return e;
  if ((e = prepare_one<12, 1>()) != cudaSuccess) return e;
  if ((e = prepare_one<13, 1>()) != cudaSuccess) return e;
  if ((e = prepare_one<14, 1>()) != cudaSuccess) return e;
  if ((e = prepare_one<13, 4>()) != cudaSuccess) return e;
  if ((e = prepare_one<13, 8>()) != cudaSuccess) return e;
  if ((e = prepare_one<13, 16>()) != cudaSuccess) return e;
  if ((e = prepare_one<14, 8>()) != cudaSuccess) return e;
  if ((e = prepare_one<13, 32>()) != cudaSuccess) return e;
  return prepare_one<14, 16>();
}

cudaError_t launch_fsk_fwd(int logN, int logM, const FskFwdParams& p, cudaStream_t s) {
  if (p.n_items <= 0) return cudaSuccess;
  if (!fsk_plan_supported(logN, logM)) return cudaErrorInvalidValue;
  switch (logN) {
    case 10: return fwd_one<10, 1>(p, s);
    case 11: return fwd_one<11, 1>(p, s);
    case 12: return fwd_one<12, 1>(p, s);
    case 13: return fwd_one<13, 1>(p, s);
    case 14: return fwd_one<14, 1>(p, s);
    case 15: return fwd_one<13, 4>(p, s);
    case 16: return fwd_one<13, 8>(p, s);
    case 17: return logM == 14 ? fwd_one<14, 8>(p, s) : fwd_one<13, 16>(p, s);
    case 18: return logM == 14 ? fwd_one<14, 16>(p, s) : fwd_one<13, 32>(p, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_fsk_corr(int logN, int logM, const FskCorrParams& p, cudaStream_t s) {
  if (p.nw <= 0 || p.Cg <= 0) return cudaSuccess;
  if (!fsk_plan_supported(logN, logM)) return cudaErrorInvalidValue;
  switch (logN) {
    case 10: return corr_one<10, 1>(p, s);
    case 11: return corr_one<11, 1>(p, s);
    case 12: return corr_one<12, 1>(p, s);
    case 13: return corr_one<13, 1>(p, s);
    case 14: return corr_one<14, 1>(p, s);
    case 15: return corr_one<13, 4>(p, s);
    case 16: return corr_one<13, 8>(p, s);
    case 17: return logM == 14 ? corr_one<14, 8>(p, s) : corr_one<13, 16>(p, s);
    case 18: return logM == 14 ? corr_one<14, 16>(p, s) : corr_one<13, 32>(p, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace atlas
