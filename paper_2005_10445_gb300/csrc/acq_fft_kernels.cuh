// acq_fft_kernels.cuh -- the transform kernels of the search, templated on the
// transform size (LOGM) and on the tile shape (LOGE: 2^LOGE complex values per
// thread, 2^(LOGM-LOGE) threads per block).  Instantiated once per LOGE in
// acq_fft_e4.cu / acq_fft_e5.cu; the host picks the tile shape per size
// (autotuned or default).
//
//   k_window_fft<LOGM, LOGE>        G = FFT_M(B) in place, one block per (rho, k, window)
//   k_corr<LOGM, LOGE>              G * conj(C) / M -> IFFT_M -> |.|^2 -> floor sum, argmax
//   k_window_fft_split<LOGH, LOGE>  M = 2^(LOGH+1): a 2-block cluster, block h transforms the
//                                   even (h = 0) or odd (h = 1) samples of the row; the row
//                                   becomes [E | O] (decimation in time)
//   k_corr_split<LOGH, LOGE>        rebuilds G from E and O on load, multiplies by the code
//                                   spectrum, takes one radix-2 decimation-in-frequency step
//                                   and inverse-transforms one half: block h produces the
//                                   lags q = 2k + h
//   k_corr_dif<14, SPLIT>           the default correlation for M = 2^14 (one block per
//                                   item, warp-private second and third passes) and, with
//                                   SPLIT, for M = 2^15: each half h of k_corr_split's
//                                   decomposition as one 2^14-point item, its input formed
//                                   as E A_h + O B_h from three precomputed code tables
// Section 4.1 computes cross-correlations with FFTs; the split forms are the
// same transforms with one radix-2 stage folded into the global loads, so
// transforms of 2^15 points need no more shared memory than 2^14.
#pragma once

#include <cooperative_groups.h>

#include <algorithm>

#include "acq_common.cuh"

namespace atlas {

template <int LOGM, int LOGE>
constexpr int fft_threads() { return (1 << LOGM) >> LOGE; }

// dynamic shared memory: padded transform buffer, twiddle tables of the
// transform, the 32 x 32 second-pass table, the tables of the split stage,
// reduction scratch for up to 32 warps
template <int LOGM>
constexpr size_t fft_smem() {
  return sizeof(float2) * (BlockFFT<LOGM, 5, -1>::SMEM_ELEMS + TwTables<LOGM>::N + 1024 + TwTables<LOGM + 1>::N) +
         32 * sizeof(float4) + sizeof(float2) * (kMaxSps + 1);
}

// valid lags of window w (Section 2.1 overlap rule): [0, hop) before the last
// window, [0, min(hop, S - L - w*hop)] in the last.
__device__ __forceinline__ int valid_lags(const CorrParams& p, int w) {
  int nvalid = p.hop;
  if (w == p.W - 1) {
    const int64_t lim = p.S - p.L - (int64_t)w * p.hop;
    nvalid = (int)(lim < p.hop ? lim : p.hop) + 1;
  }
  return nvalid;
}

// The index of a correlation item in the mixed radix (h: 2 for split rows,
// else 1; rho: sps; bin: K; code: Cg; then the window of the launch group,
// or the listed pair), kept as digits.  Advancing by the grid stride adds
// digit by digit with one carry each: the item loop needs no integer
// division (sps is a power of two).
struct ItemCursor {
  int h, rho, k, c;
  int64_t w;
  __device__ __forceinline__ void set(const CorrParams& p, bool split, int lsps, int64_t v) {
    h = split ? (int)(v & 1) : 0;
    if (split) v >>= 1;
    rho = (int)(v & ((1 << lsps) - 1));
    v >>= lsps;
    k = p.pairs ? 0 : (int)(v % p.K);
    if (!p.pairs) v /= p.K;
    c = p.pairs ? 0 : (int)(v % p.Cg);
    w = p.pairs ? v : v / p.Cg;
  }
  __device__ __forceinline__ void advance(const CorrParams& p, bool split, const ItemCursor& s) {
    int cy = 0;
    if (split) {
      h += s.h;
      cy = h >= 2;
      h -= 2 * cy;
    }
    rho += s.rho + cy;
    cy = rho >= p.sps;
    rho -= cy * p.sps;
    if (p.pairs) {
      w += s.w + cy;
      return;
    }
    k += s.k + cy;
    cy = k >= p.K;
    k -= cy * p.K;
    c += s.c + cy;
    cy = c >= p.Cg;
    c -= cy * p.Cg;
    w += s.w + cy;
  }
  // the item's window-spectrum row, window, code and partial-result index
  __device__ __forceinline__ void locate(const CorrParams& p, int64_t& row, int& win, int& code, int64_t& out) const {
    if (p.pairs) {
      const int4 pr = p.pairs[w];
      row = (int64_t)pr.x * p.sps + rho;
      code = pr.y;
      win = pr.z;
      out = w * p.sps + rho;
    } else {
      row = (w * p.K + k) * p.sps + rho;
      code = c;
      win = p.w0 + (int)w;
      out = ((w * p.Cg + c) * p.K + k) * p.sps + rho;
    }
  }
};

// Persistent over its rows (block b takes rows b, b + gridDim.x, ...).
template <int LOGM, int LOGE>
__global__ void __launch_bounds__(fft_threads<LOGM, LOGE>()) k_window_fft(WindowFftParams p) {
  using FFT = BlockFFT<LOGM, LOGE, -1, true>;
  extern __shared__ float4 smem_raw[];
  float2* sm = reinterpret_cast<float2*>(smem_raw);
  float2* sm_tw = sm + FFT::SMEM_ELEMS;
  load_tables<LOGM>(sm_tw, p.tw);
  __syncthreads();
  build_tw32<LOGM>(sm_tw);
  const int64_t rows = (int64_t)p.nw * p.K * p.sps;
  for (int64_t row = blockIdx.x; row < rows; row += gridDim.x) {
    __syncthreads();  // tables ready; the previous row's shared-memory reads are done
    // every input value is read into registers/shared memory before the first
    // output is written (the passes are separated by block barriers), so the
    // transform can overwrite its own input row
    float2* G = p.G + row * FFT::M;
    // the block's next row (written by the mix kernel, in device memory) is
    // fetched into L2 while this one is transformed, so its loads hit L2
    if (row + gridDim.x < rows) {
      const char* nxt = reinterpret_cast<const char*>(G + (int64_t)gridDim.x * FFT::M);
      for (int off = 128 * (int)threadIdx.x; off < FFT::M * (int)sizeof(float2); off += 128 * (int)blockDim.x)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(nxt + off));
    }
    auto load = [&](int i) { return G[i]; };
    auto emit = [&](int i, float2 v) { G[i] = v; };
    FFT::run(sm, sm_tw, load, emit);
  }
}

// Persistent over its cells: block b takes cells b, b + gridDim.x, ...  (the
// launch order of a one-cell-per-block grid: rho fastest, then bin, then
// window and code), so the twiddle tables are loaded once per block and the
// per-cell prologue is a barrier.
template <int LOGM, int LOGE>
__global__ void __launch_bounds__(fft_threads<LOGM, LOGE>()) k_corr(CorrParams p) {
  using FFT = BlockFFT<LOGM, LOGE, +1, true>;
  extern __shared__ float4 smem_raw[];
  float2* sm = reinterpret_cast<float2*>(smem_raw);
  float2* sm_tw = sm + FFT::SMEM_ELEMS;
  float4* red = reinterpret_cast<float4*>(sm_tw + TwTables<LOGM>::N + 1024 + TwTables<LOGM + 1>::N);

  const int sps = p.sps;
  load_tables<LOGM>(sm_tw, p.tw);
  __syncthreads();
  build_tw32<LOGM>(sm_tw);
  const int64_t n_items = p.pairs ? (int64_t)p.n_pairs * sps : (int64_t)sps * p.K * p.nw * p.Cg;
  const int lsps = __ffs(sps) - 1;  // sps is a power of two
  ItemCursor cur, stride;
  cur.set(p, false, lsps, blockIdx.x);
  stride.set(p, false, lsps, gridDim.x);
  for (int64_t item = blockIdx.x; item < n_items; item += gridDim.x, cur.advance(p, false, stride)) {
    __syncthreads();  // tables ready; the previous cell's shared-memory reads are done
    const int rho = cur.rho;
    int64_t row, out;  // G row and partial-result index of this cell
    int c, w;
    cur.locate(p, row, w, c, out);
    const int nvalid = valid_lags(p, w);
    const float2* G = p.G + row * FFT::M;
    const float2* D = p.D + (int64_t)c * FFT::M;
    auto load = [&](int i) { return cmul(G[i], D[i]); };
    // lag tau = sps*q + rho is valid iff q < qlim; a thread's outputs arrive in
    // increasing q, so the first maximum is the smallest lag
    const int qlim = (nvalid - rho + sps - 1) >> lsps;
    float sum = 0.f, best = -1.f;
    int bq = 0x7fffffff;
    auto emit = [&](int q, float2 v) {
      const float P = fmaf(v.x, v.x, v.y * v.y);
      sum += P;
      if (q < qlim && P > best) {
        best = P;
        bq = q;
      }
    };
    FFT::run(sm, sm_tw, load, emit);
    int bt = bq == 0x7fffffff ? bq : bq * sps + rho;
    block_reduce_stats(sum, best, bt, red);
    if (threadIdx.x == 0) p.part[out] = make_float4(sum, best, __int_as_float(bt), 0.f);
  }
}

// ---------------------------------------------------------------------------
// k_corr_dif: the per-code correlation of M = 2^12, 2^13 or 2^14 points with
// warp-private second and third passes (written out below for M = 2^14; a
// smaller M has NCH = M / 1024 chunks, NCH warps and NCH-point step-A DFTs,
// each thread taking 16 / NCH column pairs).
//
// The inverse transform is split by decimation in frequency, M = 16 x 1024:
// with i = j + 1024 m and q = m' + 16 k,
//   corr[q] = sum_j W_1024^{jk} (W_M^{j m'} sum_m Z[j + 1024 m] W_16^{m m'}),   W = exp(+2 pi i / .)
// Step A (whole block): thread t loads Z[j + 1024 m] = G * conj(C)/M for the
// two columns j = t and j' = 1024 - t (thread 0: 0 and 512), takes their
// 16-point DFTs over m, multiplies output m' by W_M^{j m'} and stores it at
// position j of chunk m'.  The code spectrum of +/-1 chips is Hermitian,
// D[M - i] = conj(D[i]), and M - (j + 1024 m) = j' + 1024 (15 - m), so column
// j' takes column j's code spectrum in reverse order, conjugated: the thread
// loads one column of D instead of two.  Its twiddles are
// W_M^{j' m'} = W_16^{m'} conj(W_M^{j m'}); the W_16^{m'} factor is a cyclic
// shift of the DFT's inputs by one (free), so column j' reuses column j's
// twiddle, conjugated.  Columns 0 and 512 are each their own mirror.
// Step B (warp w alone): chunk w is an independent 1024-point inverse DFT,
// taken as two radix-32 Stockham passes through the chunk's own shared memory
// (only __syncwarp between them; the transpose is written as 16-byte pairs and
// the second pass's twiddles W_1024^{lane r} are read from the lane's row of a
// table as 16-byte pairs), then |.|^2, the floor sum and the argmax over the
// lags q = w + 16 k, k = lane + 32 r.  When hop <= N/2 no valid lag has r >= 16:
// the second pass then forms only its outputs r < 16, and the floor's sum over
// all lags comes from that pass's inputs by Parseval (sum |X|^2 = 32 sum |x|^2).
// A block meets only twice per item: before step A writes the chunks (the
// previous item's chunks are read) and after (the chunks are complete).  In
// between, warps run out of step: one warp's shared-memory traffic, global
// loads and arithmetic overlap the others'.  The 16 per-warp partial results
// are combined by warp 0 after the next item's first barrier.
// ---------------------------------------------------------------------------

constexpr int kDifChunk = 1024;                          // points per warp transform
constexpr int kDifChunkPad = kDifChunk + kDifChunk / 16;  // chunk pitch (float2): 2 pad elements per 32
constexpr int kDifTwPitch = 34;                          // row pitch of the step-B twiddle table

// chunks of 1024 points (= warps, = points of the step-A DFT) and threads of
// the block for a transform of 2^LOGM points
template <int LOGM>
constexpr int dif_chunks() { return 1 << (LOGM - 10); }
template <int LOGM>
constexpr int dif_threads() { return 32 * dif_chunks<LOGM>(); }

template <int LOGM>
constexpr size_t dif_smem() {
  return sizeof(float2) * ((size_t)dif_chunks<LOGM>() * kDifChunkPad + TwTables<LOGM>::N + 32 * kDifTwPitch) +
         2 * dif_chunks<LOGM>() * sizeof(float4);
}

// position of point j in a chunk: two pad elements after every 32, so that
// both a warp's 32 consecutive points and the 16-byte stores of step B's
// transpose (rows of 32 at a pitch of 34) are free of bank conflicts
__device__ __forceinline__ int dif_pos(int j) { return j + 2 * (j >> 5); }

// W_1024^{l r} (forward) at [34 l + r], l, r < 32: a thread reads its row as 16-byte pairs
template <int LOGM>
__device__ __forceinline__ void build_dif_tw(float2* tw) {
  for (int i = threadIdx.x; i < 32 * kDifTwPitch; i += blockDim.x) {
    const int l = i / kDifTwPitch, r = i % kDifTwPitch;
    if (r < 32) tw[TwTables<LOGM>::N + i] = twiddle<LOGM, -1>(tw, ((l * r) & 1023) << (LOGM - 10));
  }
}

__device__ __forceinline__ void warp_reduce_stats(float& sum, float& best, int& bt) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float s2 = __shfl_down_sync(0xffffffffu, sum, o);
    const float b2 = __shfl_down_sync(0xffffffffu, best, o);
    const int t2 = __shfl_down_sync(0xffffffffu, bt, o);
    sum += s2;
    better(best, bt, b2, t2);
  }
}

// Step A's twiddles for output m' = MP of the column pair (j, 1024 - j):
// W_M^{j m'} for column j and its conjugate for the mirror column (after the
// shift of its DFT inputs); W_M^{j m'} by repeated multiplication with W_M^j
// (at most 15 steps, a few FP32 ulps; a table read at m' = 8 would be an
// 8-way bank conflict, the lanes' indices 8 j being 64 bytes apart).
template <int LOGM, int MP>
__device__ __forceinline__ void dif_twiddle_one(float2* a, float2* b, float2& wt, const float2& wt1,
                                                const float2* tw, int j) {
  if constexpr (MP > 1) wt = cmul(wt, wt1);
  a[MP] = cmul(a[MP], wt);
  b[MP] = cmul_conj(b[MP], wt);
}

template <int LOGM, int... Ms>
__device__ __forceinline__ void dif_twiddles(float2* a, float2* b, const float2* tw, int j,
                                             std::integer_sequence<int, Ms...>) {
  const float2 wt1 = twiddle<LOGM, +1>(tw, j);
  float2 wt = wt1;
  (dif_twiddle_one<LOGM, Ms + 1>(a, b, wt, wt1, tw, j), ...);
}

// column 512 (the mirror of itself): W_M^{512 m'} = W_{2 NCH}^{m'}, i.e.
// W_{2 NCH}^{-m'} after the shift by W_NCH^{m'}
template <int NCH, int... Ms>
__device__ __forceinline__ void dif_twiddle_col512(float2* b, std::integer_sequence<int, Ms...>) {
  ((b[Ms + 1] = cmul(b[Ms + 1], make_float2(Tw<Ms + 1, 2 * NCH, -1>::re, Tw<Ms + 1, 2 * NCH, -1>::im))), ...);
}

// One block of 32 NCH threads per item (NCH = M / 1024 chunks, one warp per
// chunk in step B).  Thread t takes the column pairs (j, 1024 - j) with
// j = t + 32 NCH i, i < 16 / NCH (the pair j = 0 is the columns 0 and 512).
// SPLIT (M = 2^14 blocks of a 2^15-point row): the rows hold the spectra as
// [E | O] (k_window_fft_split) and item h = 0, 1 of a (cell, rho) takes the
// lags q = 2 q' + h as the 2^14-point inverse transform of Y_h = E A_h + O B_h
// (the code tables D3, k_code_split_tables).
template <int LOGM, bool SPLIT = false>
__global__ void __launch_bounds__(dif_threads<LOGM>(), 16 / dif_chunks<LOGM>()) k_corr_dif(CorrParams p) {
  constexpr int NCH = dif_chunks<LOGM>();
  constexpr int T = 32 * NCH;
  constexpr int NP = 512 / T;  // column pairs per thread
  static_assert(LOGM >= 12 && LOGM <= 14, "4, 8 or 16 chunks of 1024 points");
  static_assert(!SPLIT || LOGM == 14, "split rows: halves of 2^15 points");
  constexpr int H = 1 << LOGM;
  extern __shared__ float4 smem_raw[];
  float2* sm = reinterpret_cast<float2*>(smem_raw);
  float2* sm_tw = sm + NCH * kDifChunkPad;
  const float2* trow = sm_tw + TwTables<LOGM>::N + kDifTwPitch * (threadIdx.x & 31);  // W_1024^{lane r}
  float4* red = reinterpret_cast<float4*>(sm_tw + TwTables<LOGM>::N + 32 * kDifTwPitch);  // [2][NCH]

  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int sps = p.sps;
  const bool half = 2 * p.hop <= p.N;  // no valid lag in the upper half of any row
  load_tables<LOGM>(sm_tw, p.tw);
  __syncthreads();
  build_dif_tw<LOGM>(sm_tw);

  const int64_t n_items = (SPLIT ? 2 : 1) * (p.pairs ? (int64_t)p.n_pairs * sps : (int64_t)sps * p.K * p.nw * p.Cg);
  const int lsps = __ffs(sps) - 1;  // sps is a power of two
  ItemCursor cur, stride;
  cur.set(p, SPLIT, lsps, blockIdx.x);
  stride.set(p, SPLIT, lsps, gridDim.x);
  int64_t prev_out = -1;
  int par = 0;
  for (int64_t item = blockIdx.x;; item += gridDim.x) {
    const bool have = item < n_items;
    int64_t out = 0;
    int rho = 0, qlim = 0, h = 0;
    float2 a[NP][NCH], b[NP][NCH];
    if (have) {
      h = cur.h;
      rho = cur.rho;
      int64_t row;
      int c, w;
      cur.locate(p, row, w, c, out);
      const int nvalid = valid_lags(p, w);
      qlim = (nvalid - rho + sps - 1) >> lsps;
      if (SPLIT) {  // lags q = 2 q' + h: count the q' with 2 q' + h < qlim
        qlim = qlim > h ? (qlim - h + 1) >> 1 : 0;
        out = 2 * out + h;
      }
      const float2* G = p.G + row * (SPLIT ? 2 * H : H);
      const float2* D = SPLIT ? p.D3 + ((int64_t)c * 3 + (h ? 2 : 0)) * H : p.D + (int64_t)c * H;
      // step A: each pair's two NCH-point DFTs and the twiddles of the split.
      // a[i] first holds the code spectrum of column j (pair 0 of thread 0:
      // column 512, the mirror of its second column), read back reversed and
      // conjugated for column jb; b[i] takes its products one slot ahead (the
      // W_NCH shift)
#pragma unroll
      for (int i = 0; i < NP; ++i) {
        const int j = t + T * i;
        const bool p0 = (i == 0 && t == 0);
        const int jb = p0 ? 512 : 1024 - j;
        const int jd = p0 ? 512 : j;
#pragma unroll
        for (int m = 0; m < NCH; ++m) a[i][m] = D[jd + 1024 * m];
#pragma unroll
        for (int m = 0; m < NCH; ++m) b[i][(m + 1) % NCH] = cmul_conj(G[jb + 1024 * m], a[i][NCH - 1 - m]);
        if (p0) {
#pragma unroll
          for (int m = 0; m < NCH; ++m) a[i][m] = D[1024 * m];
        }
#pragma unroll
        for (int m = 0; m < NCH; ++m) a[i][m] = cmul(G[j + 1024 * m], a[i][m]);
        if (SPLIT) {  // + O B_h: the second table, read the same way
          const float2* O = G + H;
          const float2* B = p.D3 + ((int64_t)c * 3 + (h ? 0 : 1)) * H;
          float2 d[NCH];
#pragma unroll
          for (int m = 0; m < NCH; ++m) d[m] = B[jd + 1024 * m];
#pragma unroll
          for (int m = 0; m < NCH; ++m)
            b[i][(m + 1) % NCH] = cfma_conj(b[i][(m + 1) % NCH], O[jb + 1024 * m], d[NCH - 1 - m]);
          if (p0) {
#pragma unroll
            for (int m = 0; m < NCH; ++m) d[m] = B[1024 * m];
          }
#pragma unroll
          for (int m = 0; m < NCH; ++m) a[i][m] = cfma(a[i][m], O[j + 1024 * m], d[m]);
        }
        dft_reg<NCH, +1>(a[i]);
        dft_reg<NCH, +1>(b[i]);
        dif_twiddles<LOGM>(a[i], b[i], sm_tw, j, std::make_integer_sequence<int, NCH - 1>{});
        if (p0) dif_twiddle_col512<NCH>(b[i], std::make_integer_sequence<int, NCH - 1>{});
      }
    }
    __syncthreads();  // (1) the previous item's chunks are read and its partial results written
    if (prev_out >= 0 && warp == 0) {
      float4 r = lane < NCH ? red[(par ^ 1) * NCH + lane] : make_float4(0.f, -1.f, __int_as_float(0x7fffffff), 0.f);
      float sum = r.x, best = r.y;
      int bt = __float_as_int(r.z);
      warp_reduce_stats(sum, best, bt);
      if (lane == 0) p.part[prev_out] = make_float4(sum, best, __int_as_float(bt), 0.f);
    }
    if (!have) break;
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      const int j = t + T * i;
      const int jb = (i == 0 && t == 0) ? 512 : 1024 - j;
#pragma unroll
      for (int m = 0; m < NCH; ++m) {
        sm[m * kDifChunkPad + dif_pos(j)] = a[i][m];
        sm[m * kDifChunkPad + dif_pos(jb)] = b[i][m];
      }
    }
    __syncthreads();  // (2) every chunk is complete

    // step B: warp `warp` transforms chunk `warp` (1024 points) on its own
    float2* ch = sm + warp * kDifChunkPad;
    float2 x[32];
#pragma unroll
    for (int r = 0; r < 32; ++r) x[r] = ch[dif_pos(lane + 32 * r)];
    __syncwarp();
    dft_reg<32, +1>(x);
    // transpose: point 32 lane + r, as 16-byte pairs (r, r + 1)
    float4* row = reinterpret_cast<float4*>(ch + dif_pos(32 * lane));
#pragma unroll
    for (int r = 0; r < 32; r += 2) row[r / 2] = make_float4(x[r].x, x[r].y, x[r + 1].x, x[r + 1].y);
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
    // epilogue: lag tau = sps q + rho with q = warp + NCH (lane + 32 r), increasing in r
    constexpr int QS = 32 * NCH;  // q step per r
    float sum, best = -1.f;
    int bq = 0x7fffffff;
    const int q0 = warp + NCH * lane;
    auto argmax = [&](auto nr, bool all_valid) {
#pragma unroll
      for (int r = 0; r < decltype(nr)::value; ++r) {
        const float P = fmaf(x[r].x, x[r].x, x[r].y * x[r].y);
        if ((all_valid || q0 + QS * r < qlim) && P > best) {
          best = P;
          bq = q0 + QS * r;
        }
      }
    };
    if (half) {
      // hop <= N/2: every valid lag has r < 16.  The floor's sum over all
      // lags comes from the DFT's inputs (Parseval: sum |X_r|^2 = 32 sum |x_r|^2)
      // and only the outputs r < 16 are formed
      float e0 = 0.f, e1 = 0.f;
#pragma unroll
      for (int r = 0; r < 32; r += 2) {
        e0 = fmaf(x[r].x, x[r].x, fmaf(x[r].y, x[r].y, e0));
        e1 = fmaf(x[r + 1].x, x[r + 1].x, fmaf(x[r + 1].y, x[r + 1].y, e1));
      }
      sum = 32.f * (e0 + e1);
      dft_reg_low<32, +1>(x);
      if (q0 + QS * 15 < qlim) argmax(std::integral_constant<int, 16>{}, true);
      else argmax(std::integral_constant<int, 16>{}, false);
    } else {
      dft_reg<32, +1>(x);
      float s0 = 0.f, s1 = 0.f;
#pragma unroll
      for (int r = 0; r < 32; r += 2) {
        s0 += fmaf(x[r].x, x[r].x, x[r].y * x[r].y);
        s1 += fmaf(x[r + 1].x, x[r + 1].x, x[r + 1].y * x[r + 1].y);
      }
      sum = s0 + s1;
      if (q0 + QS * 31 < qlim) argmax(std::integral_constant<int, 32>{}, true);
      else argmax(std::integral_constant<int, 32>{}, false);
    }
    int bt = bq == 0x7fffffff ? bq : (SPLIT ? 2 * bq + h : bq) * sps + rho;
    warp_reduce_stats(sum, best, bt);
    if (lane == 0) red[par * NCH + warp] = make_float4(sum, best, __int_as_float(bt), 0.f);
    prev_out = out;
    par ^= 1;
    cur.advance(p, SPLIT, stride);
  }
}

template <int LOGH, int LOGE>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(fft_threads<LOGH, LOGE>())
    k_window_fft_split(WindowFftParams p) {
  using FFT = BlockFFT<LOGH, LOGE, -1>;
  constexpr int H = 1 << LOGH;
  extern __shared__ float4 smem_raw[];
  float2* sm = reinterpret_cast<float2*>(smem_raw);
  float2* sm_tw = sm + FFT::SMEM_ELEMS;
  load_tables<LOGH>(sm_tw, p.tw);
  __syncthreads();
  const int rho = blockIdx.x >> 1, h = blockIdx.x & 1;
  float2* row = p.G + (((int64_t)blockIdx.z * p.K + blockIdx.y) * p.sps + rho) * (2 * H);
  auto load = [&](int i) { return row[2 * i + h]; };
  auto emit = [&](int k, float2 v) { row[h * H + k] = v; };
  // both blocks of the cluster have read the whole row before either writes
  auto hook = [] { cooperative_groups::this_cluster().sync(); };
  FFT::run(sm, sm_tw, load, emit, hook);
}

template <int LOGH, int LOGE>
__global__ void __launch_bounds__(fft_threads<LOGH, LOGE>()) k_corr_split(CorrParams p) {
  using FFT = BlockFFT<LOGH, LOGE, +1>;
  constexpr int H = 1 << LOGH;
  extern __shared__ float4 smem_raw[];
  float2* sm = reinterpret_cast<float2*>(smem_raw);
  float2* sm_tw = sm + FFT::SMEM_ELEMS;
  float2* sm_tw2 = sm_tw + TwTables<LOGH>::N;
  float4* red = reinterpret_cast<float4*>(sm_tw2 + TwTables<LOGH + 1>::N);

  const int rho = blockIdx.x >> 1, h = blockIdx.x & 1, k = blockIdx.y;
  const int wl = blockIdx.z / p.Cg, c = blockIdx.z % p.Cg;
  const int sps = p.sps;
  load_tables<LOGH>(sm_tw, p.tw);
  load_tables<LOGH + 1>(sm_tw2, p.tw2);
  __syncthreads();
  const int nvalid = valid_lags(p, p.w0 + wl);

  const float2* E = p.G + (((int64_t)wl * p.K + k) * sps + rho) * (2 * H);
  const float2* O = E + H;
  const float2* D = p.D + (int64_t)c * (2 * H);
  // G[i] = E[i] + W^i O[i], G[i + H] = E[i] - W^i O[i]   (W = exp(-2 pi i / 2H));
  // h = 0: Z[i] + Z[i + H];  h = 1: (Z[i] - Z[i + H]) W^-i   (Z = G * D)
  auto load = [&](int i) {
    const float2 w = twiddle<LOGH + 1, -1>(sm_tw2, i);
    const float2 wo = cmul(w, O[i]);
    const float2 e = E[i];
    const float2 z0 = cmul(make_float2(e.x + wo.x, e.y + wo.y), D[i]);
    const float2 z1 = cmul(make_float2(e.x - wo.x, e.y - wo.y), D[i + H]);
    if (h == 0) return make_float2(z0.x + z1.x, z0.y + z1.y);
    return cmul(make_float2(z0.x - z1.x, z0.y - z1.y), make_float2(w.x, -w.y));
  };
  const int qlim = (nvalid - rho + sps - 1) / sps;
  float sum = 0.f, best = -1.f;
  int bq = 0x7fffffff;
  auto emit = [&](int kk, float2 v) {  // increasing kk, so increasing q
    const int q = 2 * kk + h;
    const float P = fmaf(v.x, v.x, v.y * v.y);
    sum += P;
    if (q < qlim && P > best) {
      best = P;
      bq = q;
    }
  };
  FFT::run(sm, sm_tw, load, emit);
  int bt = bq == 0x7fffffff ? bq : bq * sps + rho;
  block_reduce_stats(sum, best, bt, red);
  if (threadIdx.x == 0) {
    p.part[(((int64_t)wl * p.Cg + c) * p.K + k) * (2 * sps) + 2 * rho + h] =
        make_float4(sum, best, __int_as_float(bt), 0.f);
  }
}

// ---------------------------------------------------------------------------
// launchers for one tile shape
// ---------------------------------------------------------------------------

template <int LOGE>
struct FftLaunch {
  template <int LOGM>
  static cudaError_t prepare_one() {
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_window_fft<LOGM, LOGE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)fft_smem<LOGM>())) != cudaSuccess)
      return e;
    return cudaFuncSetAttribute(k_corr<LOGM, LOGE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)fft_smem<LOGM>());
  }

  template <int LOGH>
  static cudaError_t prepare_split() {
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_window_fft_split<LOGH, LOGE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)fft_smem<LOGH>())) != cudaSuccess)
      return e;
    return cudaFuncSetAttribute(k_corr_split<LOGH, LOGE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)fft_smem<LOGH>());
  }

  static cudaError_t prepare() {
    cudaError_t e;
    if (LOGE == 5) {
      void (*d12)(CorrParams) = k_corr_dif<12, false>;
      void (*d13)(CorrParams) = k_corr_dif<13, false>;
      void (*d14)(CorrParams) = k_corr_dif<14, false>;
      void (*d14s)(CorrParams) = k_corr_dif<14, true>;
      const cudaFuncAttribute attr = cudaFuncAttributeMaxDynamicSharedMemorySize;
      if ((e = cudaFuncSetAttribute(d12, attr, (int)dif_smem<12>())) != cudaSuccess ||
          (e = cudaFuncSetAttribute(d13, attr, (int)dif_smem<13>())) != cudaSuccess ||
          (e = cudaFuncSetAttribute(d14, attr, (int)dif_smem<14>())) != cudaSuccess ||
          (e = cudaFuncSetAttribute(d14s, attr, (int)dif_smem<14>())) != cudaSuccess)
        return e;
    }
    if ((e = prepare_one<10>()) != cudaSuccess) return e;
    if ((e = prepare_one<11>()) != cudaSuccess) return e;
    if ((e = prepare_one<12>()) != cudaSuccess) return e;
    if ((e = prepare_one<13>()) != cudaSuccess) return e;
    if ((e = prepare_one<14>()) != cudaSuccess) return e;
    if ((e = prepare_split<13>()) != cudaSuccess) return e;
    return prepare_split<14>();
  }

  // split: the transform of M = 2^logM points as two blocks of 2^(logM-1)
  // (required for 2^15, optional for 2^14)
  static cudaError_t window_fft(int logM, bool split, const WindowFftParams& p, cudaStream_t s) {
    dim3 grid(p.sps, p.K, p.nw);
    dim3 g2(2 * p.sps, p.K, p.nw);
    if (split) {
      switch (logM) {
        case 14: k_window_fft_split<13, LOGE><<<g2, fft_threads<13, LOGE>(), fft_smem<13>(), s>>>(p); break;
        case 15: k_window_fft_split<14, LOGE><<<g2, fft_threads<14, LOGE>(), fft_smem<14>(), s>>>(p); break;
        default: return cudaErrorInvalidValue;
      }
      return cudaGetLastError();
    }
    switch (logM) {
      case 10: return window_persistent<10>(p, s);
      case 11: return window_persistent<11>(p, s);
      case 12: return window_persistent<12>(p, s);
      case 13: return window_persistent<13>(p, s);
      case 14: return window_persistent<14>(p, s);
      default: return cudaErrorInvalidValue;
    }
  }

  template <class K>
  static cudaError_t resident_blocks(K kernel, int threads, size_t smem, int* out) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem);
    if (e == cudaSuccess) *out = std::max(1, sms * std::max(per_sm, 1));
    return e;
  }

  // k_window_fft with as many blocks as fit on the device at once (at most one per row)
  template <int LOGM>
  static cudaError_t window_persistent(const WindowFftParams& p, cudaStream_t s) {
    static int resident = 0;
    if (resident == 0) {
      const cudaError_t e = resident_blocks(k_window_fft<LOGM, LOGE>, fft_threads<LOGM, LOGE>(), fft_smem<LOGM>(),
                                            &resident);
      if (e != cudaSuccess) return e;
    }
    const int64_t rows = (int64_t)p.nw * p.K * p.sps;
    const unsigned blocks = (unsigned)std::min<int64_t>(rows, resident);
    k_window_fft<LOGM, LOGE><<<blocks, fft_threads<LOGM, LOGE>(), fft_smem<LOGM>(), s>>>(p);
    return cudaGetLastError();
  }

  static cudaError_t corr(int logM, bool split, const CorrParams& p, cudaStream_t s) {
    if (p.pairs && (split || logM > 14)) return cudaErrorInvalidValue;  // listed cells: single-block sizes
    dim3 grid(p.sps, p.pairs ? 1 : p.K, p.pairs ? p.n_pairs : p.nw * p.Cg);
    dim3 g2(2 * p.sps, p.K, p.nw * p.Cg);
    if (split && LOGE == 5 && logM == 15 && p.D3) return corr_dif<14, true>(p, s);
    if (split) {
      switch (logM) {
        case 14: k_corr_split<13, LOGE><<<g2, fft_threads<13, LOGE>(), fft_smem<13>(), s>>>(p); break;
        case 15: k_corr_split<14, LOGE><<<g2, fft_threads<14, LOGE>(), fft_smem<14>(), s>>>(p); break;
        default: return cudaErrorInvalidValue;
      }
      return cudaGetLastError();
    }
    if (LOGE == 5 && logM == 12) return corr_dif<12, false>(p, s);
    if (LOGE == 5 && logM == 13) return corr_dif<13, false>(p, s);
    if (LOGE == 5 && logM == 14) return corr_dif<14, false>(p, s);
    switch (logM) {
      case 10: return corr_persistent<10>(p, s);
      case 11: return corr_persistent<11>(p, s);
      case 12: return corr_persistent<12>(p, s);
      case 13: return corr_persistent<13>(p, s);
      case 14: return corr_persistent<14>(p, s);
      default: return cudaErrorInvalidValue;
    }
  }

  // k_corr_dif with as many blocks as fit on the device at once (at most one per item)
  template <int LOGM, bool SPLIT>
  static cudaError_t corr_dif(const CorrParams& p, cudaStream_t s) {
    static int resident = 0;
    if (resident == 0) {
      void (*kern)(CorrParams) = k_corr_dif<LOGM, SPLIT>;
      const cudaError_t e = resident_blocks(kern, dif_threads<LOGM>(), dif_smem<LOGM>(), &resident);
      if (e != cudaSuccess) return e;
    }
    const int64_t items = (SPLIT ? 2 : 1) *
                          (p.pairs ? (int64_t)p.n_pairs * p.sps : (int64_t)p.sps * p.K * p.nw * p.Cg);
    const unsigned blocks = (unsigned)std::min<int64_t>(items, resident);
    k_corr_dif<LOGM, SPLIT><<<blocks, dif_threads<LOGM>(), dif_smem<LOGM>(), s>>>(p);
    return cudaGetLastError();
  }

  // k_corr with as many blocks as fit on the device at once (at most one per cell)
  template <int LOGM>
  static cudaError_t corr_persistent(const CorrParams& p, cudaStream_t s) {
    static int resident = 0;  // blocks resident on the whole device (computed once per process)
    if (resident == 0) {
      const cudaError_t e = resident_blocks(k_corr<LOGM, LOGE>, fft_threads<LOGM, LOGE>(), fft_smem<LOGM>(),
                                            &resident);
      if (e != cudaSuccess) return e;
    }
    const int64_t items = p.pairs ? (int64_t)p.n_pairs * p.sps : (int64_t)p.sps * p.K * p.nw * p.Cg;
    const unsigned blocks = (unsigned)std::min<int64_t>(items, resident);
    k_corr<LOGM, LOGE><<<blocks, fft_threads<LOGM, LOGE>(), fft_smem<LOGM>(), s>>>(p);
    return cudaGetLastError();
  }
};

}  // namespace atlas
