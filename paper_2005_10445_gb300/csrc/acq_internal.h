// acq_internal.h -- parameter blocks shared by the host side of the library
// and its kernels (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "atlas_acq.h"

namespace atlas {

constexpr int kMinLogM = 10;
constexpr int kMaxLogM = 15;  // 2^15 via the split (two-block) transforms
constexpr int kMaxSps = 16;

// Device status word bits (the kernels OR these in; 0 = all checks passed).
enum : int {
  kStatusBadIndex = 1,
};

// Mix + box sum + decimation: one block per (tile of q, group of bins, window).
struct MixParams {
  const float2* x;          // stream [S]
  int64_t S;
  int N, M, sps, hop;       // window length, M = N / sps, samples/chip, hop
  int w0, nw;               // first window of the launch group, windows in it
  int K;
  const uint64_t* inc;      // [K] phase increment per sample, turns * 2^64 (two's complement)
  float2* B;                // out [nw][K][sps][M]: B_rho[q] = sum_s y[(sps q + rho + s) mod N]
  const int2* items = nullptr;  // optional (window, bin) list: then B is [n_items][sps][M]
  int n_items = 0;
};

// Window FFT: one block per (rho, k, window in the launch group), in place.
struct WindowFftParams {
  int M, sps, K, nw;
  const float2* tw;         // twiddle tables for log2(M)
  float2* G;                // in: B, out: FFT_M(B) [nw][K][sps][M]
};

// Per-code inverse FFT and epilogue: one block per (rho, k, window, code).
struct CorrParams {
  const float2* G;          // [nw][K][sps][M]
  const float2* D;          // [Cg][M] conj(FFT_M(chips)) / M
  // M = 2^15 only: per code the three half-length tables of the split
  // correlation, [Cg][3][M/2] = {D[i] + D[i + M/2], W^i (D[i] - D[i + M/2]),
  // W^-i (D[i] - D[i + M/2])}, W = exp(-2 pi i / M) (null: not built)
  const float2* D3 = nullptr;
  const float2* tw;         // twiddle tables of the block transform
  const float2* tw2 = nullptr;  // tables of the full size M (split transforms only)
  float4* part;             // out [nw][Cg][K][sps] (x2 for split) = {sum P, P*, tau*, 0}
  int64_t S;
  int N, M, sps, hop, W, L;
  int w0, nw, K, Cg;
  int* status;
  const int4* pairs = nullptr;  // optional list of (G row, code, window, -): then part is [n_pairs][sps]
  int n_pairs = 0;
};

// Per listed cell: combine the sps partial results into {score, P*, lag, floor}.
struct PairStatsParams {
  const float4* part;       // [n][sps]
  int n, sps, N;
  float4* out;              // [n] = {P* / floor, P*, lag (as int bits), floor}
};

// Bin selection, threshold and ordered compaction for one launch group.
struct SelectParams {
  const float4* part;       // [nw][Cg][K][sps]
  const int* codes;         // [Cg] global code ids of the group
  int Cg, C, K, sps, N, W, w0, nw;  // sps here: partial results per cell
  float threshold;
  atlas_detection* out;
  int capacity;
  int* count;               // running count (device)
  atlas_cell* cells;        // optional [Wmax][C][K]
  // optional workspace of [nw * Cg] per-pair results: with it the pairs are
  // evaluated by many blocks and then compacted in order by one (the same
  // records as the single-block selection)
  int* tmp_flags = nullptr;
  atlas_detection* tmp_recs = nullptr;
};

// FP64 direct recompute at a-1, a, a+1 and parabolic refinement.
struct RefineParams {
  const float2* x;
  int64_t S;
  const int8_t* chips;      // concatenated
  const int64_t* chip_off;  // [C]
  const int* chips_per_code;// [C]
  const int* hop;           // [C]
  const uint64_t* inc;      // [K]
  int sps;
  atlas_detection* out;
  int capacity;
  const int* count;
};

// Code bank: conj(FFT_M(chips zero padded)) / M per code of a group.
struct CodeBankParams {
  const int8_t* chips;
  const int64_t* chip_off;  // [Cg] offsets of the group's codes
  const int* n_chips;       // [Cg]
  const float2* tw;
  float2* D;                // [Cg][M]
  float2* D3 = nullptr;     // M = 2^15: [Cg][3][M/2] tables of the split correlation (see CorrParams)
  int M;
  float scale;              // 1 / M
};

cudaError_t launch_code_bank(int logM, const CodeBankParams& p, int n_codes, cudaStream_t s);
cudaError_t launch_mix(const MixParams& p, cudaStream_t s);
// loge: log2 of the complex values per thread of the transform kernels (4 or 5);
// split: the transform as two blocks of half the size (required for 2^15,
// available for 2^14)
cudaError_t launch_window_fft(int logM, int loge, bool split, const WindowFftParams& p, cudaStream_t s);
cudaError_t launch_corr(int logM, int loge, bool split, const CorrParams& p, cudaStream_t s);
cudaError_t prepare_fft_e4();
cudaError_t prepare_fft_e5();
cudaError_t launch_window_fft_e4(int logM, bool split, const WindowFftParams& p, cudaStream_t s);
cudaError_t launch_window_fft_e5(int logM, bool split, const WindowFftParams& p, cudaStream_t s);
cudaError_t launch_corr_e4(int logM, bool split, const CorrParams& p, cudaStream_t s);
cudaError_t launch_corr_e5(int logM, bool split, const CorrParams& p, cudaStream_t s);
cudaError_t launch_select(const SelectParams& p, cudaStream_t s);
int select_launches(const SelectParams& p);  // kernels launch_select starts for p
cudaError_t launch_pair_stats(const PairStatsParams& p, cudaStream_t s);
cudaError_t launch_refine(const RefineParams& p, int grid, cudaStream_t s);
cudaError_t prepare_kernels();  // raises the dynamic shared-memory limits once per process
// per-code correlation with the inverse transform on the tensor cores
// (precision 1: FP16 operands, 2: BF16; FP32 accumulation), M = 2^14 only:
// tcgen05.mma with TMEM accumulators (acq_tc5.cu)
cudaError_t launch_corr_tc5(int precision, const CorrParams& p, cudaStream_t s);
cudaError_t prepare_tc5();

}  // namespace atlas
