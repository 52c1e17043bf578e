// fsk_internal.h -- kernel parameters and launchers of the FSK front end
// (Section 3 steps 1-8 for frequency-shift keying; Section 4.1 for the
// FFT filters and cross-correlation).  Host code in atlas_fsk_host.cu.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "acq_internal.h"
#include "atlas_acq.h"
#include "atlas_fsk.h"

namespace atlas {

constexpr int kFskLogB = 12;          // demodulation block: 4096-point transforms
constexpr int kFskMaxTaps = 1024;     // composed filter taps T (<= B / 4)
constexpr int kFskMinLogN = 10;
constexpr int kFskMaxLogN = 18;
constexpr int kFskLogMBlock = 14;     // largest transform one block holds alone

// Points per block (log2) of a transform of 2^logN points: the whole transform
// up to 2^14; beyond, 2^13 (three blocks per SM) up to 2^17 and 2^14 (one
// block per SM) at 2^18.
constexpr int fsk_default_log_m(int logN) { return logN <= kFskLogMBlock ? logN : (logN <= 17 ? 13 : 14); }
// The (logN, logM) pairs with compiled kernels.  Plans of more than 16 blocks
// or of blocks of 2^14 points have the two-pass form only.
constexpr bool fsk_plan_supported(int logN, int logM) {
  return logN <= kFskLogMBlock ? logM == logN
                               : ((logM == 13 && logN <= 18) || (logM == 14 && (logN == 17 || logN == 18)));
}
constexpr bool fsk_plan_has_cluster_form(int logN, int logM) {
  return logN <= kFskLogMBlock || (logM == 13 && logN <= 17);
}
constexpr int kFskStatsSlices = 32;   // slices of the support per candidate in the peak sums

// Steps 1-5 over an index range of the stream (or of a replica): conversion,
// LO mix, both composed filters by overlap-save with B-point transforms,
// magnitudes, d and u.  Output index i in [start, start + count) is written to
// d[i - start], u[i - start]; i < 0 or i >= S_out gives 0.
struct FskDemodParams {
  const int16_t* iq = nullptr;  // int16 [S][2] input, or
  const float2* xf = nullptr;   // float2 [S] input (replicas)
  int64_t S;                    // input samples (reads outside [0, S) are 0)
  int64_t S_out;                // demodulated-stream length (outputs at or past it are 0)
  int64_t start, count;
  int T;                        // composed filter taps
  uint64_t lo_inc;              // LO phase per sample, turns * 2^64 (x * exp(-j 2 pi f_lo i / fs))
  int64_t lo_first = 0;         // absolute stream index of input sample 0 (the LO phase continues across calls)
  // Cyclic-buffer input (tracking tasks): when ring is set, input sample i is
  // ring[(*ring_start + i) mod ring_cap] and lo_first is *ring_start (both read on
  // the device, so a captured graph can be replayed for any block).
  const int16_t* ring = nullptr;
  int64_t ring_cap = 0;
  const int64_t* ring_start = nullptr;
  const float2* G1;             // [B] FFT_B(g_1 zero padded) / B
  const float2* G0;             // [B]
  const float2* tw;             // twiddle tables of B
  float* d;
  float* u;                     // may be null (not written)
};

// Replica of each code (step 6): r[n] = exp(+j 2 pi phase(n)), phase exact in
// turns * 2^64 from the number of earlier samples on each tone.
struct FskReplicaParams {
  const int8_t* chips;          // the codes' chips, concatenated
  const int64_t* chip_off;      // [n] offset of each code's chips
  const int64_t* ones_before;   // concatenated like chips: +1 chips before chip i of its code
  int n_chips, sps;
  uint64_t inc1, inc0;          // tone increments per sample
  float2* r;                    // out [n][L]
};

// Forward N-point transforms (N = R * M) into the permuted spectrum layout
// X[r * M + k2] = DFT_N(x)[R * k2 + r].  Items are window pairs (x = d_{w} +
// j d_{w+1}) or, in code mode, single rows (x = row, zero padded).
struct FskFwdParams {
  const float* d;               // window mode: demodulated stream held for indices [base, base + len)
  int64_t base, len;
  int hop, w0, nw;              // windows [w0, w0 + nw) of the launch group, in pairs
  const float* rows = nullptr;  // code mode: [n_items][ld] rows of n_valid values
  int ld = 0, n_valid = 0;
  int n_items;
  const float2* tw;             // tables of M
  const float2* twN;            // tables of N (R > 1)
  float2* X;                    // out [n_items][N]
  float scale;                  // applied to the output
  int conj_out;                 // 1: write conj(X) * scale
  // Two-pass form (R > 1): scratch of chunk_items items x N values between the
  // R-point and the M-point stages; null selects the cluster form.
  float2* scratch = nullptr;
  int chunk_items = 0;
};

// Per (window pair, code): Z = X * C, inverse N-point transform, corr^2,
// floor sum and argmax over the valid lags of both windows (real part: the
// pair's first window, imaginary part: its second).
struct FskCorrParams {
  const float2* X;              // [pairs][N]
  const float2* C;              // [Cg][N] conj(DFT_N(d_c)) / N, permuted like X
  const float2* tw;
  const float2* twN;
  float4* part;                 // out [nw][Cg][R] = {sum P, P*, lag (int bits), 0}
  int64_t S;
  int N, hop, W, n_c;
  int w0, nw, Cg;
  const int* sel = nullptr;     // optional [Cg] group-local indices of the searched codes
  // Two-pass form of the exchange (no cluster): scratch of chunk_items items
  // x N values that holds the blocks' twiddled inverse transforms between the
  // passes; null selects the cluster form.
  float2* scratch = nullptr;
  int chunk_items = 0;
};

// Per candidate of a launch group: the direct sums at the peak (FP32 within a
// warp's few terms per thread and its shuffle tree, FP64 beyond) and the
// parabolic arrival time (step 8); appends to the caller's list.
struct FskStatsParams {
  const atlas_detection* cand;  // group's candidates (k_select output)
  const int* n_cand;
  const float* d;               // demodulated stream held for [base, base + len)
  const float* u;
  int64_t base, len;
  const float* dc;              // [C][ld] the codes' d_c rows
  int ld, n_c, hop;
  int64_t S;
  atlas_fsk_detection* out;
  int capacity;
  int* count;                   // running count: read as the base index, advanced by k_fsk_advance
  double* part;                 // [max_cand][kFskStatsSlices][5] partial sums
};

cudaError_t fsk_prepare();      // raises the shared-memory limits of every FSK kernel
cudaError_t fsk_prepare_fft();  // (the transform kernels; called by fsk_prepare)
cudaError_t launch_fsk_demod(const FskDemodParams& p, cudaStream_t s);
int64_t fsk_demod_outputs_per_block(int T);
cudaError_t launch_fsk_replica(const FskReplicaParams& p, int n_codes, int L, cudaStream_t s);
// N = 2^logN points as 2^(logN - logM) blocks of 2^logM (fsk_plan_supported)
cudaError_t launch_fsk_fwd(int logN, int logM, const FskFwdParams& p, cudaStream_t s);
cudaError_t launch_fsk_corr(int logN, int logM, const FskCorrParams& p, cudaStream_t s);
// selection of a launch group (SelectParams with K = 1, sps = R partials per
// cell); *p.count receives the group's candidate count (not accumulated)
cudaError_t launch_fsk_select(const SelectParams& p, cudaStream_t s);
// the peak sums of up to max_cand candidates, then *p.count += *p.n_cand: in
// the final stage's single block when max_cand <= kFskStatsFinalOneBlock,
// else by a separate one-thread launch
constexpr int kFskStatsFinalOneBlock = 32;
cudaError_t launch_fsk_stats(const FskStatsParams& p, int max_cand, cudaStream_t s);

}  // namespace atlas
