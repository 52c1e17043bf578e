/*
 * atlas_acq.h -- C ABI of the GB300 acquisition-mode time-of-arrival search.
 *
 * The search (Rubinpur & Toledo, "Signal Processing for a Reverse-GPS Wildlife
 * Tracking System", arXiv 2005.10445) detects which tag codes appear in a
 * block of complex baseband samples and estimates a sub-sample time of
 * arrival for each (Section 2, problem statement; Section 3, steps 1-8).
 * This library runs the coherent form of that search over every code and a
 * grid of carrier-frequency offsets:
 *
 *   for every overlapping window w (Section 2.1: blocks overlap so that each
 *   transmission lies entirely in one block; here hop = N - L), every code c
 *   and every frequency bin k:
 *     y[m]      = x[w*hop + m] * exp(-j 2 pi f_k m / fs)        (Section 3 step 2,
 *                                                                one LO mix per bin)
 *     corr[tau] = sum_{n<L} y[(tau+n) mod N] * r_c[n]           (step 7; computed with
 *                                                                FFTs, Section 4.1)
 *     P = |corr|^2, floor = mean_{tau<N} P, (P*, tau*) = argmax over the window's
 *     valid lags (smallest lag on ties)                          (step 8)
 *   per (w, c): the bin with the largest score P_max / floor (smallest bin on
 *   ties) is a detection when score >= threshold; its peak is then refined
 *   ("interpolated", step 8) by recomputing |corr|^2 directly in FP64 at the
 *   absolute lags a-1, a, a+1 and taking the vertex of the parabola.
 *
 * r_c[n] = chip_c[n / sps] for n < L = chips_c * sps (the replica, step 6).
 * Samples are interleaved float32 (re, im) pairs ("complex64").
 *
 * Threading: a context may be used from one host thread at a time.  All
 * device work is stream-ordered on the stream the caller passes.
 * Errors: every call returns ATLAS_OK (0) or a negative ATLAS_ERR_* code;
 * atlas_acq_strerror() gives a message.  After ATLAS_ERR_CUDA the CUDA error
 * string is available from atlas_acq_last_error().
 */
#ifndef ATLAS_ACQ_H_
#define ATLAS_ACQ_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  ATLAS_OK = 0,
  ATLAS_ERR_INVALID_ARG = -1,  /* null pointer, non-positive count, stream shorter than a code ... */
  ATLAS_ERR_CUDA = -2,         /* a CUDA runtime call failed; see atlas_acq_last_error() */
  ATLAS_ERR_NO_MEMORY = -3,    /* device or host allocation failed (create time only) */
  ATLAS_ERR_UNSUPPORTED = -4,  /* a size outside what the kernels support (see atlas_acq_create) */
  ATLAS_ERR_TIMEOUT = -5,      /* reserved for a bounded device-side wait that gives up; no kernel of
                                  this library waits on another block, stream or device, so no call
                                  returns it at present */
  ATLAS_ERR_DEVICE = -6        /* a kernel reported an internal check failure (device status word) */
};

typedef struct atlas_acq_ctx* atlas_acq_t;

/* One detection (32 bytes).  Written by the library into caller-owned memory. */
typedef struct {
  int32_t code;       /* code index, 0 .. n_codes-1 */
  int32_t window;     /* window index w; the window starts at sample w*hop_c */
  int32_t lag;        /* window-relative lag tau*; absolute lag a = window*hop_c + lag */
  int32_t freq_bin;   /* index k into the frequency grid */
  float   score;      /* P_max / floor of the chosen (w, c, k) cell (FP32 FFT path) */
  float   peak_power; /* |corr|^2 at absolute lag a, recomputed directly in FP64 */
  double  toa;        /* a + delta, samples from the stream start (FP64) */
} atlas_detection;

/* Per-cell statistics (16 bytes), for inspection and testing. */
typedef struct {
  float   p_max;      /* P* over the window's valid lags */
  float   floor;      /* mean of P over all N circular lags */
  int32_t lag;        /* tau* (smallest on ties) */
  int32_t valid;      /* 1 if this (w, c) window exists for the code, else 0 */
} atlas_cell;

typedef struct {
  float   threshold;       /* detection threshold on P_max / floor; default 25 */
  int32_t fft_len;         /* N for every code; 0 = 2 * nextpow2(L_c) per code */
  int32_t windows_per_launch; /* windows processed per launch group; 0 = automatic */
  int32_t tile_log2;       /* complex values per thread of the transform kernels: 4 -> 16, 5 -> 32;
                              0 = default (32) or the autotuned choice */
  int32_t split;           /* 1: run transforms of N/sps = 2^14 as two blocks of 2^13 (always done
                              for 2^15); 0 = default */
  int32_t precision;       /* 0: FP32 (default); 1 / 2: the per-code inverse transforms of codes with
                              N/sps = 2^14 as tensor-core (tcgen05) contractions, DFT stages of
                              16, 32 and 32 points, with FP16 / BF16 operands, FP32 accumulation
                              and per-stage power-of-two scaling
                              (other sizes stay FP32); window transforms and the refinement are
                              unchanged */
  int32_t reserved[2];
} atlas_acq_opts;

/* Fill *opts with the defaults. */
void atlas_acq_default_opts(atlas_acq_opts* opts);

/*
 * Create a search context on the current CUDA device.
 *   chips           host, n_codes concatenated +/-1 int8 chip sequences (copied)
 *   chips_per_code  host, [n_codes] chip counts (each >= 1)
 *   samples_per_chip  sps: a power of two, 1 .. 16
 *   fs_hz           sample rate (> 0)
 *   freq_offsets_hz host, [n_freq] carrier offsets f_k in Hz (copied)
 *   opts            NULL for defaults
 * Builds the stored, conjugated code spectra on the device (Section 4.2: the
 * transformed replicas are computed once and kept), allocates every
 * workspace the searches need (Section 4.2: preallocated, size-keyed arrays
 * that are reused), and synchronises the device before returning.
 * Supported sizes: N a power of two with N > L_c, N/sps between 2^10 and
 * 2^15; otherwise ATLAS_ERR_UNSUPPORTED.  Ownership: *out is owned by the
 * caller and released with atlas_acq_destroy().
 */
int atlas_acq_create(atlas_acq_t* out, const int8_t* chips, const int32_t* chips_per_code,
                     int32_t n_codes, int32_t samples_per_chip, double fs_hz,
                     const double* freq_offsets_hz, int32_t n_freq, const atlas_acq_opts* opts);

/* Window plan of code `code` for a stream of n_samples (pure query, no device
 * work): W = max(1, ceil((S - N) / hop) + 1), hop = N - L (Section 2.1). */
int atlas_acq_windows(atlas_acq_t ctx, int32_t code, int64_t n_samples, int32_t* n_windows,
                      int32_t* hop, int32_t* fft_len);

/*
 * Run the search on a device-resident stream.
 *   stream     cudaStream_t (as void*); NULL = the legacy default stream
 *   d_iq       device, [n_samples][2] float32 interleaved (re, im), caller-owned
 *   n_samples  S >= the longest code length L
 *   d_out      device, [capacity] atlas_detection, caller-owned
 *   capacity   >= 0
 *   d_count    device, one int32: receives the number of detections found
 *              (may exceed capacity; only the first `capacity` are written)
 * Detections are ordered by (code length group, window, code) -- by (window,
 * code) when all codes have the same length -- so repeated runs are
 * bit-identical.  Asynchronous: results are valid after the caller
 * synchronises `stream`.  Allocates nothing.  Returns ATLAS_ERR_INVALID_ARG
 * for bad pointers or sizes or when the current CUDA device is not the one the
 * context was created on, ATLAS_ERR_CUDA if a launch fails.
 */
int atlas_acq_run(atlas_acq_t ctx, void* stream, const float* d_iq, int64_t n_samples,
                  atlas_detection* d_out, int32_t capacity, int32_t* d_count);

/*
 * Same search with per-cell statistics: d_cells (device, caller-owned) gets
 * [max_windows][n_codes][n_freq] atlas_cell, where max_windows is the largest
 * W over the codes (atlas_acq_windows); cells of windows a code does not have
 * are written with valid = 0.  d_out/d_count behave as in atlas_acq_run.
 */
int atlas_acq_run_cells(atlas_acq_t ctx, void* stream, const float* d_iq, int64_t n_samples,
                        atlas_cell* d_cells, atlas_detection* d_out, int32_t capacity,
                        int32_t* d_count);

/*
 * End-to-end form on HOST buffers: copies h_iq to the device, runs the search
 * and copies the count and the first min(count, capacity) detections back,
 * then synchronises `stream`.  The samples past the first launch group are
 * copied on a stream of the context's own, overlapping that group's work
 * (ordered after the caller's earlier work on `stream`).  h_iq, h_out and h_count are host memory (pinned
 * memory makes the copies asynchronous DMA).  The device staging buffer for
 * the samples is allocated on first use for a given size and kept by the
 * context (Section 4.2 memoization); *h_count receives the full count.
 */
int atlas_acq_run_host(atlas_acq_t ctx, void* stream, const float* h_iq, int64_t n_samples,
                       atlas_detection* h_out, int32_t capacity, int32_t* h_count);

/*
 * Autotune the transform tile shape (16 or 32 complex values per thread), the
 * split of 2^14-point transforms into two blocks, and the windows per launch
 * group of every code-length group of the context, by
 * timing each candidate on the caller's stream over the given device samples
 * (Section 4.2 plans FFTs for fixed sizes; this plans our own kernels).  With
 * cache_path (a JSON-lines file, one object per tuned shape keyed by GPU name,
 * N, M, samples/chip, bins and codes) cached choices are applied without
 * timing and new ones appended; NULL = no cache.  Allocates a few temporary
 * buffers; synchronises the stream.  Results of later runs do not depend on
 * the choice beyond FP32 rounding.
 */
int atlas_acq_autotune(atlas_acq_t ctx, void* stream, const float* d_iq, int64_t n_samples,
                       const char* cache_path);

/* The tile shape (log2 of values per thread), windows per launch group and
 * split flag (two-block transforms) in use for the group of code `code`. */
int atlas_acq_tuning(atlas_acq_t ctx, int32_t code, int32_t* tile_log2, int32_t* windows_per_launch,
                     int32_t* split);

/*
 * Batched search over many receiver streams (Section 4.3 batches many
 * correlations per call).  Each stream i has its own context ctxs[i] (codes,
 * samples/chip, sample rate, frequency grid; contexts must be distinct because
 * each owns its workspace) and its own device samples d_iq[i] of n_samples[i].
 * The whole batch -- every stream's launch sequence on its own branch -- is
 * captured once into a CUDA graph bound to these buffers (Section 4.2: plans
 * refer to fixed arrays); atlas_acq_batch_run launches that graph.
 *   d_out    device, [n_streams][capacity] atlas_detection, caller-owned
 *   d_count  device, [n_streams] int32, caller-owned; count of stream i
 * The contexts' tuning (atlas_acq_autotune) is frozen into the graph at
 * creation.  A context must not run other searches while a graph that uses it
 * executes.  Results equal those of atlas_acq_run on each stream.
 */
typedef struct atlas_acq_batch* atlas_acq_batch_t;
int atlas_acq_batch_create(atlas_acq_batch_t* out, const atlas_acq_t* ctxs, int32_t n_streams,
                           const float* const* d_iq, const int64_t* n_samples, atlas_detection* d_out,
                           int32_t capacity, int32_t* d_count);

/* Launch the batch's graph on `stream` (asynchronous). */
int atlas_acq_batch_run(atlas_acq_batch_t batch, void* stream);

/* Number of kernel launches in one run of the batch's graph. */
int64_t atlas_acq_batch_kernels(atlas_acq_batch_t batch);

/* Release the graph, its streams and events.  NULL is a no-op. */
void atlas_acq_batch_destroy(atlas_acq_batch_t batch);

/* ------------------------------------------------------------------------
 * Learned (code, bin) proposal.  The paper has no learned component; the
 * proposal prunes its exhaustive search (every code correlated in every
 * block, Sections 2.1 and 3): a small network looks at a window's Welch power
 * spectrum (segments of 4096 samples, Hann taper, log10, mean removed) and
 * ranks (code, bin) candidates; only the top-k are correlated, and windows
 * where it is not confident fall back to the exhaustive search, which also
 * labels the training data.
 * Features per window: one row of 4096 + n_bins floats -- the Welch spectrum,
 * then n_bins carrier-line values: for +/-1 chips the squared transmission is a
 * pure tone at twice the carrier offset, so L[k] = log10(|DFT of x^2 at 2 f_k|^2
 * / sum |x|^4 + 1) shows the bin of a tag (about 0.3 for noise).
 * Network: conv1d (8 channels, kernel 16, stride 8) + ReLU on the spectrum,
 * dense 4096 -> 48 + ReLU, heads: code logits [n_codes], bin logits [n_bins]
 * (+ a L[k]), presence logit (+ c max_k L[k]).
 * Parameters: one FP32 array in the order conv_w [8][16], conv_b [8],
 * w1 [4096][48], b1 [48], wc [48][n_codes], bc [n_codes], wb [48][n_bins],
 * bb [n_bins], wp [48], bp [1], wl [2] = (a, c); inference uses an FP16 copy
 * (FP32 accumulate).
 * ------------------------------------------------------------------------ */
typedef struct atlas_prop* atlas_prop_t;

/* Create a network with seeded He-uniform weights, zero biases and the
 * carrier-line weights (a, c) = (4, 1) (1 <= n_codes, n_bins <= 256). */
int atlas_prop_create(atlas_prop_t* out, int32_t n_codes, int32_t n_bins, uint64_t seed);
int64_t atlas_prop_num_params(atlas_prop_t p);
/* Copy the FP32 parameters out to / in from host memory (set resets Adam). */
int atlas_prop_get_params(atlas_prop_t p, float* h_params);
int atlas_prop_set_params(atlas_prop_t p, const float* h_params);

/* Checkpoint: the FP32 parameters, the Adam moments and the step count in one
 * file (little-endian): a 40-byte header -- magic "ATLPROP1", uint32 version 2,
 * int32 n_codes, int32 n_bins, uint32 CRC-32 (IEEE 802.3) of the payload,
 * int64 n_params, int64 step -- then params, m, v as float32 [n_params] each.
 * Load checks the magic, version, shapes, length and CRC and returns
 * ATLAS_ERR_INVALID_ARG on any mismatch, leaving the network unchanged;
 * training resumes exactly where the saved run stood.  Synchronous. */
int atlas_prop_save(atlas_prop_t p, const char* path);
int atlas_prop_load(atlas_prop_t p, const char* path);

/* Frequency grid of the carrier-line features: fs_hz and the n_freq (= n_bins)
 * offsets, read during the call (host).  Until it is set the line features are 0. */
int atlas_prop_set_grid(atlas_prop_t p, double fs_hz, const double* freq_offsets_hz, int32_t n_freq);
/* Floats in one window's feature row: 4096 + n_bins. */
int32_t atlas_prop_feature_len(atlas_prop_t p);

/* Features of n_windows windows of window_len samples (a multiple of 4096) starting at
 * first_sample + w * stride of the device stream d_iq [n_samples][2]; samples outside
 * the stream read as zero; the carrier-line phase is window-relative.
 * d_feat: device [n_windows][atlas_prop_feature_len(p)]. */
int atlas_prop_features(atlas_prop_t p, void* stream, const float* d_iq, int64_t n_samples, int64_t first_sample,
                        int64_t stride, int32_t window_len, int32_t n_windows, float* d_feat);

/* Mean loss over the batch into *d_loss (device float) and the gradient of every
 * parameter into d_grad (device, [num_params]; NULL = the network's own buffer).
 * d_code / d_bin: device [batch] labels, code < 0 for a window without a detection. */
int atlas_prop_loss_grad(atlas_prop_t p, void* stream, const float* d_feat, const int32_t* d_code,
                         const int32_t* d_bin, int32_t batch, float* d_loss, float* d_grad);

/* One Adam step (beta 0.9 / 0.999, eps 1e-8, bias-corrected) with the given gradient
 * (NULL = the network's own buffer); refreshes the FP16 copy. */
int atlas_prop_adam(atlas_prop_t p, void* stream, const float* d_grad, float lr);

/* Logits of a batch (any pointer may be NULL): FP16 weights when half_weights != 0. */
int atlas_prop_logits(atlas_prop_t p, void* stream, const float* d_feat, int32_t batch, int32_t half_weights,
                      float* d_zc, float* d_zb, float* d_zp);

/* Top-k (code, bin) candidates per window by log p(code) + log p(bin) (ties to the
 * smaller code*n_bins + bin), FP16 weights.  d_cand: [n_windows][topk][2] int32
 * (code, bin); d_conf: [n_windows][2] = {probability of the top pair, presence
 * probability}.  1 <= topk <= 32. */
int atlas_prop_candidates(atlas_prop_t p, void* stream, const float* d_feat, int32_t n_windows, int32_t topk,
                          int32_t* d_cand, float* d_conf);

/* Top n_top bins per window by the bin head (ties to the smaller bin), FP16
 * weights: d_bins [n_windows][n_top] int32; d_conf [n_windows][2] = {probability
 * mass of the chosen bins, presence probability}.  1 <= n_top <= min(32, n_bins). */
int atlas_prop_bin_candidates(atlas_prop_t p, void* stream, const float* d_feat, int32_t n_windows, int32_t n_top,
                              int32_t* d_bins, float* d_conf);

/*
 * Search with the proposal: features and candidates for every window of the
 * context's single code length; each window where the network is confident --
 * max(probability of its top pair, 1 - presence probability) >= tau_fb -- is
 * searched only over its top-k (code, bin) candidates (per code, the best of
 * its candidate bins), every other window by the exhaustive search.
 * Output as atlas_acq_run (ordered by window, then code; refined ToA).
 * h_n_fallback (host, may be NULL) receives the number of exhaustive windows.
 * Synchronous: it reads the candidates on the host to build the work lists, and
 * grows its workspaces on first use for a given number of windows.  tau_fb = 0
 * never falls back; tau_fb > 1 always does (the exhaustive search).
 */
int atlas_acq_run_proposed(atlas_acq_t ctx, atlas_prop_t prop, void* stream, const float* d_iq,
                           int64_t n_samples, int32_t topk, float tau_fb, atlas_detection* d_out, int32_t capacity,
                           int32_t* d_count, int32_t* h_n_fallback);

/*
 * The same search with bin proposals: a confident window -- probability mass of
 * its top n_top bins >= tau_fb -- is searched over every code in its top n_top
 * bins only (n_top of the context's bins, 1 <= n_top <= 32); every other window
 * by the exhaustive search.  The presence head does not skip windows here: a
 * weak tag and an empty window have the same features.  The proposal's
 * carrier-line grid is set from the context.  Otherwise as
 * atlas_acq_run_proposed.
 */
int atlas_acq_run_proposed_bins(atlas_acq_t ctx, atlas_prop_t prop, void* stream, const float* d_iq,
                                int64_t n_samples, int32_t n_top, float tau_fb, atlas_detection* d_out,
                                int32_t capacity, int32_t* d_count, int32_t* h_n_fallback);

const char* atlas_prop_last_error(atlas_prop_t p);
void atlas_prop_destroy(atlas_prop_t p);

/* Kernel timing collected by the library between atlas_acq_profile_begin and
 * atlas_acq_profile_end. */
typedef struct {
  int64_t launches;       /* kernels of this library launched while profiling */
  int64_t corr_launches;  /* launches of the per-code correlation kernel (the dominant one) */
  double  corr_ms;        /* summed device time of those launches (CUDA events on the run's stream) */
  int64_t corr_units;     /* (window, code, bin) cells those launches processed */
  int64_t timed_launches; /* correlation launches that had an event pair (<= the pool size) */
} atlas_acq_profile;

/*
 * Start collecting kernel timing: allocates a pool of max_timed CUDA event
 * pairs (so call it outside any timed region) and resets the counters.
 * While active, every run records an event pair around each launch of the
 * correlation kernel on the run's stream; launches past the pool size are
 * counted but not timed.
 */
int atlas_acq_profile_begin(atlas_acq_t ctx, int32_t max_timed);

/* Synchronise the device, sum the recorded times into *out, free the events
 * and stop collecting. */
int atlas_acq_profile_end(atlas_acq_t ctx, atlas_acq_profile* out);

/*
 * Search for one code without a context and without allocating device
 * memory.  The paper has no counterpart: it exists for callers that cannot
 * call cudaMalloc when they need a search -- code under a framework whose
 * caching allocator owns device memory and forbids raw allocations, plug-ins
 * that must not grow the process's footprint, or a real-time loop that cannot
 * afford an allocation's implicit synchronisation.
 *   stream, d_iq, n_samples, d_out, capacity, d_count  as in atlas_acq_run
 *   d_chips        device, [n_chips] +/-1 int8 chips of the one code (caller-owned).
 *                  They are not checked (they are device memory): other values
 *                  give scores that do not match atlas_acq_run.
 *   samples_per_chip, fs_hz  as in atlas_acq_create
 *   freq_offsets_hz  host, [n_freq] carrier offsets in Hz (read during the call)
 *   fft_len        N; 0 = 2 * nextpow2(n_chips * samples_per_chip)
 *   threshold      detection threshold on P_max / floor
 * All intermediate arrays live in one static device array of 4,342,016 bytes
 * (about 4.14 MiB).  A GPU holds it from the time the library's device code
 * is loaded there (with CUDA's lazy module loading, the first call on that
 * device) until the process exits.  Limits: N <= 16384, n_freq <= 32,
 * samples_per_chip a power of two <= 16, N / samples_per_chip >= 1024; beyond
 * them the call returns ATLAS_ERR_UNSUPPORTED and does no device work.  A
 * stream longer than atlas_acq_run accepts (8 * INT32_MAX samples) returns
 * ATLAS_ERR_INVALID_ARG.  The first call on a device looks up the array's
 * device address (and sets kernel attributes); make that first call before
 * any stream capture.  Every call reuses the same array and rewrites what it
 * reads; calls whose device work may overlap (other host threads, or streams
 * not ordered with this one) race on it.  The records equal atlas_acq_run's
 * for the same code bit for bit; the call is asynchronous on `stream`.
 */
int atlas_acq_run_static(void* stream, const float* d_iq, int64_t n_samples, const int8_t* d_chips,
                         int32_t n_chips, int32_t samples_per_chip, double fs_hz,
                         const double* freq_offsets_hz, int32_t n_freq, int32_t fft_len, float threshold,
                         atlas_detection* d_out, int32_t capacity, int32_t* d_count);

/* Device status word of the last run (0 = no kernel-side check failed).
 * Synchronises the device. */
int atlas_acq_last_device_status(atlas_acq_t ctx);

/* Text of the last CUDA error seen by this context ("" if none). */
const char* atlas_acq_last_error(atlas_acq_t ctx);

/* Release every device and host resource of the context.  NULL is a no-op. */
void atlas_acq_destroy(atlas_acq_t ctx);

/* Static message for a status code. */
const char* atlas_acq_strerror(int status);

#ifdef __cplusplus
}
#endif

#endif /* ATLAS_ACQ_H_ */
