/*
 * atlas_fsk.h -- C ABI of the FSK acquisition front end.
 *
 * The front end of Section 3 (steps 1-8, stated there for frequency-shift
 * keying) with the filter composition and cross-correlation identity of
 * Section 4.1.  For a stream of int16 (I, Q) pairs:
 *
 *   1. x[i] = I[i] + j Q[i]
 *   2. x[i] <- x[i] * exp(-j 2 pi f_lo i / fs)          (i: absolute sample index)
 *   3-4. f_b[i] = sum_{t<T} g_b[t] x[i-t], x[i<0] = 0, b in {1, 0}, with the
 *        composed filters g_b = h_bp * m_b (band-pass, then the matched filter
 *        of one chip of tone f_b: m_b[t] = exp(-j 2 pi f_b (sps-1-t) / fs))
 *   5. d = (|f_1| - |f_0|) / (|f_1| + |f_0|) (0 where both vanish), u = |f_1| - |f_0|;
 *      d and u have the stream's length (zero at and past its end)
 *   6. the same steps (no LO mix) on the replica of each code -- a
 *      continuous-phase FSK packet, chip +1 on tone f_1, chip -1 on tone f_0,
 *      phase 0 at its first sample -- give d_c, nonzero on n_c = L + T - 1
 *      samples (L = chips * sps)
 *   7. per overlapping window w (hop = N - n_c, window w covers samples
 *      [w hop, w hop + N)): corr[tau] = sum_{n<n_c} d_c[n] d[w hop + (tau+n) mod N]
 *   8. j = argmax over the window's valid lags of |corr| (smallest on ties);
 *      score = corr[j]^2 / mean_{tau<N} corr[tau]^2; a detection when
 *      score >= threshold, with w_c = sum d_c[n] d[a+n], q = sum d[a+n]^2,
 *      p_c = sum d_c[n] u[a+n] (n < n_c, a = w hop + j, direct sums) and
 *      the arrival time a + delta, delta the vertex of the parabola through
 *      corr^2 at a-1, a, a+1 (0 at the stream ends).
 *
 * Valid lags: [0, hop) in every window but the last, [0, min(hop, S - n_c -
 * w hop)] in the last, so every absolute lag 0 .. S - n_c is searched once.
 *
 * Threading, streams and errors as for atlas_acq.h (ATLAS_OK or a negative
 * ATLAS_ERR_* code; atlas_fsk_last_error() after ATLAS_ERR_CUDA).
 */
#ifndef ATLAS_FSK_H_
#define ATLAS_FSK_H_

#include <stdint.h>

#include "atlas_acq.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct atlas_fsk_ctx* atlas_fsk_t;

/* One FSK detection (48 bytes), written into caller-owned memory. */
typedef struct {
  int32_t code;    /* code index */
  int32_t window;  /* window index w; the window starts at sample w * hop_c */
  int32_t lag;     /* window-relative lag j; absolute lag a = window * hop_c + lag */
  float   score;   /* corr[j]^2 / floor (FP32 transform path) */
  double  toa;     /* a + delta, samples from the stream start */
  double  w_c;     /* sum_n d_c[n] d[a+n]  (direct sums of the FP32 d, u, d_c: FP32 within a warp,
                      at most 32 x 9 terms, FP64 beyond) */
  double  q;       /* sum_n d[a+n]^2 */
  double  p_c;     /* sum_n d_c[n] u[a+n] */
} atlas_fsk_detection;

typedef struct {
  float   threshold;          /* on corr[j]^2 / floor; default 49 */
  int32_t fft_len;            /* N for every code; 0 = 2 * nextpow2(L_c) per code */
  int32_t windows_per_launch; /* windows per launch group, rounded up to an even count; 0 = 128 */
  int32_t exchange;           /* transforms of more than 2^14 points: 0 = default (two passes
                                 through a device scratch of up to 1 GiB), 1 = one pass over a thread-block
                                 cluster exchanging through distributed shared memory, 2 = two
                                 passes; every form gives bit-identical results */
  int32_t block_log2;         /* transforms of more than 2^14 points: log2 of the points per block,
                                 0 = default (13 up to N = 2^17, 14 at 2^18), 13 or 14 (N = 2^17
                                 or 2^18 only); 32 blocks of 2^13 (N = 2^18) and blocks of 2^14 have
                                 the two-pass form only */
  int32_t reserved[3];
} atlas_fsk_opts;

void atlas_fsk_default_opts(atlas_fsk_opts* opts);

/*
 * Create an FSK search context on the current CUDA device.
 *   chips, chips_per_code, n_codes  as atlas_acq_create (host, +/-1 int8, copied)
 *   samples_per_chip  sps >= 1
 *   fs_hz             sample rate (> 0)
 *   f1_hz, f0_hz      tones of chips +1 and -1, relative to the band centre
 *   f_lo_hz           band centre relative to the receiver's centre (step 2)
 *   h_bp              host, [n_bp][2] double (re, im) band-pass taps (copied)
 *   n_bp              1 .. 1024 - sps + 1 (the composed filters have T = n_bp + sps - 1 taps)
 * Composes the filters in FP64 on the host, transforms them, builds every
 * code's replica, d_c and stored conjugated spectrum on the device (Section
 * 4.2: computed once and kept), allocates the workspaces and synchronises.
 * Supported: N a power of two, 2^10 .. 2^18, N > n_c; otherwise
 * ATLAS_ERR_UNSUPPORTED.  *out is released with atlas_fsk_destroy().
 */
int atlas_fsk_create(atlas_fsk_t* out, const int8_t* chips, const int32_t* chips_per_code, int32_t n_codes,
                     int32_t samples_per_chip, double fs_hz, double f1_hz, double f0_hz, double f_lo_hz,
                     const double* h_bp, int32_t n_bp, const atlas_fsk_opts* opts);

/* Plan of code `code` for n_samples (no device work): window count, hop,
 * transform length N and the support n_c of d_c. */
int atlas_fsk_windows(atlas_fsk_t ctx, int32_t code, int64_t n_samples, int32_t* n_windows, int32_t* hop,
                      int32_t* fft_len, int32_t* support);

/*
 * Run the search on a device-resident stream.
 *   stream     cudaStream_t (as void*); NULL = the legacy default stream
 *   d_iq       device, [n_samples][2] int16 (I, Q), caller-owned
 *   n_samples  S >= the largest support n_c
 *   d_out      device, [capacity] atlas_fsk_detection, caller-owned
 *   d_count    device, one int32: the number of detections (may exceed capacity;
 *              only the first `capacity` records are written)
 * Detections are ordered by (code length group, window, code).  Asynchronous
 * and stream-ordered; allocates nothing.  ATLAS_ERR_INVALID_ARG for bad
 * pointers or sizes or when the current CUDA device is not the context's.
 */
int atlas_fsk_run(atlas_fsk_t ctx, void* stream, const int16_t* d_iq, int64_t n_samples,
                  atlas_fsk_detection* d_out, int32_t capacity, int32_t* d_count);

/*
 * The search restricted to a subset of the codes, on a block of a longer
 * stream.
 *   first_sample  absolute index of d_iq[0] in the receiver's stream: the LO
 *                 phase of step 2 continues from it (windows, lags and ToAs
 *                 stay relative to d_iq)
 *   h_codes       host, n_sel distinct code indices (read before the call
 *                 returns); NULL searches every code; n_sel = 0 with a
 *                 non-NULL list searches nothing and writes *d_count = 0
 *   n_samples     >= the largest support n_c of the listed codes
 * Detections are ordered by (code length group, window, code).  Used for the
 * tracking tasks (one code, a block around a predicted arrival) and for the
 * searching queue of the scheduler (atlas_rt_*).
 */
int atlas_fsk_run_codes(atlas_fsk_t ctx, void* stream, const int16_t* d_iq, int64_t n_samples,
                        int64_t first_sample, const int32_t* h_codes, int32_t n_sel, atlas_fsk_detection* d_out,
                        int32_t capacity, int32_t* d_count);

/* The same with host buffers: copies h_iq in, searches, copies the records and
 * the count out, and synchronises.  Device staging buffers, a copy stream and
 * its events are made on first use and kept.  The input goes in four copies
 * on the copy stream and the demodulation of each part starts when its copy
 * is done, so the copy overlaps the computation; the records are those of
 * atlas_fsk_run on the same samples.  h_iq is read until the call returns. */
int atlas_fsk_run_host(atlas_fsk_t ctx, void* stream, const int16_t* h_iq, int64_t n_samples,
                       atlas_fsk_detection* h_out, int32_t capacity, int32_t* h_count);

/* Steps 1-5 alone: d and u of stream indices [start, start + count) into the
 * device arrays d_d and d_u (caller-owned, `count` floats each; d_u may be
 * NULL).  For inspection and testing. */
int atlas_fsk_demod(atlas_fsk_t ctx, void* stream, const int16_t* d_iq, int64_t n_samples, int64_t start,
                    int64_t count, float* d_d, float* d_u);

/* Copy code `code`'s stored d_c (n_c floats) to host memory h_dc of `cap`
 * floats; *n gets n_c. */
int atlas_fsk_code_demod(atlas_fsk_t ctx, int32_t code, float* h_dc, int32_t cap, int32_t* n);

/*
 * Tracking task as a single launch.  A tracker replays one CUDA graph, captured
 * at creation, that searches one code on a block of n_samples samples taken
 * straight out of a cyclic buffer of int16 (I, Q) pairs: absolute sample i is
 * d_ring[i mod ring_samples].  The block's start, and with it the LO phase of
 * step 2, and the code are written into a 16-byte device descriptor by the
 * graph's first node.  A tracker serves the codes whose length equals `code`'s.
 *   d_ring        device, caller-owned, must outlive the tracker
 *   n_samples     block length, >= the codes' support n_c
 * atlas_fsk_tracker_run is synchronous: one graph launch on `stream`, one
 * synchronisation; h_out (host, capacity records) receives the detections
 * (windows, lags and ToAs relative to block_start), *h_count their number.
 * The tracker uses the context's workspaces: it and the context's other calls
 * must be ordered on one stream.
 */
typedef struct atlas_fsk_tracker* atlas_fsk_tracker_t;
int atlas_fsk_tracker_create(atlas_fsk_tracker_t* out, atlas_fsk_t ctx, int32_t code, int64_t n_samples,
                             const int16_t* d_ring, int64_t ring_samples);
int atlas_fsk_tracker_run(atlas_fsk_tracker_t t, void* stream, int32_t code, int64_t block_start,
                          atlas_fsk_detection* h_out, int32_t capacity, int32_t* h_count);
/* Kernel launches one atlas_fsk_tracker_run makes (the kernel nodes of its
 * graph); -1 for a null tracker. */
int32_t atlas_fsk_tracker_kernels(atlas_fsk_tracker_t t);
void atlas_fsk_tracker_destroy(atlas_fsk_tracker_t t);

/* Device-time profile of the runs between begin and end: CUDA events on the
 * run's stream around the demodulation and correlation launches (at most
 * max_timed of each kind are timed; the counts cover every launch). */
typedef struct {
  int64_t launches;        /* kernels the profiled runs launched */
  int64_t corr_launches;   /* correlation launches (inverse transform, corr^2, floor, argmax) */
  int64_t corr_units;      /* (window, code) cells they processed */
  int64_t corr_timed;
  double  corr_ms;         /* summed device time of the timed correlation launches */
  int64_t demod_launches;  /* demodulation launches (steps 1-5) */
  int64_t demod_samples;   /* samples they demodulated */
  int64_t demod_timed;
  double  demod_ms;        /* summed device time of the timed demodulation launches */
} atlas_fsk_profile;

int atlas_fsk_profile_begin(atlas_fsk_t ctx, int32_t max_timed);
int atlas_fsk_profile_end(atlas_fsk_t ctx, atlas_fsk_profile* out);

const char* atlas_fsk_last_error(atlas_fsk_t ctx);
void atlas_fsk_destroy(atlas_fsk_t ctx);

#ifdef __cplusplus
}
#endif

#endif /* ATLAS_FSK_H_ */
