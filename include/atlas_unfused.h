/*
 * atlas_unfused.h -- the comparison pipeline: the coherent search of
 * atlas_acq.h computed the way the paper's GPU implementation is organised
 * (Section 4.4: cuFFT plans plus separate element-wise kernels, every
 * intermediate in device memory).  Per launch group of windows:
 *
 *   mix kernel      y_{w,k}[m] = x[w hop + m] exp(-j 2 pi f_k m / fs)   -> HBM
 *   cuFFT           Y = FFT_N(y), batched over windows and bins        -> HBM
 *   multiply kernel Z_{w,c,k} = Y_{w,k} conj(C_c) / N for every code  -> HBM
 *   cuFFT           corr = IFFT_N(Z), batched, in place                -> HBM
 *   power kernel    P = |corr|^2, floor, argmax over the valid lags (reads the surface)
 *
 * then the same selection and FP64 refinement as the fused search, so both
 * produce the same detections.  It is a baseline for measurement only: the
 * fused search never calls it.  Codes of one length only.
 */
#ifndef ATLAS_UNFUSED_H_
#define ATLAS_UNFUSED_H_

#include <stdint.h>

#include "atlas_acq.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct atlas_unfused* atlas_unfused_t;

/*
 * chips, chips_per_code (all equal), n_codes, samples_per_chip, fs_hz,
 * freq_offsets_hz, n_freq: as atlas_acq_create.  fft_len: N (0 = 2 nextpow2(L)),
 * a power of two with N > L.  threshold: on P_max / floor.
 * windows_per_launch: windows per launch group, 0 = 16 (the surface of one
 * group, windows x codes x bins x N complex values, is held in device memory).
 * Builds the full N-point code spectra with cuFFT and plans the transforms.
 */
int atlas_unfused_create(atlas_unfused_t* out, const int8_t* chips, const int32_t* chips_per_code,
                         int32_t n_codes, int32_t samples_per_chip, double fs_hz, const double* freq_offsets_hz,
                         int32_t n_freq, int32_t fft_len, float threshold, int32_t windows_per_launch);

/* As atlas_acq_run (device stream of [n_samples][2] float32). */
int atlas_unfused_run(atlas_unfused_t ctx, void* stream, const float* d_iq, int64_t n_samples,
                      atlas_detection* d_out, int32_t capacity, int32_t* d_count);

const char* atlas_unfused_last_error(atlas_unfused_t ctx);
void atlas_unfused_destroy(atlas_unfused_t ctx);

#ifdef __cplusplus
}
#endif

#endif /* ATLAS_UNFUSED_H_ */
