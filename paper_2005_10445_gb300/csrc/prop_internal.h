// prop_internal.h -- state of a proposal network (not part of the public ABI).
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <string>

#include "atlas_acq.h"

namespace atlas {
namespace prop {

// offsets (in floats) of each parameter tensor in the flat parameter array
struct Layout {
  int C = 0, K = 0;
  size_t conv_w = 0, conv_b = 0, w1 = 0, b1 = 0, wc = 0, bc = 0, wb = 0, bb = 0, wp = 0, bp = 0, wl = 0, total = 0;
};

// length (floats) of one window's feature row: 4096 spectrum values, then K carrier-line values
int feature_len(int K);
Layout make_layout(int C, int K);

}  // namespace prop
}  // namespace atlas

struct atlas_prop {
  atlas::prop::Layout lay;
  float* params = nullptr;  // FP32 master weights
  __half* half = nullptr;   // FP16 copy used for inference
  float* grad = nullptr;
  float* m = nullptr;       // Adam moments
  float* v = nullptr;
  int64_t step = 0;
  // activations and their gradients for batches up to max_batch
  float *a1p = nullptr, *x1 = nullptr, *dx1 = nullptr, *hp = nullptr, *h = nullptr, *dh = nullptr;
  float *zc = nullptr, *zb = nullptr, *zp = nullptr, *dzc = nullptr, *dzb = nullptr, *dzp = nullptr, *loss = nullptr;
  int max_batch = 0;
  float2* tw = nullptr;     // 4096-point twiddle tables
  uint64_t* inc2 = nullptr; // [K] phase increment of 2 f_k per sample (turns * 2^64); null until a grid is set
  // proposal-search workspace (features, candidates, confidences for up to ws_windows windows)
  float* feat = nullptr;
  int* cand = nullptr;
  float* conf = nullptr;
  int ws_windows = 0;
  std::string last_error;
};
