// acq_common.cuh -- device helpers shared by the search kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "acq_internal.h"
#include "fft_block.cuh"

namespace atlas {

constexpr int kLogE = 5;  // 32 complex values per thread

// phase (turns * 2^64) -> exp(-2 pi i turns) in FP32.  The top 32 bits give the
// angle as a fraction of a half turn in [-1, 1).
__device__ __forceinline__ float2 expi_neg(uint64_t ph) {
  const float h = (float)(int32_t)(ph >> 32) * 4.656612873077392578125e-10f;  // 2^-31
  float s, c;
  sincospif(h, &s, &c);
  return make_float2(c, -s);
}

template <int LOGM>
__device__ __forceinline__ void load_tables(float2* sm_tw, const float2* tw) {
  for (int i = threadIdx.x; i < TwTables<LOGM>::N; i += blockDim.x) sm_tw[i] = tw[i];
}

// Block-wide deterministic reduction of (sum, max, argmax) with the smallest
// lag on ties.  Result valid in thread 0.
__device__ __forceinline__ void better(float& best, int& bt, float p, int t) {
  if (p > best || (p == best && t < bt)) {
    best = p;
    bt = t;
  }
}

__device__ __forceinline__ void block_reduce_stats(float& sum, float& best, int& bt, float4* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float s2 = __shfl_down_sync(0xffffffffu, sum, o);
    const float b2 = __shfl_down_sync(0xffffffffu, best, o);
    const int t2 = __shfl_down_sync(0xffffffffu, bt, o);
    sum += s2;
    better(best, bt, b2, t2);
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) red[warp] = make_float4(sum, best, __int_as_float(bt), 0.f);
  __syncthreads();
  if (warp == 0) {
    const int nw = blockDim.x >> 5;
    float4 r = lane < nw ? red[lane] : make_float4(0.f, -1.f, __int_as_float(0x7fffffff), 0.f);
    sum = r.x;
    best = r.y;
    bt = __float_as_int(r.z);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float s2 = __shfl_down_sync(0xffffffffu, sum, o);
      const float b2 = __shfl_down_sync(0xffffffffu, best, o);
      const int t2 = __shfl_down_sync(0xffffffffu, bt, o);
      sum += s2;
      better(best, bt, b2, t2);
    }
  }
}

}  // namespace atlas
