// host_util.h -- host-side helpers shared by the search contexts.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

namespace atlas {

// turns * 2^64 of f/fs, reduced to [-1/2, 1/2) turns, as two's complement.
uint64_t phase_increment(double f_hz, double fs_hz);

// W_M^t = exp(-2 pi i t / M) as the two-level tables of the block transforms:
// HI[i] = W^{i << LB} then LO[i] = W^i, FP64 then rounded.
std::vector<float2> twiddle_tables(int logM);

}  // namespace atlas
