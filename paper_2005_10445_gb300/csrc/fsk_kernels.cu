// fsk_kernels.cu -- the FSK front end's element-wise and per-detection kernels:
//
//   k_fsk_demod    Section 3 steps 1-5 over a range of the stream: int16 (I, Q)
//                  to float, the LO mix with an exact fixed-point phase, both
//                  composed filters H_BP H_1 and H_BP H_0 (Section 4.1) by
//                  overlap-save with 4096-point transforms in shared memory
//                  (one forward, two inverse per block of 4096 - T + 1
//                  outputs), magnitudes, d and u
//   k_fsk_replica  step 6: the continuous-phase FSK replica of each code
//   k_fsk_stats_part / _final
//                  step 8 per candidate: w_c, q, p_c and the three
//                  correlation values around the peak as direct sums over the
//                  support (32 slices; FP32 within a warp's few terms per
//                  thread and its shuffle tree, FP64 across warps and slices,
//                  in a fixed order), the parabolic
//                  arrival time, the record appended to the caller's list
//   k_fsk_select   per (window, code): combines the cluster's partial results,
//                  score, threshold, ordered compaction by a block prefix sum
//   k_fsk_advance  advances the caller's running count by the group's candidates
#include <cuda_runtime.h>
#include <stdint.h>

#include "acq_common.cuh"
#include "fsk_internal.h"

namespace atlas {

constexpr int kFskLogE = 4;  // 16 values per thread in the demodulation transforms
constexpr int kFskDemodThreads = (1 << kFskLogB) >> kFskLogE;

// padded work buffer, the block's spectrum, twiddle tables (67 KB: three
// blocks per SM)
constexpr size_t fsk_demod_smem() {
  return sizeof(float2) * (BlockFFT<kFskLogB, kFskLogE, -1>::SMEM_ELEMS + (1 << kFskLogB) + TwTables<kFskLogB>::N);
}

__global__ void __launch_bounds__(kFskDemodThreads, 3) k_fsk_demod(FskDemodParams p) {
  using FWD = BlockFFT<kFskLogB, kFskLogE, -1>;
  using INV = BlockFFT<kFskLogB, kFskLogE, +1>;
  constexpr int B = 1 << kFskLogB;
  // The last pass of INV is one radix-E transform per thread: thread t emits
  // the outputs t + j T, j < E, in increasing j, the same in both inverse
  // transforms, so |f_1| waits for |f_0| in registers, indexed by j.
  static_assert(INV::T == kFskDemodThreads && (kFskLogB % kFskLogE) == 0, "one radix-E last pass per thread");
  constexpr int kLogT = kFskLogB - kFskLogE;
  extern __shared__ float4 smem_raw[];
  float2* sm = reinterpret_cast<float2*>(smem_raw);
  float2* Xs = sm + FWD::SMEM_ELEMS;
  float2* sm_tw = Xs + B;
  load_tables<kFskLogB>(sm_tw, p.tw);
  const int T = p.T;
  const int64_t per = B - (T - 1);
  // blocks sit on a grid fixed in stream coordinates (block b holds outputs
  // [b per, (b+1) per)), so every output is computed the same way whatever
  // range is asked for
  const int64_t first = (p.start >= 0 ? p.start / per : -((-p.start + per - 1) / per)) * per;
  const int64_t end = p.start + p.count;
  const int64_t n_blocks = (end - first + per - 1) / per;
  const short2* iq = reinterpret_cast<const short2*>(p.iq);
  const short2* ring = reinterpret_cast<const short2*>(p.ring);
  const int64_t ring_base = ring ? *p.ring_start : 0;
  const int64_t lo_first = ring ? ring_base : p.lo_first;
  for (int64_t blk = blockIdx.x; blk < n_blocks; blk += gridDim.x) {
    __syncthreads();  // tables ready; the previous block is done with Xs
    // transform position n holds input sample i0 + n; outputs n >= T - 1 are
    // the linear convolution at i0 + n (no wrap-around)
    const int64_t i0 = first + blk * per - (T - 1);
    auto load = [&](int n) -> float2 {
      const int64_t i = i0 + n;
      if (i < 0 || i >= p.S) return make_float2(0.f, 0.f);
      float2 x;
      if (ring) {
        const short2 v = ring[(ring_base + i) % p.ring_cap];
        x = make_float2((float)v.x, (float)v.y);
      } else if (iq) {
        const short2 v = iq[i];
        x = make_float2((float)v.x, (float)v.y);
      } else {
        x = p.xf[i];
      }
      if (p.lo_inc) x = cmul(x, expi_neg((uint64_t)(i + lo_first) * p.lo_inc));
      return x;
    };
    auto keep = [&](int k, float2 v) { Xs[k] = v; };
    FWD::run(sm, sm_tw, load, keep);
    __syncthreads();  // the block's spectrum is complete
    auto load1 = [&](int k) { return cmul(Xs[k], p.G1[k]); };
    float a1[1 << kFskLogE];
    auto mag1 = [&](int n, float2 v) { a1[(n - (int)threadIdx.x) >> kLogT] = sqrtf(fmaf(v.x, v.x, v.y * v.y)); };
    INV::run(sm, sm_tw, load1, mag1);
    auto load0 = [&](int k) { return cmul(Xs[k], p.G0[k]); };
    auto out = [&](int n, float2 v) {
      const int64_t i = i0 + n;
      if (n < T - 1 || i < p.start || i >= end) return;
      float dd = 0.f, uu = 0.f;
      if (i >= 0 && i < p.S_out) {
        const float m1 = a1[(n - (int)threadIdx.x) >> kLogT];
        const float a0 = sqrtf(fmaf(v.x, v.x, v.y * v.y));
        const float s = m1 + a0;
        uu = m1 - a0;
        dd = s > 0.f ? uu / s : 0.f;
      }
      p.d[i - p.start] = dd;
      if (p.u) p.u[i - p.start] = uu;
    };
    INV::run(sm, sm_tw, load0, out);
  }
}

__global__ void k_fsk_replica(FskReplicaParams p, int L) {
  const int c = blockIdx.y;
  const int64_t off = p.chip_off[c];
  for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < L; n += gridDim.x * blockDim.x) {
    const int ci = n / p.sps;
    const int within = n - ci * p.sps;
    const int64_t ones = p.ones_before[off + ci] * p.sps + (p.chips[off + ci] > 0 ? within : 0);
    const uint64_t ph = (uint64_t)ones * p.inc1 + (uint64_t)(n - ones) * p.inc0;
    p.r[(int64_t)c * L + n] = expi_neg(0ull - ph);  // exp(+j 2 pi phase)
  }
}

__device__ __forceinline__ float warp_sumf(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

constexpr int kFskStatsThreads = 256;

// Stage 1: candidate b's five sums over slice s of n (n in [s*chunk, (s+1)*chunk));
// persistent over (candidate, slice).
__global__ void __launch_bounds__(kFskStatsThreads) k_fsk_stats_part(FskStatsParams p) {
  __shared__ double red[5][kFskStatsThreads / 32];
  const int n_items = *p.n_cand * kFskStatsSlices;
  const int chunk = (p.n_c + kFskStatsSlices - 1) / kFskStatsSlices;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
    const int b = item / kFskStatsSlices, sl = item % kFskStatsSlices;
    const atlas_detection cd = p.cand[b];
    const int64_t a = (int64_t)cd.window * p.hop + cd.lag;
    const float* dc = p.dc + (int64_t)cd.code * p.ld;
    auto dv = [&](int64_t i) -> float {
      const int64_t k = i - p.base;
      return (k >= 0 && k < p.len) ? p.d[k] : 0.f;
    };
    // each thread sums its few terms (a slice of chunk <= 2100 over 256 threads)
    // in FP32
    float fm = 0.f, f0 = 0.f, fp = 0.f, fq = 0.f, fu = 0.f;
    const int n1 = min(p.n_c, (sl + 1) * chunk);
    for (int n = sl * chunk + threadIdx.x; n < n1; n += blockDim.x) {
      const float g = dc[n];
      const float d0 = dv(a + n);
      const int64_t k = a + n - p.base;
      const float u0 = (k >= 0 && k < p.len) ? p.u[k] : 0.f;
      fm = fmaf(g, dv(a - 1 + n), fm);
      f0 = fmaf(g, d0, f0);
      fp = fmaf(g, dv(a + 1 + n), fp);
      fq = fmaf(d0, d0, fq);
      fu = fmaf(g, u0, fu);
    }
    // a warp's partial sums (at most 32 x 9 terms) by an FP32 shuffle tree;
    // FP64 across the warps and slices
    const double cm = warp_sumf(fm);
    const double c0 = warp_sumf(f0);
    const double cp = warp_sumf(fp);
    const double q = warp_sumf(fq);
    const double pc = warp_sumf(fu);
    __syncthreads();  // the previous item's reduction has been read
    if (lane == 0) {
      red[0][warp] = cm;
      red[1][warp] = c0;
      red[2][warp] = cp;
      red[3][warp] = q;
      red[4][warp] = pc;
    }
    __syncthreads();
    if (threadIdx.x < 5) {
      double v = 0.0;
      for (int w = 0; w < kFskStatsThreads / 32; ++w) v += red[threadIdx.x][w];
      p.part[((int64_t)b * kFskStatsSlices + sl) * 5 + threadIdx.x] = v;
    }
  }
}

// Stage 2: one warp per candidate: lane s takes slice s, the slices are summed
// by a fixed shuffle tree (deterministic, and log-depth where a sequential
// FP64 chain was latency-bound), then the parabolic arrival time and the
// record appended to the caller's list.
static_assert(kFskStatsSlices == 32, "one slice per lane");

// ADVANCE (a one-block launch): the block also advances the caller's running
// count once every record is written, in place of k_fsk_advance.
template <bool ADVANCE>
__global__ void __launch_bounds__(kFskStatsThreads) k_fsk_stats_final(FskStatsParams p) {
  const int nc = *p.n_cand;
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; b < nc; b += warps) {
    const double* pv = p.part + ((int64_t)b * kFskStatsSlices + lane) * 5;
    double v[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) v[k] = warp_sum(pv[k]);
    if (lane != 0) continue;
    const atlas_detection cd = p.cand[b];
    const int64_t a = (int64_t)cd.window * p.hop + cd.lag;
    const double cm = v[0], c0 = v[1], cp = v[2];
    double delta = 0.0;
    if (a - 1 >= 0 && a + 1 <= p.S - p.n_c) {
      const double pm = cm * cm, p0 = c0 * c0, pp = cp * cp;
      const double den = pm - 2.0 * p0 + pp;
      if (den < 0.0) {
        delta = 0.5 * (pm - pp) / den;
        delta = delta > 0.5 ? 0.5 : (delta < -0.5 ? -0.5 : delta);
      }
    }
    const int idx = *p.count + b;
    if (idx < p.capacity) {
      atlas_fsk_detection o;
      o.code = cd.code;
      o.window = cd.window;
      o.lag = cd.lag;
      o.score = cd.score;
      o.toa = (double)a + delta;
      o.w_c = c0;
      o.q = v[3];
      o.p_c = v[4];
      p.out[idx] = o;
    }
  }
  if constexpr (ADVANCE) {
    __syncthreads();  // every record has read the old count
    if (threadIdx.x == 0) *p.count += nc;
  }
}

__global__ void k_fsk_advance(int* count, const int* n) { *count += *n; }

// Selection of a launch group (Section 3 step 8): per (window, code) the
// R partial results of the cluster's blocks are combined (floor = sum / N,
// the maximum with the smallest lag on ties), score = P* / floor, and the
// cells at or above the threshold are appended in (window, code) order by
// a block-wide prefix sum, kFskSelectThreads cells per round.
constexpr int kFskSelectThreads = 1024;

__global__ void __launch_bounds__(kFskSelectThreads) k_fsk_select(SelectParams p) {
  __shared__ int warp_tot[kFskSelectThreads / 32];
  __shared__ int base_sh;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) base_sh = 0;  // a launch group's candidate list starts empty
  const int n_pairs = p.nw * p.Cg;
  for (int p0 = 0; p0 < n_pairs; p0 += kFskSelectThreads) {
    const int pi = p0 + threadIdx.x;
    int flag = 0;
    atlas_detection d;
    if (pi < n_pairs) {
      const float4* pr = p.part + (int64_t)pi * p.sps;
      float sum = 0.f, best = -1.f;
      int bt = 0x7fffffff;
      for (int r = 0; r < p.sps; ++r) {
        const float4 v = pr[r];
        sum += v.x;
        better(best, bt, v.y, __float_as_int(v.z));
      }
      const float floor_ = sum / (float)p.N;
      const float score = floor_ > 0.f ? best / floor_ : 0.f;
      flag = score >= p.threshold ? 1 : 0;
      d.code = p.codes[pi % p.Cg];
      d.window = p.w0 + pi / p.Cg;
      d.lag = bt;
      d.freq_bin = 0;
      d.score = score;
      d.peak_power = best;
      d.toa = 0.0;
    }
    // exclusive prefix sum of the flags over the block
    const unsigned m = __ballot_sync(0xffffffffu, flag);
    const int in_warp = __popc(m & ((1u << lane) - 1u));
    if (lane == 0) warp_tot[warp] = __popc(m);
    __syncthreads();
    if (warp == 0) {
      const int v = warp_tot[lane];
      int x = v;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
      }
      warp_tot[lane] = x - v;  // exclusive
    }
    __syncthreads();
    const int base = base_sh;
    if (flag) {
      const int idx = base + warp_tot[warp] + in_warp;
      if (idx < p.capacity) p.out[idx] = d;
    }
    __syncthreads();  // every thread has read base_sh and warp_tot
    if (threadIdx.x == kFskSelectThreads - 1) base_sh = base + warp_tot[warp] + in_warp + flag;
    __syncthreads();
  }
  if (threadIdx.x == 0) *p.count = base_sh;
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------

int64_t fsk_demod_outputs_per_block(int T) { return (int64_t)(1 << kFskLogB) - (T - 1); }

namespace {

// Co-resident blocks of `kern` on the current device (occupancy query, cached per device).
template <class K>
int resident_blocks(K kern, int threads, size_t smem) {
  constexpr int kMaxDevices = 64;
  static int cache[kMaxDevices] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < kMaxDevices && cache[dev] > 0) return cache[dev];
  int sms = 0, per_sm = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
  const int n = (sms > 0 ? sms : 1) * (per_sm > 0 ? per_sm : 1);
  if (dev >= 0 && dev < kMaxDevices) cache[dev] = n;
  return n;
}

}  // namespace

cudaError_t fsk_prepare() {
  cudaError_t e = cudaFuncSetAttribute(k_fsk_demod, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)fsk_demod_smem());
  if (e != cudaSuccess) return e;
  return fsk_prepare_fft();
}

cudaError_t launch_fsk_demod(const FskDemodParams& p, cudaStream_t s) {
  if (p.count <= 0) return cudaSuccess;
  if (p.T < 1 || p.T > kFskMaxTaps) return cudaErrorInvalidValue;
  const int64_t per = fsk_demod_outputs_per_block(p.T);
  const int64_t blocks = (p.count + per - 1) / per + 1;  // the grid of blocks may straddle one more
  const int resident = resident_blocks(k_fsk_demod, kFskDemodThreads, fsk_demod_smem());
  const int grid = (int)(blocks < resident ? blocks : resident);
  k_fsk_demod<<<grid, kFskDemodThreads, fsk_demod_smem(), s>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_fsk_replica(const FskReplicaParams& p, int n_codes, int L, cudaStream_t s) {
  if (n_codes <= 0 || L <= 0) return cudaSuccess;
  dim3 grid((unsigned)((L + 255) / 256 < 1024 ? (L + 255) / 256 : 1024), (unsigned)n_codes);
  k_fsk_replica<<<grid, 256, 0, s>>>(p, L);
  return cudaGetLastError();
}

cudaError_t launch_fsk_select(const SelectParams& p, cudaStream_t s) {
  k_fsk_select<<<1, kFskSelectThreads, 0, s>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_fsk_stats(const FskStatsParams& p, int max_cand, cudaStream_t s) {
  if (max_cand > 0) {
    const int items = max_cand * kFskStatsSlices;
    const int resident = resident_blocks(k_fsk_stats_part, kFskStatsThreads, 0);
    k_fsk_stats_part<<<items < resident ? items : resident, kFskStatsThreads, 0, s>>>(p);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    constexpr int warps_per_block = kFskStatsThreads / 32;
    static_assert(kFskStatsFinalOneBlock <= 4 * warps_per_block, "a few candidates per warp");
    if (max_cand <= kFskStatsFinalOneBlock) {  // small groups (tracking tasks): one block that also advances
      k_fsk_stats_final<true><<<1, kFskStatsThreads, 0, s>>>(p);
      return cudaGetLastError();
    }
    k_fsk_stats_final<false><<<(max_cand + warps_per_block - 1) / warps_per_block, kFskStatsThreads, 0, s>>>(p);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  k_fsk_advance<<<1, 1, 0, s>>>(p.count, p.n_cand);
  return cudaGetLastError();
}

}  // namespace atlas
