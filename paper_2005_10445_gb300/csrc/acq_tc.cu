// acq_tc.cu -- the per-code correlation with its inverse transform on the
// tensor cores (reduced-precision mode; transforms of M = 2^14 points).
//
// The inverse FFT of 16384 points is taken as radix 16 x 16 x 16 x 4
// (self-sorting Stockham order, as in fft_block.cuh).  Each radix-16 stage is
// a dense contraction: the 1024 sub-transforms of a stage are the rows of a
// [1024 x 32] real matrix [Re x | Im x], multiplied by the real form of the
// 16-point DFT matrix F (F[a][b] = exp(+2 pi i a b / 16)):
//
//   [Re y | Im y] = [Re x | Im x] * [[Re F, Im F], [-Im F, Re F]]   (32 x 32)
//
// run as mma.sync m16n8k16 with FP16 or BF16 operands and FP32 accumulation
// (a warp covers 64 rows: 4 row tiles x 4 column tiles x 2 k-steps).  Before
// each contraction the whole transform is scaled by a power of two 2^-e
// (e from the block-wide maximum magnitude) so the operands sit in [-1, 1];
// the scales are exact and are undone in FP32 on |.|^2.  Inter-stage twiddles
// and the last radix-4 stage are FP32; the epilogue (|.|^2, floor sum,
// argmax over valid lags) is the FP32 kernel's.
//
// Data exchange between stages goes through shared memory with one padding
// rule, index i -> i + 2 * (i / 1024), under which the fragment-ordered
// loads of a stage (8 rows x 4 columns per quarter warp) hit distinct banks.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "acq_common.cuh"
#include "acq_internal.h"

namespace atlas {
namespace tc {

constexpr int kLogM = 14;
constexpr int kM = 1 << kLogM;
constexpr int kThreads = 512;
constexpr int kWarps = kThreads / 32;
constexpr int kSmemElems = kM + 2 * (kM / 1024);

__device__ __forceinline__ int tpad(int i) { return i + 2 * (i >> 10); }

// cos and sin of 2 pi m / 16, m = 0 .. 15 (the 16-point DFT matrix entries)
__constant__ float kCos16[16] = {1.000000000f,  0.923879533f,  0.707106781f,  0.382683432f,
                                 0.000000000f,  -0.382683432f, -0.707106781f, -0.923879533f,
                                 -1.000000000f, -0.923879533f, -0.707106781f, -0.382683432f,
                                 0.000000000f,  0.382683432f,  0.707106781f,  0.923879533f};
__constant__ float kSin16[16] = {0.000000000f,  0.382683432f,  0.707106781f,  0.923879533f,
                                 1.000000000f,  0.923879533f,  0.707106781f,  0.382683432f,
                                 0.000000000f,  -0.382683432f, -0.707106781f, -0.923879533f,
                                 -1.000000000f, -0.923879533f, -0.707106781f, -0.382683432f};

template <int PREC>
struct Op;
template <>
struct Op<1> {  // FP16
  __device__ static uint32_t pack(float lo, float hi) {
    __half2 h = __floats2half2_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&h);
  }
  __device__ static void mma(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
  }
};
template <>
struct Op<2> {  // BF16
  __device__ static uint32_t pack(float lo, float hi) {
    __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&h);
  }
  __device__ static void mma(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
  }
};

// block-wide maximum (every thread gets it)
__device__ __forceinline__ float block_max(float v, float* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  float m = red[0];
#pragma unroll
  for (int i = 1; i < kWarps; ++i) m = fmaxf(m, red[i]);
  return m;
}

// exponent e with m * 2^-e <= 1 (0 for m == 0)
__device__ __forceinline__ int scale_exp(float m) {
  int e = 0;
  if (m > 0.f) frexpf(m, &e);
  return e;
}

// One radix-16 stage on the tensor cores for the 4 row tiles of this warp.
// x[mt][g2][c]: row g2 (0: row g, 1: row g + 8) of tile mt, column c (0..3 ->
// columns 2t, 2t+1, 2t+8, 2t+9), already scaled; y receives the outputs in
// the same positions.
template <int PREC>
__device__ __forceinline__ void stage_mma(float2 (&x)[4][2][4], const uint32_t (&bf)[2][4][2]) {
#pragma unroll
  for (int mt = 0; mt < 4; ++mt) {
    uint32_t a[2][4];  // k-step 0: real parts, k-step 1: imaginary parts
#pragma unroll
    for (int ks = 0; ks < 2; ++ks) {
      auto part = [&](int g2, int c) { return ks == 0 ? x[mt][g2][c].x : x[mt][g2][c].y; };
      a[ks][0] = Op<PREC>::pack(part(0, 0), part(0, 1));
      a[ks][1] = Op<PREC>::pack(part(1, 0), part(1, 1));
      a[ks][2] = Op<PREC>::pack(part(0, 2), part(0, 3));
      a[ks][3] = Op<PREC>::pack(part(1, 2), part(1, 3));
    }
    float d[4][4];
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
#pragma unroll
      for (int i = 0; i < 4; ++i) d[nt][i] = 0.f;
#pragma unroll
      for (int ks = 0; ks < 2; ++ks) Op<PREC>::mma(d[nt], a[ks], bf[ks][nt][0], bf[ks][nt][1]);
    }
    // n-tiles 0, 1: real parts of output columns 2t(+1) and 2t+8(+9); 2, 3: imaginary
#pragma unroll
    for (int g2 = 0; g2 < 2; ++g2) {
      x[mt][g2][0] = make_float2(d[0][2 * g2 + 0], d[2][2 * g2 + 0]);
      x[mt][g2][1] = make_float2(d[0][2 * g2 + 1], d[2][2 * g2 + 1]);
      x[mt][g2][2] = make_float2(d[1][2 * g2 + 0], d[3][2 * g2 + 0]);
      x[mt][g2][3] = make_float2(d[1][2 * g2 + 1], d[3][2 * g2 + 1]);
    }
  }
}

template <int PREC>
__global__ void __launch_bounds__(kThreads) k_corr_tc(CorrParams p) {
  extern __shared__ float4 smem_raw[];
  float2* sm = reinterpret_cast<float2*>(smem_raw);
  float2* sm_tw = sm + kSmemElems;
  float* red = reinterpret_cast<float*>(sm_tw + TwTables<kLogM>::N);
  float4* red4 = reinterpret_cast<float4*>(red + 32);

  const int rho = blockIdx.x, k = blockIdx.y, sps = p.sps;
  const int wl = blockIdx.z / p.Cg, c = blockIdx.z % p.Cg;
  const int w = p.w0 + wl;
  load_tables<kLogM>(sm_tw, p.tw);

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, t4 = lane & 3;
  // DFT matrix fragments: B[ks][nt] = rows 16 ks + {2t, 2t+1, 2t+8, 2t+9}, column 8 nt + g
  // of [[Re F, Im F], [-Im F, Re F]], F[a][b] = exp(+2 pi i a b / 16)
  uint32_t bf[2][4][2];
#pragma unroll
  for (int ks = 0; ks < 2; ++ks)
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
      float v[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int a = 2 * t4 + (q & 1) + ((q >> 1) << 3);  // row within the k-step
        const int b = (8 * nt + g) & 15;                   // column within the quadrant
        const float s = kSin16[(a * b) & 15], co = kCos16[(a * b) & 15];
        const bool im_out = nt >= 2;
        v[q] = ks == 0 ? (im_out ? s : co) : (im_out ? co : -s);
      }
      bf[ks][nt][0] = Op<PREC>::pack(v[0], v[1]);
      bf[ks][nt][1] = Op<PREC>::pack(v[2], v[3]);
    }
  __syncthreads();

  int nvalid = p.hop;
  if (w == p.W - 1) {
    const int64_t lim = p.S - p.L - (int64_t)w * p.hop;
    nvalid = (int)(lim < p.hop ? lim : p.hop) + 1;
  }
  const float2* G = p.G + (((int64_t)wl * p.K + k) * sps + rho) * kM;
  const float2* D = p.D + (int64_t)c * kM;

  float2 x[4][2][4];
  int etot = 0;
  // ---- stage 0: rows j = 64 warp + 16 mt + g (+8), columns r; input index j + 1024 r
  float mx = 0.f;
#pragma unroll
  for (int mt = 0; mt < 4; ++mt)
#pragma unroll
    for (int g2 = 0; g2 < 2; ++g2)
#pragma unroll
      for (int cc = 0; cc < 4; ++cc) {
        const int j = 64 * warp + 16 * mt + g + 8 * g2;
        const int r = 2 * t4 + (cc & 1) + ((cc >> 1) << 3);
        const int i = j + 1024 * r;
        const float2 z = cmul(G[i], D[i]);
        x[mt][g2][cc] = z;
        mx = fmaxf(mx, fmaxf(fabsf(z.x), fabsf(z.y)));
      }
  // ---- three radix-16 stages: Ns = 1, 16, 256
#pragma unroll
  for (int st = 0; st < 3; ++st) {
    const int Ns = 1 << (4 * st);
    const int e = scale_exp(block_max(mx, red));
    etot += e;
    const float sc = ldexpf(1.f, -e);
#pragma unroll
    for (int mt = 0; mt < 4; ++mt)
#pragma unroll
      for (int g2 = 0; g2 < 2; ++g2)
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) x[mt][g2][cc] = make_float2(x[mt][g2][cc].x * sc, x[mt][g2][cc].y * sc);
    stage_mma<PREC>(x, bf);
    // outputs: o = (j / Ns) * 16 Ns + (j % Ns) + n * Ns; stored for the next stage
    __syncthreads();  // the previous stage's loads are complete
    mx = 0.f;
#pragma unroll
    for (int mt = 0; mt < 4; ++mt)
#pragma unroll
      for (int g2 = 0; g2 < 2; ++g2) {
        const int j = 64 * warp + 16 * mt + g + 8 * g2;
        const int ob = (j / Ns) * 16 * Ns + (j % Ns);
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) {
          const int n = 2 * t4 + (cc & 1) + ((cc >> 1) << 3);
          sm[tpad(ob + n * Ns)] = x[mt][g2][cc];
        }
      }
    __syncthreads();
    if (st < 2) {
      // next radix-16 stage: rows j, inputs j + 1024 r, twiddle W_{16 Ns'}^{(j mod Ns') r}
      const int Ns2 = Ns * 16;
      const int sh = kLogM - 4 * (st + 1) - 4;  // W_M exponent multiplier: M / (16 Ns2)
#pragma unroll
      for (int mt = 0; mt < 4; ++mt)
#pragma unroll
        for (int g2 = 0; g2 < 2; ++g2) {
          const int j = 64 * warp + 16 * mt + g + 8 * g2;
          const int jm = j & (Ns2 - 1);
          // W^{jm r} for r = 2t, 2t+1, 2t+8, 2t+9: two table values, two products by W^{jm}
          const float2 w1 = twiddle<kLogM, +1>(sm_tw, jm << sh);
          const float2 wa = twiddle<kLogM, +1>(sm_tw, (jm * 2 * t4) << sh);
          const float2 wb = twiddle<kLogM, +1>(sm_tw, (jm * (2 * t4 + 8)) << sh);
          const float2 tw4[4] = {wa, cmul(wa, w1), wb, cmul(wb, w1)};
#pragma unroll
          for (int cc = 0; cc < 4; ++cc) {
            const int r = 2 * t4 + (cc & 1) + ((cc >> 1) << 3);
            const float2 v = cmul(sm[tpad(j + 1024 * r)], tw4[cc]);
            x[mt][g2][cc] = v;
            mx = fmaxf(mx, fmaxf(fabsf(v.x), fabsf(v.y)));
          }
        }
    }
  }
  // ---- last stage: radix 4 in FP32, Ns = 4096; 4096 sub-transforms, 8 per thread
  const float unscale = ldexpf(1.f, 2 * etot);
  const int qlim = (nvalid - rho + sps - 1) / sps;
  float sum = 0.f, best = -1.f;
  int bq = 0x7fffffff;
#pragma unroll
  for (int s = 0; s < 8; ++s) {
    const int j = threadIdx.x + kThreads * s;
    float2 v[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      v[r] = sm[tpad(j + 4096 * r)];
      if (r) v[r] = cmul(v[r], twiddle<kLogM, +1>(sm_tw, j * r));
    }
    dft_reg<4, +1>(v);
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int q = j + 4096 * r;
      const float P = fmaf(v[r].x, v[r].x, v[r].y * v[r].y) * unscale;
      sum += P;
      if (q < qlim) better(best, bq, P, q);
    }
  }
  int bt = bq == 0x7fffffff ? bq : bq * sps + rho;
  block_reduce_stats(sum, best, bt, red4);
  if (threadIdx.x == 0)
    p.part[(((int64_t)wl * p.Cg + c) * p.K + k) * sps + rho] = make_float4(sum, best, __int_as_float(bt), 0.f);
}

constexpr size_t kSmem =
    sizeof(float2) * (kSmemElems + TwTables<kLogM>::N) + 32 * sizeof(float) + 32 * sizeof(float4);

}  // namespace tc

cudaError_t prepare_tc() {
  cudaError_t e = cudaFuncSetAttribute(tc::k_corr_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc::kSmem);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(tc::k_corr_tc<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc::kSmem);
}

cudaError_t launch_corr_tc(int precision, const CorrParams& p, cudaStream_t s) {
  if (p.M != tc::kM || p.pairs) return cudaErrorInvalidValue;
  dim3 grid(p.sps, p.K, p.nw * p.Cg);
  if (precision == 1) tc::k_corr_tc<1><<<grid, tc::kThreads, tc::kSmem, s>>>(p);
  else if (precision == 2) tc::k_corr_tc<2><<<grid, tc::kThreads, tc::kSmem, s>>>(p);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

}  // namespace atlas
