// acq_tc5.cu -- the per-code correlation of M = 2^14 points (reduced-precision
// mode) with every DFT stage on the fifth-generation tensor cores: tcgen05.mma
// with FP16 or BF16 operands in shared memory and FP32 accumulators in tensor
// memory (TMEM), issued by one thread, completion signalled on an mbarrier.
//
// The inverse transform follows the decimation in frequency of k_corr_dif,
// M = 16 x 32 x 32 (Section 4.1 computes the correlation with FFTs; the
// stages here are dense contractions instead of butterflies):
//
//   stage A  the 1024 columns j of Z = G * conj(C)/M as the rows of a
//            [1024 x 32] real operand (16 complex inputs m, interleaved re/im;
//            a thread loads the adjacent columns 2t and 2t + 1 with 16-byte loads)
//            times the real form of the 16-point DFT matrix (32 x 32);
//            outputs m' times W_M^{j m'} (FP32) form chunk m' (1024 points);
//   stage B1 each chunk's 32 columns l (inputs x[l + 32 r]) as rows: a
//            warpgroup holds four chunks, [128 x 64] times the real 32-point
//            DFT matrix (64 x 64); outputs r' times W_1024^{l r'} (FP32);
//   stage B2 the transposed 32 x 32 blocks (row r', column l) times the same
//            matrix: outputs k = l' + 32 r'' of chunk m' are the correlation at
//            q = m' + 16 k, then |.|^2, the floor sum and the argmax (FP32).
//
// Operands are scaled by exact powers of two before the conversion: per row in
// stages A and B1 (a row is one thread's values) and per warp (one chunk) in
// stage B2, mapping the largest magnitude into [2^13, 2^14); the scale is
// undone in FP32 on the accumulators.
//
// Operand layout in shared memory: K-major, no swizzle, 8-row x 16-byte core
// matrices; LBO = byte distance of core matrices adjacent in K, SBO = of core
// matrices adjacent in rows.  Stage B2's operand uses LBO = 144 bytes so that
// the transposing 4-byte stores of a warp fall in 32 distinct banks.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "acq_fft_kernels.cuh"
#include "acq_internal.h"

namespace atlas {
namespace tc5 {

constexpr int kThreads = 512;
constexpr int kLogM = 14;

// shared memory (bytes)
constexpr uint32_t kOffChunks = 0;                            // [16][1024] float2; B1 operands alias (per warpgroup)
constexpr uint32_t kOffOpnd = 16 * 1024 * 8;                  // stage-A operand (64 KB) / B2 operands (4 x kB2Bytes)
constexpr uint32_t kB1Region = 4 * 1024 * 8;                  // a warpgroup's four chunks (32 KB); its B1 operand is 16 KB
constexpr uint32_t kB2Bytes = 16 * 1152;                      // 128 rows: 16 row groups x 1152 B
constexpr uint32_t kOffFA = kOffOpnd + 4 * kB2Bytes;          // 16-point DFT, real form: 32 x 32 halves
constexpr uint32_t kOffFB = kOffFA + 2048;                    // 32-point DFT, real form: 64 x 64 halves
constexpr uint32_t kOffUndo = kOffFB + 8192;                  // [1024] float: stage-A row scales to undo
constexpr uint32_t kOffTw = kOffUndo + 4096;                  // tables of 2^14 (256) + W_1024 table (1024), float2
constexpr uint32_t kOffRed = kOffTw + (256 + 1024) * 8;       // [16] float4 per-warp partial results
constexpr uint32_t kOffBar = kOffRed + 16 * 16;               // 9 mbarriers, TMEM address, abort flag
constexpr uint32_t kSmem = kOffBar + 128;
static_assert(kSmem <= 232448, "one block per SM");
constexpr int kTmemCols = 512;
constexpr int kWaitLimit = 1 << 20;

__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

// kind::f16 instruction descriptor: FP32 accumulators, A and B of type PREC
// (1: FP16, 2: BF16), both K-major, M x N
template <int PREC>
__device__ __forceinline__ constexpr uint32_t idesc(int M, int N) {
  return (1u << 4) | ((PREC == 2 ? 1u : 0u) << 7) | ((PREC == 2 ? 1u : 0u) << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

template <int PREC>
__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
  if constexpr (PREC == 2) {
    __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&h);
  } else {
    __half2 h = __floats2half2_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&h);
  }
}

__device__ __forceinline__ void mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(id), "r"(acc));
}

__device__ __forceinline__ void commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(bar)));
}

// Bounded wait for phase `parity` of an mbarrier; false if the limit ran out.
__device__ __forceinline__ bool wait_bar(uint64_t* bar, uint32_t parity) {
  uint32_t done = 0;
  for (int it = 0; it < kWaitLimit && !done; ++it) {
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(saddr(bar)), "r"(parity));
  }
  return done != 0;
}

__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void group_sync(int g) { asm volatile("bar.sync %0, 128;" ::"r"(1 + g) : "memory"); }

// 32 consecutive FP32 columns of this thread's TMEM lane (the warp's 32-lane quadrant)
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// scale 2^(13 - e) and its inverse for the largest magnitude m = 2^e * f (1 <= f < 2)
__device__ __forceinline__ void pow2_scale(float m, float& s, float& undo) {
  int e = m > 0.f ? ((__float_as_int(m) >> 23) & 0xff) - 127 : 0;
  e = min(max(e, -100), 100);
  s = __int_as_float((127 + 13 - e) << 23);
  undo = __int_as_float((127 - 13 + e) << 23);
}

// byte offsets inside the operands (K index in halves; two halves per complex value)
__device__ __forceinline__ uint32_t off_a(int row, int kg) { return (row >> 3) * 512 + (row & 7) * 16 + kg * 128; }
__device__ __forceinline__ uint32_t off_b1(int row, int kg) { return (row >> 3) * 1024 + (row & 7) * 16 + kg * 128; }
__device__ __forceinline__ uint32_t off_b2(int row, int l) {
  return (row >> 3) * 1152 + (row & 7) * 16 + (l >> 2) * 144 + (l & 3) * 4;
}

// real form of the R-point inverse DFT as the B operand (N = K = 2R rows x
// columns, K-major): row n = 2 m' + co, column k = 2 m + ci, W = exp(+2 pi i m m'/R)
template <int PREC, int R>
__device__ __forceinline__ void build_dft(unsigned char* dst, int sbo) {
  for (int i = threadIdx.x; i < 4 * R * R; i += blockDim.x) {
    const int n = i / (2 * R), k = i % (2 * R);
    const int mo = n >> 1, co = n & 1, mi = k >> 1, ci = k & 1;
    float sn, cs;
    sincospif(2.f * (float)((mo * mi) % R) / (float)R, &sn, &cs);
    const float v = (co == ci) ? cs : (co == 0 ? -sn : sn);
    const uint32_t off = (n >> 3) * sbo + (n & 7) * 16 + (k >> 3) * 128 + (k & 7) * 2;
    if constexpr (PREC == 2) *reinterpret_cast<__nv_bfloat16*>(dst + off) = __float2bfloat16_rn(v);
    else *reinterpret_cast<__half*>(dst + off) = __float2half_rn(v);
  }
}

template <int PREC>
__global__ void __launch_bounds__(kThreads, 1) k_corr_tc5(CorrParams p, int* status) {
  extern __shared__ __align__(1024) unsigned char smem[];
  float2* chunks = reinterpret_cast<float2*>(smem + kOffChunks);
  unsigned char* opnd = smem + kOffOpnd;
  float* undo_a = reinterpret_cast<float*>(smem + kOffUndo);
  float2* sm_tw = reinterpret_cast<float2*>(smem + kOffTw);
  const float2* t32 = sm_tw + TwTables<kLogM>::N;
  float4* red = reinterpret_cast<float4*>(smem + kOffRed);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + kOffBar);  // [0] A, [1..4] B1, [5..8] B2
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + kOffBar + 72);
  int* abort_flag = reinterpret_cast<int*>(smem + kOffBar + 76);

  const int t = threadIdx.x, lane = t & 31, warp = t >> 5, q = warp & 3, g = warp >> 2;
  const uint32_t base = saddr(smem);
  load_tables<kLogM>(sm_tw, p.tw);
  build_dft<PREC, 16>(smem + kOffFA, 512);
  build_dft<PREC, 32>(smem + kOffFB, 1024);
  if (t == 0) {
    for (int i = 0; i < 9; ++i) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(bars + i)));
    asm volatile("fence.mbarrier_init.release.cluster;");
    *abort_flag = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(tmem_slot)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  __syncthreads();
  build_tw32<kLogM>(sm_tw);
  fence_async();
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;
  constexpr uint32_t id_a = idesc<PREC>(128, 32), id_b = idesc<PREC>(128, 64);
  // hop <= N/2: no valid lag has output r >= 16 of stage B2, which then forms
  // only outputs 0..15 (N = 32: the first 32 rows of the DFT matrix); the
  // floor's sum comes from B2's FP32 inputs by Parseval (sum |X|^2 = 32 sum |x|^2)
  const bool half = 2 * p.hop <= p.N;

  const int sps = p.sps;
  const int64_t n_items = p.pairs ? (int64_t)p.n_pairs * sps : (int64_t)sps * p.K * p.nw * p.Cg;
  uint32_t ph = 0;
  for (int64_t item = blockIdx.x; item < n_items; item += gridDim.x, ph ^= 1) {
    const int rho = (int)(item % sps);
    const int64_t rest = item / sps;
    int64_t row, out;
    int c, w;
    if (p.pairs) {
      const int4 pr = p.pairs[rest];
      row = (int64_t)pr.x * sps + rho;
      c = pr.y;
      w = pr.z;
      out = rest * sps + rho;
    } else {
      const int k = (int)(rest % p.K);
      const int z = (int)(rest / p.K);
      const int wl = z / p.Cg;
      c = z % p.Cg;
      w = p.w0 + wl;
      row = ((int64_t)wl * p.K + k) * sps + rho;
      out = (((int64_t)wl * p.Cg + c) * p.K + k) * sps + rho;
    }
    const int qlim = (valid_lags(p, w) - rho + sps - 1) / sps;
    const float2* G = p.G + row * (1 << kLogM);
    const float2* D = p.D + (int64_t)c * (1 << kLogM);

    // ---- stage A operand: rows j = t and jb = 1024 - t (thread 0: 0 and 512),
    // each scaled by a power of two.  The code spectrum of +/-1 chips is
    // Hermitian and M - (j + 1024 m) = jb + 1024 (15 - m): row jb takes row j's
    // code spectrum reversed and conjugated, so a thread loads one column of
    // it (a quarter fewer bytes from L2 than two columns)
    {
      const int jb = t ? 1024 - t : 512, jd = t ? t : 512;
      float2 z0[16], z1[16];
#pragma unroll
      for (int m = 0; m < 16; ++m) z0[m] = D[jd + 1024 * m];
#pragma unroll
      for (int m = 0; m < 16; ++m) z1[m] = cmul_conj(G[jb + 1024 * m], z0[15 - m]);
      if (t == 0) {
#pragma unroll
        for (int m = 0; m < 16; ++m) z0[m] = D[1024 * m];
      }
      float mx0 = 0.f, mx1 = 0.f;
#pragma unroll
      for (int m = 0; m < 16; ++m) {
        z0[m] = cmul(G[t + 1024 * m], z0[m]);
        mx0 = fmaxf(mx0, fmaxf(fabsf(z0[m].x), fabsf(z0[m].y)));
        mx1 = fmaxf(mx1, fmaxf(fabsf(z1[m].x), fabsf(z1[m].y)));
      }
      float s0, u0, s1, u1;
      pow2_scale(mx0, s0, u0);
      pow2_scale(mx1, s1, u1);
      undo_a[t] = u0;
      undo_a[jb] = u1;
#pragma unroll
      for (int kg = 0; kg < 4; ++kg) {
        uint4 v;
        v.x = pack2<PREC>(z0[4 * kg].x * s0, z0[4 * kg].y * s0);
        v.y = pack2<PREC>(z0[4 * kg + 1].x * s0, z0[4 * kg + 1].y * s0);
        v.z = pack2<PREC>(z0[4 * kg + 2].x * s0, z0[4 * kg + 2].y * s0);
        v.w = pack2<PREC>(z0[4 * kg + 3].x * s0, z0[4 * kg + 3].y * s0);
        *reinterpret_cast<uint4*>(opnd + off_a(t, kg)) = v;
        v.x = pack2<PREC>(z1[4 * kg].x * s1, z1[4 * kg].y * s1);
        v.y = pack2<PREC>(z1[4 * kg + 1].x * s1, z1[4 * kg + 1].y * s1);
        v.z = pack2<PREC>(z1[4 * kg + 2].x * s1, z1[4 * kg + 2].y * s1);
        v.w = pack2<PREC>(z1[4 * kg + 3].x * s1, z1[4 * kg + 3].y * s1);
        *reinterpret_cast<uint4*>(opnd + off_a(jb, kg)) = v;
      }
    }
    fence_async();
    fence_before();
    __syncthreads();  // the stage-A operand is complete (and the previous item is finished)
    fence_after();
    if (t == 0) {
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int kk = 0; kk < 2; ++kk)
          mma(tmem + 32 * i, desc(base + kOffOpnd + 8192 * i + 256 * kk, 128, 512),
              desc(base + kOffFA + 256 * kk, 128, 512), id_a, kk);
      commit(&bars[0]);
    }
    if (!wait_bar(&bars[0], ph)) *abort_flag = 1;
    fence_after();

    // ---- stage A results: rows j of tiles 2g, 2g+1 (this warp's lane quadrant), twiddles, chunks
#pragma unroll 1
    for (int ii = 0; ii < 2; ++ii) {
      const int i = 2 * g + ii;
      const int j = 128 * i + 32 * q + lane;
      float v[32];
      tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + 32 * i, v);
      // the row's scale is undone inside the twiddle: wt = u W_M^{j m}, by
      // repeated multiplication (15 steps: a few FP32 ulps, far below the
      // operands' FP16 / BF16 rounding)
      const float u = undo_a[j];
      const float2 w1 = twiddle<kLogM, +1>(sm_tw, j);
      float2 wt = make_float2(u, 0.f);
#pragma unroll
      for (int m = 0; m < 16; ++m) {
        if (m > 0) wt = cmul(wt, w1);
        chunks[m * 1024 + j] = cmul(make_float2(v[2 * m], v[2 * m + 1]), wt);
      }
    }
    fence_before();
    __syncthreads();  // every chunk is complete; every stage-A accumulator is read
    fence_after();

    // ---- stage B1: row (32 q + lane) of warpgroup g = column l = lane of chunk `warp`
    float2 x[32];
    {
      float mx = 0.f;
#pragma unroll
      for (int r = 0; r < 32; ++r) {
        x[r] = chunks[warp * 1024 + lane + 32 * r];
        mx = fmaxf(mx, fmaxf(fabsf(x[r].x), fabsf(x[r].y)));
      }
      float s, u1;
      pow2_scale(mx, s, u1);
      group_sync(g);  // the group's chunks are read: its B1 operand overwrites them
      unsigned char* op1 = smem + kOffChunks + g * kB1Region;
      const int rw = 32 * q + lane;
#pragma unroll
      for (int kg = 0; kg < 8; ++kg) {
        uint4 v;
        v.x = pack2<PREC>(x[4 * kg].x * s, x[4 * kg].y * s);
        v.y = pack2<PREC>(x[4 * kg + 1].x * s, x[4 * kg + 1].y * s);
        v.z = pack2<PREC>(x[4 * kg + 2].x * s, x[4 * kg + 2].y * s);
        v.w = pack2<PREC>(x[4 * kg + 3].x * s, x[4 * kg + 3].y * s);
        *reinterpret_cast<uint4*>(op1 + off_b1(rw, kg)) = v;
      }
      fence_async();
      fence_before();
      group_sync(g);
      fence_after();
      if (lane == 0 && q == 0) {
#pragma unroll
        for (int kk = 0; kk < 4; ++kk)
          mma(tmem + 256 + 64 * g, desc(base + kOffChunks + g * kB1Region + 256 * kk, 128, 1024),
              desc(base + kOffFB + 256 * kk, 128, 1024), id_b, kk);
        commit(&bars[1 + g]);
      }
      if (!wait_bar(&bars[1 + g], ph)) *abort_flag = 1;
      fence_after();
      // outputs r' of column l, undo, W_1024^{l r'}
      float v[32];
      const uint32_t ta = tmem + ((uint32_t)(32 * q) << 16) + 256 + 64 * g;
      tmem_ld32(ta, v);
#pragma unroll
      for (int r = 0; r < 16; ++r) x[r] = make_float2(v[2 * r] * u1, v[2 * r + 1] * u1);
      tmem_ld32(ta + 32, v);
#pragma unroll
      for (int r = 0; r < 16; ++r) x[16 + r] = make_float2(v[2 * r] * u1, v[2 * r + 1] * u1);
#pragma unroll
      for (int r = 1; r < 32; ++r) {
        float2 wv = t32[32 * r + lane];
        wv.y = -wv.y;
        x[r] = cmul(x[r], wv);
      }
    }

    // ---- stage B2: the warp's 32 x 32 block transposed (row r', column l), one scale per warp
    float energy = 0.f;  // sum of |x|^2 over this thread's B2 inputs (half)
    {
      if (half) {
        float e0 = 0.f, e1 = 0.f;
#pragma unroll
        for (int r = 0; r < 32; r += 2) {
          e0 = fmaf(x[r].x, x[r].x, fmaf(x[r].y, x[r].y, e0));
          e1 = fmaf(x[r + 1].x, x[r + 1].x, fmaf(x[r + 1].y, x[r + 1].y, e1));
        }
        energy = 32.f * (e0 + e1);
      }
      float mx = 0.f;
#pragma unroll
      for (int r = 0; r < 32; ++r) mx = fmaxf(mx, fmaxf(fabsf(x[r].x), fabsf(x[r].y)));
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      float s, u2;
      pow2_scale(mx, s, u2);
      unsigned char* op2 = opnd + g * kB2Bytes;
#pragma unroll
      for (int r = 0; r < 32; ++r)
        *reinterpret_cast<uint32_t*>(op2 + off_b2(32 * q + r, lane)) = pack2<PREC>(x[r].x * s, x[r].y * s);
      fence_async();
      fence_before();
      group_sync(g);
      fence_after();
      if (lane == 0 && q == 0) {
#pragma unroll
        for (int kk = 0; kk < 4; ++kk)
          mma(tmem + 64 * g, desc(base + kOffOpnd + g * kB2Bytes + 288 * kk, 144, 1152),
              desc(base + kOffFB + 256 * kk, 128, 1024), half ? id_a : id_b, kk);
        commit(&bars[5 + g]);
      }
      if (!wait_bar(&bars[5 + g], ph)) *abort_flag = 1;
      fence_after();
      float v[32];
      const uint32_t ta = tmem + ((uint32_t)(32 * q) << 16) + 64 * g;
      tmem_ld32(ta, v);
#pragma unroll
      for (int r = 0; r < 16; ++r) x[r] = make_float2(v[2 * r] * u2, v[2 * r + 1] * u2);
      if (!half) {
        tmem_ld32(ta + 32, v);
#pragma unroll
        for (int r = 0; r < 16; ++r) x[16 + r] = make_float2(v[2 * r] * u2, v[2 * r + 1] * u2);
      }
    }

    // ---- epilogue: lag tau = sps q + rho with q = warp + 16 (lane + 32 r), increasing in r
    float s0 = 0.f, s1 = 0.f, best = -1.f;
    int bq = 0x7fffffff;
    const int q0 = warp + 16 * lane;
    float sum;
    if (half) {
#pragma unroll
      for (int r = 0; r < 16; ++r) {
        const float P = fmaf(x[r].x, x[r].x, x[r].y * x[r].y);
        if (q0 + 512 * r < qlim && P > best) {
          best = P;
          bq = q0 + 512 * r;
        }
      }
      sum = energy;
    } else {
#pragma unroll
      for (int r = 0; r < 32; ++r) {
        const float P = fmaf(x[r].x, x[r].x, x[r].y * x[r].y);
        if (r & 1) s1 += P;
        else s0 += P;
        if (q0 + 512 * r < qlim && P > best) {
          best = P;
          bq = q0 + 512 * r;
        }
      }
      sum = s0 + s1;
    }
    int bt = bq == 0x7fffffff ? bq : bq * sps + rho;
    warp_reduce_stats(sum, best, bt);
    if (lane == 0) red[warp] = make_float4(sum, best, __int_as_float(bt), 0.f);
    fence_before();
    __syncthreads();  // partial results written; every accumulator of this item is read
    fence_after();
    if (warp == 0) {
      float4 r = lane < 16 ? red[lane] : make_float4(0.f, -1.f, __int_as_float(0x7fffffff), 0.f);
      float sm2 = r.x, bs = r.y;
      int bt2 = __float_as_int(r.z);
      warp_reduce_stats(sm2, bs, bt2);
      if (lane == 0) p.part[out] = make_float4(sm2, bs, __int_as_float(bt2), 0.f);
    }
    if (*abort_flag) break;
  }
  fence_before();
  __syncthreads();
  if (t == 0 && *abort_flag && status) atomicOr(status, kStatusBadIndex);
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
}

}  // namespace tc5

cudaError_t prepare_tc5() {
  cudaError_t e = cudaFuncSetAttribute(tc5::k_corr_tc5<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc5::kSmem);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(tc5::k_corr_tc5<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc5::kSmem);
}

cudaError_t launch_corr_tc5(int precision, const CorrParams& p, cudaStream_t s) {
  if (p.M != (1 << tc5::kLogM) || (precision != 1 && precision != 2)) return cudaErrorInvalidValue;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int64_t items = p.pairs ? (int64_t)p.n_pairs * p.sps : (int64_t)p.sps * p.K * p.nw * p.Cg;
  const unsigned blocks = (unsigned)std::min<int64_t>(items, sms);  // one block per SM (shared memory, TMEM)
  if (precision == 1) tc5::k_corr_tc5<1><<<blocks, tc5::kThreads, tc5::kSmem, s>>>(p, p.status);
  else tc5::k_corr_tc5<2><<<blocks, tc5::kThreads, tc5::kSmem, s>>>(p, p.status);
  return cudaGetLastError();
}

}  // namespace atlas
