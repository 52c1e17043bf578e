// fft_block.cuh -- one complex FFT of M = 2^LOGM points per thread block,
// held in shared memory, for the on-chip correlation (Section 4.1 computes
// cross-correlations with FFTs; here every transform stays on chip).
//
// Structure: self-sorting Stockham passes.  Pass p has radix R = 2^RB and
// follows passes whose radices multiply to Ns = 2^D.  Sub-transform j reads
// the R values j + r*M/R, multiplies value r by W_{Ns*R}^{(j mod Ns)*r}, does
// an R-point DFT in registers and writes value r to
// (j / Ns)*Ns*R + (j mod Ns) + r*Ns.  Outputs end in natural order, so no
// bit reversal pass is needed.  The first pass takes its inputs from a
// caller functor (global loads fused with the preceding elementwise work) and
// the last pass hands its outputs to a caller functor (fused epilogue), so a
// transform costs (passes - 1) round trips through shared memory.
//
// Every thread owns E = 2^LOGE values (T = M / E threads).  Shared memory is
// padded by one element per 32 (index i lives at i + i/32) so that the strided
// writes of the first pass are free of bank conflicts.
//
// Twiddles W_M^t come from two small tables, W_M^t = HI[t >> LB] * LO[t & (2^LB - 1)],
// each entry the correctly rounded FP32 value of a FP64 evaluation; within a
// pass a thread takes every eighth power of its base twiddle from the tables
// and the powers in between by repeated multiplication.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <utility>

namespace atlas {

// ---------------------------------------------------------------------------
// compile-time constants
// ---------------------------------------------------------------------------

constexpr double kPi = 3.14159265358979323846264338327950288;

constexpr int ct_log2(int x) { return x <= 1 ? 0 : 1 + ct_log2(x >> 1); }

constexpr int ct_brev(int x, int bits) {
  int r = 0;
  for (int i = 0; i < bits; ++i) r = (r << 1) | ((x >> i) & 1);
  return r;
}

// sin / cos of x in [-2 pi, 2 pi] by their Maclaurin series (compile time only).
constexpr double ct_sin(double x) {
  double term = x, sum = x;
  for (int n = 1; n < 40; ++n) {
    term *= -x * x / ((2.0 * n) * (2.0 * n + 1.0));
    sum += term;
  }
  return sum;
}
constexpr double ct_cos(double x) {
  double term = 1.0, sum = 1.0;
  for (int n = 1; n < 40; ++n) {
    term *= -x * x / ((2.0 * n - 1.0) * (2.0 * n));
    sum += term;
  }
  return sum;
}

// W_LEN^K for direction DIR (-1: exp(-2 pi i K / LEN), +1: exp(+2 pi i K / LEN)).
template <int K, int LEN, int DIR>
struct Tw {
  static constexpr double a = DIR * 2.0 * kPi * K / LEN;
  static constexpr float re = (float)ct_cos(a);
  static constexpr float im = (float)ct_sin(a);
};

// ---------------------------------------------------------------------------
// complex helpers
// ---------------------------------------------------------------------------

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__device__ __forceinline__ float2 cmul_conj(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -(a.x * b.y)));
}
// acc + a * b and acc + a * conj(b)
__device__ __forceinline__ float2 cfma(float2 acc, float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, fmaf(-a.y, b.y, acc.x)), fmaf(a.x, b.y, fmaf(a.y, b.x, acc.y)));
}
__device__ __forceinline__ float2 cfma_conj(float2 acc, float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, fmaf(a.y, b.y, acc.x)), fmaf(a.y, b.x, fmaf(-a.x, b.y, acc.y)));
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }

// ---------------------------------------------------------------------------
// R-point DFT in registers: radix-2 decimation in time, bit-reversed input
// order produced by a compile-time register permutation, natural output.
// ---------------------------------------------------------------------------

template <int DIR, int LEN, int K>
__device__ __forceinline__ void bfly(float2& a, float2& b) {
  if constexpr (K != 0 && 4 * K != LEN) {
    // a + w b by four fused multiply-adds, then a - w b = 2a - (a + w b) by two more
    constexpr float wr = Tw<K, LEN, DIR>::re;
    constexpr float wi = Tw<K, LEN, DIR>::im;
    const float px = fmaf(b.x, wr, fmaf(-b.y, wi, a.x));
    const float py = fmaf(b.x, wi, fmaf(b.y, wr, a.y));
    b = make_float2(fmaf(2.f, a.x, -px), fmaf(2.f, a.y, -py));
    a = make_float2(px, py);
  } else if constexpr (K == 0) {
    // w = 1: two packed FP32x2 operations; a - b = fma(b, -1, a) exactly
    const float2 s = __fadd2_rn(a, b);
    b = __ffma2_rn(b, make_float2(-1.f, -1.f), a);
    a = s;
  } else {
    // w = -/+ i (a swap of the parts)
    const float2 t = (DIR < 0) ? make_float2(b.y, -b.x) : make_float2(-b.y, b.x);
    b = make_float2(a.x - t.x, a.y - t.y);
    a = make_float2(a.x + t.x, a.y + t.y);
  }
}

template <int R, int DIR, int LEN, int... Ks>
__device__ __forceinline__ void dit_stage(float2* v, std::integer_sequence<int, Ks...>) {
#pragma unroll
  for (int i = 0; i < R; i += LEN) {
    (bfly<DIR, LEN, Ks>(v[i + Ks], v[i + Ks + LEN / 2]), ...);
  }
}

template <int R, int DIR, int LEN>
__device__ __forceinline__ void dit_stages(float2* v) {
  if constexpr (LEN <= R) {
    dit_stage<R, DIR, LEN>(v, std::make_integer_sequence<int, LEN / 2>{});
    dit_stages<R, DIR, LEN * 2>(v);
  }
}

template <int R, int... Is>
__device__ __forceinline__ void brev_perm(float2* v, std::integer_sequence<int, Is...>) {
  float2 t[R] = {v[ct_brev(Is, ct_log2(R))]...};
  ((v[Is] = t[Is]), ...);
}

template <int R, int DIR>
__device__ __forceinline__ void dft_reg(float2* v) {
  if constexpr (R > 1) {
    brev_perm<R>(v, std::make_integer_sequence<int, R>{});
    dit_stages<R, DIR, 2>(v);
  }
}

// The first R/2 outputs only: every stage but the last, then the last stage's
// a + w b halves (the same operations as in bfly, so these outputs equal
// dft_reg's bit for bit); v[R/2 ..] is left undefined.
template <int DIR, int LEN, int K>
__device__ __forceinline__ void bfly_sum(float2& a, const float2& b) {
  if constexpr (K != 0 && 4 * K != LEN) {
    constexpr float wr = Tw<K, LEN, DIR>::re;
    constexpr float wi = Tw<K, LEN, DIR>::im;
    a = make_float2(fmaf(b.x, wr, fmaf(-b.y, wi, a.x)), fmaf(b.x, wi, fmaf(b.y, wr, a.y)));
  } else if constexpr (K == 0) {
    a = __fadd2_rn(a, b);
  } else {
    const float2 t = (DIR < 0) ? make_float2(b.y, -b.x) : make_float2(-b.y, b.x);
    a = make_float2(a.x + t.x, a.y + t.y);
  }
}

template <int R, int DIR, int LEN>
__device__ __forceinline__ void dit_stages_below(float2* v) {
  if constexpr (LEN < R) {
    dit_stage<R, DIR, LEN>(v, std::make_integer_sequence<int, LEN / 2>{});
    dit_stages_below<R, DIR, LEN * 2>(v);
  }
}

template <int R, int DIR, int... Ks>
__device__ __forceinline__ void last_stage_low(float2* v, std::integer_sequence<int, Ks...>) {
  (bfly_sum<DIR, R, Ks>(v[Ks], v[Ks + R / 2]), ...);
}

template <int R, int DIR>
__device__ __forceinline__ void dft_reg_low(float2* v) {
  static_assert(R >= 2, "at least one stage");
  brev_perm<R>(v, std::make_integer_sequence<int, R>{});
  dit_stages_below<R, DIR, 2>(v);
  last_stage_low<R, DIR>(v, std::make_integer_sequence<int, R / 2>{});
}

// ---------------------------------------------------------------------------
// block FFT
// ---------------------------------------------------------------------------

__device__ __forceinline__ int spad(int i) { return i + (i >> 5); }

template <int LOGM>
struct TwTables {
  static constexpr int LB = LOGM / 2;            // low bits
  static constexpr int HB = LOGM - LB;           // high bits
  static constexpr int NLO = 1 << LB;
  static constexpr int NHI = 1 << HB;
  static constexpr int N = NLO + NHI;            // float2 entries (HI first, then LO)
};

// W_M^t for 0 <= t < M from the shared tables (hi first, lo after), conjugated for DIR = +1.
template <int LOGM, int DIR>
__device__ __forceinline__ float2 twiddle(const float2* tw, int t);

// W_1024^{a b} for a, b < 32 at tw[N + 32 b + a] (forward), built from the
// two-level tables of size 2^LOGM (LOGM >= 10) already in shared memory; the
// caller synchronises before and after.
template <int LOGM>
__device__ __forceinline__ void build_tw32(float2* tw) {
  for (int i = threadIdx.x; i < 1024; i += blockDim.x) {
    const int a = i & 31, b = i >> 5;
    tw[TwTables<LOGM>::N + i] = twiddle<LOGM, -1>(tw, ((a * b) & 1023) << (LOGM - 10));
  }
}

template <int LOGM, int DIR>
__device__ __forceinline__ float2 twiddle(const float2* tw, int t) {
  using TT = TwTables<LOGM>;
  float2 w = cmul(tw[t >> TT::LB], tw[TT::NHI + (t & (TT::NLO - 1))]);
  if (DIR > 0) w.y = -w.y;
  return w;
}

// T32: the pass over bits [5, 10) takes its twiddles W_1024^{jm r} (jm = lane,
// r < 32) from a 32 x 32 table that follows the two-level tables in shared
// memory ([r][jm], forward direction; see build_tw32) instead of the
// recurrence.
template <int LOGM, int LOGE, int DIR, bool T32 = false>
struct BlockFFT {
  static constexpr int M = 1 << LOGM;
  static constexpr int E = 1 << LOGE;
  static constexpr int T = M / E;
  static constexpr int SMEM_ELEMS = M + M / 32;  // padded buffer

  // Pass over bits [D, D + RB).  FIRST: inputs from `load(i)`; LAST: outputs to
  // `emit(i, value)`; otherwise through the shared buffer.
  template <int D, int RB, bool FIRST, bool LAST, class Load, class Emit>
  __device__ __forceinline__ static void pass(float2* sm, const float2* tw, Load& load, Emit& emit) {
    constexpr int R = 1 << RB;
    constexpr int S = E / R;        // sub-transforms per thread
    constexpr int STRIDE = M / R;   // input stride (a multiple of 32)
    static_assert(STRIDE % 32 == 0 && T % 32 == 0, "padding arithmetic needs 32-multiples");
    // padded shared index spad(i) = i + i/32 of every access below is a
    // per-thread base plus a compile-time offset (outputs with 0 < D < 5 excepted)
    constexpr int PSTRIDE = STRIDE + STRIDE / 32;
    constexpr int PT = T + T / 32;
    constexpr bool OUT_CLOSED = (D == 0 || D >= 5);
    constexpr int POUT = D == 0 ? 1 : (D >= 5 ? (1 << D) + (1 << (D - 5)) : 0);
    const int t = threadIdx.x;
    float2 v[E];
    if constexpr (FIRST) {
#pragma unroll
      for (int s = 0; s < S; ++s)
#pragma unroll
        for (int r = 0; r < R; ++r) v[s * R + r] = load(t + T * s + r * STRIDE);
    } else {
      const float2* src = sm + spad(t);
#pragma unroll
      for (int s = 0; s < S; ++s)
#pragma unroll
        for (int r = 0; r < R; ++r) v[s * R + r] = src[s * PT + r * PSTRIDE];
      __syncthreads();  // every value of this pass is in registers
    }
#pragma unroll
    for (int s = 0; s < S; ++s) {
      const int j = t + T * s;
      if constexpr (T32 && D == 5 && RB == 5) {
        const float2* t32 = tw + TwTables<LOGM>::N + (j & 31);
#pragma unroll
        for (int r = 1; r < R; ++r) {
          float2 w = t32[r * 32];
          if (DIR > 0) w.y = -w.y;
          v[s * R + r] = cmul(v[s * R + r], w);
        }
      } else if constexpr (D > 0) {
        // W^{jm r}: every eighth power from the tables, the others by one to
        // seven multiplications by W^{jm} (a few ulps at most)
        const int jm = j & ((1 << D) - 1);
        constexpr int SH = LOGM - D - RB;
        const float2 w1 = twiddle<LOGM, DIR>(tw, jm << SH);
        float2 w = w1;
#pragma unroll
        for (int r = 1; r < R; ++r) {
          if (r > 1) w = (r & 7) == 0 ? twiddle<LOGM, DIR>(tw, (jm * r) << SH) : cmul(w, w1);
          v[s * R + r] = cmul(v[s * R + r], w);
        }
      }
      dft_reg<R, DIR>(v + s * R);
      const int ob = ((j >> D) << (D + RB)) + (j & ((1 << D) - 1));
      if constexpr (LAST) {
        // emitted below, in increasing output index
      } else if constexpr (OUT_CLOSED) {
        float2* dst = sm + spad(ob);
#pragma unroll
        for (int r = 0; r < R; ++r) dst[r * POUT] = v[s * R + r];
      } else {
#pragma unroll
        for (int r = 0; r < R; ++r) sm[spad(ob + (r << D))] = v[s * R + r];
      }
    }
    if constexpr (LAST) {
      // the last pass's outputs of this thread are j_s + r * 2^D with
      // j_s = t + T s < 2^D: emitting r-major, s-minor gives increasing indices
#pragma unroll
      for (int r = 0; r < R; ++r)
#pragma unroll
        for (int s = 0; s < S; ++s) emit(t + T * s + (r << D), v[s * R + r]);
    } else {
      __syncthreads();
    }
  }

  template <int D, class Load, class Emit, class Hook>
  __device__ __forceinline__ static void passes_from(float2* sm, const float2* tw, Load& load, Emit& emit,
                                                     Hook& hook) {
    constexpr int RB = (LOGM - D) < LOGE ? (LOGM - D) : LOGE;
    constexpr bool LAST = (D + RB == LOGM);
    pass<D, RB, D == 0, LAST>(sm, tw, load, emit);
    if constexpr (D == 0) hook();
    if constexpr (!LAST) passes_from<D + RB>(sm, tw, load, emit, hook);
  }

  // Full transform: x[i] = load(i) for i < M; emit(k, X[k]) for k < M, unnormalised,
  // X[k] = sum_i x[i] exp(DIR * 2 pi i * i k / M).  hook() runs once every input
  // has been read (after the first pass), before any output is emitted.  Each
  // thread emits its outputs in increasing k.
  template <class Load, class Emit, class Hook>
  __device__ __forceinline__ static void run(float2* sm, const float2* tw, Load& load, Emit& emit, Hook& hook) {
    passes_from<0>(sm, tw, load, emit, hook);
  }
  template <class Load, class Emit>
  __device__ __forceinline__ static void run(float2* sm, const float2* tw, Load& load, Emit& emit) {
    auto none = [] {};
    passes_from<0>(sm, tw, load, emit, none);
  }
};

}  // namespace atlas
