// common.cuh -- device building blocks shared by the libgwx kernels.
//
// * complex helpers on float2 (interleaved re, im);
// * per-translation-unit constant tables in device memory (FFT twiddles and
//   powers of the bin index), filled once per device from host FP64 values;
// * Philox4x32-10 (Salmon et al., SC'11), the counter-based generator used for
//   the prior draws and the background noise;
// * double-float ("hi + lo" float pairs) products for the large phase terms;
// * a Stockham auto-sort FFT over shared memory (radix 8 passes, one radix 4 or
//   2 pass for the remainder), executed by n/8 threads per transform of n
//   complex points, forward (e^{-2 pi i}) or inverse (e^{+2 pi i}, unscaled).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "gwx_internal.h"

namespace gwx {

// ---------------------------------------------------------------- debug index checks
// In the debug build (GWX_DEBUG_CHECKS) the hot kernels check the indices of their global
// loads and stores: an index outside its array is not accessed (loads give zero) and the
// first such event of the translation unit is recorded as (site << 48) | (index & 2^47-1)
// | 2^47, for gwx_debug_status.  In the normal build the checks compile to nothing.
#ifdef GWX_DEBUG_CHECKS
static __device__ unsigned long long g_dbg_first_bad;
__device__ __forceinline__ bool dbg_in(int64_t i, int64_t n, unsigned site) {
  if (i >= 0 && i < n) return true;
  atomicCAS(&g_dbg_first_bad, 0ull,
            ((unsigned long long)(site & 0xFFFFu) << 48) | (1ull << 47) | ((unsigned long long)i & ((1ull << 47) - 1)));
  return false;
}
#define GWX_IDX_OK(i, n, site) ::gwx::dbg_in((int64_t)(i), (int64_t)(n), (site))
// This translation unit's record (read and cleared), on the current device.
static inline cudaError_t dbg_take_this_tu(unsigned long long* v) {
  cudaError_t e = cudaMemcpyFromSymbol(v, g_dbg_first_bad, sizeof(*v));
  if (e != cudaSuccess) return e;
  const unsigned long long zero = 0;
  return cudaMemcpyToSymbol(g_dbg_first_bad, &zero, sizeof(zero));
}
#else
#define GWX_IDX_OK(i, n, site) true
static inline cudaError_t dbg_take_this_tu(unsigned long long* v) {
  *v = 0;
  return cudaSuccess;
}
#endif

// ---------------------------------------------------------------- complex
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// The same product with one explicit rounding per partial product, so that it is fused
// the same way wherever it is inlined.
__device__ __forceinline__ float2 cmul_rn(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -__fmul_rn(a.y, b.y)), fmaf(a.x, b.y, __fmul_rn(a.y, b.x)));
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// multiply by -i (forward) or +i (inverse)
template <bool INV>
__device__ __forceinline__ float2 mul_mi(float2 a) {
  return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// ---------------------------------------------------------------- tables
// Twiddles e^{-2 pi i m / TWN}, m < TWN; covers complex FFTs up to TWN/2 points
// and the real-FFT pack twiddles e^{-2 pi i k/N} for N <= TWN.
constexpr int TWN = 16384;
// Powers of the bin index k <= KMAX: k^{-5/3} (hi, lo), k^{-2/3} (hi, lo), and
// k^{-1/3}, ln k (hi, lo).
constexpr int KMAX = 16384;

// Per-pass twiddles of the Stockham passes, laid out [pass][row][jm] so that the
// butterflies of consecutive threads (consecutive jm) read consecutive entries.
// A radix-R pass keeps rows r = 1 .. R-1; one set for every stride Ns = 2, 4, ..., 4096
// of each radix 8, 4 and 2.
__host__ __device__ constexpr int twp_rows(int R) { return R - 1; }   // rows r = 1 .. R-1
constexpr int TWP_NSETS = 12;                                    // Ns = 2 .. 4096
__host__ __device__ constexpr int twp_ns(int q) { return 2 << q; }
__host__ __device__ constexpr int twp_size(int R) { return twp_rows(R) * ((2 << TWP_NSETS) - 2); }
__host__ __device__ constexpr int twp_base(int R) { return R == 8 ? 0 : (R == 4 ? twp_size(8) : twp_size(8) + twp_size(4)); }
__host__ __device__ constexpr int twp_offset(int R, int Ns) { return twp_base(R) + twp_rows(R) * (Ns - 2); }
constexpr int TWP_TOTAL = twp_size(8) + twp_size(4) + twp_size(2);

namespace {
__device__ float2 g_twp[TWP_TOTAL];
__device__ float2 g_tw[TWN];
__device__ float4 g_kp53[KMAX + 1];   // k^-5/3 hi, lo, k^-2/3 hi, lo
__device__ float4 g_kq[KMAX + 1];     // k^-1/3, ln k hi, ln k lo, k^-7/6
}

__device__ __forceinline__ float2 twiddle(int m) { return __ldg(&g_tw[m]); }

// Fill this translation unit's tables on the current device (host side).
// Values are computed in FP64 on the host and rounded; the double-float
// entries keep the rounding error in a second float.
// Twiddle m: of the float pairs next to (cos a, -sin a) pick the one whose squared
// magnitude is closest to 1 (then the closest in value).  Nearest rounding of the
// two parts alone leaves |w|^2 - 1 at about -7e-9 on average over the entries an
// FFT uses, which would shrink the energy of every transform by a few 1e-8.
static inline float2 unit_twiddle(double a) {
  const double c = cos(a), s = -sin(a);
  const float fc = (float)c, fs = (float)s;
  const float cc[3] = {fc, nextafterf(fc, 2.f), nextafterf(fc, -2.f)};
  const float ss[3] = {fs, nextafterf(fs, 2.f), nextafterf(fs, -2.f)};
  float2 best = make_float2(fc, fs);
  double bm = 1e300, bd = 1e300;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      const double m = fabs((double)cc[i] * cc[i] + (double)ss[j] * ss[j] - 1.0);
      const double dist = fabs((double)cc[i] - c) + fabs((double)ss[j] - s);
      if (m < bm || (m == bm && dist < bd)) {
        bm = m;
        bd = dist;
        best = make_float2(cc[i], ss[j]);
      }
    }
  return best;
}

static inline cudaError_t fill_tables_for_this_tu() {
  static float2 tw[TWN];
  static float2 twp[TWP_TOTAL];
  static float4 kp[KMAX + 1];
  static float4 kq[KMAX + 1];
  static bool built = false;
  if (!built) {
    const double two_pi = 6.283185307179586476925286766559;
    for (int m = 0; m < TWN; ++m) tw[m] = unit_twiddle(two_pi * (double)m / (double)TWN);
    const int radices[3] = {8, 4, 2};
    for (int ri = 0; ri < 3; ++ri) {
      const int R = radices[ri];
      for (int q = 0; q < TWP_NSETS; ++q) {
        const int Ns = twp_ns(q);
        const int off = twp_offset(R, Ns);
        for (int row = 0; row < twp_rows(R); ++row)
          for (int jm = 0; jm < Ns; ++jm)
            twp[off + row * Ns + jm] =
                unit_twiddle(two_pi * (double)jm * (double)(row + 1) / ((double)Ns * (double)R));
      }
    }
    kp[0] = make_float4(0.f, 0.f, 0.f, 0.f);
    kq[0] = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int k = 1; k <= KMAX; ++k) {
      double p53 = pow((double)k, -5.0 / 3.0);
      double p23 = pow((double)k, -2.0 / 3.0);
      double p13 = pow((double)k, -1.0 / 3.0);
      double lk = log((double)k);
      float h53 = (float)p53, h23 = (float)p23, hlk = (float)lk;
      kp[k] = make_float4(h53, (float)(p53 - (double)h53), h23, (float)(p23 - (double)h23));
      kq[k] = make_float4((float)p13, hlk, (float)(lk - (double)hlk), (float)pow((double)k, -7.0 / 6.0));
    }
    built = true;
  }
  cudaError_t e = cudaMemcpyToSymbol(g_tw, tw, sizeof(tw));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_twp, twp, sizeof(twp));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_kp53, kp, sizeof(kp));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_kq, kq, sizeof(kq));
  return e;
}

// ---------------------------------------------------------------- Philox
struct u32x4 { uint32_t x, y, z, w; };

__device__ __forceinline__ u32x4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                                uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
    uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
    uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
    uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
  }
  return {c0, c1, c2, c3};
}

constexpr uint32_t TAG_PRIOR = 1u;
constexpr uint32_t TAG_NOISE = 2u;

// (x + 1/2) 2^-52 from the top 52 bits of (hi, lo): exact in binary64.
__device__ __forceinline__ double uniform52(uint32_t hi, uint32_t lo) {
  uint64_t x = ((uint64_t)hi << 20) | (uint64_t)(lo >> 12);
  return ((double)x + 0.5) * 0x1p-52;
}
// ((w >> 8) + 1/2) 2^-24: exact in binary32.
__device__ __forceinline__ float uniform24(uint32_t w) { return ((float)(w >> 8) + 0.5f) * 0x1p-24f; }

// ---------------------------------------------------------------- double-float
// Product of (ah + al) and (bh + bl) as an unnormalised pair (p, e) with
// p = fl(ah bh) and e carrying the rounding error of p plus the cross terms
// (Dekker 1971; error-free fma product, Ogita-Rump-Oishi 2005).
__device__ __forceinline__ float2 df_mul(float ah, float al, float bh, float bl) {
  float p = ah * bh;
  float e = fmaf(ah, bh, -p);
  e = fmaf(ah, bl, e);
  e = fmaf(al, bh, e);
  return make_float2(p, e);
}
// Fractional part of a double-float value in turns, in [-1, 1): the integer part
// of the high word is removed exactly (|p| < 2^23) before the low word is added.
__device__ __forceinline__ float df_frac(float2 v) { return (v.x - rintf(v.x)) + v.y; }

// ---------------------------------------------------------------- FFT
// Shared-memory layout of every FFT buffer: element i is stored at sw(i), an XOR
// swizzle of bits 0-3 by bits 3-6.  It is a bijection on [0, n) for any power of two
// n, and it makes the strided stores of the first two radix-8 Stockham passes (stride
// 8 and 64 complex values) as well as the contiguous loads free of bank conflicts for
// 64-bit accesses (checked exhaustively for n = 2^10 .. 2^13).
__device__ __forceinline__ int sw(int i) { return i ^ ((i >> 3) & 1) ^ (((i >> 4) & 7) << 1); }

template <bool INV>
__device__ __forceinline__ void dft2(float2& a, float2& b) {
  float2 t = a;
  a = cadd(t, b);
  b = csub(t, b);
}

template <bool INV>
__device__ __forceinline__ void dft4(float2& a0, float2& a1, float2& a2, float2& a3) {
  float2 s02 = cadd(a0, a2), d02 = csub(a0, a2);
  float2 s13 = cadd(a1, a3), d13 = csub(a1, a3);
  float2 t = mul_mi<INV>(d13);
  a0 = cadd(s02, s13);
  a2 = csub(s02, s13);
  a1 = cadd(d02, t);
  a3 = csub(d02, t);
}

// x sqrt(1/2), correctly rounded in almost all cases: the exact error of x hi (an
// fma) and x lo are added before the single final rounding.  A plain product with
// the nearest float to sqrt(1/2) (about 1.7e-8 low) would bias the energy of every
// radix-8 transform.
__device__ __forceinline__ float mul_rsqrt2(float x) {
  const float hi = 0.707106769084930419921875f;   // nearest float to sqrt(1/2)
  const float lo = 1.2101617222470066e-08f;       // sqrt(1/2) - hi
  const float p = x * hi;
  return p + fmaf(x, lo, fmaf(x, hi, -p));
}

// (hi + lo) x rounded once, for a double-float constant and a float x.
__device__ __forceinline__ float df_scale(float hi, float lo, float x) {
  const float p = hi * x;
  return p + fmaf(lo, x, fmaf(hi, x, -p));
}

// Radix-8 butterfly.  EXACT: the products by sqrt(1/2) are rounded once from their
// exact values (mul_rsqrt2), which removes the ~6e-8 energy loss per transform that the
// nearest-float constant leaves (it would bias a likelihood built on the transform by
// ~1e-3); otherwise the constant product is fused into the final additions.
template <bool INV, bool EXACT = true>
__device__ __forceinline__ void dft8(float2* v) {
  // even/odd split: E = DFT4(v0, v2, v4, v6), O = DFT4(v1, v3, v5, v7)
  dft4<INV>(v[0], v[2], v[4], v[6]);
  dft4<INV>(v[1], v[3], v[5], v[7]);
  // O_k *= w8^{-+k}, w8 = e^{2 pi i/8}
  const float2 p = v[3], q = v[7];
  const float2 e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6], o0 = v[1];
  const float2 o2 = mul_mi<INV>(v[5]);
  v[0] = cadd(e0, o0); v[4] = csub(e0, o0);
  v[2] = cadd(e2, o2); v[6] = csub(e2, o2);
  if constexpr (EXACT) {
    const float2 o1 = INV ? make_float2(mul_rsqrt2(p.x - p.y), mul_rsqrt2(p.x + p.y))
                          : make_float2(mul_rsqrt2(p.x + p.y), mul_rsqrt2(p.y - p.x));
    const float2 o3 = INV ? make_float2(-mul_rsqrt2(q.x + q.y), mul_rsqrt2(q.x - q.y))
                          : make_float2(mul_rsqrt2(q.y - q.x), -mul_rsqrt2(q.x + q.y));
    v[1] = cadd(e1, o1); v[5] = csub(e1, o1);
    v[3] = cadd(e3, o3); v[7] = csub(e3, o3);
  } else {
    constexpr float c = 0.707106769084930419921875f;   // nearest float to sqrt(1/2)
    // o1 = c (a1x, a1y), o3 = c (a3x, a3y)
    const float a1x = INV ? p.x - p.y : p.x + p.y, a1y = INV ? p.x + p.y : p.y - p.x;
    const float a3x = INV ? -(q.x + q.y) : q.y - q.x, a3y = INV ? q.x - q.y : -(q.x + q.y);
    v[1] = make_float2(fmaf(c, a1x, e1.x), fmaf(c, a1y, e1.y));
    v[5] = make_float2(fmaf(-c, a1x, e1.x), fmaf(-c, a1y, e1.y));
    v[3] = make_float2(fmaf(c, a3x, e3.x), fmaf(c, a3y, e3.y));
    v[7] = make_float2(fmaf(-c, a3x, e3.x), fmaf(-c, a3y, e3.y));
  }
}

template <int R, bool INV, bool EXACT = true>
__device__ __forceinline__ void dftR(float2* v) {
  if constexpr (R == 8) dft8<INV, EXACT>(v);
  else if constexpr (R == 4) dft4<INV>(v[0], v[1], v[2], v[3]);
  else dft2<INV>(v[0], v[1]);
}

// One Stockham pass of radix R over x[0..n) in shared memory, Ns = product of
// the radices of the previous passes.  Butterfly j reads x[j + r n/R],
// multiplies by e^{-+2 pi i (j mod Ns) r/(Ns R)}, transforms, and writes
// x[(j div Ns) Ns R + (j mod Ns) + r Ns] (Govindaraju et al., SC'08).  Thread t of
// the n/8 threads owns butterflies t + i n/8, i < 8/R, and all of them are read
// before any is written (the two barriers make the pass in place).
// Shared-memory accesses by 32-bit shared-window address (explicit ld/st.shared, so the
// FFT keeps native shared-memory instructions although it is a separate function).
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ float2 lds2(uint32_t a) {
  float2 v;
  asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(a) : "memory");
  return v;
}
__device__ __forceinline__ void sts2(uint32_t a, float2 v) {
  asm volatile("st.shared.v2.f32 [%0], {%1, %2};" ::"r"(a), "f"(v.x), "f"(v.y) : "memory");
}
__device__ __forceinline__ float4 lds4(uint32_t a) {
  float4 v;
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(a) : "memory");
  return v;
}
__device__ __forceinline__ void sts4(uint32_t a, float4 v) {
  asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(a), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w) : "memory");
}

// One Stockham pass of radix R over x[0..n) in shared memory, Ns = product of
// the radices of the previous passes.  Butterfly j reads x[j + r n/R],
// multiplies by e^{-+2 pi i (j mod Ns) r/(Ns R)}, transforms, and writes
// x[(j div Ns) Ns R + (j mod Ns) + r Ns] (Govindaraju et al., SC'08).  Thread t of
// the n/8 threads owns butterflies t + i n/8, i < 8/R, and all of them are read
// before any is written (the two barriers make the pass in place).  x is the
// shared-window address of element 0; element i lives at x + 8 sw(i).
template <int LOGN, int R, int Ns, bool INV>
__device__ __forceinline__ void fft_pass(uint32_t x, int t) {
  static_assert(Ns == 1 || (Ns >= 2 && Ns <= 4096), "no twiddle table for this pass");
  constexpr int n = 1 << LOGN;
  constexpr int NB = 8 / R;
  constexpr int nR = n / R;
  float2 v[NB][R];
#pragma unroll
  for (int i = 0; i < NB; ++i) {
    const int j = t + i * (n / 8);
    if constexpr (nR % 128 == 0) {
      // r nR leaves bits 0-6 alone, so sw(j + r nR) = sw(j) + r nR
      const uint32_t b = x + 8u * (uint32_t)sw(j);
#pragma unroll
      for (int r = 0; r < R; ++r) v[i][r] = lds2(b + 8u * (uint32_t)(r * nR));
    } else {
#pragma unroll
      for (int r = 0; r < R; ++r) v[i][r] = lds2(x + 8u * (uint32_t)sw(j + r * nR));
    }
    const int jm = j & (Ns - 1);
    if (Ns > 1) {
      // e^{-2 pi i jm r/(Ns R)} from the per-pass table (coalesced across threads)
      const float2* tp = g_twp + twp_offset(R, Ns) + jm;
      float2 w[R];
#pragma unroll
      for (int r = 1; r < R; ++r) w[r] = __ldg(tp + (r - 1) * Ns);
#pragma unroll
      for (int r = 1; r < R; ++r) v[i][r] = cmul(v[i][r], INV ? cconj(w[r]) : w[r]);
    }
    dftR<R, INV>(v[i]);
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < NB; ++i) {
    const int j = t + i * (n / 8);
    const int jm = j & (Ns - 1);
    const int idx = (j - jm) * R + jm;
    // Closed forms of sw(idx + r Ns) for the strides that occur (checked exhaustively).
    if constexpr (Ns % 128 == 0) {
      const uint32_t b = x + 8u * (uint32_t)sw(idx);
#pragma unroll
      for (int r = 0; r < R; ++r) sts2(b + 8u * (uint32_t)(r * Ns), v[i][r]);
    } else if constexpr (Ns == 64 && R == 8) {
      // idx has bits 6-8 clear; bit 6 of idx + 64 r is r & 1, which flips bit 3
      const int se = sw(idx), so = se ^ 8;
#pragma unroll
      for (int r = 0; r < R; ++r) sts2(x + 8u * (uint32_t)(((r & 1) ? so : se) + 64 * r), v[i][r]);
    } else if constexpr (Ns == 8 && R == 8) {
      // idx has bits 3-5 clear: r fills them; bit 6 of idx flips bit 3
      const int b6 = ((idx >> 6) & 1) << 3;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int kr = (r & 1) ^ (((r >> 1) & 3) << 1);
        sts2(x + 8u * (uint32_t)((idx + 8 * r) ^ (kr ^ b6)), v[i][r]);
      }
    } else if constexpr (Ns == 1 && R == 8) {
      // idx = 8 j: r fills bits 0-2; bits 3-6 come from j
      const int c = (j & 1) ^ (((j >> 1) & 7) << 1);
      const int base = (8 * j) ^ (c & 8), lo = c & 7;
#pragma unroll
      for (int r = 0; r < R; ++r) sts2(x + 8u * (uint32_t)(base | (r ^ lo)), v[i][r]);
    } else {
#pragma unroll
      for (int r = 0; r < R; ++r) sts2(x + 8u * (uint32_t)sw(idx + r * Ns), v[i][r]);
    }
  }
  __syncthreads();
}

template <int LOGN, int DONE, bool INV>
struct FftPasses {
  static __device__ __forceinline__ void run(uint32_t x, int t) {
    constexpr int REM = LOGN - DONE;
    constexpr int LR = REM >= 3 ? 3 : REM;
    fft_pass<LOGN, (1 << LR), (1 << DONE), INV>(x, t);
    FftPasses<LOGN, DONE + LR, INV>::run(x, t);
  }
};
template <int LOGN, bool INV>
struct FftPasses<LOGN, LOGN, INV> {
  static __device__ __forceinline__ void run(uint32_t, int) {}
};

// Complex FFT of n = 2^LOGN points held in shared memory at x (swizzled layout, see
// sw) by threads t = 0 .. n/8-1.  Every thread of the block must call it (it
// contains __syncthreads).  Starts and ends with the data in x.  Kept out of line:
// inlined into a loop over transforms, the compiler keeps the addresses of all
// passes live at once and spills.
template <int LOGN, bool INV>
__device__ __noinline__ void fft_smem_at(uint32_t x, int t) {
  static_assert(LOGN >= 3 && LOGN <= 13, "FFT size out of range");
  FftPasses<LOGN, 0, INV>::run(x, t);
}

template <int LOGN, bool INV>
__device__ __forceinline__ void fft_smem(float2* x, int t) {
  fft_smem_at<LOGN, INV>(smem_addr(x), t);
}

// ------------------------------------------------ real <-> half-length complex
// Forward: z_m = x_2m + i x_2m+1, Z = FFT_n(z).  For 1 <= k <= n/2 returns the
// real-input spectrum X_k and X_{n-k}:
//   E = (Z_k + conj Z_{n-k})/2, O = -i (Z_k - conj Z_{n-k})/2,
//   X_k = E + w^k O, X_{n-k} = conj(E - w^k O),  w = e^{-2 pi i/N}.
__device__ __forceinline__ void unpack_pair(float2 zk, float2 znk, float2 wk, float2& xk, float2& xnk) {
  float2 bc = cconj(znk);
  float2 E = cscale(cadd(zk, bc), 0.5f);
  float2 O = cscale(mul_mi<false>(csub(zk, bc)), 0.5f);
  float2 wO = cmul(wk, O);
  xk = cadd(E, wO);
  xnk = cconj(csub(E, wO));
}
// Inverse: from Y_k and Y_{n-k} builds Z_k, Z_{n-k} such that IFFT_n(Z)/n packs
// irfft(Y) as (y_2m, y_2m+1):  E_k = (Y_k + conj Y_{n-k})/2,
// O_k = (Y_k - conj Y_{n-k}) w^{-k}/2, Z_k = E_k + i O_k, and the same with k
// replaced by n-k (w^{-(n-k)} = -w^k).
__device__ __forceinline__ void pack_pair(float2 yk, float2 ynk, float2 wk, float2& zk, float2& znk) {
  float2 E = cscale(cadd(yk, cconj(ynk)), 0.5f);
  float2 O = cscale(cmul(csub(yk, cconj(ynk)), cconj(wk)), 0.5f);
  zk = cadd(E, mul_mi<true>(O));
  float2 E2 = cconj(E);
  float2 O2 = cscale(cmul(csub(ynk, cconj(yk)), make_float2(-wk.x, -wk.y)), 0.5f);
  znk = cadd(E2, mul_mi<true>(O2));
}

// Twiddle w^k = e^{-2 pi i k/N} for N <= TWN, N a power of two.
__device__ __forceinline__ float2 pack_twiddle(int k, int logN) { return twiddle(k << (14 - logN)); }

// Host helper: call f(std::integral_constant<int, lg>) for a runtime lg in [LO, HI].
template <int LO, int HI, typename Fn>
static inline cudaError_t dispatch_log(int lg, Fn&& f) {
  if constexpr (LO > HI) {
    (void)lg;
    (void)f;
    return cudaErrorInvalidValue;
  } else {
    if (lg == LO) return f(std::integral_constant<int, LO>{});
    return dispatch_log<LO + 1, HI>(lg, f);
  }
}

static inline int ilog2_exact(int64_t v) {
  int l = 0;
  while (((int64_t)1 << l) < v) ++l;
  return l;
}

}  // namespace gwx
