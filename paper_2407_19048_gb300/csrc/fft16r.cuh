// fft16r.cuh -- radix-16 Stockham passes with one 16-point butterfly per thread (n/16
// threads per transform of n points), for the fused per-draw kernel when log2 n is not
// a multiple of 4.  The forward transform runs A = floor(log2 n / 4) radix-16 passes
// and ends with the short radix RL = 2^(log2 n mod 4) (2, 4 or 8); the inverse runs the
// same radices in reverse order.  Against radix-8 passes this saves one pass each way
// for n = 2^13 (16 16 16 2 instead of 8 8 8 8 2), 2^11 and 2^10, i.e. one shared-memory
// round trip of the whole window and one barrier per direction.
//
// Shared memory uses the swizzle sw16(i) = i ^ ((i >> 4) & 15): every 16 consecutive
// elements stay in 16 distinct 8-byte bank pairs, and so do the strided stores of the
// radix-16 passes (stride 16 x Ns elements): each 16-lane phase of a 64-bit access is
// free of bank conflicts (checked exhaustively for n = 2^9 .. 2^13), except the
// mirrored butterflies of the short-radix pass, whose phases straddle two 16-element
// groups (two lanes share a bank pair).
#pragma once

#include "common.cuh"

namespace gwx {

__device__ __forceinline__ int sw16(int i) { return i ^ ((i >> 4) & 15); }

// ---------------------------------------------------------------- twiddles
// e^{-2 pi i jm/(16 Ns)} for every stride Ns = 2, 4, ..., 512, laid out [Ns][jm] so that
// consecutive butterflies read consecutive entries; the powers r = 2 .. 15 a butterfly
// needs are formed in registers (three squarings and eleven products), which keeps the
// table at 1022 entries (8 KB, resident in L1) instead of fifteen rows per stride.
constexpr int TW16_NSETS = 9;   // Ns = 2 .. 512
__host__ __device__ constexpr int tw16_offset(int Ns) { return Ns - 2; }
constexpr int TW16_TOTAL = (2 << TW16_NSETS) - 2;

namespace {
__device__ float2 g_tw16[TW16_TOTAL];
}

static inline cudaError_t fill_tw16_for_this_tu() {
  static float2 tw[TW16_TOTAL];
  static bool built = false;
  if (!built) {
    const double two_pi = 6.283185307179586476925286766559;
    for (int q = 0; q < TW16_NSETS; ++q) {
      const int Ns = 2 << q;
      for (int jm = 0; jm < Ns; ++jm) tw[tw16_offset(Ns) + jm] = unit_twiddle(two_pi * (double)jm / (16.0 * Ns));
    }
    built = true;
  }
  return cudaMemcpyToSymbol(g_tw16, tw, sizeof(tw));
}

__device__ __forceinline__ float2 csquare(float2 a) {
  return make_float2(fmaf(a.x, a.x, -__fmul_rn(a.y, a.y)), __fmul_rn(2.f * a.x, a.y));
}

// w[r] = w[1]^r for r = 2 .. 15 from w[1].  The products are written with explicit
// roundings, so every kernel that inlines this rounds them alike.
__device__ __forceinline__ void tw16_powers(float2* w) {
  w[2] = csquare(w[1]);
  w[4] = csquare(w[2]);
  w[8] = csquare(w[4]);
  w[3] = cmul_rn(w[1], w[2]);
#pragma unroll
  for (int l = 1; l < 4; ++l) w[4 + l] = cmul_rn(w[4], w[l]);
#pragma unroll
  for (int l = 1; l < 8; ++l) w[8 + l] = cmul_rn(w[8], w[l]);
}

// w[r] = e^{-+2 pi i jm r/(16 Ns)}, r = 1 .. 15 (w[0] unused).
template <int Ns, bool INV>
__device__ __forceinline__ void tw16(int jm, float2* w) {
  static_assert(Ns >= 2 && Ns <= 512, "no radix-16 twiddle set for this stride");
  w[1] = __ldg(g_tw16 + tw16_offset(Ns) + jm);
  if constexpr (INV) w[1] = cconj(w[1]);
  tw16_powers(w);
}

// ---------------------------------------------------------------- butterfly
// x e^{-+2 pi i q/16} for the constant q of the 16-point transform.
template <int q, bool INV>
__device__ __forceinline__ float2 rot16(float2 x) {
  constexpr float h = 0.707106769084930419921875f;   // nearest float to sqrt(1/2)
  constexpr float c1 = 0.92387950420379638671875f;   // nearest float to cos(pi/8)
  constexpr float s1 = 0.3826834261417388916015625f; // nearest float to sin(pi/8)
  if constexpr (q == 4) {
    return mul_mi<INV>(x);
  } else if constexpr (q == 2) {
    return INV ? make_float2(h * (x.x - x.y), h * (x.x + x.y)) : make_float2(h * (x.x + x.y), h * (x.y - x.x));
  } else if constexpr (q == 6) {
    return INV ? make_float2(-h * (x.x + x.y), h * (x.x - x.y)) : make_float2(h * (x.y - x.x), -h * (x.x + x.y));
  } else {
    // (c, s) = (cos, sin)(2 pi q/16) for q = 1, 3, 9
    constexpr float c = q == 1 ? c1 : (q == 3 ? s1 : -c1);
    constexpr float s = q == 1 ? s1 : (q == 3 ? c1 : -s1);
    // forward x (c - i s), inverse x (c + i s)
    return INV ? make_float2(fmaf(x.x, c, -x.y * s), fmaf(x.y, c, x.x * s))
               : make_float2(fmaf(x.x, c, x.y * s), fmaf(x.y, c, -x.x * s));
  }
}

// 16-point DFT in registers, natural order in and out: v[k] <- sum_m v[m] e^{-+2 pi i m k/16}.
// With m = 4a + b and k = c + 4d: four 4-point DFTs over a, the factors e^{-+2 pi i b c/16},
// four 4-point DFTs over b; the result V[c + 4d] lands in v[4c + d] and is renamed back.
template <bool INV>
__device__ __forceinline__ void dft16(float2* v) {
#pragma unroll
  for (int b = 0; b < 4; ++b) dft4<INV>(v[b], v[4 + b], v[8 + b], v[12 + b]);
  v[5] = rot16<1, INV>(v[5]);
  v[9] = rot16<2, INV>(v[9]);
  v[13] = rot16<3, INV>(v[13]);
  v[6] = rot16<2, INV>(v[6]);
  v[10] = rot16<4, INV>(v[10]);
  v[14] = rot16<6, INV>(v[14]);
  v[7] = rot16<3, INV>(v[7]);
  v[11] = rot16<6, INV>(v[11]);
  v[15] = rot16<9, INV>(v[15]);
#pragma unroll
  for (int c = 0; c < 4; ++c) dft4<INV>(v[4 * c], v[4 * c + 1], v[4 * c + 2], v[4 * c + 3]);
  float2 o[16];
#pragma unroll
  for (int c = 0; c < 4; ++c) {
#pragma unroll
    for (int d = 0; d < 4; ++d) o[c + 4 * d] = v[4 * c + d];
  }
#pragma unroll
  for (int k = 0; k < 16; ++k) v[k] = o[k];
}

// ---------------------------------------------------------------- shared memory
// The passes address x[a + b] with a per-thread part a and b = r 2^s, r < 16, a constant
// once the callers' loops over r unroll, whose bits do not overlap a's.  The swizzle mask of
// such a sum is the XOR of the parts' masks: sw16(a + b) = sw16(a) ^ b ^ ((b >> 4) & 15), one
// XOR with a constant per access.  When sw16(a) < 2^s as well (a < 2^s, or 2^s >= 16 with a's
// bits all above the field of b), this is (sw16(a) ^ ((b >> 4) & 15)) + b, b's mask being
// below 2^s as r < 16: few distinct constants, and b an immediate offset.
__device__ __forceinline__ uint32_t sw16_add(uint32_t sa8, int b) {   // 8 sw16(a + b) from 8 sw16(a)
  return (sa8 ^ (8u * (uint32_t)((b >> 4) & 15))) + 8u * (uint32_t)b;
}
__device__ __forceinline__ uint32_t sw16_xor(uint32_t sa8, int b) {
  return sa8 ^ (8u * (uint32_t)(b ^ ((b >> 4) & 15)));
}

// Load x[j + r nR], r < R, j < nR (swizzled sw16).
template <int R, int nR>
__device__ __forceinline__ void load_strided16(uint32_t x, int j, float2* v) {
  const uint32_t sj8 = 8u * (uint32_t)sw16(j);
#pragma unroll
  for (int r = 0; r < R; ++r) v[r] = lds2(x + sw16_add(sj8, r * nR));
}

// Store the outputs of butterfly j < n/R of a pass (R, Ns) to x[idx + r Ns],
// idx = (j - jm) R + jm: idx has no bits in the field of r Ns (below it, jm < Ns; above
// it, (j - jm) R); for Ns < 16 sw16(idx)'s mask reaches into that field.
template <int R, int Ns>
__device__ __forceinline__ void store_pass16(uint32_t x, int j, const float2* v) {
  const int jm = j & (Ns - 1);
  const uint32_t si8 = 8u * (uint32_t)sw16((j - jm) * R + jm);
#pragma unroll
  for (int r = 0; r < R; ++r) {
    if constexpr (Ns >= 16) sts2(x + sw16_add(si8, r * Ns), v[r]);
    else sts2(x + sw16_xor(si8, r * Ns), v[r]);
  }
}

// One radix-16 pass out of place (src -> dst, one barrier) or in place (two barriers);
// thread t owns butterfly t.
template <int LOGN, int Ns, bool INV, bool PP>
__device__ __forceinline__ void pass_r16(uint32_t src, uint32_t dst, int t) {
  constexpr int nR = (1 << LOGN) / 16;
  float2 v[16];
  load_strided16<16, nR>(src, t, v);
  if constexpr (Ns > 1) {
    float2 w[16];
    tw16<Ns, INV>(t & (Ns - 1), w);
#pragma unroll
    for (int r = 1; r < 16; ++r) v[r] = cmul(v[r], w[r]);
  }
  dft16<INV>(v);
  if constexpr (!PP) __syncthreads();
  store_pass16<16, Ns>(dst, t, v);
  __syncthreads();
}

// Middle passes; run(a, b) starts from a and returns the buffer that holds the result
// (b == a for the in-place form).
// Forward: Ns = 16^p, p = 1 .. PMAX.
template <int LOGN, int p, int PMAX, bool PP>
struct FwdMiddle16 {
  static __device__ __forceinline__ uint32_t run(uint32_t a, uint32_t b, int t) {
    if constexpr (p <= PMAX) {
      pass_r16<LOGN, (1 << (4 * p)), false, PP>(a, PP ? b : a, t);
      return FwdMiddle16<LOGN, p + 1, PMAX, PP>::run(PP ? b : a, PP ? a : b, t);
    } else {
      return a;
    }
  }
};

// Inverse: Ns = RL 16^(p-1), p = 1 .. PMAX.
template <int LOGN, int p, int PMAX, int RL, bool PP>
struct InvMiddle16 {
  static __device__ __forceinline__ uint32_t run(uint32_t a, uint32_t b, int t) {
    if constexpr (p <= PMAX) {
      pass_r16<LOGN, RL * (1 << (4 * (p - 1))), true, PP>(a, PP ? b : a, t);
      return InvMiddle16<LOGN, p + 1, PMAX, RL, PP>::run(PP ? b : a, PP ? a : b, t);
    } else {
      return a;
    }
  }
};

}  // namespace gwx
