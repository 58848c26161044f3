// fft16.cuh -- Stockham passes with 16 complex values per thread (n/16 threads per
// transform of n points), used by the fused per-draw kernel.
//
// The forward transform runs radix-8 passes and ends with the short radix RL
// (2, 4 or 8 so that n = 8^(P-1) RL); the inverse transform runs the same radices
// in reverse order, starting with RL.  Because the last forward pass and the first
// inverse pass then touch the same elements (x[j + r n/RL] for butterfly j), a
// thread that owns butterflies j and n/RL - j holds both bins k and n - k of every
// real-FFT pair and can do the frequency-domain step and the first inverse pass in
// registers; the first forward pass reads its input from global memory and the last
// inverse pass writes its output there.  Shared memory uses the swizzled layout sw().
#pragma once

#include "common.cuh"

namespace gwx {

template <int LOGN>
struct Plan16 {
  static constexpr int n = 1 << LOGN;
  static constexpr int T = n / 16;                                       // threads per transform
  static constexpr int P = (LOGN + 2) / 3;                               // passes
  static constexpr int RL = (LOGN % 3 == 0) ? 8 : (LOGN % 3 == 1 ? 2 : 4); // short radix
  static constexpr int NB = n / RL;                                      // butterflies of that pass
  static constexpr int SLOTS = 8 / RL;                                   // butterfly pairs per thread
};

// w^r, r = 1 .. R-1, of butterfly jm in a pass (R, Ns): e^{-2 pi i jm r/(Ns R)}
template <int R, int Ns, bool INV>
__device__ __forceinline__ void pass_twiddles(int jm, float2* w) {
  const float2* tp = g_twp + twp_offset(R, Ns) + jm;
#pragma unroll
  for (int r = 1; r < R; ++r) w[r] = __ldg(tp + (r - 1) * Ns);
  if (INV) {
#pragma unroll
    for (int r = 1; r < R; ++r) w[r] = cconj(w[r]);
  }
}

// Load x[j + r nR], r < R (shared, swizzled).
template <int R, int nR>
__device__ __forceinline__ void load_strided(uint32_t x, int j, float2* v) {
  if constexpr (nR % 128 == 0) {
    const uint32_t b = x + 8u * (uint32_t)sw(j);
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = lds2(b + 8u * (uint32_t)(r * nR));
  } else {
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = lds2(x + 8u * (uint32_t)sw(j + r * nR));
  }
}

// Store the outputs of butterfly j of a pass (R, Ns) to x[idx + r Ns],
// idx = (j - jm) R + jm, using closed forms of sw() where they exist.
template <int R, int Ns>
__device__ __forceinline__ void store_pass(uint32_t x, int j, const float2* v) {
  const int jm = j & (Ns - 1);
  const int idx = (j - jm) * R + jm;
  if constexpr (Ns % 128 == 0) {
    const uint32_t b = x + 8u * (uint32_t)sw(idx);
#pragma unroll
    for (int r = 0; r < R; ++r) sts2(b + 8u * (uint32_t)(r * Ns), v[r]);
  } else if constexpr (Ns == 64 && R == 8) {
    const int se = sw(idx), so = se ^ 8;
#pragma unroll
    for (int r = 0; r < R; ++r) sts2(x + 8u * (uint32_t)(((r & 1) ? so : se) + 64 * r), v[r]);
  } else if constexpr (Ns == 8 && R == 8) {
    const int b6 = ((idx >> 6) & 1) << 3;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int kr = (r & 1) ^ (((r >> 1) & 3) << 1);
      sts2(x + 8u * (uint32_t)((idx + 8 * r) ^ (kr ^ b6)), v[r]);
    }
  } else if constexpr (Ns == 1 && R == 8) {
    const int c = (j & 1) ^ (((j >> 1) & 7) << 1);
    const int base = (8 * j) ^ (c & 8), lo = c & 7;
#pragma unroll
    for (int r = 0; r < R; ++r) sts2(x + 8u * (uint32_t)(base | (r ^ lo)), v[r]);
  } else {
#pragma unroll
    for (int r = 0; r < R; ++r) sts2(x + 8u * (uint32_t)sw(idx + r * Ns), v[r]);
  }
}

// One shared-memory-to-shared-memory pass; thread t owns butterflies t + i n/16.
template <int LOGN, int R, int Ns, bool INV>
__device__ __forceinline__ void pass16(uint32_t x, int t) {
  constexpr int n = 1 << LOGN;
  constexpr int NBT = 16 / R;
  constexpr int nR = n / R;
  float2 v[NBT][R];
#pragma unroll
  for (int i = 0; i < NBT; ++i) {
    const int j = t + i * (n / 16);
    load_strided<R, nR>(x, j, v[i]);
    if constexpr (Ns > 1) {
      float2 w[R];
      pass_twiddles<R, Ns, INV>(j & (Ns - 1), w);
#pragma unroll
      for (int r = 1; r < R; ++r) v[i][r] = cmul(v[i][r], w[r]);
    }
    dftR<R, INV, false>(v[i]);
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < NBT; ++i) store_pass<R, Ns>(x, t + i * (n / 16), v[i]);
  __syncthreads();
}

// The same pass out of place: reads src, writes dst, one barrier (the two buffers
// alternate, so no thread can overwrite an element another has yet to read).
template <int LOGN, int R, int Ns, bool INV>
__device__ __forceinline__ void pass16_pp(uint32_t src, uint32_t dst, int t) {
  constexpr int n = 1 << LOGN;
  constexpr int NBT = 16 / R;
  constexpr int nR = n / R;
  float2 v[NBT][R];
#pragma unroll
  for (int i = 0; i < NBT; ++i) {
    const int j = t + i * (n / 16);
    load_strided<R, nR>(src, j, v[i]);
    if constexpr (Ns > 1) {
      float2 w[R];
      pass_twiddles<R, Ns, INV>(j & (Ns - 1), w);
#pragma unroll
      for (int r = 1; r < R; ++r) v[i][r] = cmul(v[i][r], w[r]);
    }
    dftR<R, INV, false>(v[i]);
  }
#pragma unroll
  for (int i = 0; i < NBT; ++i) store_pass<R, Ns>(dst, t + i * (n / 16), v[i]);
  __syncthreads();
}

// Middle passes alternating between two buffers; run(a, b) starts from a and returns the
// buffer that holds the result.
template <int LOGN, int p, int PMAX>
struct FwdMiddlePP {
  static __device__ __forceinline__ uint32_t run(uint32_t a, uint32_t b, int t) {
    if constexpr (p <= PMAX) {
      pass16_pp<LOGN, 8, (1 << (3 * p)), false>(a, b, t);
      return FwdMiddlePP<LOGN, p + 1, PMAX>::run(b, a, t);
    } else {
      return a;
    }
  }
};

template <int LOGN, int p, int PMAX, int RL>
struct InvMiddlePP {
  static __device__ __forceinline__ uint32_t run(uint32_t a, uint32_t b, int t) {
    if constexpr (p <= PMAX) {
      pass16_pp<LOGN, 8, RL * (1 << (3 * (p - 1))), true>(a, b, t);
      return InvMiddlePP<LOGN, p + 1, PMAX, RL>::run(b, a, t);
    } else {
      return a;
    }
  }
};

// Middle passes of the forward transform: radix 8 with Ns = 8^p, p = 1 .. P-2.
template <int LOGN, int p, int PMAX>
struct FwdMiddle {
  static __device__ __forceinline__ void run(uint32_t x, int t) {
    if constexpr (p <= PMAX) {
      pass16<LOGN, 8, (1 << (3 * p)), false>(x, t);
      FwdMiddle<LOGN, p + 1, PMAX>::run(x, t);
    }
  }
};

// Middle passes of the inverse transform: radix 8 with Ns = RL 8^(p-1), p = 1 .. P-2.
template <int LOGN, int p, int PMAX, int RL>
struct InvMiddle {
  static __device__ __forceinline__ void run(uint32_t x, int t) {
    if constexpr (p <= PMAX) {
      pass16<LOGN, 8, RL * (1 << (3 * (p - 1))), true>(x, t);
      InvMiddle<LOGN, p + 1, PMAX, RL>::run(x, t);
    }
  }
};

}  // namespace gwx
