// k_spectral.cu -- Welch PSD (A5), whitening filter and whitening (A7), crop and
// injection (A6), and row-wise real FFTs.  Every transform is a shared-memory
// Stockham FFT of n = N/2 complex points (the real window packed as
// z_m = x_2m + i x_2m+1) run by n/8 threads per row; several rows share a block
// when n/8 < 256.
#include "common.cuh"

namespace gwx {

cudaError_t init_tables_spectral() { return fill_tables_for_this_tu(); }

template <int LOGN>
struct RowGeom {
  static constexpr int n = 1 << LOGN;
  static constexpr int TPR = n / 8;                         // threads per row
  static constexpr int G = TPR >= 256 ? 1 : 256 / TPR;      // rows per block
  static constexpr int THREADS = TPR * G;
  static constexpr size_t SMEM = (size_t)G * n * sizeof(float2);
};

template <typename K>
static cudaError_t launch_rows(K kernel, int64_t rows, int G, int threads, size_t smem, cudaStream_t s,
                               auto... args) {
  if (rows <= 0) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kernel<<<(unsigned)((rows + G - 1) / G), threads, smem, s>>>(args...);
  return cudaGetLastError();
}

// ----------------------------------------------------------------- A5 Welch
// One block per (segment, detector): Hann-windowed segment -> FFT -> |X_k|^2 (FP64)
// into part[d][s][k], k = 0 .. M/2.
template <int LOGN>
__global__ void __launch_bounds__(RowGeom<LOGN>::TPR) k_welch_seg(const float* __restrict__ x, int64_t L,
                                                                   int64_t stride, int K, double* __restrict__ part) {
  constexpr int n = 1 << LOGN;
  constexpr int M = 2 * n;
  extern __shared__ float2 sm[];
  const int s = blockIdx.x, d = blockIdx.y, t = threadIdx.x;
  const float* seg = x + (int64_t)d * L + (int64_t)s * stride;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int m = t + i * (n / 8);
    const float w0 = 0.5f - 0.5f * cospif((float)(2 * m) * (2.0f / (float)M));
    const float w1 = 0.5f - 0.5f * cospif((float)(2 * m + 1) * (2.0f / (float)M));
    sm[sw(m)] = make_float2(seg[2 * m] * w0, seg[2 * m + 1] * w1);
  }
  __syncthreads();
  fft_smem<LOGN, false>(sm, t);
  double* P = part + ((int64_t)d * K + s) * (n + 1);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int k = t + i * (n / 8);
    if (k == 0) {
      const float2 z0 = sm[0];
      const double x0 = (double)z0.x + z0.y, xn = (double)z0.x - z0.y;
      P[0] = x0 * x0;
      P[n] = xn * xn;
      continue;
    }
    float2 xk, xnk;
    unpack_pair(sm[sw(k)], sm[sw(n - k)], pack_twiddle(k, LOGN + 1), xk, xnk);
    P[k] = (double)xk.x * xk.x + (double)xk.y * xk.y;
    P[n - k] = (double)xnk.x * xnk.x + (double)xnk.y * xnk.y;
  }
  if (t == 0) {
    float2 xh, xh2;
    unpack_pair(sm[sw(n / 2)], sm[sw(n / 2)], pack_twiddle(n / 2, LOGN + 1), xh, xh2);
    P[n / 2] = (double)xh.x * xh.x + (double)xh.y * xh.y;
  }
}

// psd[d][k] = c_k / (fs sum w^2) / K * sum_s part[d][s][k].  A block covers 32 bins
// of one detector with 8 lanes per bin; lane l sums the segments s = l mod 8 and the
// eight partial sums are combined in a fixed order (deterministic result).
__global__ void __launch_bounds__(256) k_welch_reduce(const double* __restrict__ part, int D, int K, int nb,
                                                      double scale_mid, double scale_end, double* __restrict__ psd) {
  __shared__ double red[8][33];
  const int d = blockIdx.y;
  const int kk = threadIdx.x & 31, lane = threadIdx.x >> 5;
  const int k = blockIdx.x * 32 + kk;
  double acc = 0.0;
  if (k < nb) {
    const double* p = part + (int64_t)d * K * nb + k;
    for (int s = lane; s < K; s += 8) acc += p[(int64_t)s * nb];
  }
  red[lane][kk] = acc;
  __syncthreads();
  if (lane == 0 && k < nb) {
    double t = 0.0;
#pragma unroll
    for (int l = 0; l < 8; ++l) t += red[l][kk];
    psd[(int64_t)d * nb + k] = t * ((k == 0 || k == nb - 1) ? scale_end : scale_mid);
  }
}

size_t welch_ws(int D, int64_t L, int64_t M, int64_t stride) {
  const int64_t K = (L - M) / stride + 1;
  return (size_t)D * (size_t)K * (size_t)(M / 2 + 1) * sizeof(double);
}

cudaError_t launch_welch(const float* x, int D, int64_t L, double fs, int64_t M, int64_t stride, double* psd,
                         void* ws, cudaStream_t s) {
  const int K = (int)((L - M) / stride + 1);
  const int logn = ilog2_exact(M / 2);
  double* part = reinterpret_cast<double*>(ws);
  cudaError_t e = dispatch_log<3, 13>(logn, [&](auto c) {
    constexpr int LG = decltype(c)::value;
    const size_t smem = RowGeom<LG>::n * sizeof(float2);
    cudaError_t err = cudaFuncSetAttribute(k_welch_seg<LG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    k_welch_seg<LG><<<dim3((unsigned)K, (unsigned)D), RowGeom<LG>::TPR, smem, s>>>(x, L, stride, K, part);
    return cudaGetLastError();
  });
  if (e != cudaSuccess) return e;
  double sw2 = 0.0;
  const double two_pi = 6.283185307179586476925286766559;
  for (int64_t i = 0; i < M; ++i) {
    const double w = 0.5 - 0.5 * cos(two_pi * (double)i / (double)M);
    sw2 += w * w;
  }
  const int nb = (int)(M / 2 + 1);
  const double scale_end = 1.0 / (fs * sw2) / (double)K;
  k_welch_reduce<<<dim3((unsigned)((nb + 31) / 32), (unsigned)D), 256, 0, s>>>(part, D, K, nb, 2.0 * scale_end,
                                                                               scale_end, psd);
  return cudaGetLastError();
}

// ----------------------------------------------------------------- whitening filter
// W[d][k] = M_k / sqrt(S~_k fs / 2), S~ the PSD linearly interpolated from the grid
// fs/M to fs/N at the exact rational position k M / N.
// W_k = M_k / sqrt(S~_k fs/2) (whitening), or M_k sqrt(S~_k fs/2) with `inverse` (the
// unwhitening filter: its inverse on the band).
__global__ void k_whiten_filter(const double* __restrict__ psd, int D, int64_t M, double fs, int k_lo, int64_t N,
                                bool inverse, float* __restrict__ W) {
  const int64_t F = N / 2 + 1;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)D * F) return;
  const int d = (int)(i / F);
  const int64_t k = i % F;
  float w = 0.f;
  if (k >= k_lo && k < N / 2) {
    const int64_t nb = M / 2 + 1;
    const int64_t num = k * M;
    const int64_t j0 = num / N;
    const int64_t j1 = j0 + 1 < nb ? j0 + 1 : nb - 1;
    const double frac = (double)(num % N) / (double)N;
    const double* p = psd + (int64_t)d * nb;
    const double S = p[j0] + (p[j1] - p[j0]) * frac;
    w = inverse ? (float)sqrt(S * fs * 0.5) : (float)(1.0 / sqrt(S * fs * 0.5));
  }
  W[i] = w;
}

cudaError_t launch_whiten_filter(const double* psd, int D, int64_t M, double fs, int k_lo, int64_t N, float* W,
                                 cudaStream_t s, bool inverse) {
  const int64_t total = (int64_t)D * (N / 2 + 1);
  k_whiten_filter<<<(unsigned)((total + 63) / 64), 64, 0, s>>>(psd, D, M, fs, k_lo, N, inverse, W);   // FP64: spread wide
  return cudaGetLastError();
}

// ----------------------------------------------------------------- row helpers
template <int LOGN>
__device__ __forceinline__ void load_real_row(float2* z, const float* row, int t, bool live) {
  constexpr int n = 1 << LOGN;
  const float2* r2 = reinterpret_cast<const float2*>(row);
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int m = t + i * (n / 8);
    z[sw(m)] = live ? r2[m] : make_float2(0.f, 0.f);
  }
}

template <int LOGN>
__device__ __forceinline__ void store_real_row(const float2* z, float* row, int t, bool live) {
  constexpr int n = 1 << LOGN;
  if (!live) return;
  float2* r2 = reinterpret_cast<float2*>(row);
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int m = t + i * (n / 8);
    __stcs(&r2[m], z[sw(m)]);
  }
}

// ----------------------------------------------------------------- A7 whiten rows
template <int LOGN>
__global__ void __launch_bounds__(RowGeom<LOGN>::THREADS) k_whiten_rows(const float* __restrict__ din,
                                                                         const float* __restrict__ W, int64_t rows,
                                                                         int D, float* __restrict__ yout) {
  using Gm = RowGeom<LOGN>;
  constexpr int n = Gm::n;
  constexpr int64_t N = 2 * n;
  constexpr int64_t F = n + 1;
  extern __shared__ float2 sm[];
  const int g = threadIdx.x / Gm::TPR, t = threadIdx.x % Gm::TPR;
  const int64_t r = (int64_t)blockIdx.x * Gm::G + g;
  const bool live = r < rows;
  float2* z = sm + g * n;
  load_real_row<LOGN>(z, din + r * N, t, live);
  __syncthreads();
  fft_smem<LOGN, false>(z, t);
  const float* Wd = W + (int64_t)(live ? (int)(r % D) : 0) * F;
  const float inv_n = 1.0f / (float)n;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int k = t + i * (n / 8);
    if (k == 0) {
      const float2 z0 = z[0];
      const float y0 = (z0.x + z0.y) * __ldg(&Wd[0]) * inv_n, yn = (z0.x - z0.y) * __ldg(&Wd[n]) * inv_n;
      z[0] = make_float2(0.5f * (y0 + yn), 0.5f * (y0 - yn));
      continue;
    }
    const float2 wk = pack_twiddle(k, LOGN + 1);
    float2 xk, xnk, zk, znk;
    unpack_pair(z[sw(k)], z[sw(n - k)], wk, xk, xnk);
    pack_pair(cscale(xk, __ldg(&Wd[k]) * inv_n), cscale(xnk, __ldg(&Wd[n - k]) * inv_n), wk, zk, znk);
    z[sw(k)] = zk;
    z[sw(n - k)] = znk;
  }
  if (t == 0) {   // k = n/2 pairs with itself
    const int h = n / 2;
    const float2 wk = pack_twiddle(h, LOGN + 1);
    float2 xk, xnk, zk, znk;
    unpack_pair(z[sw(h)], z[sw(h)], wk, xk, xnk);
    const float s_ = __ldg(&Wd[h]) * inv_n;
    pack_pair(cscale(xk, s_), cscale(xk, s_), wk, zk, znk);
    z[sw(h)] = zk;
  }
  __syncthreads();
  fft_smem<LOGN, true>(z, t);
  store_real_row<LOGN>(z, yout + r * N, t, live);
}

cudaError_t launch_whiten_rows(const float* d, const float* W, int64_t rows, int D, int64_t N, float* y,
                               cudaStream_t s) {
  return dispatch_log<4, 13>(ilog2_exact(N / 2), [&](auto c) {
    constexpr int LG = decltype(c)::value;
    using Gm = RowGeom<LG>;
    return launch_rows(k_whiten_rows<LG>, rows, Gm::G, Gm::THREADS, Gm::SMEM, s, d, W, rows, D, y);
  });
}

// ----------------------------------------------------------------- A6 inject rows
// row r = (b, dd): d = crop(noise[dd], off_b) + irfft(fs h_det[b][dd]).
template <int LOGN>
__global__ void __launch_bounds__(RowGeom<LOGN>::THREADS) k_inject_rows(const float* __restrict__ noise, int64_t L,
                                                                         const int64_t* __restrict__ offsets,
                                                                         const float2* __restrict__ h, int64_t rows,
                                                                         int D, float scale, float* __restrict__ dout) {
  using Gm = RowGeom<LOGN>;
  constexpr int n = Gm::n;
  constexpr int64_t N = 2 * n;
  constexpr int64_t F = n + 1;
  extern __shared__ float2 sm[];
  const int g = threadIdx.x / Gm::TPR, t = threadIdx.x % Gm::TPR;
  const int64_t r = (int64_t)blockIdx.x * Gm::G + g;
  const bool live = r < rows;
  float2* z = sm + g * n;
  const float2* hr = h + (live ? r : 0) * F;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int k = t + i * (n / 8);
    if (k == 0) {
      const float y0 = hr[0].x * scale, yn = hr[n].x * scale;
      z[0] = make_float2(0.5f * (y0 + yn), 0.5f * (y0 - yn));
      continue;
    }
    float2 zk, znk;
    pack_pair(cscale(hr[k], scale), cscale(hr[n - k], scale), pack_twiddle(k, LOGN + 1), zk, znk);
    z[sw(k)] = zk;
    z[sw(n - k)] = znk;
  }
  if (t == 0) {
    const int h = n / 2;
    float2 zk, znk;
    pack_pair(cscale(hr[h], scale), cscale(hr[h], scale), pack_twiddle(h, LOGN + 1), zk, znk);
    z[sw(h)] = zk;
  }
  __syncthreads();
  fft_smem<LOGN, true>(z, t);
  if (!live) return;
  const int64_t b = r / D;
  const int dd = (int)(r % D);
  int64_t off = offsets[b];
  off = off < 0 ? 0 : (off > L - N ? L - N : off);   // keep a bad offset inside the stretch
  const float* crop = noise + (int64_t)dd * L + off;
  float2* out = reinterpret_cast<float2*>(dout + r * N);
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int m = t + i * (n / 8);
    const float2 v = z[sw(m)];
    __stcs(&out[m], make_float2(v.x + crop[2 * m], v.y + crop[2 * m + 1]));
  }
}

cudaError_t launch_inject_rows(const float* noise, int D, int64_t L, const int64_t* offsets, const float2* hdet,
                               int64_t B, int64_t N, double fs, float* d, cudaStream_t s) {
  const int64_t rows = B * D;
  const float scale = (float)(fs / (double)(N / 2));
  return dispatch_log<4, 13>(ilog2_exact(N / 2), [&](auto c) {
    constexpr int LG = decltype(c)::value;
    using Gm = RowGeom<LG>;
    return launch_rows(k_inject_rows<LG>, rows, Gm::G, Gm::THREADS, Gm::SMEM, s, noise, L, offsets, hdet, rows, D,
                       scale, d);
  });
}

// Definition B injection: d[b][dd][i] = noise[dd][off_b + i] + fs h_td[b][dd][i] for the
// first N samples of each padded time series h_td (rows of N_pad samples).
__global__ void k_inject_padded(const float* __restrict__ noise, int D, int64_t L, const int64_t* __restrict__ off,
                                const float* __restrict__ htd, int64_t B, int64_t N, int64_t Np, float fs,
                                float* __restrict__ d) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B * D * N) return;
  const int64_t row = i / N, t = i - row * N;
  const int64_t b = row / D;
  const int dd = (int)(row - b * D);
  d[i] = noise[(int64_t)dd * L + __ldg(&off[b]) + t] + fs * htd[row * Np + t];
}

cudaError_t launch_inject_padded(const float* noise, int D, int64_t L, const int64_t* offsets, const float* htd,
                                 int64_t B, int64_t N, int64_t Np, double fs, float* d, cudaStream_t s) {
  const int64_t total = B * D * N;
  if (total == 0) return cudaSuccess;
  k_inject_padded<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(noise, D, L, offsets, htd, B, N, Np, (float)fs, d);
  return cudaGetLastError();
}

// ----------------------------------------------------------------- rfft / irfft rows
template <int LOGN>
__global__ void __launch_bounds__(RowGeom<LOGN>::THREADS) k_rfft_rows(const float* __restrict__ x, int64_t rows,
                                                                       float2* __restrict__ X) {
  using Gm = RowGeom<LOGN>;
  constexpr int n = Gm::n;
  constexpr int64_t N = 2 * n;
  constexpr int64_t F = n + 1;
  extern __shared__ float2 sm[];
  const int g = threadIdx.x / Gm::TPR, t = threadIdx.x % Gm::TPR;
  const int64_t r = (int64_t)blockIdx.x * Gm::G + g;
  const bool live = r < rows;
  float2* z = sm + g * n;
  load_real_row<LOGN>(z, x + r * N, t, live);
  __syncthreads();
  fft_smem<LOGN, false>(z, t);
  if (!live) return;
  float2* Xr = X + r * F;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int k = t + i * (n / 8);
    if (k == 0) {
      const float2 z0 = z[0];
      Xr[0] = make_float2(z0.x + z0.y, 0.f);
      Xr[n] = make_float2(z0.x - z0.y, 0.f);
      continue;
    }
    float2 xk, xnk;
    unpack_pair(z[sw(k)], z[sw(n - k)], pack_twiddle(k, LOGN + 1), xk, xnk);
    Xr[k] = xk;
    Xr[n - k] = xnk;
  }
  if (t == 0) {
    float2 xk, xnk;
    unpack_pair(z[sw(n / 2)], z[sw(n / 2)], pack_twiddle(n / 2, LOGN + 1), xk, xnk);
    Xr[n / 2] = xk;
  }
}

template <int LOGN>
__global__ void __launch_bounds__(RowGeom<LOGN>::THREADS) k_irfft_rows(const float2* __restrict__ X, int64_t rows,
                                                                        float* __restrict__ x) {
  using Gm = RowGeom<LOGN>;
  constexpr int n = Gm::n;
  constexpr int64_t N = 2 * n;
  constexpr int64_t F = n + 1;
  extern __shared__ float2 sm[];
  const int g = threadIdx.x / Gm::TPR, t = threadIdx.x % Gm::TPR;
  const int64_t r = (int64_t)blockIdx.x * Gm::G + g;
  const bool live = r < rows;
  float2* z = sm + g * n;
  const float2* Xr = X + (live ? r : 0) * F;
  const float inv_n = 1.0f / (float)n;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int k = t + i * (n / 8);
    if (k == 0) {
      const float y0 = Xr[0].x * inv_n, yn = Xr[n].x * inv_n;
      z[0] = make_float2(0.5f * (y0 + yn), 0.5f * (y0 - yn));
      continue;
    }
    float2 zk, znk;
    pack_pair(cscale(Xr[k], inv_n), cscale(Xr[n - k], inv_n), pack_twiddle(k, LOGN + 1), zk, znk);
    z[sw(k)] = zk;
    z[sw(n - k)] = znk;
  }
  if (t == 0) {
    const int h = n / 2;
    float2 zk, znk;
    pack_pair(cscale(Xr[h], inv_n), cscale(Xr[h], inv_n), pack_twiddle(h, LOGN + 1), zk, znk);
    z[sw(h)] = zk;
  }
  __syncthreads();
  fft_smem<LOGN, true>(z, t);
  store_real_row<LOGN>(z, x + r * N, t, live);
}

cudaError_t launch_rfft_rows(const float* x, int64_t R, int64_t N, float2* X, cudaStream_t s) {
  return dispatch_log<4, 13>(ilog2_exact(N / 2), [&](auto c) {
    constexpr int LG = decltype(c)::value;
    using Gm = RowGeom<LG>;
    return launch_rows(k_rfft_rows<LG>, R, Gm::G, Gm::THREADS, Gm::SMEM, s, x, R, X);
  });
}

cudaError_t launch_irfft_rows(const float2* X, int64_t R, int64_t N, float* x, cudaStream_t s) {
  return dispatch_log<4, 13>(ilog2_exact(N / 2), [&](auto c) {
    constexpr int LG = decltype(c)::value;
    using Gm = RowGeom<LG>;
    return launch_rows(k_irfft_rows<LG>, R, Gm::G, Gm::THREADS, Gm::SMEM, s, X, R, x);
  });
}

}  // namespace gwx
