// k_random.cu -- prior draws (A1) and the coloured Gaussian background (A4).
#include "common.cuh"

namespace gwx {

cudaError_t init_tables_random() { return fill_tables_for_this_tu(); }

// ----------------------------------------------------------------- A1
// One thread per draw.  Linear maps use the non-contracting intrinsics so the
// doubles equal a plain lo + (hi - lo) u evaluated with two roundings.
__device__ __forceinline__ double lin_map(double lo, double hi, double u) {
  return __dadd_rn(lo, __dmul_rn(__dsub_rn(hi, lo), u));
}

__global__ void k_sample_prior(gwx_prior p, uint32_t k0, uint32_t k1, uint32_t step, int64_t B, uint32_t span,
                               double* __restrict__ theta, int64_t* __restrict__ offsets) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  double u[11];
  uint32_t woff = 0;
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    const u32x4 r = philox4x32_10((uint32_t)b, (uint32_t)j, TAG_PRIOR, step, k0, k1);
    u[2 * j] = uniform52(r.x, r.y);
    if (j < 5) u[2 * j + 1] = uniform52(r.z, r.w);
    else woff = r.z;
  }
  const double two_pi = 6.283185307179586476925286766559;
  theta[GWX_M1 * B + b] = lin_map(p.m_lo, p.m_hi, u[0]);
  theta[GWX_M2 * B + b] = lin_map(p.m_lo, p.m_hi, u[1]);
  theta[GWX_CHI1 * B + b] = lin_map(p.chi_lo, p.chi_hi, u[2]);
  theta[GWX_CHI2 * B + b] = lin_map(p.chi_lo, p.chi_hi, u[3]);
  theta[GWX_DIST * B + b] = lin_map(p.d_lo, p.d_hi, u[4]);
  theta[GWX_TC * B + b] = lin_map(p.tc_lo, p.tc_hi, u[5]);
  theta[GWX_PHIC * B + b] = lin_map(p.phi_lo, p.phi_hi, u[6]);
  theta[GWX_THETAJN * B + b] = acos(__dsub_rn(1.0, __dmul_rn(2.0, u[7])));
  theta[GWX_PSI * B + b] = lin_map(p.psi_lo, p.psi_hi, u[8]);
  theta[GWX_RA * B + b] = __dmul_rn(two_pi, u[9]);
  theta[GWX_DEC * B + b] = asin(__dsub_rn(__dmul_rn(2.0, u[10]), 1.0));
  offsets[b] = (int64_t)(((uint64_t)woff * (uint64_t)span) >> 32);
}

cudaError_t launch_sample_prior(const gwx_prior& p, uint64_t seed, uint32_t step, int64_t B, int64_t L, int64_t N,
                                double* theta, int64_t* offsets, cudaStream_t s) {
  if (B <= 0) return cudaSuccess;
  const int T = 32;   // FP64 acos/asin: spread the draws over many SMs
  k_sample_prior<<<(unsigned)((B + T - 1) / T), T, 0, s>>>(p, (uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32),
                                                           step, B, (uint32_t)(L - N + 1), theta, offsets);
  return cudaGetLastError();
}

// ----------------------------------------------------------------- A4
// Analytic aLIGO fit times 1e49, at max(f, f_lo).
__device__ __forceinline__ float aligo_psd_e49(float f, float f_lo) {
  const float x = fmaxf(f, f_lo) * (1.0f / 215.0f);
  const float x2 = x * x;
  return exp2f(-4.14f * log2f(x)) - 5.0f / x2 + 111.0f * (1.0f - x2 + 0.5f * x2 * x2) / (1.0f + 0.5f * x2);
}

// Spectrum bin k (0 <= k <= L/2) of detector d, scaled by 1/n (n = L/2).
__device__ __forceinline__ float2 noise_bin(uint32_t k0, uint32_t k1, uint32_t step, int d, int64_t k, int64_t L,
                                            float fs, float f_lo, float sig_scale) {
  if (k == 0) return make_float2(0.f, 0.f);
  const u32x4 r = philox4x32_10((uint32_t)(k >> 1), (uint32_t)d, TAG_NOISE, step, k0, k1);
  const uint32_t wa = (k & 1) ? r.z : r.x;
  const uint32_t wb = (k & 1) ? r.w : r.y;
  const float u1 = uniform24(wa), u2 = uniform24(wb);
  const float rad = sqrtf(-2.0f * logf(u1));
  float sn, cs;
  sincospif(2.0f * u2, &sn, &cs);
  const float f = (float)k * (fs / (float)L);
  // sigma = sqrt(L fs S / 4) with S = 1e-49 S'; sig_scale = sqrt(L fs 1e-49 / 4) / n
  float sigma = sqrtf(aligo_psd_e49(f, f_lo)) * sig_scale;
  if (2 * k == L) return make_float2(1.41421356237309505f * sigma * rad * cs, 0.f);
  return make_float2(sigma * rad * cs, sigma * rad * sn);
}

// Packed spectrum element Z_k (0 <= k < n) of the background, generated on the fly:
// Z_k = E_k + i O_k from X_k and X_{n-k} (see pack_pair), w = e^{-2 pi i/L}.
__device__ __forceinline__ float2 noise_packed(uint32_t k0, uint32_t k1, uint32_t step, int d, int64_t k, int64_t L,
                                               float fs, float f_lo, float sig_scale) {
  const int64_t n = L / 2;
  if (k == 0) {
    const float2 xn = noise_bin(k0, k1, step, d, n, L, fs, f_lo, sig_scale);   // X_0 = 0
    return make_float2(0.5f * xn.x, -0.5f * xn.x);
  }
  const float2 xk = noise_bin(k0, k1, step, d, k, L, fs, f_lo, sig_scale);
  const float2 xnk = noise_bin(k0, k1, step, d, n - k, L, fs, f_lo, sig_scale);
  float sn, cs;
  sincospif(2.0f * (float)k / (float)L, &sn, &cs);
  float2 zk, znk;
  pack_pair(xk, xnk, make_float2(cs, -sn), zk, znk);
  return zk;
}

// Four-step inverse FFT of length n = n1 n2 (Bailey 1990): with k = k1 + n1 k2 and
// m = n2 m1 + m2, z_m = sum_k1 e^{2 pi i k1 m1/n1} [e^{2 pi i k1 m2/n} sum_k2 e^{2 pi i k2 m2/n2} Z_k].
// Pass A: for a tile of TK consecutive k1, inverse FFTs of length n2 over k2, then the
// twiddle; writes G[k1][m2].  The input elements Z_k are generated here.
template <int LOGN2>
__global__ void k_fourstep_a(uint32_t key0, uint32_t key1, uint32_t step, int64_t L, float fs, float f_lo,
                             float sig_scale, int n1, int TK, float2* __restrict__ G) {
  constexpr int n2 = 1 << LOGN2;
  extern __shared__ float2 sm[];
  const int64_t n = L / 2;
  const int d = blockIdx.y;
  const int k1_0 = blockIdx.x * TK;
  float2* Gd = G + (int64_t)d * n;
  const int stride = n2 + 1;
  for (int e = threadIdx.x; e < TK * n2; e += blockDim.x) {
    const int g = e % TK, k2 = e / TK;
    sm[g * stride + sw(k2)] =
        noise_packed(key0, key1, step, d, (int64_t)(k1_0 + g) + (int64_t)n1 * k2, L, fs, f_lo, sig_scale);
  }
  __syncthreads();
  const int g = threadIdx.x / (n2 / 8), t = threadIdx.x % (n2 / 8);
  fft_smem<LOGN2, true>(sm + g * stride, t);
  const float two_over_n = 2.0f / (float)n;   // exact: n is a power of two
  for (int e = threadIdx.x; e < TK * n2; e += blockDim.x) {
    const int gg = e / n2, m2 = e % n2;
    const int k1 = k1_0 + gg;
    float sn, cs;
    sincospif((float)(k1 * m2) * two_over_n, &sn, &cs);   // k1 m2 < n <= 2^23: exact
    Gd[(int64_t)k1 * n2 + m2] = cmul(sm[gg * stride + sw(m2)], make_float2(cs, sn));
  }
}

// Pass B: for a tile of TM consecutive m2, inverse FFTs of length n1 over k1; writes
// x_2m = Re z_m, x_2m+1 = Im z_m with m = n2 m1 + m2.
template <int LOGN1>
__global__ void k_fourstep_b(const float2* __restrict__ G, int64_t n, int n2, int TM, float* __restrict__ x) {
  constexpr int n1 = 1 << LOGN1;
  extern __shared__ float2 sm[];
  const int d = blockIdx.y;
  const int m2_0 = blockIdx.x * TM;
  const float2* Gd = G + (int64_t)d * n;
  float2* xd = reinterpret_cast<float2*>(x + (int64_t)d * 2 * n);
  const int stride = n1 + 1;
  for (int e = threadIdx.x; e < TM * n1; e += blockDim.x) {
    const int g = e % TM, k1 = e / TM;
    sm[g * stride + sw(k1)] = Gd[(int64_t)k1 * n2 + m2_0 + g];
  }
  __syncthreads();
  const int g = threadIdx.x / (n1 / 8), t = threadIdx.x % (n1 / 8);
  fft_smem<LOGN1, true>(sm + g * stride, t);
  for (int e = threadIdx.x; e < TM * n1; e += blockDim.x) {
    const int gg = e % TM, m1 = e / TM;
    xd[(int64_t)n2 * m1 + m2_0 + gg] = sm[gg * stride + sw(m1)];
  }
}

size_t colored_noise_ws(int D, int64_t L) { return (size_t)D * (size_t)(L / 2) * sizeof(float2); }

struct NoiseArgs {
  uint32_t k0, k1, step;
  int64_t L;
  float fs, f_lo, sig_scale;
};
template <int LOG>
static cudaError_t run_pass_a(int lg, const NoiseArgs& a, int n1, int D, float2* G, cudaStream_t s);
template <int LOG>
static cudaError_t run_pass_b(int lg, const float2* G, int64_t n, int n2, int D, float* x, cudaStream_t s);

template <int LOG>
static cudaError_t run_pass_a(int lg, const NoiseArgs& a, int n1, int D, float2* G, cudaStream_t s) {
  if constexpr (LOG > 13) {
    return cudaErrorInvalidValue;
  } else {
    if (lg != LOG) return run_pass_a<LOG + 1>(lg, a, n1, D, G, s);
    constexpr int n2 = 1 << LOG;
    const int per = n2 / 8;
    int TK = 1024 / per;
    if (TK > 4) TK = 4;   // small tiles: many blocks for a transform done once per step
    if (TK > n1) TK = n1;
    const size_t smem = (size_t)TK * (n2 + 1) * sizeof(float2);
    cudaError_t e = cudaFuncSetAttribute(k_fourstep_a<LOG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)(n1 / TK), (unsigned)D);
    k_fourstep_a<LOG><<<grid, TK * per, smem, s>>>(a.k0, a.k1, a.step, a.L, a.fs, a.f_lo, a.sig_scale, n1, TK, G);
    return cudaGetLastError();
  }
}

template <int LOG>
static cudaError_t run_pass_b(int lg, const float2* G, int64_t n, int n2, int D, float* x, cudaStream_t s) {
  if constexpr (LOG > 13) {
    return cudaErrorInvalidValue;
  } else {
    if (lg != LOG) return run_pass_b<LOG + 1>(lg, G, n, n2, D, x, s);
    constexpr int n1 = 1 << LOG;
    const int per = n1 / 8;
    int TM = 1024 / per;
    if (TM > 4) TM = 4;
    if (TM > n2) TM = n2;
    const size_t smem = (size_t)TM * (n1 + 1) * sizeof(float2);
    cudaError_t e = cudaFuncSetAttribute(k_fourstep_b<LOG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)(n2 / TM), (unsigned)D);
    k_fourstep_b<LOG><<<grid, TM * per, smem, s>>>(G, n, n2, TM, x);
    return cudaGetLastError();
  }
}

cudaError_t launch_colored_noise(uint64_t seed, uint32_t step, int D, int64_t L, double fs, double f_lo,
                                 float* noise, void* ws, cudaStream_t s) {
  const int64_t n = L / 2;
  int logn = 0;
  while (((int64_t)1 << logn) < n) ++logn;
  const int log1 = logn / 2, log2 = logn - log1;   // n1 <= n2, both >= 2^3 for L >= 1024... checked by caller
  const int n1 = 1 << log1, n2 = 1 << log2;
  float2* G = reinterpret_cast<float2*>(ws);
  const NoiseArgs a{(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32), step, L, (float)fs, (float)f_lo,
                    (float)(sqrt((double)L * fs * 1e-49 / 4.0) / (double)n)};
  cudaError_t e = run_pass_a<3>(log2, a, n1, D, G, s);
  if (e != cudaSuccess) return e;
  return run_pass_b<3>(log1, G, n, n2, D, noise, s);
}

}  // namespace gwx
