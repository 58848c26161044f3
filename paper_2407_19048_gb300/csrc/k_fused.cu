// k_fused.cu -- the per-batch pass of Sec. 3.2 fused per draw: for each draw b and
// detector d,
//   y[b][d] = irfft( (rfft(noise[d][off_b : off_b + N]) + fs h_d(theta_b)) W_d )
// which equals whiten(inject(...)) because the injection is linear.  One block per
// draw (persistent over draws): the D windows live in shared memory as n = N/2
// complex points each; the waveform of a bin is evaluated once and projected onto
// all D detectors, so the frequency-domain stage costs one phase/amplitude
// evaluation per bin plus one complex exponential per detector.
#include "waveform.cuh"

namespace gwx {

cudaError_t init_tables_fused() { return fill_tables_for_this_tu(); }

// Frequency-domain step of one bin pair (k, n-k), 0 < k < n/2, for every detector:
// unpack the real spectra, add the projected waveform, whiten, repack.
__device__ __forceinline__ void fd_pair(float2* sm, int n, int D, int k, const DrawCoef& c, int k_lo,
                                        const float* __restrict__ W, int64_t F, float inv_n, int logN) {
  const int nk = n - k;
  const float2 wk = pack_twiddle(k, logN);
  float ak = 0.f, tk = 0.f, ank = 0.f, tnk = 0.f;
  if (k >= k_lo && k <= c.kcut) tk = waveform_turns(c, k, ak);
  if (nk != k && nk >= k_lo && nk <= c.kcut) tnk = waveform_turns(c, nk, ank);
  for (int d = 0; d < D; ++d) {
    float2* z = sm + d * n;
    float2 xk, xnk;
    unpack_pair(z[sw(k)], z[sw(nk)], wk, xk, xnk);
    const float2 gd = make_float2(c.g[d].x, c.g[d].z);
    if (ak != 0.f) xk = cadd(xk, cscale(cmul(gd, expm2pi(tk + lin_turns(c.nu[d], k))), ak));
    if (ank != 0.f) xnk = cadd(xnk, cscale(cmul(gd, expm2pi(tnk + lin_turns(c.nu[d], nk))), ank));
    const float* Wd = W + (int64_t)d * F;
    float2 zk, znk;
    pack_pair(cscale(xk, __ldg(&Wd[k]) * inv_n), cscale(xnk, __ldg(&Wd[nk]) * inv_n), wk, zk, znk);
    z[sw(k)] = zk;
    if (nk != k) z[sw(nk)] = znk;
  }
}

template <int LOGN>
__global__ void __launch_bounds__((1 << LOGN) / 8, LOGN >= 13 ? 1 : 2)
    k_simulate(const DrawCoef* __restrict__ coef, const float* __restrict__ noise, int64_t L,
               const int64_t* __restrict__ offsets, const float* __restrict__ W, int k_lo, int D, int64_t B,
               float* __restrict__ y) {
  constexpr int n = 1 << LOGN;
  constexpr int64_t N = 2 * n;
  constexpr int64_t F = n + 1;
  constexpr int NT = n / 8;
  extern __shared__ float2 sm[];
  __shared__ DrawCoef sc;
  const int t = threadIdx.x;
  const float inv_n = 1.0f / (float)n;
  for (int64_t b = blockIdx.x; b < B; b += gridDim.x) {
    if (t < (int)(sizeof(DrawCoef) / 16))
      reinterpret_cast<int4*>(&sc)[t] = __ldg(reinterpret_cast<const int4*>(coef + b) + t);
    int64_t off = __ldg(&offsets[b]);
    off = off < 0 ? 0 : (off > L - N ? L - N : off);   // keep a bad offset inside the stretch
    // Crop: aligned float2 loads of (x[a + 2m], x[a + 2m + 1]) with a = off rounded
    // down to even; for an odd offset each value pair is (own .y, next lane's .x).
    const int64_t a = off & ~(int64_t)1;
    const bool odd = (off & 1) != 0;
    const int lane = t & 31;
    for (int d = 0; d < D; ++d) {
      const float* row = noise + (int64_t)d * L + a;
      const float2* row2 = reinterpret_cast<const float2*>(row);
      float2* z = sm + d * n;
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int m = t + i * NT;
        const float2 p = __ldg(&row2[m]);
        float2 v = p;
        if (odd) {
          float nx;
          if constexpr (NT >= 32) {   // full warps: the next pair comes from lane + 1
            nx = __shfl_down_sync(0xffffffffu, p.x, 1);
            if (lane == 31) nx = __ldg(&row[2 * m + 2]);
          } else {
            nx = __ldg(&row[2 * m + 2]);
          }
          v = make_float2(p.y, nx);
        }
        z[sw(m)] = v;
      }
    }
    __syncthreads();
    for (int d = 0; d < D; ++d) fft_smem<LOGN, false>(sm + d * n, t);
    const DrawCoef& c = sc;
#pragma unroll 1
    for (int i = 0; i < 4; ++i) {
      const int k = t + i * NT;
      if (k == 0) {   // DC and Nyquist: real parts, both outside the whitening band in practice
        for (int d = 0; d < D; ++d) {
          const float2 z0 = sm[d * n];
          const float* Wd = W + (int64_t)d * F;
          const float y0 = (z0.x + z0.y) * __ldg(&Wd[0]) * inv_n, yn = (z0.x - z0.y) * __ldg(&Wd[n]) * inv_n;
          sm[d * n] = make_float2(0.5f * (y0 + yn), 0.5f * (y0 - yn));
        }
      } else {
        fd_pair(sm, n, D, k, c, k_lo, W, F, inv_n, LOGN + 1);
      }
    }
    if (t == 0) fd_pair(sm, n, D, n / 2, c, k_lo, W, F, inv_n, LOGN + 1);
    __syncthreads();
    for (int d = 0; d < D; ++d) fft_smem<LOGN, true>(sm + d * n, t);
    for (int d = 0; d < D; ++d) {
      float2* out = reinterpret_cast<float2*>(y + (b * D + d) * N);
      const float2* z = sm + d * n;
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int m = t + i * NT;
        __stcs(&out[m], z[sw(m)]);
      }
    }
    __syncthreads();
  }
}

cudaError_t launch_simulate_fused(const DrawCoef* coef, const float* noise, int64_t L, const int64_t* offsets,
                                  const float* W, int k_lo, int D, int64_t B, int64_t N, double fs, float* y,
                                  cudaStream_t s) {
  if (B <= 0) return cudaSuccess;
  return dispatch_log<4, 13>(ilog2_exact(N / 2), [&](auto cst) {
    constexpr int LG = decltype(cst)::value;
    constexpr int NT = (1 << LG) / 8;
    const size_t smem = (size_t)D * (1 << LG) * sizeof(float2);
    cudaError_t e = cudaFuncSetAttribute(k_simulate<LG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_simulate<LG>, NT, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    int64_t grid = (int64_t)sms * per_sm;
    if (grid > B) grid = B;
    k_simulate<LG><<<(unsigned)grid, NT, smem, s>>>(coef, noise, L, offsets, W, k_lo, D, B, y);
    return cudaGetLastError();
  });
}

}  // namespace gwx
