// k_resnet.cu -- the pieces of the ResNet-1D data summary of Sec. 4 around its
// convolutions: 1-D convolutions are im2col rows (channels-last activations, all taps of
// all channels per output time) times the weights on the tensor cores
// (gwx_dense_bf16 / gwx_dense_bf16_backward); these kernels build the rows (k_im2col,
// k_im2col_cf for the channels-first input strain), fold row gradients back (k_col2im),
// normalise per sample and channel group (k_gn_stats, k_gn_apply, with the residual
// addition and the ReLU fused) and take the gradient of that (k_gn_bwd_stats,
// k_gn_bwd_apply, k_gn_param_part / k_gn_param_finish, k_relu_mask), and pool (k_maxpool, k_mean_time and
// their backward).
#include <cuda_bf16.h>

#include "gwx_internal.h"

namespace gwx {

namespace {

constexpr float GN_EPS = 1e-5f;

inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// cols[(b To + t) K + j C + c] = x[b][s t + j - p][c] (zero outside the series and for
// columns >= k C); one thread per 8 columns (C % 8 == 0, so a chunk stays in one tap).
__global__ void k_im2col(const __nv_bfloat16* __restrict__ x, int64_t B, int T, int C, int k, int s, int p, int To,
                         int K, __nv_bfloat16* __restrict__ cols) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int ch = K / 8;
  if (i >= B * To * ch) return;
  const int64_t row = i / ch;
  const int q = (int)(i - row * ch);
  const int64_t b = row / To;
  const int t = (int)(row - b * To);
  const int col = 8 * q, j = col / C, c0 = col - j * C;
  uint4 v = make_uint4(0u, 0u, 0u, 0u);
  const int src = s * t + j - p;
  if (j < k && src >= 0 && src < T) v = *reinterpret_cast<const uint4*>(x + ((b * T + src) * C + c0));
  reinterpret_cast<uint4*>(cols + row * K)[q] = v;
}

// The same rows from channels-first FP32 input y [B][D][N] (the whitened strain).
__global__ void k_im2col_cf(const float* __restrict__ y, int64_t B, int D, int N, int k, int s, int p, int To, int K,
                            __nv_bfloat16* __restrict__ cols) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B * To * K) return;
  const int64_t row = i / K;
  const int col = (int)(i - row * K);
  const int64_t b = row / To;
  const int t = (int)(row - b * To);
  float v = 0.f;
  if (col < k * D) {
    const int j = col / D, c = col - j * D, src = s * t + j - p;
    if (src >= 0 && src < N) v = y[(b * D + c) * N + src];
  }
  cols[i] = __float2bfloat16_rn(v);
}

// dx[b][t][c] = (addend) + sum over taps j with s t_out = t + p - j of dcols[b, t_out][j C + c]
__global__ void k_col2im(const float* __restrict__ dcols, int64_t B, int T, int C, int k, int s, int p, int To, int K,
                         const float* __restrict__ addend, float* __restrict__ dx) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B * T * C) return;
  const int64_t bt = i / C;
  const int c = (int)(i - bt * C);
  const int64_t b = bt / T;
  const int t = (int)(bt - b * T);
  float acc = addend ? addend[i] : 0.f;
  for (int j = 0; j < k; ++j) {
    const int num = t + p - j;
    if (num < 0 || num % s) continue;
    const int to = num / s;
    if (to < To) acc += dcols[(b * To + to) * K + j * C + c];
  }
  dx[i] = acc;
}

// Per (sample, group): mean and 1 / sqrt(var + eps) over T x C/G values (FP64 sums).
__global__ void __launch_bounds__(256) k_gn_stats(const float* __restrict__ z, int T, int C, int G,
                                                  float* __restrict__ ms) {
  __shared__ double r1[256], r2[256];
  const int64_t b = blockIdx.x / G;
  const int g = blockIdx.x % G, cg = C / G;
  const int n = T * cg;
  double s1 = 0.0, s2 = 0.0;
  for (int e = threadIdx.x; e < n; e += blockDim.x) {
    const int t = e / cg, c = g * cg + e % cg;
    const double v = z[(b * T + t) * C + c];
    s1 += v;
    s2 += v * v;
  }
  r1[threadIdx.x] = s1;
  r2[threadIdx.x] = s2;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      r1[threadIdx.x] += r1[threadIdx.x + o];
      r2[threadIdx.x] += r2[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double mean = r1[0] / n, var = fmax(r2[0] / n - mean * mean, 0.0);
    ms[2 * blockIdx.x] = (float)mean;
    ms[2 * blockIdx.x + 1] = (float)(1.0 / sqrt(var + (double)GN_EPS));
  }
}

// out = act(gamma_c (z - mean) rstd + beta_c + residual), bfloat16 or FP32 out; residual
// FP32 (res32) or bfloat16 (res16) or none.
__global__ void k_gn_apply(const float* __restrict__ z, int64_t B, int T, int C, int G, const float* __restrict__ ms,
                           const float* __restrict__ gamma, const float* __restrict__ beta,
                           const float* __restrict__ res32, const __nv_bfloat16* __restrict__ res16, int relu,
                           __nv_bfloat16* __restrict__ out16, float* __restrict__ out32) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B * T * C) return;
  const int64_t bt = i / C;
  const int c = (int)(i - bt * C);
  const int64_t b = bt / T;
  const int g = c / (C / G);
  const float mean = ms[2 * (b * G + g)], rstd = ms[2 * (b * G + g) + 1];
  float v = fmaf((z[i] - mean) * rstd, gamma[c], beta[c]);
  if (res32) v += res32[i];
  if (res16) v += __bfloat162float(res16[i]);
  if (relu) v = fmaxf(v, 0.f);
  if (out16) out16[i] = __float2bfloat16_rn(v);
  if (out32) out32[i] = v;
}

// dsum = dy [out > 0]
__global__ void k_relu_mask(const float* __restrict__ dy, const __nv_bfloat16* __restrict__ out, int64_t n,
                            float* __restrict__ d) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) d[i] = __bfloat162float(out[i]) > 0.f ? dy[i] : 0.f;
}

// Per (sample, group): the means of dxh = dy gamma and dxh xhat (FP64 sums).
__global__ void __launch_bounds__(256) k_gn_bwd_stats(const float* __restrict__ dy, const float* __restrict__ z,
                                                      int T, int C, int G, const float* __restrict__ ms,
                                                      const float* __restrict__ gamma, float* __restrict__ mm) {
  __shared__ double r1[256], r2[256];
  const int64_t b = blockIdx.x / G;
  const int g = blockIdx.x % G, cg = C / G;
  const int n = T * cg;
  const float mean = ms[2 * blockIdx.x], rstd = ms[2 * blockIdx.x + 1];
  double s1 = 0.0, s2 = 0.0;
  for (int e = threadIdx.x; e < n; e += blockDim.x) {
    const int t = e / cg, c = g * cg + e % cg;
    const int64_t i = (b * T + t) * C + c;
    const double dxh = (double)dy[i] * gamma[c];
    s1 += dxh;
    s2 += dxh * (double)((z[i] - mean) * rstd);
  }
  r1[threadIdx.x] = s1;
  r2[threadIdx.x] = s2;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      r1[threadIdx.x] += r1[threadIdx.x + o];
      r2[threadIdx.x] += r2[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    mm[2 * blockIdx.x] = (float)(r1[0] / n);
    mm[2 * blockIdx.x + 1] = (float)(r2[0] / n);
  }
}

// dz = rstd (dy gamma - m1 - xhat m2)
__global__ void k_gn_bwd_apply(const float* __restrict__ dy, const float* __restrict__ z, int64_t B, int T, int C,
                               int G, const float* __restrict__ ms, const float* __restrict__ mm,
                               const float* __restrict__ gamma, float* __restrict__ dz) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B * T * C) return;
  const int64_t bt = i / C;
  const int c = (int)(i - bt * C);
  const int64_t bg = (bt / T) * G + c / (C / G);
  const float mean = ms[2 * bg], rstd = ms[2 * bg + 1];
  const float xh = (z[i] - mean) * rstd;
  dz[i] = rstd * (dy[i] * gamma[c] - mm[2 * bg] - xh * mm[2 * bg + 1]);
}

// dgamma_c = sum dy xhat, dbeta_c = sum dy over samples and times, in two deterministic
// passes: block (channel tile of 32, row slice) sums its slice (8 row lanes, FP64) into
// part[slice][c][2]; k_gn_param_finish adds the slices.
constexpr int GN_SLICES = 64;

__global__ void __launch_bounds__(256) k_gn_param_part(const float* __restrict__ dy, const float* __restrict__ z,
                                                       int64_t rows, int T, int C, int G,
                                                       const float* __restrict__ ms, double* __restrict__ part) {
  __shared__ double a[8][33], bb[8][33];
  const int cx = threadIdx.x & 31, ry = threadIdx.x >> 5;
  const int c = blockIdx.x * 32 + cx;
  const int64_t per = (rows + GN_SLICES - 1) / GN_SLICES;
  const int64_t r0 = blockIdx.y * per, r1 = min(rows, r0 + per);
  double sg = 0.0, sb = 0.0;
  if (c < C)
    for (int64_t r = r0 + ry; r < r1; r += 8) {
      const int64_t i = r * C + c;
      const int64_t bg = (r / T) * G + c / (C / G);
      const double xh = (double)((z[i] - ms[2 * bg]) * ms[2 * bg + 1]);
      sg += (double)dy[i] * xh;
      sb += (double)dy[i];
    }
  a[ry][cx] = sg;
  bb[ry][cx] = sb;
  __syncthreads();
  if (ry == 0 && c < C) {
    double tg = 0.0, tb = 0.0;
    for (int k = 0; k < 8; ++k) {
      tg += a[k][cx];
      tb += bb[k][cx];
    }
    part[((int64_t)blockIdx.y * C + c) * 2] = tg;
    part[((int64_t)blockIdx.y * C + c) * 2 + 1] = tb;
  }
}

__global__ void k_gn_param_finish(const double* __restrict__ part, int C, float* __restrict__ dgamma,
                                  float* __restrict__ dbeta) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= C) return;
  double tg = 0.0, tb = 0.0;
  for (int s = 0; s < GN_SLICES; ++s) {
    tg += part[((int64_t)s * C + c) * 2];
    tb += part[((int64_t)s * C + c) * 2 + 1];
  }
  dgamma[c] = (float)tg;
  dbeta[c] = (float)tb;
}

// k 3, s 2, p 1 max pool over time (first maximum of a window), and its backward.
__global__ void k_maxpool(const __nv_bfloat16* __restrict__ x, int64_t B, int T, int C, int To,
                          __nv_bfloat16* __restrict__ y, uint8_t* __restrict__ arg) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B * To * C) return;
  const int64_t bt = i / C;
  const int c = (int)(i - bt * C);
  const int64_t b = bt / To;
  const int t = (int)(bt - b * To);
  float best = -INFINITY;
  int a = 0;
  for (int j = 0; j < 3; ++j) {
    const int src = 2 * t + j - 1;
    if (src < 0 || src >= T) continue;
    const float v = __bfloat162float(x[(b * T + src) * C + c]);
    if (v > best) {
      best = v;
      a = j;
    }
  }
  y[i] = __float2bfloat16_rn(best);
  arg[i] = (uint8_t)a;
}

__global__ void k_maxpool_back(const float* __restrict__ dy, const uint8_t* __restrict__ arg, int64_t B, int T, int C,
                               int To, float* __restrict__ dx) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B * T * C) return;
  const int64_t bt = i / C;
  const int c = (int)(i - bt * C);
  const int64_t b = bt / T;
  const int t = (int)(bt - b * T);
  float acc = 0.f;
  for (int to = t / 2; to <= (t + 1) / 2; ++to) {
    if (to >= To) continue;
    const int64_t o = (b * To + to) * C + c;
    if (2 * to - 1 + (int)arg[o] == t) acc += dy[o];
  }
  dx[i] = acc;
}

__global__ void k_mean_time(const __nv_bfloat16* __restrict__ x, int64_t B, int T, int C,
                            __nv_bfloat16* __restrict__ m) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B * C) return;
  const int64_t b = i / C;
  const int c = (int)(i - b * C);
  float acc = 0.f;
  for (int t = 0; t < T; ++t) acc += __bfloat162float(x[(b * T + t) * C + c]);
  m[i] = __float2bfloat16_rn(acc / T);
}

__global__ void k_mean_time_back(const float* __restrict__ dm, int64_t B, int T, int C, float* __restrict__ dx) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B * T * C) return;
  const int64_t b = i / ((int64_t)T * C);
  const int c = (int)(i % C);
  dx[i] = dm[b * C + c] / T;
}

}  // namespace

cudaError_t launch_im2col(const void* x, int64_t B, int T, int C, int k, int s, int p, int K, void* cols,
                          cudaStream_t st) {
  const int To = (T + 2 * p - k) / s + 1;
  k_im2col<<<nblk(B * To * (K / 8), 256), 256, 0, st>>>(reinterpret_cast<const __nv_bfloat16*>(x), B, T, C, k, s, p,
                                                        To, K, reinterpret_cast<__nv_bfloat16*>(cols));
  return cudaGetLastError();
}

cudaError_t launch_im2col_cf(const float* y, int64_t B, int D, int N, int k, int s, int p, int K, void* cols,
                             cudaStream_t st) {
  const int To = (N + 2 * p - k) / s + 1;
  k_im2col_cf<<<nblk(B * To * K, 256), 256, 0, st>>>(y, B, D, N, k, s, p, To, K,
                                                     reinterpret_cast<__nv_bfloat16*>(cols));
  return cudaGetLastError();
}

cudaError_t launch_col2im(const float* dcols, int64_t B, int T, int C, int k, int s, int p, int K, const float* addend,
                          float* dx, cudaStream_t st) {
  const int To = (T + 2 * p - k) / s + 1;
  k_col2im<<<nblk(B * T * C, 256), 256, 0, st>>>(dcols, B, T, C, k, s, p, To, K, addend, dx);
  return cudaGetLastError();
}

cudaError_t launch_group_norm(const float* z, int64_t B, int T, int C, int G, const float* gamma, const float* beta,
                              const float* res32, const void* res16, int relu, void* out16, float* out32, float* ms,
                              cudaStream_t st) {
  k_gn_stats<<<(unsigned)(B * G), 256, 0, st>>>(z, T, C, G, ms);
  k_gn_apply<<<nblk(B * T * C, 256), 256, 0, st>>>(z, B, T, C, G, ms, gamma, beta, res32,
                                                   reinterpret_cast<const __nv_bfloat16*>(res16), relu,
                                                   reinterpret_cast<__nv_bfloat16*>(out16), out32);
  return cudaGetLastError();
}

size_t group_norm_backward_scratch(int64_t B, int C, int G) {
  return (size_t)B * G * 2 * sizeof(float) + 256 + (size_t)GN_SLICES * C * 2 * sizeof(double);
}

cudaError_t launch_group_norm_backward(const float* dy, const float* z, int64_t B, int T, int C, int G,
                                       const float* ms, const float* gamma, void* scratch, float* dz, float* dgamma,
                                       float* dbeta, cudaStream_t st) {
  float* mm = reinterpret_cast<float*>(scratch);
  double* part = reinterpret_cast<double*>(reinterpret_cast<char*>(scratch) +
                                           (((size_t)B * G * 2 * sizeof(float) + 255) & ~(size_t)255));
  k_gn_bwd_stats<<<(unsigned)(B * G), 256, 0, st>>>(dy, z, T, C, G, ms, gamma, mm);
  k_gn_bwd_apply<<<nblk(B * T * C, 256), 256, 0, st>>>(dy, z, B, T, C, G, ms, mm, gamma, dz);
  k_gn_param_part<<<dim3(nblk(C, 32), GN_SLICES), 256, 0, st>>>(dy, z, B * T, T, C, G, ms, part);
  k_gn_param_finish<<<nblk(C, 128), 128, 0, st>>>(part, C, dgamma, dbeta);
  return cudaGetLastError();
}

cudaError_t launch_relu_mask(const float* dy, const void* out, int64_t n, float* d, cudaStream_t st) {
  k_relu_mask<<<nblk(n, 256), 256, 0, st>>>(dy, reinterpret_cast<const __nv_bfloat16*>(out), n, d);
  return cudaGetLastError();
}

cudaError_t launch_maxpool(const void* x, int64_t B, int T, int C, void* y, uint8_t* arg, cudaStream_t st) {
  const int To = (T + 2 - 3) / 2 + 1;
  k_maxpool<<<nblk(B * To * C, 256), 256, 0, st>>>(reinterpret_cast<const __nv_bfloat16*>(x), B, T, C, To,
                                                   reinterpret_cast<__nv_bfloat16*>(y), arg);
  return cudaGetLastError();
}

cudaError_t launch_maxpool_back(const float* dy, const uint8_t* arg, int64_t B, int T, int C, float* dx,
                                cudaStream_t st) {
  const int To = (T + 2 - 3) / 2 + 1;
  k_maxpool_back<<<nblk(B * T * C, 256), 256, 0, st>>>(dy, arg, B, T, C, To, dx);
  return cudaGetLastError();
}

cudaError_t launch_mean_time(const void* x, int64_t B, int T, int C, void* m, cudaStream_t st) {
  k_mean_time<<<nblk(B * C, 256), 256, 0, st>>>(reinterpret_cast<const __nv_bfloat16*>(x), B, T, C,
                                                reinterpret_cast<__nv_bfloat16*>(m));
  return cudaGetLastError();
}

cudaError_t launch_mean_time_back(const float* dm, int64_t B, int T, int C, float* dx, cudaStream_t st) {
  k_mean_time_back<<<nblk(B * T * C, 256), 256, 0, st>>>(dm, B, T, C, dx);
  return cudaGetLastError();
}

}  // namespace gwx
