// k_resnet.cu -- the pieces of the ResNet-1D data summary of Sec. 4 around its
// convolutions: 1-D convolutions are im2col rows (channels-last activations, all taps of
// all channels per output time) times the weights on the tensor cores
// (gwx_dense_bf16 / gwx_dense_bf16_backward); these kernels build the rows (k_im2col,
// k_im2col_cf for the channels-first input strain), fold row gradients back (k_col2im),
// normalise per sample and channel group (k_gn_stats, k_gn_apply, with the residual
// addition and the ReLU fused) and take the gradient of that (k_gn_bwd_stats,
// k_gn_bwd_apply, k_gn_param_part / k_gn_param_finish, k_relu_mask), and pool (k_maxpool, k_mean_time and
// their backward).
#include <stdint.h>

#include <algorithm>

#include <cuda_bf16.h>

#include "gwx_internal.h"

namespace gwx {

namespace {

constexpr float GN_EPS = 1e-5f;

inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// Index arithmetic: every kernel runs on a grid whose y coordinate is the sample b and
// whose x threads cover one sample's elements, so the divisions below are 32-bit (the
// C-ABI keeps T C below 2^31 and B below 65536); sums are FP32 per thread over a few
// dozen terms and FP64 across threads (GB300's FP64 rate is a small fraction of FP32).

// cols[(b To + t) K + j C + c] = x[b][s t + j - p][c] (zero outside the series and for
// columns >= k C); one thread per 8 columns (C % 8 == 0, so a chunk stays in one tap).
__global__ void k_im2col(const __nv_bfloat16* __restrict__ x, int T, int C, int k, int s, int p, int To, int K,
                         __nv_bfloat16* __restrict__ cols) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int ch = K / 8;
  if (i >= To * ch) return;
  const int64_t b = blockIdx.y;
  const int t = i / ch, q = i - t * ch;
  const int col = 8 * q, j = col / C, c0 = col - j * C;
  uint4 v = make_uint4(0u, 0u, 0u, 0u);
  const int src = s * t + j - p;
  if (j < k && src >= 0 && src < T) v = *reinterpret_cast<const uint4*>(x + ((b * T + src) * C + c0));
  reinterpret_cast<uint4*>(cols + (b * To + t) * K)[q] = v;
}

// The same rows from channels-first FP32 input y [B][D][N] (the whitened strain).
__global__ void k_im2col_cf(const float* __restrict__ y, int D, int N, int k, int s, int p, int To, int K,
                            __nv_bfloat16* __restrict__ cols) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= To * K) return;
  const int64_t b = blockIdx.y;
  const int t = i / K, col = i - t * K;
  float v = 0.f;
  if (col < k * D) {
    const int j = col / D, c = col - j * D, src = s * t + j - p;
    if (src >= 0 && src < N) v = y[(b * D + c) * N + src];
  }
  cols[(b * To + t) * K + col] = __float2bfloat16_rn(v);
}

// dx[b][t][c] = (addend) + sum over taps j with s t_out = t + p - j of dcols[b, t_out][j C + c]
__global__ void k_col2im(const float* __restrict__ dcols, int T, int C, int k, int s, int p, int To, int K,
                         const float* __restrict__ addend, float* __restrict__ dx) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= T * C) return;
  const int64_t b = blockIdx.y;
  const int t = i / C, c = i - t * C;
  const int64_t o = b * T * C + i;
  float acc = addend ? addend[o] : 0.f;
  for (int j = 0; j < k; ++j) {
    const int num = t + p - j;
    if (num < 0 || num % s) continue;
    const int to = num / s;
    if (to < To) acc += dcols[(b * To + to) * K + j * C + c];
  }
  dx[o] = acc;
}

// The same with KT taps known at compile time and four channels per thread: all taps'
// float4 loads are issued before the sums (in tap order, as above).
template <int KT>
__global__ void k_col2im4(const float* __restrict__ dcols, int T, int C, int s, int p, int To, int K,
                          const float* __restrict__ addend, float* __restrict__ dx) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= T * C / 4) return;
  const int64_t b = blockIdx.y;
  const int t = (4 * i) / C, c = 4 * i - t * C;
  float4 v[KT];
#pragma unroll
  for (int j = 0; j < KT; ++j) {
    const int num = t + p - j;
    const int to = num / s;
    v[j] = (num >= 0 && num - to * s == 0 && to < To)
               ? __ldg(reinterpret_cast<const float4*>(dcols + (b * To + to) * K + j * C + c))
               : make_float4(0.f, 0.f, 0.f, 0.f);
  }
  const int64_t o = b * T * C + 4 * (int64_t)i;
  float4 acc = addend ? *reinterpret_cast<const float4*>(addend + o) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
  for (int j = 0; j < KT; ++j) {
    acc.x += v[j].x;
    acc.y += v[j].y;
    acc.z += v[j].z;
    acc.w += v[j].w;
  }
  *reinterpret_cast<float4*>(dx + o) = acc;
}

// Block sums of two FP32 per-thread partials in FP64 (warp shuffles, then the warps in
// order); the totals land in thread 0.
__device__ __forceinline__ void block_sum2(double& a, double& b2) {
  __shared__ double r[2][32];
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b2 += __shfl_down_sync(0xffffffffu, b2, o);
  }
  const int w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  if ((threadIdx.x & 31) == 0) {
    r[0][w] = a;
    r[1][w] = b2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    a = 0.0;
    b2 = 0.0;
    for (int k = 0; k < nw; ++k) {
      a += r[0][k];
      b2 += r[1][k];
    }
  }
}

// Per (sample, group): mean and 1 / sqrt(var + eps) over T x C/G values.  The values are
// shifted by the group's first value before squaring, so the FP32 partial sums do not
// cancel when the mean is large against the spread.  VEC values per load (4 when C/G is a
// multiple of 4).
template <int VEC>
__global__ void __launch_bounds__(256) k_gn_stats(const float* __restrict__ z, int T, int C, int G,
                                                  float* __restrict__ ms) {
  const int b = blockIdx.x / G, g = blockIdx.x - (blockIdx.x / G) * G, cg = C / G, cv = cg / VEC;
  const float* zb = z + (int64_t)b * T * C + g * cg;
  const float k0 = __ldg(zb);
  float s1 = 0.f, s2 = 0.f;
#pragma unroll 4
  for (int e = threadIdx.x; e < T * cv; e += blockDim.x) {
    const int t = e / cv, c = (e - t * cv) * VEC;
    if constexpr (VEC == 4) {
      const float4 v = __ldg(reinterpret_cast<const float4*>(zb + (int64_t)t * C + c));
      const float d0 = v.x - k0, d1 = v.y - k0, d2 = v.z - k0, d3 = v.w - k0;
      s1 += (d0 + d1) + (d2 + d3);
      s2 += (d0 * d0 + d1 * d1) + (d2 * d2 + d3 * d3);
    } else {
      const float d = __ldg(zb + (int64_t)t * C + c) - k0;
      s1 += d;
      s2 += d * d;
    }
  }
  double a = s1, q = s2;
  block_sum2(a, q);
  if (threadIdx.x == 0) {
    const double n = (double)T * cg, m = a / n, var = fmax(q / n - m * m, 0.0);
    ms[2 * blockIdx.x] = (float)((double)k0 + m);
    ms[2 * blockIdx.x + 1] = (float)(1.0 / sqrt(var + (double)GN_EPS));
  }
}

// Per-sample variants of the two statistics kernels for C / 4 dividing 256: one block of
// 256 threads reads sample b's whole [T][C] slab with coalesced float4 loads (thread
// (row lane l, column quad q) reads rows l, l + 256 / (C / 4), ... of channels 4 q ..
// 4 q + 3), FP32 sums over runs of 16 rows added into FP64; then the row lanes of each
// column quad and the column quads of each group are added in order.
__device__ __forceinline__ void sample_group_sums(double a, double q, int cq, int rl, int cg, int G, double* out) {
  __shared__ double r1[256], r2[256];
  const int tid = threadIdx.x;
  r1[tid] = a;
  r2[tid] = q;
  __syncthreads();
  if (tid < cq) {
    double x = 0.0, y = 0.0;
    for (int l = 0; l < rl; ++l) {
      x += r1[l * cq + tid];
      y += r2[l * cq + tid];
    }
    r1[tid] = x;
    r2[tid] = y;
  }
  __syncthreads();
  if (tid < G) {
    double x = 0.0, y = 0.0;
    for (int k = tid * (cg / 4); k < (tid + 1) * (cg / 4); ++k) {
      x += r1[k];
      y += r2[k];
    }
    out[2 * tid] = x;
    out[2 * tid + 1] = y;
  }
}

__global__ void __launch_bounds__(256) k_gn_stats_s(const float* __restrict__ z, int T, int C, int G,
                                                    float* __restrict__ ms) {
  __shared__ double sums[64];
  const int cq = C / 4, rl = 256 / cq, cg = C / G;
  const int q4 = threadIdx.x % cq, l0 = threadIdx.x / cq;
  const float* zb = z + (int64_t)blockIdx.x * T * C;
  const float k0 = __ldg(zb + ((4 * q4) / cg) * cg);
  double a = 0.0, q = 0.0;
  for (int t0 = l0; t0 < T; t0 += 16 * rl) {
    float s1 = 0.f, s2 = 0.f;
#pragma unroll 4
    for (int t = t0; t < min(T, t0 + 16 * rl); t += rl) {
      const float4 v = __ldg(reinterpret_cast<const float4*>(zb + (int64_t)t * C) + q4);
      const float d0 = v.x - k0, d1 = v.y - k0, d2 = v.z - k0, d3 = v.w - k0;
      s1 += (d0 + d1) + (d2 + d3);
      s2 += (d0 * d0 + d1 * d1) + (d2 * d2 + d3 * d3);
    }
    a += s1;
    q += s2;
  }
  sample_group_sums(a, q, cq, rl, cg, G, sums);
  if ((int)threadIdx.x < G) {
    const int g = threadIdx.x;
    const double n = (double)T * cg, m = sums[2 * g] / n, var = fmax(sums[2 * g + 1] / n - m * m, 0.0);
    ms[2 * ((int64_t)blockIdx.x * G + g)] = (float)((double)__ldg(zb + g * cg) + m);
    ms[2 * ((int64_t)blockIdx.x * G + g) + 1] = (float)(1.0 / sqrt(var + (double)GN_EPS));
  }
}

// part (optional, [B][C][2] doubles): this sample's sums of dy xhat and dy per channel (FP32
// over runs of at most 16 rows, FP64 across runs and, in a fixed order, across the threads
// that share the channels), the partials of dgamma and dbeta that k_gn_param_finish adds.
__global__ void __launch_bounds__(256, 4) k_gn_bwd_stats_s(const float* __restrict__ dy, const float* __restrict__ z,
                                                        int T, int C, int G, const float* __restrict__ ms,
                                                        const float* __restrict__ gamma, float* __restrict__ mm,
                                                        double* __restrict__ part) {
  __shared__ double sums[64];
  __shared__ double pr[256 * 8];
  const int cq = C / 4, rl = 256 / cq, cg = C / G;
  const int q4 = threadIdx.x % cq, l0 = threadIdx.x / cq, g = (4 * q4) / cg;
  const int64_t off = (int64_t)blockIdx.x * T * C;
  const float mean = ms[2 * ((int64_t)blockIdx.x * G + g)], rstd = ms[2 * ((int64_t)blockIdx.x * G + g) + 1];
  const float4 gm = make_float4(__ldg(&gamma[4 * q4]), __ldg(&gamma[4 * q4 + 1]), __ldg(&gamma[4 * q4 + 2]),
                                __ldg(&gamma[4 * q4 + 3]));
  double a = 0.0, q = 0.0;
  double pg[4] = {0.0, 0.0, 0.0, 0.0}, pb[4] = {0.0, 0.0, 0.0, 0.0};
  for (int t0 = l0; t0 < T; t0 += 16 * rl) {
    float s1 = 0.f, s2 = 0.f;
    float fg[4] = {0.f, 0.f, 0.f, 0.f}, fb[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 4
    for (int t = t0; t < min(T, t0 + 16 * rl); t += rl) {
      const float4 d = __ldg(reinterpret_cast<const float4*>(dy + off + (int64_t)t * C) + q4);
      const float4 x = __ldg(reinterpret_cast<const float4*>(z + off + (int64_t)t * C) + q4);
      const float a0 = d.x * gm.x, a1 = d.y * gm.y, a2 = d.z * gm.z, a3 = d.w * gm.w;
      const float h0 = (x.x - mean) * rstd, h1 = (x.y - mean) * rstd, h2 = (x.z - mean) * rstd,
                  h3 = (x.w - mean) * rstd;
      s1 += (a0 + a1) + (a2 + a3);
      s2 += (a0 * h0 + a1 * h1) + (a2 * h2 + a3 * h3);
      if (part) {
        fg[0] += d.x * h0;
        fg[1] += d.y * h1;
        fg[2] += d.z * h2;
        fg[3] += d.w * h3;
        fb[0] += d.x;
        fb[1] += d.y;
        fb[2] += d.z;
        fb[3] += d.w;
      }
    }
    a += s1;
    q += s2;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      pg[m] += fg[m];
      pb[m] += fb[m];
    }
  }
  sample_group_sums(a, q, cq, rl, cg, G, sums);
  if ((int)threadIdx.x < G) {
    const double n = (double)T * cg;
    mm[2 * ((int64_t)blockIdx.x * G + threadIdx.x)] = (float)(sums[2 * threadIdx.x] / n);
    mm[2 * ((int64_t)blockIdx.x * G + threadIdx.x) + 1] = (float)(sums[2 * threadIdx.x + 1] / n);
  }
  if (part) {
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      pr[threadIdx.x * 8 + m] = pg[m];
      pr[threadIdx.x * 8 + 4 + m] = pb[m];
    }
    __syncthreads();
    // thread tid < C: channel tid, summed over the rl threads l = 0 .. rl-1 in order
    for (int c = threadIdx.x; c < C; c += blockDim.x) {
      const int qq = c / 4, m = c % 4;
      double sg = 0.0, sb = 0.0;
      for (int l = 0; l < rl; ++l) {
        sg += pr[(l * cq + qq) * 8 + m];
        sb += pr[(l * cq + qq) * 8 + 4 + m];
      }
      part[((int64_t)blockIdx.x * C + c) * 2] = sg;
      part[((int64_t)blockIdx.x * C + c) * 2 + 1] = sb;
    }
  }
}

// out = act(gamma_c (z - mean) rstd + beta_c + residual), bfloat16 or FP32 out; residual
// FP32 (res32) or bfloat16 (res16) or none.  VEC consecutive channels per thread.
template <int VEC>
__global__ void k_gn_apply(const float* __restrict__ z, int T, int C, int G, const float* __restrict__ ms,
                           const float* __restrict__ gamma, const float* __restrict__ beta,
                           const float* __restrict__ res32, const __nv_bfloat16* __restrict__ res16, int relu,
                           __nv_bfloat16* __restrict__ out16, float* __restrict__ out32) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= T * C / VEC) return;
  const int b = blockIdx.y;
  const int c = (j * VEC) % C, g = c / (C / G);
  const int64_t i = (int64_t)b * T * C + (int64_t)j * VEC;
  const float mean = ms[2 * (b * G + g)], rstd = ms[2 * (b * G + g) + 1];
  float v[VEC];
  if constexpr (VEC == 4) {
    const float4 q = *reinterpret_cast<const float4*>(z + i);
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
  } else {
    v[0] = z[i];
  }
#pragma unroll
  for (int u = 0; u < VEC; ++u) v[u] = fmaf((v[u] - mean) * rstd, __ldg(&gamma[c + u]), __ldg(&beta[c + u]));
  if (res32) {
    if constexpr (VEC == 4) {
      const float4 q = *reinterpret_cast<const float4*>(res32 + i);
      v[0] += q.x; v[1] += q.y; v[2] += q.z; v[3] += q.w;
    } else {
      v[0] += res32[i];
    }
  }
  if (res16) {
    if constexpr (VEC == 4) {
      const uint2 q = *reinterpret_cast<const uint2*>(res16 + i);
      const float2 lo = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&q.x));
      const float2 hi = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&q.y));
      v[0] += lo.x; v[1] += lo.y; v[2] += hi.x; v[3] += hi.y;
    } else {
      v[0] += __bfloat162float(res16[i]);
    }
  }
  if (relu) {
#pragma unroll
    for (int u = 0; u < VEC; ++u) v[u] = fmaxf(v[u], 0.f);
  }
  if constexpr (VEC == 4) {
    if (out16) {
      __nv_bfloat162 lo = __floats2bfloat162_rn(v[0], v[1]), hi = __floats2bfloat162_rn(v[2], v[3]);
      uint2 q;
      q.x = *reinterpret_cast<uint32_t*>(&lo);
      q.y = *reinterpret_cast<uint32_t*>(&hi);
      *reinterpret_cast<uint2*>(out16 + i) = q;
    }
    if (out32) *reinterpret_cast<float4*>(out32 + i) = make_float4(v[0], v[1], v[2], v[3]);
  } else {
    if (out16) out16[i] = __float2bfloat16_rn(v[0]);
    if (out32) out32[i] = v[0];
  }
}

// dsum = dy [out > 0]
__global__ void k_relu_mask(const float* __restrict__ dy, const __nv_bfloat16* __restrict__ out, int64_t n,
                            float* __restrict__ d) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) d[i] = __bfloat162float(out[i]) > 0.f ? dy[i] : 0.f;
}

// The same, four elements per thread (n4 = n / 4 groups).
__global__ void k_relu_mask4(const float* __restrict__ dy, const __nv_bfloat16* __restrict__ out, int64_t n4,
                             float* __restrict__ d) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n4) return;
  const float4 g = __ldg(reinterpret_cast<const float4*>(dy) + i);
  const uint2 q = __ldg(reinterpret_cast<const uint2*>(out) + i);
  const float2 lo = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&q.x));
  const float2 hi = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&q.y));
  reinterpret_cast<float4*>(d)[i] = make_float4(lo.x > 0.f ? g.x : 0.f, lo.y > 0.f ? g.y : 0.f,
                                                hi.x > 0.f ? g.z : 0.f, hi.y > 0.f ? g.w : 0.f);
}

// Per (sample, group): the means of dxh = dy gamma and dxh xhat.
template <int VEC>
__global__ void __launch_bounds__(256) k_gn_bwd_stats(const float* __restrict__ dy, const float* __restrict__ z,
                                                      int T, int C, int G, const float* __restrict__ ms,
                                                      const float* __restrict__ gamma, float* __restrict__ mm) {
  const int b = blockIdx.x / G, g = blockIdx.x - (blockIdx.x / G) * G, cg = C / G, cv = cg / VEC;
  const int64_t base = (int64_t)b * T * C + g * cg;
  const float mean = ms[2 * blockIdx.x], rstd = ms[2 * blockIdx.x + 1];
  float s1 = 0.f, s2 = 0.f;
#pragma unroll 4
  for (int e = threadIdx.x; e < T * cv; e += blockDim.x) {
    const int t = e / cv, c = (e - t * cv) * VEC;
    const int64_t i = base + (int64_t)t * C + c;
    if constexpr (VEC == 4) {
      const float4 d = __ldg(reinterpret_cast<const float4*>(dy + i));
      const float4 x = __ldg(reinterpret_cast<const float4*>(z + i));
      const float4 gm = make_float4(__ldg(&gamma[g * cg + c]), __ldg(&gamma[g * cg + c + 1]),
                                    __ldg(&gamma[g * cg + c + 2]), __ldg(&gamma[g * cg + c + 3]));
      const float a0 = d.x * gm.x, a1 = d.y * gm.y, a2 = d.z * gm.z, a3 = d.w * gm.w;
      s1 += (a0 + a1) + (a2 + a3);
      s2 += (a0 * ((x.x - mean) * rstd) + a1 * ((x.y - mean) * rstd)) +
            (a2 * ((x.z - mean) * rstd) + a3 * ((x.w - mean) * rstd));
    } else {
      const float a = __ldg(dy + i) * __ldg(&gamma[g * cg + c]);
      s1 += a;
      s2 += a * ((__ldg(z + i) - mean) * rstd);
    }
  }
  double a = s1, q = s2;
  block_sum2(a, q);
  if (threadIdx.x == 0) {
    const double n = (double)T * cg;
    mm[2 * blockIdx.x] = (float)(a / n);
    mm[2 * blockIdx.x + 1] = (float)(q / n);
  }
}

// dz = rstd (dy gamma - m1 - xhat m2)
template <int VEC>
__global__ void k_gn_bwd_apply(const float* __restrict__ dy, const float* __restrict__ z, int T, int C, int G,
                               const float* __restrict__ ms, const float* __restrict__ mm,
                               const float* __restrict__ gamma, float* __restrict__ dz) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= T * C / VEC) return;
  const int b = blockIdx.y;
  const int c = (j * VEC) % C, bg = b * G + c / (C / G);
  const int64_t i = (int64_t)b * T * C + (int64_t)j * VEC;
  const float mean = ms[2 * bg], rstd = ms[2 * bg + 1], m1 = mm[2 * bg], m2 = mm[2 * bg + 1];
  if constexpr (VEC == 4) {
    const float4 d = *reinterpret_cast<const float4*>(dy + i);
    const float4 x = *reinterpret_cast<const float4*>(z + i);
    float4 o;
    o.x = rstd * (d.x * __ldg(&gamma[c]) - m1 - (x.x - mean) * rstd * m2);
    o.y = rstd * (d.y * __ldg(&gamma[c + 1]) - m1 - (x.y - mean) * rstd * m2);
    o.z = rstd * (d.z * __ldg(&gamma[c + 2]) - m1 - (x.z - mean) * rstd * m2);
    o.w = rstd * (d.w * __ldg(&gamma[c + 3]) - m1 - (x.w - mean) * rstd * m2);
    *reinterpret_cast<float4*>(dz + i) = o;
  } else {
    dz[i] = rstd * (dy[i] * gamma[c] - m1 - (z[i] - mean) * rstd * m2);
  }
}

// dgamma_c = sum dy xhat, dbeta_c = sum dy over samples and times, in two deterministic
// passes: block (channel tile of 32, row slice of about 256 rows) sums its slice (8 row
// lanes; FP32 over runs of 64 rows, FP64 across runs) into part[slice][c][2];
// k_gn_param_finish adds the slices in order.
constexpr int GN_MAX_SLICES = 1024;

int gn_slices(int64_t rows) { return (int)std::min<int64_t>(GN_MAX_SLICES, std::max<int64_t>(1, (rows + 255) / 256)); }

__global__ void __launch_bounds__(256) k_gn_param_part(const float* __restrict__ dy, const float* __restrict__ z,
                                                       int rows, int T, int C, int G,
                                                       const float* __restrict__ ms, double* __restrict__ part) {
  __shared__ double a[8][33], bb[8][33];
  const int cx = threadIdx.x & 31, ry = threadIdx.x >> 5;
  const int c = blockIdx.x * 32 + cx;
  const int per = (rows + gridDim.y - 1) / gridDim.y;
  const int r0 = blockIdx.y * per, r1 = min(rows, r0 + per);
  double sg = 0.0, sb = 0.0;
  if (c < C) {
    const int g = c / (C / G);
    int r = r0 + ry, b = r / T, t = r - b * T;
    while (r < r1) {
      float fg = 0.f, fb = 0.f;
      for (int n = 0; n < 64 && r < r1; ++n) {
        const int64_t i = (int64_t)r * C + c;
        const float d = __ldg(dy + i);
        fg += d * ((__ldg(z + i) - ms[2 * (b * G + g)]) * ms[2 * (b * G + g) + 1]);
        fb += d;
        r += 8;
        t += 8;
        while (t >= T) {
          t -= T;
          ++b;
        }
      }
      sg += fg;
      sb += fb;
    }
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

// Slices in order: block (32 channels) x (32 lanes), lane y summing slices y, y + 32, ...,
// then the 32 lanes in order.
__global__ void __launch_bounds__(1024) k_gn_param_finish(const double* __restrict__ part, int slices, int C,
                                                          float* __restrict__ dgamma, float* __restrict__ dbeta) {
  __shared__ double rg[32][33], rb[32][33];
  const int c = blockIdx.x * 32 + threadIdx.x;
  double tg = 0.0, tb = 0.0;
  if (c < C)
    for (int s = threadIdx.y; s < slices; s += 32) {
      tg += part[((int64_t)s * C + c) * 2];
      tb += part[((int64_t)s * C + c) * 2 + 1];
    }
  rg[threadIdx.y][threadIdx.x] = tg;
  rb[threadIdx.y][threadIdx.x] = tb;
  __syncthreads();
  if (threadIdx.y == 0 && c < C) {
    double g = 0.0, bsum = 0.0;
    for (int y = 0; y < 32; ++y) {
      g += rg[y][threadIdx.x];
      bsum += rb[y][threadIdx.x];
    }
    dgamma[c] = (float)g;
    dbeta[c] = (float)bsum;
  }
}

// k 3, s 2, p 1 max pool over time (first maximum of a window), and its backward.
__global__ void k_maxpool(const __nv_bfloat16* __restrict__ x, int T, int C, int To, __nv_bfloat16* __restrict__ y,
                          uint8_t* __restrict__ arg) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= To * C) return;
  const int64_t b = blockIdx.y;
  const int t = i / C, c = i - t * C;
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
  y[b * To * C + i] = __float2bfloat16_rn(best);
  arg[b * To * C + i] = (uint8_t)a;
}

__global__ void k_maxpool_back(const float* __restrict__ dy, const uint8_t* __restrict__ arg, int T, int C, int To,
                               float* __restrict__ dx) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= T * C) return;
  const int64_t b = blockIdx.y;
  const int t = i / C, c = i - t * C;
  float acc = 0.f;
  for (int to = t / 2; to <= (t + 1) / 2; ++to) {
    if (to >= To) continue;
    const int64_t o = (b * To + to) * C + c;
    if (2 * to - 1 + (int)arg[o] == t) acc += dy[o];
  }
  dx[b * T * C + i] = acc;
}

// The same for four consecutive channels per thread (C % 4 == 0, 16-byte aligned dy, dx):
// float4 gradients, 4-byte argument groups; identical sums.
__global__ void k_maxpool_back4(const float* __restrict__ dy, const uint8_t* __restrict__ arg, int T, int C, int To,
                                float* __restrict__ dx) {
  const int i4 = blockIdx.x * blockDim.x + threadIdx.x;
  if (i4 >= T * C / 4) return;
  const int64_t b = blockIdx.y;
  const int t = (4 * i4) / C, c = 4 * i4 - t * C;
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int to = t / 2; to <= (t + 1) / 2; ++to) {
    if (to >= To) continue;
    const int64_t o = (b * To + to) * C + c;
    const float4 d = __ldg(reinterpret_cast<const float4*>(dy + o));
    const uchar4 a = __ldg(reinterpret_cast<const uchar4*>(arg + o));
    const int base = 2 * to - 1;
    if (base + (int)a.x == t) acc.x += d.x;
    if (base + (int)a.y == t) acc.y += d.y;
    if (base + (int)a.z == t) acc.z += d.z;
    if (base + (int)a.w == t) acc.w += d.w;
  }
  reinterpret_cast<float4*>(dx + b * T * C)[i4] = acc;
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

__global__ void k_mean_time_back(const float* __restrict__ dm, int T, int C, float* __restrict__ dx) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= T * C) return;
  const int64_t b = blockIdx.y;
  dx[b * T * C + i] = dm[b * C + i % C] / T;
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }
// the per-sample statistics kernels: C / 4 divides 256, at most 32 groups of whole quads
bool per_sample_ok(int C, int G) { return C % 4 == 0 && 256 % (C / 4) == 0 && (C / G) % 4 == 0 && G <= 32; }
bool aligned8(const void* p) { return ((uintptr_t)p & 7u) == 0; }

}  // namespace

cudaError_t launch_im2col(const void* x, int64_t B, int T, int C, int k, int s, int p, int K, void* cols,
                          cudaStream_t st) {
  const int To = (T + 2 * p - k) / s + 1;
  k_im2col<<<dim3(nblk((int64_t)To * (K / 8), 256), (unsigned)B), 256, 0, st>>>(
      reinterpret_cast<const __nv_bfloat16*>(x), T, C, k, s, p, To, K, reinterpret_cast<__nv_bfloat16*>(cols));
  return cudaGetLastError();
}

cudaError_t launch_im2col_cf(const float* y, int64_t B, int D, int N, int k, int s, int p, int K, void* cols,
                             cudaStream_t st) {
  const int To = (N + 2 * p - k) / s + 1;
  k_im2col_cf<<<dim3(nblk((int64_t)To * K, 256), (unsigned)B), 256, 0, st>>>(y, D, N, k, s, p, To, K,
                                                                             reinterpret_cast<__nv_bfloat16*>(cols));
  return cudaGetLastError();
}

cudaError_t launch_col2im(const float* dcols, int64_t B, int T, int C, int k, int s, int p, int K, const float* addend,
                          float* dx, cudaStream_t st) {
  const int To = (T + 2 * p - k) / s + 1;
  const bool v4 = C % 4 == 0 && K % 4 == 0 && aligned16(dcols) && aligned16(addend) && aligned16(dx);
  const dim3 g4(nblk((int64_t)T * C / 4, 256), (unsigned)B);
  if (v4 && k == 1) {
    k_col2im4<1><<<g4, 256, 0, st>>>(dcols, T, C, s, p, To, K, addend, dx);
  } else if (v4 && k == 5) {
    k_col2im4<5><<<g4, 256, 0, st>>>(dcols, T, C, s, p, To, K, addend, dx);
  } else if (v4 && k == 7) {
    k_col2im4<7><<<g4, 256, 0, st>>>(dcols, T, C, s, p, To, K, addend, dx);
  } else {
    k_col2im<<<dim3(nblk((int64_t)T * C, 256), (unsigned)B), 256, 0, st>>>(dcols, T, C, k, s, p, To, K, addend, dx);
  }
  return cudaGetLastError();
}

cudaError_t launch_group_norm(const float* z, int64_t B, int T, int C, int G, const float* gamma, const float* beta,
                              const float* res32, const void* res16, int relu, void* out16, float* out32, float* ms,
                              cudaStream_t st) {
  const bool v4 = (C / G) % 4 == 0 && aligned16(z) && aligned16(res32) && aligned8(res16) && aligned8(out16) &&
                  aligned16(out32);
  const auto r16 = reinterpret_cast<const __nv_bfloat16*>(res16);
  const auto o16 = reinterpret_cast<__nv_bfloat16*>(out16);
  if (v4 && per_sample_ok(C, G)) {
    k_gn_stats_s<<<(unsigned)B, 256, 0, st>>>(z, T, C, G, ms);
    k_gn_apply<4><<<dim3(nblk((int64_t)T * C / 4, 256), (unsigned)B), 256, 0, st>>>(z, T, C, G, ms, gamma, beta, res32,
                                                                                    r16, relu, o16, out32);
  } else if (v4) {
    k_gn_stats<4><<<(unsigned)(B * G), 256, 0, st>>>(z, T, C, G, ms);
    k_gn_apply<4><<<dim3(nblk((int64_t)T * C / 4, 256), (unsigned)B), 256, 0, st>>>(z, T, C, G, ms, gamma, beta, res32,
                                                                                    r16, relu, o16, out32);
  } else {
    k_gn_stats<1><<<(unsigned)(B * G), 256, 0, st>>>(z, T, C, G, ms);
    k_gn_apply<1><<<dim3(nblk((int64_t)T * C, 256), (unsigned)B), 256, 0, st>>>(z, T, C, G, ms, gamma, beta, res32,
                                                                                r16, relu, o16, out32);
  }
  return cudaGetLastError();
}

size_t group_norm_backward_scratch(int64_t B, int C, int G) {
  return (size_t)B * G * 2 * sizeof(float) + 256 + (size_t)GN_MAX_SLICES * C * 2 * sizeof(double);
}

cudaError_t launch_group_norm_backward(const float* dy, const float* z, int64_t B, int T, int C, int G,
                                       const float* ms, const float* gamma, void* scratch, float* dz, float* dgamma,
                                       float* dbeta, cudaStream_t st) {
  float* mm = reinterpret_cast<float*>(scratch);
  double* part = reinterpret_cast<double*>(reinterpret_cast<char*>(scratch) +
                                           (((size_t)B * G * 2 * sizeof(float) + 255) & ~(size_t)255));
  const bool v4 = (C / G) % 4 == 0 && aligned16(dy) && aligned16(z) && aligned16(dz);
  if (v4 && per_sample_ok(C, G)) {
    // the per-channel parameter sums come out of the statistics pass, one slice per sample
    const bool fused = B <= GN_MAX_SLICES;
    k_gn_bwd_stats_s<<<(unsigned)B, 256, 0, st>>>(dy, z, T, C, G, ms, gamma, mm, fused ? part : nullptr);
    k_gn_bwd_apply<4><<<dim3(nblk((int64_t)T * C / 4, 256), (unsigned)B), 256, 0, st>>>(dy, z, T, C, G, ms, mm, gamma,
                                                                                        dz);
    if (fused) {
      k_gn_param_finish<<<nblk(C, 32), dim3(32, 32), 0, st>>>(part, (int)B, C, dgamma, dbeta);
      return cudaGetLastError();
    }
  } else if (v4) {
    k_gn_bwd_stats<4><<<(unsigned)(B * G), 256, 0, st>>>(dy, z, T, C, G, ms, gamma, mm);
    k_gn_bwd_apply<4><<<dim3(nblk((int64_t)T * C / 4, 256), (unsigned)B), 256, 0, st>>>(dy, z, T, C, G, ms, mm, gamma,
                                                                                        dz);
  } else {
    k_gn_bwd_stats<1><<<(unsigned)(B * G), 256, 0, st>>>(dy, z, T, C, G, ms, gamma, mm);
    k_gn_bwd_apply<1><<<dim3(nblk((int64_t)T * C, 256), (unsigned)B), 256, 0, st>>>(dy, z, T, C, G, ms, mm, gamma, dz);
  }
  const int slices = gn_slices(B * T);
  k_gn_param_part<<<dim3(nblk(C, 32), slices), 256, 0, st>>>(dy, z, (int)(B * T), T, C, G, ms, part);
  k_gn_param_finish<<<nblk(C, 32), dim3(32, 32), 0, st>>>(part, slices, C, dgamma, dbeta);
  return cudaGetLastError();
}

cudaError_t launch_relu_mask(const float* dy, const void* out, int64_t n, float* d, cudaStream_t st) {
  if (n % 4 == 0 && aligned16(dy) && aligned8(out) && aligned16(d))
    k_relu_mask4<<<nblk(n / 4, 256), 256, 0, st>>>(dy, reinterpret_cast<const __nv_bfloat16*>(out), n / 4, d);
  else
    k_relu_mask<<<nblk(n, 256), 256, 0, st>>>(dy, reinterpret_cast<const __nv_bfloat16*>(out), n, d);
  return cudaGetLastError();
}

cudaError_t launch_maxpool(const void* x, int64_t B, int T, int C, void* y, uint8_t* arg, cudaStream_t st) {
  const int To = (T + 2 - 3) / 2 + 1;
  k_maxpool<<<dim3(nblk((int64_t)To * C, 256), (unsigned)B), 256, 0, st>>>(
      reinterpret_cast<const __nv_bfloat16*>(x), T, C, To, reinterpret_cast<__nv_bfloat16*>(y), arg);
  return cudaGetLastError();
}

cudaError_t launch_maxpool_back(const float* dy, const uint8_t* arg, int64_t B, int T, int C, float* dx,
                                cudaStream_t st) {
  const int To = (T + 2 - 3) / 2 + 1;
  if (C % 4 == 0 && aligned16(dy) && aligned16(dx) && ((uintptr_t)arg & 3u) == 0)
    k_maxpool_back4<<<dim3(nblk((int64_t)T * C / 4, 256), (unsigned)B), 256, 0, st>>>(dy, arg, T, C, To, dx);
  else
    k_maxpool_back<<<dim3(nblk((int64_t)T * C, 256), (unsigned)B), 256, 0, st>>>(dy, arg, T, C, To, dx);
  return cudaGetLastError();
}

cudaError_t launch_mean_time(const void* x, int64_t B, int T, int C, void* m, cudaStream_t st) {
  k_mean_time<<<nblk(B * C, 256), 256, 0, st>>>(reinterpret_cast<const __nv_bfloat16*>(x), B, T, C,
                                                reinterpret_cast<__nv_bfloat16*>(m));
  return cudaGetLastError();
}

cudaError_t launch_mean_time_back(const float* dm, int64_t B, int T, int C, float* dx, cudaStream_t st) {
  k_mean_time_back<<<dim3(nblk((int64_t)T * C, 256), (unsigned)B), 256, 0, st>>>(dm, T, C, dx);
  return cudaGetLastError();
}

}  // namespace gwx
