// k_learn.cu -- elementwise kernels of the learned proposal (the network of Sec. 4/5 is
// trained on the simulated batches with AdamW and its samples are judged by the
// likelihood of Sec. 6).  The first learned proposal is the simplest conditional flow,
// one affine (Gaussian) layer over chirp mass Mc, total mass M and distance D:
// - k_features: log of the mean power |Y_k|^2 / N over groups of G bins of the whitened
//   strain's spectrum, per detector, as bfloat16 network input;
// - k_targets: standardised (Mc, M, D) of each draw;
// - k_gauss_nll: per-row Gaussian negative log-density and its gradient;
// - k_adamw: one AdamW step on FP32 master weights with their bfloat16 copy;
// - k_proposal: importance-sampling draws of (m1, m2, D) from the network's Gaussian (or
//   from the prior), with the other parameters drawn as the prior does or taken from the
//   event, and ln prior - ln proposal.
#include <cuda_bf16.h>

#include "common.cuh"

namespace gwx {

namespace {

constexpr uint32_t TAG_PROPOSAL = 3u;
constexpr double PI_L = 3.141592653589793238462643383279502884;

__global__ void k_features(const float2* __restrict__ Y, int D, int64_t F, int N, int k_lo, int G, int ng, int F_pad,
                           int64_t B, __nv_bfloat16* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B * F_pad) return;
  const int64_t b = i / F_pad;
  const int col = (int)(i % F_pad);
  float v = 0.f;
  if (col < D * ng) {
    const int d = col / ng, g = col % ng;
    const float2* y = Y + (b * D + d) * F + k_lo + (int64_t)g * G;
    float s = 0.f;
    for (int k = 0; k < G; ++k) s = fmaf(y[k].x, y[k].x, fmaf(y[k].y, y[k].y, s));
    v = logf(s / ((float)N * (float)G));
  }
  out[i] = __float2bfloat16_rn(v);
}

// Normalised cross spectrum of detector pair p (pairs (a, b), a < b, in row-major
// order) over group g: rho = sum Y_a conj(Y_b) / sqrt(sum |Y_a|^2 sum |Y_b|^2); Re rho
// to column col0 + 2 p ng + g, Im rho to col0 + (2 p + 1) ng + g.
__global__ void k_cross_features(const float2* __restrict__ Y, int D, int64_t F, int k_lo, int G, int ng, int F_pad,
                                 int col0, int64_t B, __nv_bfloat16* __restrict__ out) {
  const int P = D * (D - 1) / 2;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B * P * ng) return;
  const int64_t b = i / (P * ng);
  const int rem = (int)(i - b * P * ng);
  const int p = rem / ng, g = rem % ng;
  int a = 0, c = 1, q = p;
  while (q >= D - 1 - a) {   // p-th pair in (0,1), (0,2), .., (1,2), .. order
    q -= D - 1 - a;
    ++a;
  }
  c = a + 1 + q;
  const float2* ya = Y + (b * D + a) * F + k_lo + (int64_t)g * G;
  const float2* yb = Y + (b * D + c) * F + k_lo + (int64_t)g * G;
  float re = 0.f, im = 0.f, na = 0.f, nb = 0.f;
  for (int k = 0; k < G; ++k) {
    const float2 u = ya[k], v = yb[k];
    re = fmaf(u.x, v.x, fmaf(u.y, v.y, re));
    im = fmaf(u.y, v.x, fmaf(-u.x, v.y, im));
    na = fmaf(u.x, u.x, fmaf(u.y, u.y, na));
    nb = fmaf(v.x, v.x, fmaf(v.y, v.y, nb));
  }
  const float inv = rsqrtf(na * nb);
  __nv_bfloat16* row = out + b * F_pad + col0;
  row[2 * p * ng + g] = __float2bfloat16_rn(re * inv);
  row[(2 * p + 1) * ng + g] = __float2bfloat16_rn(im * inv);
}

// Normalised lag-one spectral product of detector d over group g:
// lam = sum Y_k conj(Y_{k+1}) / sqrt(sum |Y_k|^2 sum |Y_{k+1}|^2); Re lam to column
// col0 + 2 d ng + g, Im lam to col0 + (2 d + 1) ng + g.
__global__ void k_lag_features(const float2* __restrict__ Y, int D, int64_t F, int k_lo, int G, int ng, int F_pad,
                               int col0, int64_t B, __nv_bfloat16* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B * D * ng) return;
  const int64_t b = i / (D * ng);
  const int rem = (int)(i - b * D * ng);
  const int d = rem / ng, g = rem % ng;
  const float2* y = Y + (b * D + d) * F + k_lo + (int64_t)g * G;
  float re = 0.f, im = 0.f, na = 0.f, nb = 0.f;
  float2 u = y[0];
  for (int k = 0; k < G; ++k) {
    const float2 v = y[k + 1];
    re = fmaf(u.x, v.x, fmaf(u.y, v.y, re));
    im = fmaf(u.y, v.x, fmaf(-u.x, v.y, im));
    na = fmaf(u.x, u.x, fmaf(u.y, u.y, na));
    nb = fmaf(v.x, v.x, fmaf(v.y, v.y, nb));
    u = v;
  }
  const float inv = rsqrtf(na * nb);
  __nv_bfloat16* row = out + b * F_pad + col0;
  row[2 * d * ng + g] = __float2bfloat16_rn(re * inv);
  row[(2 * d + 1) * ng + g] = __float2bfloat16_rn(im * inv);
}

struct Std3 {
  double mean[3], scale[3];
};

__global__ void k_targets(const double* __restrict__ theta, int64_t B, Std3 st, float* __restrict__ t) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  const double m1 = theta[b], m2 = theta[B + b], D = theta[4 * B + b];
  const double M = m1 + m2;
  const double Mc = pow(m1 * m2, 0.6) / pow(M, 0.2);
  t[b * 3 + 0] = (float)((Mc - st.mean[0]) / st.scale[0]);
  t[b * 3 + 1] = (float)((M - st.mean[1]) / st.scale[1]);
  t[b * 3 + 2] = (float)((D - st.mean[2]) / st.scale[2]);
}

// One block: per-row loss, its FP64 batch mean (deterministic), gradient of the mean.
__global__ void __launch_bounds__(256) k_gauss_nll(const float* __restrict__ out, int ldo, const float* __restrict__ t,
                                                   int P, int B, float* __restrict__ loss, double* __restrict__ mean,
                                                   float* __restrict__ grad) {
  __shared__ double red[256];
  double acc = 0.0;
  for (int b = threadIdx.x; b < B; b += blockDim.x) {
    float lb = 0.f;
    for (int c = 0; c < ldo; ++c) grad[(int64_t)b * ldo + c] = 0.f;
    for (int p = 0; p < P; ++p) {
      const float mu = out[(int64_t)b * ldo + p], s = out[(int64_t)b * ldo + P + p];
      const float d = t[(int64_t)b * P + p] - mu;
      const float e = expf(-s);
      const float r = d * e;
      lb += 0.5f * r * r + s;
      grad[(int64_t)b * ldo + p] = -d * e * e / (float)B;
      grad[(int64_t)b * ldo + P + p] = (1.f - r * r) / (float)B;
    }
    loss[b] = lb;
    acc += lb;
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *mean = red[0] / (double)B;
}

__global__ void k_adamw(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                        float* __restrict__ v, int64_t n, float lr, float b1, float b2, float eps, float wd, float c1,
                        float c2, __nv_bfloat16* __restrict__ p16) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float pi = p[i] - lr * ((mi / c1) / (sqrtf(vi / c2) + eps) + wd * p[i]);
  p[i] = pi;
  if (p16) p16[i] = __float2bfloat16_rn(pi);
}

// k_adamw with the step number read from the device (the counter a captured training step
// advances before its updates): each block's first thread forms the bias corrections in
// FP64, as the host does for k_adamw.
__global__ void k_adamw_at(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                           float* __restrict__ v, int64_t n, float lr, float b1, float b2, float eps, float wd,
                           double b1d, double b2d, const int64_t* __restrict__ step, __nv_bfloat16* __restrict__ p16) {
  __shared__ float cs[2];
  if (threadIdx.x == 0) {
    const double k = (double)*step;
    cs[0] = (float)(1.0 - pow(b1d, k));
    cs[1] = (float)(1.0 - pow(b2d, k));
  }
  __syncthreads();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float c1 = cs[0], c2 = cs[1];
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float pi = p[i] - lr * ((mi / c1) / (sqrtf(vi / c2) + eps) + wd * p[i]);
  p[i] = pi;
  if (p16) p16[i] = __float2bfloat16_rn(pi);
}

// Gradient-norm clipping: per-block partial sums of g^2 (FP64), then one block turns
// them into the factor min(1, clip / |g|) that k_adamw_scaled applies to every gradient.
constexpr int CLIP_BLOCKS = 256;

__global__ void __launch_bounds__(256) k_sumsq(const float* __restrict__ g, int64_t n, double* __restrict__ part) {
  __shared__ double red[256];
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    acc += (double)g[i] * (double)g[i];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void __launch_bounds__(256) k_clip_scale(const double* __restrict__ part, int nparts, double clip,
                                                    float* __restrict__ scale) {
  __shared__ double red[256];
  double acc = 0.0;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) acc += part[i];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double norm = sqrt(red[0]);
    *scale = (float)(norm > clip ? clip / norm : 1.0);
  }
}

// The step counter on the device (CUDA-graph replays): advance it and write the bias
// corrections 1 - beta^step of the update that follows; with clip <= 0 the gradient
// scale is 1.
__global__ void k_adam_step(int64_t* __restrict__ counter, double b1, double b2, float* __restrict__ coef,
                            float* __restrict__ scale, int set_scale) {
  const int64_t step = *counter + 1;
  *counter = step;
  coef[0] = (float)(1.0 - pow(b1, (double)step));
  coef[1] = (float)(1.0 - pow(b2, (double)step));
  if (set_scale) *scale = 1.f;
}

__global__ void k_adamw_scaled(float* __restrict__ p, const float* __restrict__ g, const float* __restrict__ gscale,
                               float* __restrict__ m, float* __restrict__ v, int64_t n, float lr, float b1, float b2,
                               float eps, float wd, float c1, float c2, const float* __restrict__ coef,
                               __nv_bfloat16* __restrict__ p16) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (coef) {
    c1 = __ldg(coef);
    c2 = __ldg(coef + 1);
  }
  const float gi = g[i] * __ldg(gscale);
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float pi = p[i] - lr * ((mi / c1) / (sqrtf(vi / c2) + eps) + wd * p[i]);
  p[i] = pi;
  if (p16) p16[i] = __float2bfloat16_rn(pi);
}

__global__ void k_proposal(const float* __restrict__ net, int ldn, Std3 st, gwx_prior pr,
                           const double* __restrict__ truth, int64_t E, const int64_t* __restrict__ off, int64_t S,
                           uint32_t k0, uint32_t k1, uint32_t counter, int fix_angles, double* __restrict__ theta,
                           double* __restrict__ lratio) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= S) return;
  int64_t lo = 0, hi = E;   // event of sample s: largest e with off[e] <= s
  while (hi - lo > 1) {
    const int64_t mid = (lo + hi) >> 1;
    if (__ldg(&off[mid]) <= s) lo = mid; else hi = mid;
  }
  const int64_t e = lo;
  double u[10];
#pragma unroll
  for (int j = 0; j < 5; ++j) {
    const u32x4 w = philox4x32_10((uint32_t)s, (uint32_t)j, TAG_PROPOSAL, counter, k0, k1);
    u[2 * j] = uniform52(w.x, w.y);
    u[2 * j + 1] = uniform52(w.z, w.w);
  }
  double* th = theta;
  th[2 * S + s] = truth[2 * E + e];
  th[3 * S + s] = truth[3 * E + e];
  th[5 * S + s] = truth[5 * E + e];
  th[6 * S + s] = pr.phi_lo + (pr.phi_hi - pr.phi_lo) * u[5];
  th[8 * S + s] = pr.psi_lo + (pr.psi_hi - pr.psi_lo) * u[6];
  th[7 * S + s] = acos(2.0 * u[7] - 1.0);
  th[9 * S + s] = 2.0 * PI_L * u[8];
  th[10 * S + s] = asin(2.0 * u[9] - 1.0);
  if (fix_angles)
    for (int r = 6; r <= 10; ++r) th[(int64_t)r * S + s] = truth[(int64_t)r * E + e];
  if (!net) {   // the prior as proposal
    th[s] = pr.m_lo + (pr.m_hi - pr.m_lo) * u[0];
    th[S + s] = pr.m_lo + (pr.m_hi - pr.m_lo) * u[2];
    th[4 * S + s] = pr.d_lo + (pr.d_hi - pr.d_lo) * u[1];
    lratio[s] = 0.0;
    return;
  }
  const double r01 = sqrt(-2.0 * log(u[0]));
  double sn, cs;
  sincos(2.0 * PI_L * u[1], &sn, &cs);
  const double z[3] = {r01 * cs, r01 * sn, sqrt(-2.0 * log(u[2])) * cos(2.0 * PI_L * u[3])};
  double x[3], sig[3];
  for (int p = 0; p < 3; ++p) {
    const double mu = net[e * ldn + p], sp = net[e * ldn + 3 + p];
    sig[p] = st.scale[p] * exp(sp);
    x[p] = st.mean[p] + st.scale[p] * (mu + exp(sp) * z[p]);
  }
  const double Mc = x[0], M = x[1], D = x[2];
  double m1 = pr.m_lo, m2 = pr.m_lo, lr = -INFINITY;
  if (M > 0.0 && Mc > 0.0) {
    const double eta = pow(Mc / M, 5.0 / 3.0);
    if (eta <= 0.25) {
      const double root = sqrt(1.0 - 4.0 * eta);
      double a = 0.5 * M * (1.0 + root), b = 0.5 * M * (1.0 - root);
      if (u[4] < 0.5) {
        const double tmp = a;
        a = b;
        b = tmp;
      }
      m1 = a;
      m2 = b;
      const bool inside = pr.m_lo <= a && a <= pr.m_hi && pr.m_lo <= b && b <= pr.m_hi && pr.d_lo <= D &&
                          D <= pr.d_hi && a != b;
      if (inside) {
        double log_qx = 0.0;
        for (int p = 0; p < 3; ++p) log_qx += -0.5 * z[p] * z[p] - log(sig[p]) - 0.5 * log(2.0 * PI_L);
        const double jac = 0.6 * Mc * fabs(a - b) / (a * b);
        const double log_box = -log((pr.m_hi - pr.m_lo) * (pr.m_hi - pr.m_lo) * (pr.d_hi - pr.d_lo));
        lr = log_box - (log_qx + log(jac) - log(2.0));
      }
    }
  }
  th[s] = m1;
  th[S + s] = m2;
  th[4 * S + s] = (D == D) ? D : pr.d_lo;
  lratio[s] = lr;
}

}  // namespace

cudaError_t launch_features(const float* y, int64_t B, int D, int64_t N, int k_lo, int G, int F_pad, void* ws,
                            void* out, cudaStream_t s) {
  const int64_t F = N / 2 + 1;
  float2* Y = reinterpret_cast<float2*>(ws);
  cudaError_t e = launch_rfft_rows(y, B * D, N, Y, s);
  if (e != cudaSuccess) return e;
  const int ng = (int)((N / 2 - k_lo) / G);
  const int64_t total = B * F_pad;
  k_features<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(Y, D, F, (int)N, k_lo, G, ng, F_pad, B,
                                                             reinterpret_cast<__nv_bfloat16*>(out));
  return cudaGetLastError();
}

cudaError_t launch_cross_from_spectrum(const void* Y, int64_t B, int D, int64_t N, int k_lo, int G, int F_pad,
                                       int col0, void* out, cudaStream_t s) {
  const int ng = (int)((N / 2 - k_lo) / G);
  const int64_t total = B * (int64_t)(D * (D - 1) / 2) * ng;
  if (total == 0) return cudaSuccess;
  k_cross_features<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(reinterpret_cast<const float2*>(Y), D, N / 2 + 1,
                                                                   k_lo, G, ng, F_pad, col0, B,
                                                                   reinterpret_cast<__nv_bfloat16*>(out));
  return cudaGetLastError();
}

cudaError_t launch_lag_from_spectrum(const void* Y, int64_t B, int D, int64_t N, int k_lo, int G, int F_pad, int col0,
                                     void* out, cudaStream_t s) {
  const int ng = (int)((N / 2 - k_lo) / G);
  const int64_t total = B * (int64_t)D * ng;
  if (total == 0) return cudaSuccess;
  k_lag_features<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(reinterpret_cast<const float2*>(Y), D, N / 2 + 1,
                                                                 k_lo, G, ng, F_pad, col0, B,
                                                                 reinterpret_cast<__nv_bfloat16*>(out));
  return cudaGetLastError();
}

cudaError_t launch_lag_features(const float* y, int64_t B, int D, int64_t N, int k_lo, int G, int F_pad, int col0,
                                void* ws, void* out, cudaStream_t s) {
  cudaError_t e = launch_rfft_rows(y, B * D, N, reinterpret_cast<float2*>(ws), s);
  if (e != cudaSuccess) return e;
  return launch_lag_from_spectrum(ws, B, D, N, k_lo, G, F_pad, col0, out, s);
}

cudaError_t launch_cross_features(const float* y, int64_t B, int D, int64_t N, int k_lo, int G, int F_pad, int col0,
                                  void* ws, void* out, cudaStream_t s) {
  cudaError_t e = launch_rfft_rows(y, B * D, N, reinterpret_cast<float2*>(ws), s);
  if (e != cudaSuccess) return e;
  return launch_cross_from_spectrum(ws, B, D, N, k_lo, G, F_pad, col0, out, s);
}

cudaError_t launch_targets(const double* theta, int64_t B, const double* mean, const double* scale, float* t,
                           cudaStream_t s) {
  Std3 st;
  for (int i = 0; i < 3; ++i) {
    st.mean[i] = mean[i];
    st.scale[i] = scale[i];
  }
  k_targets<<<(unsigned)((B + 255) / 256), 256, 0, s>>>(theta, B, st, t);
  return cudaGetLastError();
}

cudaError_t launch_gauss_nll(const float* out, int ldo, const float* t, int P, int B, float* loss, double* mean,
                             float* grad, cudaStream_t s) {
  k_gauss_nll<<<1, 256, 0, s>>>(out, ldo, t, P, B, loss, mean, grad);
  return cudaGetLastError();
}

cudaError_t launch_adamw(float* p, const float* g, float* m, float* v, int64_t n, double lr, double b1, double b2,
                         double eps, double wd, int64_t step, void* p16, cudaStream_t s) {
  const float c1 = (float)(1.0 - pow(b1, (double)step)), c2 = (float)(1.0 - pow(b2, (double)step));
  k_adamw<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(p, g, m, v, n, (float)lr, (float)b1, (float)b2, (float)eps,
                                                      (float)wd, c1, c2, reinterpret_cast<__nv_bfloat16*>(p16));
  return cudaGetLastError();
}

cudaError_t launch_adamw_at(float* p, const float* g, float* m, float* v, int64_t n, double lr, double b1, double b2,
                            double eps, double wd, const int64_t* step, void* p16, cudaStream_t s) {
  k_adamw_at<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(p, g, m, v, n, (float)lr, (float)b1, (float)b2, (float)eps,
                                                         (float)wd, b1, b2, step, reinterpret_cast<__nv_bfloat16*>(p16));
  return cudaGetLastError();
}

size_t adamw_clip_ws() { return CLIP_BLOCKS * sizeof(double) + 256; }

cudaError_t launch_adamw_clip(float* p, const float* g, float* m, float* v, int64_t n, double lr, double b1, double b2,
                              double eps, double wd, int64_t step, double clip, void* p16, void* ws, cudaStream_t s,
                              int64_t* counter) {
  double* part = reinterpret_cast<double*>(ws);
  float* scale = reinterpret_cast<float*>(reinterpret_cast<char*>(ws) + CLIP_BLOCKS * sizeof(double));
  float* coef = scale + 4;   // 16-byte slot after the scale
  if (clip > 0.0) {
    k_sumsq<<<CLIP_BLOCKS, 256, 0, s>>>(g, n, part);
    k_clip_scale<<<1, 256, 0, s>>>(part, CLIP_BLOCKS, clip, scale);
  }
  if (counter) k_adam_step<<<1, 1, 0, s>>>(counter, b1, b2, coef, scale, clip > 0.0 ? 0 : 1);
  const float c1 = counter ? 1.f : (float)(1.0 - pow(b1, (double)step));
  const float c2 = counter ? 1.f : (float)(1.0 - pow(b2, (double)step));
  k_adamw_scaled<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(p, g, scale, m, v, n, (float)lr, (float)b1, (float)b2,
                                                             (float)eps, (float)wd, c1, c2, counter ? coef : nullptr,
                                                             reinterpret_cast<__nv_bfloat16*>(p16));
  return cudaGetLastError();
}

cudaError_t launch_proposal(const float* net, int ldn, const double* mean, const double* scale, const gwx_prior& pr,
                            const double* truth, int64_t E, const int64_t* off, int64_t S, uint64_t seed,
                            uint32_t counter, int fix_angles, double* theta, double* lratio, cudaStream_t s) {
  Std3 st;
  for (int i = 0; i < 3; ++i) {
    st.mean[i] = mean ? mean[i] : 0.0;
    st.scale[i] = scale ? scale[i] : 1.0;
  }
  k_proposal<<<(unsigned)((S + 127) / 128), 128, 0, s>>>(net, ldn, st, pr, truth, E, off, S,
                                                         (uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32),
                                                         counter, fix_angles, theta, lratio);
  return cudaGetLastError();
}

}  // namespace gwx
