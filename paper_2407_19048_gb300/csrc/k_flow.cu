// k_flow.cu -- the conditional coupling flow: the posterior estimator of Sec. 5, a
// standard normal over eight coordinates pushed through K affine coupling layers whose
// shifts and log-scales small dense networks compute from the data summary of Sec. 4.
//
// Coordinates r = (Mc, q, D_L, cos theta_JN, alpha, sin delta, psi, phi_c) with
// q = min(m1, m2) / max(m1, m2); the flow works in x = (r - mean) / scale.  Coupling
// layer l splits the eight coordinates by kSplit[l % 4] into a conditioning half a and a
// transformed half b; its conditioner maps [x_a, 0 0 0 0, context] through three dense
// layers (ReLU between them; bfloat16 operands on the tensor cores,
// gwx::launch_gemm_bf16) to o[8]:
// shift mu_j = o_j, log-scale s_j = 3 tanh(o_{4+j} / 3).  Sampling moves x_b to
// x_b e^s + mu, the density direction to (x_b - mu) e^{-s}; ln q_x(x) = ln N(z) - sum s.
//
// Elementwise kernels here: targets (theta -> x), conditioner input rows, the coupling
// step in both directions, the training loss and its gradient, the coupling step's
// backward, the conditioner-input backward, base normals and the map from flow draws to
// theta with ln prior - ln proposal.  The orchestrations below chain them with the
// spectral features, dense products, dense backward and AdamW into one training step,
// a density evaluation and the posterior sampler.
#include <cuda_bf16.h>

#include <algorithm>
#include <vector>

#include "common.cuh"

namespace gwx {

namespace {

constexpr uint32_t TAG_FLOW = 4u;
constexpr float S_MAX = 3.f;
constexpr double PI_F = 3.141592653589793238462643383279502884;
constexpr double LN_2PI = 1.8378770664093454835606594728112353;

// kSplit[p] = {a0, a1, a2, a3, b0, b1, b2, b3}
__constant__ int kSplit[4][8] = {{0, 1, 2, 3, 4, 5, 6, 7},
                                 {4, 5, 6, 7, 0, 1, 2, 3},
                                 {0, 2, 4, 6, 1, 3, 5, 7},
                                 {1, 3, 5, 7, 0, 2, 4, 6}};

struct Std8 {
  double mean[8], scale[8];
  double ln_scale_sum;
  double ln_prior0;   // the constant part of ln prior_r (set by the proposal launcher)
};

__device__ __forceinline__ void load8(const float* p, float* v) {
  const float4 a = reinterpret_cast<const float4*>(p)[0], b = reinterpret_cast<const float4*>(p)[1];
  v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
}

__device__ __forceinline__ void store8(float* p, const float* v) {
  reinterpret_cast<float4*>(p)[0] = make_float4(v[0], v[1], v[2], v[3]);
  reinterpret_cast<float4*>(p)[1] = make_float4(v[4], v[5], v[6], v[7]);
}

__device__ __forceinline__ int64_t event_of(const int64_t* __restrict__ off, int64_t E, int64_t s) {
  int64_t lo = 0, hi = E;   // largest e with off[e] <= s
  while (hi - lo > 1) {
    const int64_t mid = (lo + hi) >> 1;
    if (__ldg(&off[mid]) <= s) lo = mid; else hi = mid;
  }
  return lo;
}

__global__ void k_flow_targets(const double* __restrict__ theta, int64_t B, Std8 st, float* __restrict__ x) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  const double m1 = theta[b], m2 = theta[B + b];
  const double big = fmax(m1, m2), small = fmin(m1, m2);
  double r[8];
  r[0] = pow(m1 * m2, 0.6) / pow(m1 + m2, 0.2);
  r[1] = small / big;
  r[2] = theta[4 * B + b];
  r[3] = cos(theta[7 * B + b]);
  r[4] = theta[9 * B + b];
  r[5] = sin(theta[10 * B + b]);
  r[6] = theta[8 * B + b];
  r[7] = theta[6 * B + b];
  float v[8];
#pragma unroll
  for (int p = 0; p < 8; ++p) v[p] = (float)((r[p] - st.mean[p]) / st.scale[p]);
  store8(x + b * 8, v);
}

// One thread per (row, 16-byte chunk of the row): chunk 0 holds bf16(v_a) and four
// zeros, chunks 1 .. C/8 copy the context row (the row's own, or its event's).
__global__ void k_flow_input(int l, const float* __restrict__ v, const __nv_bfloat16* __restrict__ ctx, int C,
                             const int64_t* __restrict__ off, int64_t E, int64_t row0, int64_t B,
                             __nv_bfloat16* __restrict__ X) {
  const int chunks = 1 + C / 8;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B * chunks) return;
  const int64_t r = i / chunks;
  const int k = (int)(i - r * chunks);
  uint4* dst = reinterpret_cast<uint4*>(X + r * (int64_t)(8 + C)) + k;
  if (k == 0) {
    const int p = l & 3;
    __nv_bfloat162 h0 = __floats2bfloat162_rn(v[r * 8 + kSplit[p][0]], v[r * 8 + kSplit[p][1]]);
    __nv_bfloat162 h1 = __floats2bfloat162_rn(v[r * 8 + kSplit[p][2]], v[r * 8 + kSplit[p][3]]);
    uint4 w;
    w.x = *reinterpret_cast<uint32_t*>(&h0);
    w.y = *reinterpret_cast<uint32_t*>(&h1);
    w.z = 0u;
    w.w = 0u;
    *dst = w;
    return;
  }
  const int64_t src_row = off ? event_of(off, E, row0 + r) : r;
  *dst = reinterpret_cast<const uint4*>(ctx + src_row * (int64_t)C)[k - 1];
}

// vin and vout may be the same array (each thread reads its row before writing it).
__global__ void k_flow_coupling(int l, int dir, const float* vin, const float* __restrict__ o, int64_t B, float* vout,
                                float* __restrict__ sum_s, int init) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= B) return;
  float v[8], oo[8];
  load8(vin + r * 8, v);
  load8(o + r * 8, oo);
  const int p = l & 3;
  float acc = 0.f;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int bj = kSplit[p][4 + j];
    const float s = S_MAX * tanhf(oo[4 + j] / S_MAX);
    const float mu = oo[j];
    v[bj] = dir > 0 ? fmaf(v[bj], expf(s), mu) : (v[bj] - mu) * expf(-s);
    acc += s;
  }
  store8(vout + r * 8, v);
  sum_s[r] = init ? acc : sum_s[r] + acc;
}

// One block: per-row loss |z|^2/2 + 4 ln 2pi + sum_s, its FP64 mean, gradient z / B.
__global__ void __launch_bounds__(256) k_flow_nll(const float* __restrict__ z, const float* __restrict__ sum_s,
                                                  int64_t B, float* __restrict__ loss, double* __restrict__ mean,
                                                  float* __restrict__ grad) {
  __shared__ double red[256];
  double acc = 0.0;
  const float inv_b = 1.f / (float)B;
  for (int64_t b = threadIdx.x; b < B; b += blockDim.x) {
    float v[8];
    load8(z + b * 8, v);
    double q = 0.0;
#pragma unroll
    for (int p = 0; p < 8; ++p) {
      q += (double)v[p] * (double)v[p];
      v[p] *= inv_b;
    }
    store8(grad + b * 8, v);
    const double lb = 0.5 * q + 4.0 * LN_2PI + (double)sum_s[b];
    loss[b] = (float)lb;
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

__global__ void k_flow_coupling_backward(int l, const float* __restrict__ w, const float* __restrict__ o,
                                         const float* __restrict__ g, int64_t B, float row_weight,
                                         float* __restrict__ d_o, float* __restrict__ g_u) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= B) return;
  float ww[8], oo[8], gg[8], dd[8];
  load8(w + r * 8, ww);
  load8(o + r * 8, oo);
  load8(g + r * 8, gg);
  const int p = l & 3;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int bj = kSplit[p][4 + j];
    const float t = tanhf(oo[4 + j] / S_MAX);
    const float e = expf(-S_MAX * t);
    dd[j] = -gg[bj] * e;
    dd[4 + j] = (row_weight - gg[bj] * ww[bj]) * (1.f - t * t);
    gg[bj] *= e;
  }
  store8(d_o + r * 8, dd);
  store8(g_u + r * 8, gg);
}

// One thread per (row, column): columns 0..3 add the conditioner input's gradient into
// the conditioning half of g_u, columns 4 .. C+3 into the context gradient.
__global__ void k_flow_input_backward(int l, const float* __restrict__ dX, int C, int64_t B, float* __restrict__ g_u,
                                      float* __restrict__ d_ctx, int init) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int w = C + 4;
  if (i >= B * w) return;
  const int64_t r = i / w;
  const int c = (int)(i - r * w);
  if (c < 4) {
    g_u[r * 8 + kSplit[l & 3][c]] += dX[r * (int64_t)(8 + C) + c];
  } else {
    const float d = dX[r * (int64_t)(8 + C) + 8 + (c - 4)];
    float* t = d_ctx + r * (int64_t)C + (c - 4);
    *t = init ? d : *t + d;
  }
}

__global__ void k_flow_base(uint32_t k0, uint32_t k1, uint32_t counter, int64_t row0, int64_t n,
                            float* __restrict__ z) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const uint32_t s = (uint32_t)(row0 + r);
  float v[8];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const u32x4 w = philox4x32_10(s, (uint32_t)i, TAG_FLOW, counter, k0, k1);
    const double u0 = uniform52(w.x, w.y), u1 = uniform52(w.z, w.w);
    // radius in FP64 (the logarithm near u0 -> 0 sets the tail), angle in FP32
    const float rad = (float)sqrt(-2.0 * log(u0));
    float sn, cs;
    sincospif((float)(2.0 * u1), &sn, &cs);
    v[2 * i] = rad * cs;
    v[2 * i + 1] = rad * sn;
  }
  store8(z + r * 8, v);
}

__global__ void k_flow_proposal(const float* __restrict__ x, const float* __restrict__ z,
                                const float* __restrict__ sum_s, int64_t n, int64_t row0, int64_t S, Std8 st,
                                gwx_prior pr, uint32_t k0, uint32_t k1, uint32_t counter,
                                double* __restrict__ theta, double* __restrict__ log_q,
                                double* __restrict__ log_ratio) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t s = row0 + i;
  float xv[8], zv[8];
  load8(x + i * 8, xv);
  load8(z + i * 8, zv);
  double r[8], zz = 0.0;
#pragma unroll
  for (int p = 0; p < 8; ++p) {
    r[p] = st.mean[p] + st.scale[p] * (double)xv[p];
    zz += (double)zv[p] * (double)zv[p];
  }
  const double lq = -0.5 * zz - 4.0 * LN_2PI - (double)sum_s[i] - st.ln_scale_sum;
  const u32x4 w = philox4x32_10((uint32_t)s, 4u, TAG_FLOW, counter, k0, k1);
  const double coin = uniform52(w.x, w.y);
  // parameters the flow does not model (t_c, spins): drawn from their prior, so their
  // prior and proposal densities cancel in the log ratio
  const double u_tc = uniform52(w.z, w.w);
  const u32x4 w5 = philox4x32_10((uint32_t)s, 5u, TAG_FLOW, counter, k0, k1);
  const double u_chi1 = uniform52(w5.x, w5.y), u_chi2 = uniform52(w5.z, w5.w);
  const double Mc = r[0], q = r[1], D = r[2], ct = r[3], al = r[4], sd = r[5], psi = r[6], phi = r[7];
  double m1 = pr.m_lo, m2 = pr.m_lo, dist = pr.d_lo, lr = -INFINITY;
  if (Mc > 0.0 && q > 0.0 && q <= 1.0) {
    // m_big = Mc (1 + q)^{1/5} q^{-3/5}; ln prior_r = const + 2 ln m_big - ln Mc
    const double l_q = log(q), l_1q = log1p(q);
    const double big = Mc * exp(0.2 * l_1q - 0.6 * l_q), small = q * big;
    const bool inside = pr.m_lo <= small && big <= pr.m_hi && pr.d_lo <= D && D <= pr.d_hi && -1.0 <= ct &&
                        ct <= 1.0 && 0.0 <= al && al < 2.0 * PI_F && -1.0 <= sd && sd <= 1.0 && pr.psi_lo <= psi &&
                        psi <= pr.psi_hi && pr.phi_lo <= phi && phi <= pr.phi_hi;
    if (inside) {
      m1 = coin < 0.5 ? small : big;
      m2 = coin < 0.5 ? big : small;
      dist = D;
      const double lp = st.ln_prior0 + log(Mc) + 0.4 * l_1q - 1.2 * l_q;
      lr = lp - lq;
    }
  }
  theta[s] = m1;
  theta[S + s] = m2;
  theta[2 * S + s] = pr.chi_lo + (pr.chi_hi - pr.chi_lo) * u_chi1;
  theta[3 * S + s] = pr.chi_lo + (pr.chi_hi - pr.chi_lo) * u_chi2;
  theta[4 * S + s] = dist;
  theta[5 * S + s] = pr.tc_lo + (pr.tc_hi - pr.tc_lo) * u_tc;
  theta[6 * S + s] = phi;
  theta[7 * S + s] = acos(fmin(1.0, fmax(-1.0, ct)));
  theta[8 * S + s] = psi;
  theta[9 * S + s] = al;
  theta[10 * S + s] = asin(fmin(1.0, fmax(-1.0, sd)));
  log_q[s] = lq;
  log_ratio[s] = lr;
}

__global__ void k_flow_logq(const float* __restrict__ z, const float* __restrict__ sum_s, int64_t B, double c0,
                            double* __restrict__ log_q) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  float v[8];
  load8(z + b * 8, v);
  double q = 0.0;
#pragma unroll
  for (int p = 0; p < 8; ++p) q += (double)v[p] * (double)v[p];
  log_q[b] = -0.5 * q + c0 - (double)sum_s[b];
}

inline unsigned blocks(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

Std8 make_std(const double* mean8, const double* scale8) {
  Std8 st;
  st.ln_scale_sum = 0.0;
  st.ln_prior0 = 0.0;
  for (int p = 0; p < 8; ++p) {
    st.mean[p] = mean8[p];
    st.scale[p] = scale8[p];
    st.ln_scale_sum += log(scale8[p]);
  }
  return st;
}

// Bump allocator over a caller workspace (256-byte aligned pieces); with base NULL it
// only measures.
struct Carve {
  char* base;
  size_t used = 0;
  explicit Carve(void* b) : base(static_cast<char*>(b)) {}
  template <class T>
  T* take(int64_t count) {
    const size_t off = used;
    used += ((size_t)count * sizeof(T) + 255) & ~(size_t)255;
    return base ? reinterpret_cast<T*>(base + off) : nullptr;
  }
};

#define FL_TRY(x)                        \
  do {                                   \
    cudaError_t e_ = (x);                \
    if (e_ != cudaSuccess) return e_;    \
  } while (0)

struct FlowDims {
  int64_t F, G, He, C, K, H;
  int extra;
};

FlowDims dims_of(const gwx_flow_shape& sh) {
  return FlowDims{sh.features, sh.group, sh.embed_hidden, sh.context, sh.layers, sh.hidden, sh.extra};
}

}  // namespace

int64_t flow_layout(const gwx_flow_shape& sh, int64_t* off) {
  const FlowDims d = dims_of(sh);
  int64_t n = 0;
  int t = 0;
  auto add = [&](int64_t count) {
    if (off) off[t] = n;
    ++t;
    n += (count + 63) / 64 * 64;
  };
  add(d.He * d.F);
  add(d.He);
  add(d.He * d.He);
  add(d.He);
  add(d.C * d.He);
  add(d.C);
  for (int64_t l = 0; l < d.K; ++l) {
    add(d.H * (8 + d.C));
    add(d.H);
    add(d.H * d.H);
    add(d.H);
    add(8 * d.H);
    add(8);
  }
  return n;
}

// ---- stage launchers ----
cudaError_t launch_flow_targets(const double* theta, int64_t B, const double* mean8, const double* scale8, float* x,
                                cudaStream_t s) {
  k_flow_targets<<<blocks(B, 128), 128, 0, s>>>(theta, B, make_std(mean8, scale8), x);
  return cudaGetLastError();
}

cudaError_t launch_flow_input(int l, const float* v, const void* ctx, int C, const int64_t* off, int64_t E,
                              int64_t row0, int64_t B, void* X, cudaStream_t s) {
  k_flow_input<<<blocks(B * (1 + C / 8), 256), 256, 0, s>>>(l, v, reinterpret_cast<const __nv_bfloat16*>(ctx), C, off,
                                                            E, row0, B, reinterpret_cast<__nv_bfloat16*>(X));
  return cudaGetLastError();
}

cudaError_t launch_flow_coupling(int l, int dir, const float* vin, const float* o, int64_t B, float* vout,
                                 float* sum_s, int init, cudaStream_t s) {
  k_flow_coupling<<<blocks(B, 128), 128, 0, s>>>(l, dir, vin, o, B, vout, sum_s, init);
  return cudaGetLastError();
}

cudaError_t launch_flow_nll(const float* z, const float* sum_s, int64_t B, float* loss, double* mean, float* grad,
                            cudaStream_t s) {
  k_flow_nll<<<1, 256, 0, s>>>(z, sum_s, B, loss, mean, grad);
  return cudaGetLastError();
}

cudaError_t launch_flow_coupling_backward(int l, const float* w, const float* o, const float* g, int64_t B,
                                          float row_weight, float* d_o, float* g_u, cudaStream_t s) {
  k_flow_coupling_backward<<<blocks(B, 128), 128, 0, s>>>(l, w, o, g, B, row_weight, d_o, g_u);
  return cudaGetLastError();
}

cudaError_t launch_flow_input_backward(int l, const float* dX, int C, int64_t B, float* g_u, float* d_ctx, int init,
                                       cudaStream_t s) {
  k_flow_input_backward<<<blocks(B * (C + 4), 256), 256, 0, s>>>(l, dX, C, B, g_u, d_ctx, init);
  return cudaGetLastError();
}

cudaError_t launch_flow_base(uint64_t seed, uint32_t counter, int64_t row0, int64_t n, float* z, cudaStream_t s) {
  k_flow_base<<<blocks(n, 128), 128, 0, s>>>((uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32), counter, row0, n,
                                             z);
  return cudaGetLastError();
}

cudaError_t launch_flow_proposal(const float* x, const float* z, const float* sum_s, int64_t n, int64_t row0,
                                 int64_t S, const double* mean8, const double* scale8, const gwx_prior& pr,
                                 uint64_t seed, uint32_t counter, double* theta, double* log_q, double* log_ratio,
                                 cudaStream_t s) {
  // ln prior_r = ln 2 + 2 ln m_big - ln Mc - ln((m_hi - m_lo)^2 (d_hi - d_lo) 8 pi (psi range) (phi range))
  Std8 st = make_std(mean8, scale8);
  st.ln_prior0 = log(2.0) - 2.0 * log(pr.m_hi - pr.m_lo) - log(pr.d_hi - pr.d_lo) - log(8.0 * PI_F) -
                 log(pr.psi_hi - pr.psi_lo) - log(pr.phi_hi - pr.phi_lo);
  k_flow_proposal<<<blocks(n, 128), 128, 0, s>>>(x, z, sum_s, n, row0, S, st, pr,
                                                 (uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32), counter,
                                                 theta, log_q, log_ratio);
  return cudaGetLastError();
}

// ---- orchestrations ----
namespace {

struct Params {
  const float* p;
  const __nv_bfloat16* p16;
  std::vector<int64_t> off;
  const void* W(int t) const { return p16 + off[t]; }
  const float* b(int t) const { return p + off[t]; }
};

Params make_params(const gwx_flow_shape& sh, const float* p, const void* p16) {
  Params P;
  P.p = p;
  P.p16 = reinterpret_cast<const __nv_bfloat16*>(p16);
  P.off.resize(6 + 6 * (size_t)sh.layers);
  flow_layout(sh, P.off.data());
  return P;
}

// Embedding forward on R rows: features (bfloat16 [R][F]) -> h1, h2 -> ctx (bfloat16 [R][C]).
cudaError_t embed_forward(const FlowDims& d, const Params& P, const float* y, int64_t R, int D, int64_t N, int k_lo,
                          void* fws, __nv_bfloat16* feat, __nv_bfloat16* h1, __nv_bfloat16* h2, __nv_bfloat16* ctx,
                          cudaStream_t s) {
  FL_TRY(launch_features(y, R, D, N, k_lo, (int)d.G, (int)d.F, fws, feat, s));
  const int ng = (int)((N / 2 - k_lo) / d.G);
  int col = D * ng;
  if (d.extra & GWX_FLOW_CROSS) {
    FL_TRY(launch_cross_from_spectrum(fws, R, D, N, k_lo, (int)d.G, (int)d.F, col, feat, s));
    col += D * (D - 1) * ng;
  }
  if (d.extra & GWX_FLOW_LAG) FL_TRY(launch_lag_from_spectrum(fws, R, D, N, k_lo, (int)d.G, (int)d.F, col, feat, s));
  FL_TRY(launch_gemm_bf16(feat, P.W(0), h1, R, d.He, d.F, true, P.b(1), GWX_ACT_RELU, 0, s));
  FL_TRY(launch_gemm_bf16(h1, P.W(2), h2, R, d.He, d.He, true, P.b(3), GWX_ACT_RELU, 0, s));
  return launch_gemm_bf16(h2, P.W(4), ctx, R, d.C, d.He, true, P.b(5), GWX_ACT_NONE, 0, s);
}

// One conditioner on R rows: X -> g1, g2 -> o.
cudaError_t conditioner_forward(const FlowDims& d, const Params& P, int l, int64_t R, const __nv_bfloat16* X,
                                __nv_bfloat16* g1, __nv_bfloat16* g2, float* o, cudaStream_t s) {
  const int t = 6 + 6 * l;
  FL_TRY(launch_gemm_bf16(X, P.W(t), g1, R, d.H, 8 + d.C, true, P.b(t + 1), GWX_ACT_RELU, 0, s));
  FL_TRY(launch_gemm_bf16(g1, P.W(t + 2), g2, R, d.H, d.H, true, P.b(t + 3), GWX_ACT_RELU, 0, s));
  return launch_gemm_bf16(g2, P.W(t + 4), o, R, 8, d.H, false, P.b(t + 5), GWX_ACT_NONE, 0, s);
}

size_t dense_bw_max(const FlowDims& d, int64_t B) {
  size_t m = 0;
  const int64_t shapes[][2] = {{8, d.H}, {d.H, d.H}, {d.H, 8 + d.C}, {d.C, d.He}, {d.He, d.He}, {d.He, d.F}};
  for (auto& sh : shapes) m = std::max(m, dense_backward_ws(B, sh[0], sh[1]));
  return m;
}

struct TrainWs {
  __nv_bfloat16 *feat, *h1, *h2, *ctx, *X, *g1, *g2;
  float *xs, *o, *sum_s, *loss, *G, *Gu, *d_o, *dA, *dB, *dctx;
  void *fws, *dws, *clip;
  size_t bytes;
};

TrainWs carve_train(const FlowDims& d, int64_t B, int D, int64_t N, void* base) {
  Carve c(base);
  TrainWs w;
  const int64_t maxw = std::max(std::max(d.H, 8 + d.C), std::max(d.He, d.C));
  w.fws = c.take<char>((int64_t)((size_t)B * D * (size_t)(N / 2 + 1) * sizeof(float2)));
  w.feat = c.take<__nv_bfloat16>(B * d.F);
  w.h1 = c.take<__nv_bfloat16>(B * d.He);
  w.h2 = c.take<__nv_bfloat16>(B * d.He);
  w.ctx = c.take<__nv_bfloat16>(B * d.C);
  w.X = c.take<__nv_bfloat16>(d.K * B * (8 + d.C));
  w.g1 = c.take<__nv_bfloat16>(d.K * B * d.H);
  w.g2 = c.take<__nv_bfloat16>(d.K * B * d.H);
  w.xs = c.take<float>((d.K + 1) * B * 8);
  w.o = c.take<float>(d.K * B * 8);
  w.sum_s = c.take<float>(B);
  w.loss = c.take<float>(B);
  w.G = c.take<float>(B * 8);
  w.Gu = c.take<float>(B * 8);
  w.d_o = c.take<float>(B * 8);
  w.dA = c.take<float>(B * maxw);
  w.dB = c.take<float>(B * maxw);
  w.dctx = c.take<float>(B * d.C);
  w.dws = c.take<char>((int64_t)dense_bw_max(d, B));
  w.clip = c.take<char>((int64_t)adamw_clip_ws());
  w.bytes = c.used;
  return w;
}

struct ChainWs {   // one conditioner pass over R rows (density or sampling)
  __nv_bfloat16 *X, *g1, *g2;
  float *o, *z, *v, *sum_s;
};

ChainWs carve_chain(const FlowDims& d, int64_t R, Carve& c) {
  ChainWs w;
  w.X = c.take<__nv_bfloat16>(R * (8 + d.C));
  w.g1 = c.take<__nv_bfloat16>(R * d.H);
  w.g2 = c.take<__nv_bfloat16>(R * d.H);
  w.o = c.take<float>(R * 8);
  w.z = c.take<float>(R * 8);
  w.v = c.take<float>(R * 8);
  w.sum_s = c.take<float>(R);
  return w;
}

constexpr int64_t kSampleChunk = (int64_t)1 << 17;

}  // namespace

size_t flow_train_ws(const gwx_flow_shape& sh, int64_t B, int D, int64_t N) {
  return carve_train(dims_of(sh), B, D, N, nullptr).bytes;
}

cudaError_t flow_train_step(const gwx_flow_shape& sh, float* params, void* params_bf16, float* grads, float* m,
                            float* v, int64_t step, int64_t* step_counter, double lr, double b1, double b2, double eps, double wd, double clip,
                            const double* mean8, const double* scale8, const float* y, const double* theta, int64_t B,
                            int D, int64_t N, int k_lo, const void* ctx_in, float* d_ctx_out, double* loss_mean,
                            void* ws, cudaStream_t s) {
  const FlowDims d = dims_of(sh);
  const Params P = make_params(sh, params, params_bf16);
  const int64_t n_params = flow_layout(sh, nullptr);
  TrainWs w = carve_train(d, B, D, N, ws);
  const int64_t rows8 = B * 8;
  // the context: the built-in summary of the features, or the caller's (another summary
  // network, whose backward takes the context gradient from d_ctx_out)
  const __nv_bfloat16* ctx = ctx_in ? reinterpret_cast<const __nv_bfloat16*>(ctx_in) : w.ctx;
  if (!ctx_in) FL_TRY(embed_forward(d, P, y, B, D, N, k_lo, w.fws, w.feat, w.h1, w.h2, w.ctx, s));
  FL_TRY(launch_flow_targets(theta, B, mean8, scale8, w.xs + d.K * rows8, s));
  for (int l = (int)d.K - 1; l >= 0; --l) {
    __nv_bfloat16* X = w.X + l * B * (8 + d.C);
    __nv_bfloat16* g1 = w.g1 + l * B * d.H;
    __nv_bfloat16* g2 = w.g2 + l * B * d.H;
    float* o = w.o + l * rows8;
    FL_TRY(launch_flow_input(l, w.xs + (l + 1) * rows8, ctx, (int)d.C, nullptr, B, 0, B, X, s));
    FL_TRY(conditioner_forward(d, P, l, B, X, g1, g2, o, s));
    FL_TRY(launch_flow_coupling(l, -1, w.xs + (l + 1) * rows8, o, B, w.xs + l * rows8, w.sum_s,
                                l == (int)d.K - 1, s));
  }
  FL_TRY(launch_flow_nll(w.xs, w.sum_s, B, w.loss, loss_mean, w.G, s));
  FL_TRY(cudaMemsetAsync(grads, 0, (size_t)n_params * sizeof(float), s));
  float* G = w.G;
  float* Gu = w.Gu;
  for (int l = 0; l < (int)d.K; ++l) {
    const int t = 6 + 6 * l;
    const __nv_bfloat16* X = w.X + l * B * (8 + d.C);
    const __nv_bfloat16* g1 = w.g1 + l * B * d.H;
    const __nv_bfloat16* g2 = w.g2 + l * B * d.H;
    FL_TRY(launch_flow_coupling_backward(l, w.xs + l * rows8, w.o + l * rows8, G, B, 1.f / (float)B, w.d_o, Gu, s));
    FL_TRY(launch_dense_backward(g2, P.W(t + 4), P.b(t + 5), w.d_o, B, 8, d.H, GWX_ACT_NONE, w.dA,
                                 grads + P.off[t + 4], grads + P.off[t + 5], w.dws, 0, s));
    // the ReLU layers' masks from their stored outputs (g2, g1)
    FL_TRY(launch_dense_backward(g1, P.W(t + 2), P.b(t + 3), w.dA, B, d.H, d.H, GWX_ACT_RELU, w.dB,
                                 grads + P.off[t + 2], grads + P.off[t + 3], w.dws, 0, s, g2));
    FL_TRY(launch_dense_backward(X, P.W(t), P.b(t + 1), w.dB, B, d.H, 8 + d.C, GWX_ACT_RELU, w.dA,
                                 grads + P.off[t], grads + P.off[t + 1], w.dws, 0, s, g1));
    FL_TRY(launch_flow_input_backward(l, w.dA, (int)d.C, B, Gu, w.dctx, l == 0, s));
    std::swap(G, Gu);
  }
  if (ctx_in) {
    FL_TRY(cudaMemcpyAsync(d_ctx_out, w.dctx, (size_t)B * d.C * sizeof(float), cudaMemcpyDeviceToDevice, s));
  } else {
    FL_TRY(launch_dense_backward(w.h2, P.W(4), P.b(5), w.dctx, B, d.C, d.He, GWX_ACT_NONE, w.dA, grads + P.off[4],
                                 grads + P.off[5], w.dws, 0, s));
    FL_TRY(launch_dense_backward(w.h1, P.W(2), P.b(3), w.dA, B, d.He, d.He, GWX_ACT_RELU, w.dB, grads + P.off[2],
                                 grads + P.off[3], w.dws, 0, s, w.h2));
    FL_TRY(launch_dense_backward(w.feat, P.W(0), P.b(1), w.dB, B, d.He, d.F, GWX_ACT_RELU, nullptr,
                                 grads + P.off[0], grads + P.off[1], w.dws, 0, s, w.h1));
  }
  if (step >= 1) {
    if (step_counter)
      FL_TRY(launch_adamw_clip(params, grads, m, v, n_params, lr, b1, b2, eps, wd, step, clip, params_bf16, w.clip, s,
                               step_counter));
    else if (clip > 0.0)
      FL_TRY(launch_adamw_clip(params, grads, m, v, n_params, lr, b1, b2, eps, wd, step, clip, params_bf16, w.clip, s));
    else
      FL_TRY(launch_adamw(params, grads, m, v, n_params, lr, b1, b2, eps, wd, step, params_bf16, s));
  }
  return cudaSuccess;
}

namespace {
struct EmbedWs {
  __nv_bfloat16 *feat, *h1, *h2, *ctx;
  void* fws;
};
EmbedWs carve_embed(const FlowDims& d, int64_t R, int D, int64_t N, Carve& c) {
  EmbedWs w;
  w.fws = c.take<char>((int64_t)((size_t)R * D * (size_t)(N / 2 + 1) * sizeof(float2)));
  w.feat = c.take<__nv_bfloat16>(R * d.F);
  w.h1 = c.take<__nv_bfloat16>(R * d.He);
  w.h2 = c.take<__nv_bfloat16>(R * d.He);
  w.ctx = c.take<__nv_bfloat16>(R * d.C);
  return w;
}
}  // namespace

size_t flow_log_prob_ws(const gwx_flow_shape& sh, int64_t B, int D, int64_t N) {
  const FlowDims d = dims_of(sh);
  Carve c(nullptr);
  carve_embed(d, B, D, N, c);
  carve_chain(d, B, c);
  return c.used;
}

cudaError_t flow_log_prob(const gwx_flow_shape& sh, const float* params, const void* params_bf16, const double* mean8,
                          const double* scale8, const float* y, const double* theta, int64_t B, int D, int64_t N,
                          int k_lo, const void* ctx_in, double* log_q, void* ws, cudaStream_t s) {
  const FlowDims d = dims_of(sh);
  const Params P = make_params(sh, params, params_bf16);
  Carve c(ws);
  EmbedWs e = carve_embed(d, B, D, N, c);
  ChainWs w = carve_chain(d, B, c);
  const __nv_bfloat16* ctx = ctx_in ? reinterpret_cast<const __nv_bfloat16*>(ctx_in) : e.ctx;
  if (!ctx_in) FL_TRY(embed_forward(d, P, y, B, D, N, k_lo, e.fws, e.feat, e.h1, e.h2, e.ctx, s));
  FL_TRY(launch_flow_targets(theta, B, mean8, scale8, w.v, s));
  for (int l = (int)d.K - 1; l >= 0; --l) {
    FL_TRY(launch_flow_input(l, w.v, ctx, (int)d.C, nullptr, B, 0, B, w.X, s));
    FL_TRY(conditioner_forward(d, P, l, B, w.X, w.g1, w.g2, w.o, s));
    FL_TRY(launch_flow_coupling(l, -1, w.v, w.o, B, w.v, w.sum_s, l == (int)d.K - 1, s));
  }
  const Std8 st = make_std(mean8, scale8);
  k_flow_logq<<<blocks(B, 128), 128, 0, s>>>(w.v, w.sum_s, B, -4.0 * LN_2PI - st.ln_scale_sum, log_q);
  return cudaGetLastError();
}

size_t flow_sample_ws(const gwx_flow_shape& sh, int64_t E, int D, int64_t N, int64_t S) {
  const FlowDims d = dims_of(sh);
  Carve c(nullptr);
  carve_embed(d, E, D, N, c);
  carve_chain(d, std::min(S, kSampleChunk), c);
  return c.used;
}

cudaError_t flow_sample(const gwx_flow_shape& sh, const float* params, const void* params_bf16, const double* mean8,
                        const double* scale8, const gwx_prior& pr, const float* y, int64_t E, int D, int64_t N,
                        int k_lo, const void* ctx_in, const int64_t* off, int64_t S,
                        uint64_t seed, uint32_t counter, double* theta, double* log_q, double* log_ratio, void* ws,
                        cudaStream_t s) {
  const FlowDims d = dims_of(sh);
  const Params P = make_params(sh, params, params_bf16);
  Carve c(ws);
  EmbedWs e = carve_embed(d, E, D, N, c);
  ChainWs w = carve_chain(d, std::min(S, kSampleChunk), c);
  const __nv_bfloat16* ctx = ctx_in ? reinterpret_cast<const __nv_bfloat16*>(ctx_in) : e.ctx;
  if (!ctx_in) FL_TRY(embed_forward(d, P, y, E, D, N, k_lo, e.fws, e.feat, e.h1, e.h2, e.ctx, s));
  const bool fused = flow_fused_supported((int)d.C, (int)d.H, (int)d.K);
  for (int64_t row0 = 0; row0 < S; row0 += kSampleChunk) {
    const int64_t n = std::min(kSampleChunk, S - row0);
    FL_TRY(launch_flow_base(seed, counter, row0, n, w.z, s));
    if (fused) {
      FL_TRY(launch_flow_sample_fused(params_bf16, params, P.off.data(), (int)d.C, (int)d.H, (int)d.K, w.z, ctx,
                                      off, E, row0, n, w.v, w.sum_s, s));
      FL_TRY(launch_flow_proposal(w.v, w.z, w.sum_s, n, row0, S, mean8, scale8, pr, seed, counter, theta, log_q,
                                  log_ratio, s));
      continue;
    }
    const float* vin = w.z;
    for (int l = 0; l < (int)d.K; ++l) {
      FL_TRY(launch_flow_input(l, vin, ctx, (int)d.C, off, E, row0, n, w.X, s));
      FL_TRY(conditioner_forward(d, P, l, n, w.X, w.g1, w.g2, w.o, s));
      FL_TRY(launch_flow_coupling(l, +1, vin, w.o, n, w.v, w.sum_s, l == 0, s));
      vin = w.v;
    }
    FL_TRY(launch_flow_proposal(w.v, w.z, w.sum_s, n, row0, S, mean8, scale8, pr, seed, counter, theta, log_q,
                                log_ratio, s));
  }
  return cudaSuccess;
}

// ----------------------------------------------------------------- sky density
// The flow's density over the sky (Sec. 5: evaluated at every pixel of the map): at each
// HEALPix pixel centre (nested order) the density of the flow's coordinates with (RA,
// sin dec) at the centre and the other six held at the event's draw of largest ln q,
// normalised to unit sum over the pixels.  (RA, sin dec) have equal-area measure on the
// sphere, so with equal-area pixels this is the density per steradian up to a constant.
namespace {

constexpr int kSkyThreads = 256;

__device__ __forceinline__ uint32_t compact_bits(uint32_t v) {   // bit 2 b of v -> bit b
  v &= 0x55555555u;
  v = (v | (v >> 1)) & 0x33333333u;
  v = (v | (v >> 2)) & 0x0F0F0F0Fu;
  v = (v | (v >> 4)) & 0x00FF00FFu;
  v = (v | (v >> 8)) & 0x0000FFFFu;
  return v;
}

// Centre (longitude, cos colatitude) of nested pixel p (Gorski et al. 2005).
__device__ __forceinline__ void pix2ang_nest(int nside, int64_t p, double& phi, double& z) {
  const int jrll[12] = {2, 2, 2, 2, 3, 3, 3, 3, 4, 4, 4, 4};
  const int jpll[12] = {1, 3, 5, 7, 0, 2, 4, 6, 1, 3, 5, 7};
  const int64_t npf = (int64_t)nside * nside;
  const int f = (int)(p / npf);
  const uint32_t loc = (uint32_t)(p - f * npf);
  const int ix = (int)compact_bits(loc), iy = (int)compact_bits(loc >> 1);
  const int jr = jrll[f] * nside - ix - iy - 1;
  int nr, shift;
  if (jr < nside) {
    nr = jr;
    z = 1.0 - (double)jr * jr / (3.0 * (double)npf);
    shift = 0;
  } else if (jr > 3 * nside) {
    nr = 4 * nside - jr;
    z = -(1.0 - (double)nr * nr / (3.0 * (double)npf));
    shift = 0;
  } else {
    nr = nside;
    z = 4.0 / 3.0 - 2.0 * jr / (3.0 * nside);
    shift = (jr - nside) & 1;
  }
  int jp = (jpll[f] * nr + ix - iy + 1 + shift) / 2;
  if (jp > 4 * nr) jp -= 4 * nr;
  if (jp < 1) jp += 4 * nr;
  phi = (jp - 0.5 * (1 + shift)) * (0.5 * 3.141592653589793238462643383279502884) / nr;
}

// One block: the draw of largest log_q (first on ties) and its flow coordinates r8.
__global__ void __launch_bounds__(kSkyThreads) k_sky_pick(const double* __restrict__ theta,
                                                          const double* __restrict__ log_q, int64_t S,
                                                          double* __restrict__ r8) {
  __shared__ double bv[kSkyThreads];
  __shared__ int64_t bi[kSkyThreads];
  double v = -INFINITY;
  int64_t i = S;
  for (int64_t s = threadIdx.x; s < S; s += blockDim.x) {
    const double q = log_q[s];
    if (q > v) {
      v = q;
      i = s;
    }
  }
  bv[threadIdx.x] = v;
  bi[threadIdx.x] = i;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      const double v2 = bv[threadIdx.x + o];
      const int64_t i2 = bi[threadIdx.x + o];
      if (v2 > bv[threadIdx.x] || (v2 == bv[threadIdx.x] && i2 < bi[threadIdx.x])) {
        bv[threadIdx.x] = v2;
        bi[threadIdx.x] = i2;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const int64_t b = bi[0] < S ? bi[0] : 0;                  // every log_q -inf / NaN: the first draw
    const double m1 = theta[b], m2 = theta[S + b];
    r8[0] = pow(m1 * m2, 0.6) / pow(m1 + m2, 0.2);
    r8[1] = fmin(m1, m2) / fmax(m1, m2);
    r8[2] = theta[4 * S + b];
    r8[3] = cos(theta[7 * S + b]);
    r8[4] = theta[9 * S + b];
    r8[5] = sin(theta[10 * S + b]);
    r8[6] = theta[8 * S + b];
    r8[7] = theta[6 * S + b];
  }
}

// Standardised flow coordinates of pixels row0 .. row0 + n - 1.
__global__ void k_sky_rows(int nside, int64_t row0, int64_t n, const double* __restrict__ r8, Std8 st,
                           float* __restrict__ x) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double r[8];
#pragma unroll
  for (int p = 0; p < 8; ++p) r[p] = r8[p];
  pix2ang_nest(nside, row0 + i, r[4], r[5]);                 // RA = phi, sin dec = cos colatitude
  float v[8];
#pragma unroll
  for (int p = 0; p < 8; ++p) v[p] = (float)((r[p] - st.mean[p]) / st.scale[p]);
  store8(x + i * 8, v);
}

__global__ void k_sky_fill_offsets(int64_t* off, int64_t n) {
  if (threadIdx.x == 0) {
    off[0] = 0;
    off[1] = n;
  }
}

// One block: map = exp(lnq - max) / sum (FP64).
__global__ void __launch_bounds__(kSkyThreads) k_sky_norm(const double* __restrict__ lnq, int64_t n,
                                                          double* __restrict__ map) {
  __shared__ double red[kSkyThreads];
  double m = -INFINITY;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) m = fmax(m, lnq[i]);
  red[threadIdx.x] = m;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + o]);
    __syncthreads();
  }
  const double M = red[0];
  __syncthreads();
  double acc = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) acc += isfinite(M) ? exp(lnq[i] - M) : 0.0;
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  const double tot = red[0];
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x)
    map[i] = (isfinite(M) && tot > 0.0) ? exp(lnq[i] - M) / tot : 0.0;
}

}  // namespace

size_t flow_skymap_ws(const gwx_flow_shape& sh, int D, int64_t N, int nside) {
  const FlowDims d = dims_of(sh);
  const int64_t npix = 12 * (int64_t)nside * nside;
  Carve c(nullptr);
  carve_embed(d, 1, D, N, c);
  carve_chain(d, std::min(npix, kSampleChunk), c);
  c.take<double>(npix);
  c.take<double>(8);
  c.take<int64_t>(2);
  return c.used;
}

cudaError_t flow_skymap(const gwx_flow_shape& sh, const float* params, const void* params_bf16, const double* mean8,
                        const double* scale8, const float* y, int D, int64_t N, int k_lo, const void* ctx_in,
                        const double* theta, const double* log_q, int64_t S, int nside, double* map, void* ws,
                        cudaStream_t s) {
  const FlowDims d = dims_of(sh);
  const Params P = make_params(sh, params, params_bf16);
  const int64_t npix = 12 * (int64_t)nside * nside;
  Carve c(ws);
  EmbedWs e = carve_embed(d, 1, D, N, c);
  ChainWs w = carve_chain(d, std::min(npix, kSampleChunk), c);
  double* lnq = c.take<double>(npix);
  double* r8 = c.take<double>(8);
  int64_t* off = c.take<int64_t>(2);
  const __nv_bfloat16* ctx = ctx_in ? reinterpret_cast<const __nv_bfloat16*>(ctx_in) : e.ctx;
  if (!ctx_in) FL_TRY(embed_forward(d, P, y, 1, D, N, k_lo, e.fws, e.feat, e.h1, e.h2, e.ctx, s));
  k_sky_pick<<<1, kSkyThreads, 0, s>>>(theta, log_q, S, r8);
  k_sky_fill_offsets<<<1, 32, 0, s>>>(off, npix);
  FL_TRY(cudaGetLastError());
  const Std8 st = make_std(mean8, scale8);
  for (int64_t row0 = 0; row0 < npix; row0 += kSampleChunk) {
    const int64_t n = std::min(kSampleChunk, npix - row0);
    k_sky_rows<<<blocks(n, 128), 128, 0, s>>>(nside, row0, n, r8, st, w.v);
    FL_TRY(cudaGetLastError());
    for (int l = (int)d.K - 1; l >= 0; --l) {
      FL_TRY(launch_flow_input(l, w.v, ctx, (int)d.C, off, 1, row0, n, w.X, s));
      FL_TRY(conditioner_forward(d, P, l, n, w.X, w.g1, w.g2, w.o, s));
      FL_TRY(launch_flow_coupling(l, -1, w.v, w.o, n, w.v, w.sum_s, l == (int)d.K - 1, s));
    }
    k_flow_logq<<<blocks(n, 128), 128, 0, s>>>(w.v, w.sum_s, n, -4.0 * LN_2PI - st.ln_scale_sum, lnq + row0);
    FL_TRY(cudaGetLastError());
  }
  k_sky_norm<<<1, kSkyThreads, 0, s>>>(lnq, npix, map);
  return cudaGetLastError();
}

}  // namespace gwx
