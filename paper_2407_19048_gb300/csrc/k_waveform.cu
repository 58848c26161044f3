// k_waveform.cu -- per-draw set-up, TaylorF2 waveforms (A2), projection (A3) and
// the whitened log-likelihood (A8).
#include "waveform.cuh"

namespace gwx {

cudaError_t init_tables_waveform() { return fill_tables_for_this_tu(); }

// One thread per draw: FP64 set-up of the waveform and projection coefficients.
// One thread per draw.  The set-up is FP64-throughput bound (GB300 issues a warp's
// FP64 instruction over many cycles), so blocks are one warp wide to spread the
// draws over as many SMs as possible.
__global__ void k_draw_setup(const double* __restrict__ theta, int64_t B, double df, double df76, double fs,
                             int64_t F, DetParams dp, double gmst, DrawCoef* __restrict__ coef) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  DrawCoef c;
  double amp = 0.0;
  draw_waveform_coef(theta, B, b, df, df76, F, c, &amp);
  draw_detector_coef(theta, B, b, df, dp, gmst, c.qp, c.qc_im, fs * amp, c);
  coef[b] = c;
}

cudaError_t launch_draw_setup(const double* theta, int64_t B, int /*k_lo*/, double df, double fs, int64_t F,
                              const DetParams& dp, double gmst, DrawCoef* coef, cudaStream_t s) {
  if (B <= 0) return cudaSuccess;
  const int T = 32;
  k_draw_setup<<<(unsigned)((B + T - 1) / T), T, 0, s>>>(theta, B, df, pow(df, -7.0 / 6.0), fs, F, dp, gmst, coef);
  return cudaGetLastError();
}

// A2: one block per draw; thread 0 computes the coefficients, all threads sweep
// the bins.  hp/hc are written for every bin (zeros outside [k_lo, kcut]).
__global__ void k_generate_waveforms(const double* __restrict__ theta, int64_t B, int k_lo, double df, double df76,
                                     int64_t F, float2* __restrict__ hp, float2* __restrict__ hc) {
  __shared__ DrawCoef sc;
  const int64_t b = blockIdx.x;
  if (threadIdx.x == 0) draw_waveform_coef(theta, B, b, df, df76, F, sc);
  __syncthreads();
  const DrawCoef& c = sc;
  float2* hpb = hp + b * F;
  float2* hcb = hc + b * F;
  for (int64_t k = threadIdx.x; k < F; k += blockDim.x) {
    float2 vp = make_float2(0.f, 0.f), vc = vp;
    if (k >= k_lo && k <= c.kcut) {
      float k76;
      const float t = waveform_turns(c, (int)k, k76);
      const float A = c.amp * k76;
      const float2 e = expm2pi(t);
      vp = make_float2(A * c.qp * e.x, A * c.qp * e.y);
      // -i * qc * e
      vc = make_float2(A * c.qc_im * e.y, -A * c.qc_im * e.x);
    }
    hpb[k] = vp;
    hcb[k] = vc;
  }
}

cudaError_t launch_generate_waveforms(const double* theta, int64_t B, int k_lo, double df, int64_t F, float2* hp,
                                      float2* hc, cudaStream_t s) {
  if (B <= 0) return cudaSuccess;
  k_generate_waveforms<<<(unsigned)B, 256, 0, s>>>(theta, B, k_lo, df, pow(df, -7.0 / 6.0), F, hp, hc);
  return cudaGetLastError();
}

// A3: one block per draw; thread 0 computes F+, Fx and the fixed-point delays.
__global__ void k_project(const float2* __restrict__ hp, const float2* __restrict__ hc,
                          const double* __restrict__ theta, int64_t B, DetParams dp, double gmst, double df,
                          int64_t F, float2* __restrict__ hdet) {
  __shared__ DrawCoef sc;
  const int64_t b = blockIdx.x;
  // qp = 1, qc = -1, scale 1 makes g[d] = (F+, Fx)
  if (threadIdx.x == 0) draw_detector_coef(theta, B, b, df, dp, gmst, 1.0, -1.0, 1.0, sc);
  __syncthreads();
  const float2* hpb = hp + b * F;
  const float2* hcb = hc + b * F;
  for (int64_t k = threadIdx.x; k < F; k += blockDim.x) {
    const float2 p = hpb[k], x = hcb[k];
    for (int d = 0; d < dp.D; ++d) {
      const float fp = sc.g[d].x, fc = sc.g[d].z;
      const float2 h = make_float2(fp * p.x + fc * x.x, fp * p.y + fc * x.y);
      const float2 e = expm2pi(lin_turns(sc.nu[d], (int)k));
      hdet[(b * dp.D + d) * F + k] = cmul(h, e);
    }
  }
}

cudaError_t launch_project(const float2* hp, const float2* hc, const double* theta, int64_t B, const DetParams& dp,
                           double gmst, double df, int64_t F, float2* hdet, cudaStream_t s) {
  if (B <= 0) return cudaSuccess;
  k_project<<<(unsigned)B, 256, 0, s>>>(hp, hc, theta, B, dp, gmst, df, F, hdet);
  return cudaGetLastError();
}

// ----------------------------------------------------------------- A8
// sum_d sum_{k_lo <= k < n} |Y_e,d,k|^2 in FP64, one block per event, from the
// time-domain data by Parseval: sum_{1 <= k < n} |Y_k|^2 = (N sum y^2 - |Y_0|^2 - |Y_n|^2)/2,
// minus the few bins below k_lo.  The time-domain sum is exact to FP64 rounding,
// whereas summing FP32-transformed bins would inherit the transform's rounding.
__global__ void k_event_norm(const float* __restrict__ y, const float2* __restrict__ Y, int D, int64_t F, int k_lo,
                             int n, double* __restrict__ yy) {
  const int64_t e = blockIdx.x;
  const int64_t N = 2 * (int64_t)n;
  double ty = 0.0, low = 0.0;
  const float* ye = y + e * D * N;
  for (int64_t i = threadIdx.x; i < D * N; i += blockDim.x) {
    const double v = ye[i];
    ty += v * v;
  }
  for (int i = threadIdx.x; i < D * (k_lo + 1); i += blockDim.x) {
    const int d = i / (k_lo + 1), k = i % (k_lo + 1);
    const float2* Yd = Y + (e * D + d) * F;
    double w = 0.0;
    if (k == 0) {
      const float2 a = Yd[0], b = Yd[n];
      w = 0.5 * ((double)a.x * a.x + (double)a.y * a.y + (double)b.x * b.x + (double)b.y * b.y);
    } else if (k < k_lo) {
      const float2 a = Yd[k];
      w = (double)a.x * a.x + (double)a.y * a.y;
    }
    low += w;
  }
  double acc = 0.5 * (double)N * ty - low;
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    acc = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (threadIdx.x == 0) yy[e] = acc;
  }
}

// One warp per sample: ln L_s = -(1/N) [ |Y|^2_e + sum_support (|H|^2 - 2 Re(Y conj H)) ],
// H = fs h W.  Per-lane sums are FP32 with Kahan compensation, the warp sum FP64.
__global__ void k_loglike(const float2* __restrict__ Y, const float* __restrict__ W, const DrawCoef* __restrict__ coef,
                          const int64_t* __restrict__ ev_off, const double* __restrict__ yy, int64_t E, int D,
                          int64_t F, int n, int k_lo, int64_t S, double invN, double* __restrict__ lnl) {
  const int lane = threadIdx.x & 31;
  const int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (s >= S) return;
  // event of sample s: largest e with ev_off[e] <= s
  int64_t lo = 0, hi = E;
  while (hi - lo > 1) {
    const int64_t mid = (lo + hi) >> 1;
    if (__ldg(&ev_off[mid]) <= s) lo = mid; else hi = mid;
  }
  const int64_t e = lo;
  const DrawCoef c = coef[s];
  const int kend = min(c.kcut, n - 1);
  float sum = 0.f, comp = 0.f;
  for (int k = k_lo + lane; k <= kend; k += 32) {
    float k76;
    const float t = waveform_turns(c, k, k76);
    for (int d = 0; d < D; ++d) {
      const float x = k76 * __ldg(&W[(int64_t)d * F + k]);
      const float4 g = c.g[d];
      const float2 ph = expm2pi(t + lin_turns(c.nu[d], k));
      // per-draw constant applied with one rounding so it carries no systematic error
      const float2 H = cmul(make_float2(df_scale(g.x, g.y, x), df_scale(g.z, g.w, x)), ph);
      const float2 y = __ldg(&Y[(e * D + d) * F + k]);
      const float term = fmaf(H.x, H.x - 2.f * y.x, H.y * (H.y - 2.f * y.y));
      const float yk = term - comp;
      const float tk = sum + yk;
      comp = (tk - sum) - yk;
      sum = tk;
    }
  }
  double acc = (double)sum - (double)comp;
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if (lane == 0) lnl[s] = -(yy[e] + acc) * invN;
}

cudaError_t launch_loglike_full(const float* ydata, const float2* Ydata, const float* W, const DrawCoef* coef,
                                const int64_t* ev_off, double* yy, int64_t E, int D, int64_t N, int k_lo, int64_t S,
                                double* lnl, cudaStream_t s) {
  const int64_t F = N / 2 + 1;
  const int n = (int)(N / 2);
  if (E > 0) {
    k_event_norm<<<(unsigned)E, 256, 0, s>>>(ydata, Ydata, D, F, k_lo, n, yy);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
  }
  if (S <= 0) return cudaSuccess;
  const int T = 256;
  const int64_t warps_per_block = T / 32;
  k_loglike<<<(unsigned)((S + warps_per_block - 1) / warps_per_block), T, 0, s>>>(
      Ydata, W, coef, ev_off, yy, E, D, F, n, k_lo, S, 1.0 / (double)N, lnl);
  return cudaGetLastError();
}

}  // namespace gwx
