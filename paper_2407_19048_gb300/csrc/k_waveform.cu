// k_waveform.cu -- per-draw set-up, TaylorF2 waveforms (A2), projection (A3) and
// the whitened log-likelihood (A8).
#include "fft16.cuh"
#include "waveform.cuh"

namespace gwx {

cudaError_t init_tables_waveform() { return fill_tables_for_this_tu(); }
cudaError_t debug_take_waveform(unsigned long long* v) { return dbg_take_this_tu(v); }

// One thread per draw: FP64 set-up of the waveform and projection coefficients.
// One thread per draw.  The set-up is FP64-throughput bound (GB300 issues a warp's
// FP64 instruction over many cycles), so blocks are one warp wide to spread the
// draws over as many SMs as possible.
__global__ void k_draw_setup(const double* __restrict__ theta, int64_t B, SetupConsts kc, double fs, int64_t F,
                             DetParams dp, double gmst, DrawCoef* __restrict__ coef) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  DrawCoef c;
  double amp = 0.0;
  draw_waveform_coef(theta, B, b, kc, F, c, &amp);
  draw_detector_coef(theta, B, b, kc.df, dp, gmst, c.qp, c.qc_im, fs * amp, c);
  coef[b] = c;
}

cudaError_t launch_draw_setup(const double* theta, int64_t B, int /*k_lo*/, double df, double fs, int64_t F,
                              const DetParams& dp, double gmst, DrawCoef* coef, cudaStream_t s) {
  if (B <= 0) return cudaSuccess;
  const int T = 32;
  k_draw_setup<<<(unsigned)((B + T - 1) / T), T, 0, s>>>(theta, B, make_setup_consts(df), fs, F, dp, gmst, coef);
  return cudaGetLastError();
}

// A2: one block per draw; thread 0 computes the coefficients, all threads sweep
// the bins.  hp/hc are written for every bin (zeros outside [k_lo, kcut]).
__global__ void k_generate_waveforms(const double* __restrict__ theta, int64_t B, int k_lo, SetupConsts kc, int64_t F,
                                     float2* __restrict__ hp, float2* __restrict__ hc) {
  __shared__ DrawCoef sc;
  const int64_t b = blockIdx.x;
  if (threadIdx.x == 0) draw_waveform_coef(theta, B, b, kc, F, sc);
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
  k_generate_waveforms<<<(unsigned)B, 256, 0, s>>>(theta, B, k_lo, make_setup_consts(df), F, hp, hc);
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
// Partial sums of sum_d sum_{k_lo <= k < n} |Y_e,d,k|^2 in FP64: block (e, c) of an
// E x YY_CHUNKS grid covers chunk c of event e, so a few events still fill the GPU.
// Parseval turns the band sum into a time-domain sum that is exact to FP64 rounding:
// sum_{1 <= k < n} |Y_k|^2 = (N sum y^2 - |Y_0|^2 - |Y_n|^2)/2, minus the few bins
// below k_lo (chunk 0 subtracts those).  Summing FP32-transformed bins instead would
// inherit the transform's rounding.
constexpr int YY_CHUNKS = 8;

__global__ void k_event_norm(const float* __restrict__ y, const float2* __restrict__ Y, int D, int64_t F, int k_lo,
                             int n, double* __restrict__ yy_part) {
  const int64_t e = blockIdx.x;
  const int c = blockIdx.y;
  const int64_t N = 2 * (int64_t)n;
  const int64_t len = (int64_t)D * N;
  const int64_t i0 = len * c / YY_CHUNKS, i1 = len * (c + 1) / YY_CHUNKS;
  double ty = 0.0, low = 0.0;
  const float* ye = y + e * len;
  for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
    const double v = ye[i];
    ty = fma(v, v, ty);
  }
  if (c == 0) {
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
  }
  double acc = 0.5 * (double)N * ty - low;
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    acc = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (threadIdx.x == 0) yy_part[e * YY_CHUNKS + c] = acc;
  }
}

// (hi, lo) + (bh, bl) in double-float (Knuth's two-sum on the leading parts).
__device__ __forceinline__ void df_add(float& hi, float& lo, float bh, float bl) {
  const float s = hi + bh;
  const float v = s - hi;
  const float e = (hi - (s - v)) + (bh - v) + (lo + bl);
  hi = s + e;
  lo = e - (hi - s);
}

constexpr int LL_WARPS = 4;

// One warp per 32 consecutive samples s:
//   ln L_s = -(1/N) [ |Y|^2_e + sum_support (|H|^2 - 2 Re(Y conj H)) ],  H = fs h W.
// 1. each lane finds its sample's event and does the sample's FP64 set-up (all 32
//    lanes busy on the FP64 pipe; the warps of an SM overlap it with the FP32 work
//    of the others), keeping the coefficients in shared memory;
// 2. the warp walks its samples, lanes striding over the bins; per-lane sums are FP32
//    with Kahan compensation, the warp sum double-float through shuffles;
// 3. each lane adds its sample's FP64 data term and stores ln L (coalesced).
// ND = number of detectors, a template parameter so that per-detector constants stay
// in registers.
template <int ND>
__global__ void __launch_bounds__(LL_WARPS * 32)
k_loglike(const double* __restrict__ theta, SetupConsts kc, double fs, DetParams dp, double gmst,
          const float2* __restrict__ Y, const float* __restrict__ W, const int64_t* __restrict__ ev_off,
          const double* __restrict__ yy_part, int64_t E, int64_t F, int n, int k_lo, int64_t S, double invN,
          double* __restrict__ lnl) {
  __shared__ DrawCoef sc[LL_WARPS][32];
  __shared__ int se[LL_WARPS][32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t base = ((int64_t)blockIdx.x * LL_WARPS + wid) * 32;
  if (base >= S) return;
  const int64_t s_own = base + lane;
  int e_own = 0;
  if (s_own < S) {
    // event of sample s: largest e with ev_off[e] <= s
    int64_t lo = 0, hi = E;
    while (hi - lo > 1) {
      const int64_t mid = (lo + hi) >> 1;
      if (__ldg(&ev_off[mid]) <= s_own) lo = mid; else hi = mid;
    }
    e_own = (int)lo;
    DrawCoef c;
    double amp = 0.0;
    draw_waveform_coef(theta, S, s_own, kc, F, c, &amp);
    draw_detector_coef(theta, S, s_own, kc.df, dp, gmst, c.qp, c.qc_im, fs * amp, c);
    sc[wid][lane] = c;
    se[wid][lane] = e_own;
  }
  __syncwarp();
  const int cnt = S - base < 32 ? (int)(S - base) : 32;
  float own_hi = 0.f, own_lo = 0.f;
  for (int j = 0; j < cnt; ++j) {
    const DrawCoef c = sc[wid][j];
    const int64_t e = se[wid][j];
    const int kend = min(c.kcut, n - 1);
    // one Kahan pair per detector, so that the detectors' additions do not form one chain
    float sum[ND], comp[ND];
#pragma unroll
    for (int d = 0; d < ND; ++d) sum[d] = comp[d] = 0.f;
    for (int k = k_lo + lane; k <= kend; k += 32) {
      float k76;
      const float t = waveform_turns(c, k, k76);
#pragma unroll
      for (int d = 0; d < ND; ++d) {
        const float x = GWX_IDX_OK((int64_t)d * F + k, (int64_t)ND * F, 0x201) ? k76 * __ldg(&W[(int64_t)d * F + k]) : 0.f;
        const float4 g = c.g[d];
        const float2 ph = expm2pi(t + lin_turns(c.nu[d], k));
        // per-draw constant applied with one rounding so it carries no systematic error
        const float2 H = cmul(make_float2(df_scale(g.x, g.y, x), df_scale(g.z, g.w, x)), ph);
        const float2 yv = GWX_IDX_OK((e * ND + d) * F + k, E * ND * F, 0x202) ? __ldg(&Y[(e * ND + d) * F + k])
                                                                              : make_float2(0.f, 0.f);
        const float term = fmaf(H.x, H.x - 2.f * yv.x, H.y * (H.y - 2.f * yv.y));
        const float yk = term - comp[d];
        const float tk = sum[d] + yk;
        comp[d] = (tk - sum[d]) - yk;
        sum[d] = tk;
      }
    }
    float hi = sum[0], lo = -comp[0];
#pragma unroll
    for (int d = 1; d < ND; ++d) df_add(hi, lo, sum[d], -comp[d]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float bh = __shfl_xor_sync(0xffffffffu, hi, o);
      const float bl = __shfl_xor_sync(0xffffffffu, lo, o);
      df_add(hi, lo, bh, bl);
    }
    if (lane == j) {
      own_hi = hi;
      own_lo = lo;
    }
  }
  if (s_own < S) {
    double yy = 0.0;
#pragma unroll
    for (int c = 0; c < YY_CHUNKS; ++c) yy += yy_part[(int64_t)e_own * YY_CHUNKS + c];
    if (GWX_IDX_OK(s_own, S, 0x203)) lnl[s_own] = -(yy + ((double)own_hi + (double)own_lo)) * invN;
  }
}

size_t loglike_norm_bytes(int64_t E) { return (size_t)E * YY_CHUNKS * sizeof(double); }

cudaError_t launch_loglike_full(const float* ydata, const float2* Ydata, const float* W, const double* theta,
                                double df, double fs, const DetParams& dp, double gmst, const int64_t* ev_off,
                                double* yy_part, int64_t E, int D, int64_t N, int k_lo, int64_t S, double* lnl,
                                cudaStream_t s) {
  const int64_t F = N / 2 + 1;
  const int n = (int)(N / 2);
  if (E > 0) {
    k_event_norm<<<dim3((unsigned)E, YY_CHUNKS), 256, 0, s>>>(ydata, Ydata, D, F, k_lo, n, yy_part);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
  }
  if (S <= 0) return cudaSuccess;
  const int64_t per_block = LL_WARPS * 32;
  const unsigned grid = (unsigned)((S + per_block - 1) / per_block);
  const double invN = 1.0 / (double)N;
  const SetupConsts kc = make_setup_consts(df);
  const int T = LL_WARPS * 32;
#define GWX_LL(ND_)                                                                                                \
  k_loglike<ND_><<<grid, T, 0, s>>>(theta, kc, fs, dp, gmst, Ydata, W, ev_off, yy_part, E, F, n, k_lo, S, invN, lnl)
  switch (D) {
    case 1: GWX_LL(1); break;
    case 2: GWX_LL(2); break;
    case 3: GWX_LL(3); break;
    case 4: GWX_LL(4); break;
    default: return cudaErrorInvalidValue;
  }
#undef GWX_LL
  return cudaGetLastError();
}


// ----------------------------------------------------------------- A8, merger time integrated out
// ln L_m = ln( (1/J) sum_{j<J} exp ln L(theta, tc = tc_lo + j / (u fs)) ),  J = u n_tc.
// A merger-time shift only rotates the template's phase, so with the template H built at
// tc = tc_lo and c_k = (2/N) sum_d Y_d,k conj(H_d,k) (band bins, zero elsewhere)
//   ln L(tc_lo + (u m + r) / (u fs)) = -(|Y|^2 + |H|^2)/N + Re sum_k c_k e^{2 pi i k r/(N u)} e^{2 pi i k m/N},
// i.e. for each sub-grid offset r < u an inverse real FFT of N points of
// X_k = c_k e^{2 pi i k r/(N u)}, of which the outputs m < n_tc are used.  A block takes 32
// consecutive samples: its first warp does their FP64 set-up (one lane per sample), then
// per sample all threads build c_k in shared memory, and G groups of n/16 threads (16
// values each) run the u transforms G at a time: the first inverse pass packs X into the
// half-length complex transform as it loads (Z_m from X_m and X_{n-m}), the middle passes
// alternate between two shared buffers (one barrier each), and the last pass folds its
// outputs into a per-thread running maximum and sum of exponentials in registers; one
// block reduction per sample gives ln L_m.
constexpr int TM_SAMPLES = 32;

template <int LOGN>
struct TmGeom {
  using PL = Plan16<LOGN>;
  static constexpr int n = PL::n;                              // complex points of the packed transform
  static constexpr int TPR = PL::T;                            // threads per transform (16 values each)
  static constexpr int G = TPR >= 256 ? 1 : 256 / TPR;         // transforms in flight per block
  static constexpr int THREADS = TPR * G;
  static constexpr size_t SMEM = ((size_t)G * 2 * n + (size_t)(n + 1)) * sizeof(float2);
};

// Running log-sum-exp state (max m, sum s of exp(v - m)).
__device__ __forceinline__ void lse_add(float& m, float& s, float v) {
  if (v > m) {
    s = fmaf(s, __expf(m - v), 1.0f);
    m = v;
  } else {
    s += __expf(v - m);
  }
}
__device__ __forceinline__ void lse_merge(float& m, float& s, float m2, float s2) {
  const float M = fmaxf(m, m2);
  if (M == -INFINITY) return;
  s = s * __expf(m - M) + s2 * __expf(m2 - M);
  m = M;
}

// Elements m and n - m (0 < m < n) of the packed half-length transform of
// X_k = c_k e^{2 pi i k r/(N u)}: with X_m and X_{n-m} (whose ramp is e^{i pi r/u} times the
// conjugate of X_m's, cr = e^{i pi r/u}), pack_pair gives Z_m and Z_{n-m} together.
template <int LOGN>
__device__ __forceinline__ void tm_pair(const float2* __restrict__ cb, int m, uint32_t r, uint32_t numask,
                                        float inv_nu, float2 cr, float2& zm, float2& zn) {
  constexpr int n = 1 << LOGN;
  const float2 ph = expm2pi(-(float)(((uint32_t)m * r) & numask) * inv_nu);   // e^{+2 pi i m r/(N u)}
  const float2 xm = cmul(cb[m], ph);
  const float2 xn = cmul(cb[n - m], cmul(cr, cconj(ph)));
  pack_pair(xm, xn, pack_twiddle(m, LOGN + 1), zm, zn);
}

template <int ND, int LOGN>
__global__ void __launch_bounds__(TmGeom<LOGN>::THREADS, TmGeom<LOGN>::THREADS <= 256 ? 2 : 1)
k_loglike_tmarg(const double* __restrict__ theta, SetupConsts kc, double fs, DetParams dp, double gmst, double tc_lo,
                const float2* __restrict__ Y, const float* __restrict__ W, const int64_t* __restrict__ ev_off,
                const double* __restrict__ yy_part, int64_t E, int k_lo, int n_tc, int u, int64_t S, double invN,
                double log_J, double* __restrict__ lnl) {
  using Gm = TmGeom<LOGN>;
  using PL = typename Gm::PL;
  constexpr int n = Gm::n;
  constexpr int F = n + 1;
  constexpr int NT = Gm::THREADS;
  constexpr int NW = NT / 32 > 0 ? NT / 32 : 1;
  constexpr int TPR = Gm::TPR, RL = PL::RL, NB = PL::NB, P = PL::P;
  extern __shared__ float2 tm_smem[];
  float2* cb = tm_smem + Gm::G * 2 * n;                        // c_k, k = 0 .. n
  __shared__ DrawCoef sc[TM_SAMPLES];
  __shared__ int se[TM_SAMPLES];
  __shared__ float red_m[NW], red_s[NW];
  __shared__ double red_h[NW];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int g = tid / TPR, t = tid % TPR;
  const int64_t base = (int64_t)blockIdx.x * TM_SAMPLES;
  const int cnt = (int)min((int64_t)TM_SAMPLES, S - base);
  if (wid == 0 && lane < cnt) {
    const int64_t s_own = base + lane;
    int64_t lo = 0, hi = E;                                   // event: largest e with ev_off[e] <= s
    while (hi - lo > 1) {
      const int64_t mid = (lo + hi) >> 1;
      if (__ldg(&ev_off[mid]) <= s_own) lo = mid; else hi = mid;
    }
    DrawCoef c;
    double amp = 0.0;
    draw_waveform_coef(theta, S, s_own, kc, F, c, &amp);
    draw_detector_coef_at(theta, S, s_own, kc.df, dp, gmst, c.qp, c.qc_im, fs * amp, tc_lo, c);
    sc[lane] = c;
    se[lane] = (int)lo;
  }
  __syncthreads();
  const float two_over_N = (float)(2.0 * invN);               // a power of two: exact
  const uint32_t bufA = smem_addr(tm_smem + g * 2 * n), bufB = bufA + 8u * (uint32_t)n;
  const uint32_t numask = (uint32_t)(2 * n) * (uint32_t)u - 1u;   // N u - 1 (N u a power of two)
  const float inv_nu = 1.0f / (float)(numask + 1u);
  const float inv_2u = 0.5f / (float)u;
  for (int j = 0; j < cnt; ++j) {
    const int64_t e = se[j];
    const int kend = min(sc[j].kcut, n - 1);
    // c_k and this thread's part of sum |H|^2 (Kahan)
    float hs = 0.f, hcmp = 0.f;
    for (int k = tid; k <= n; k += NT) {
      float2 acc = make_float2(0.f, 0.f);
      if (k >= k_lo && k <= kend) {
        const DrawCoef& c = sc[j];
        float k76;
        const float tt = waveform_turns(c, k, k76);
#pragma unroll
        for (int d = 0; d < ND; ++d) {
          const float x =
              GWX_IDX_OK((int64_t)d * F + k, (int64_t)ND * F, 0x301) ? k76 * __ldg(&W[(int64_t)d * F + k]) : 0.f;
          const float4 gg = c.g[d];
          const float2 ph = expm2pi(tt + lin_turns(c.nu[d], k));
          const float2 H = cmul(make_float2(df_scale(gg.x, gg.y, x), df_scale(gg.z, gg.w, x)), ph);
          const float2 yv = GWX_IDX_OK((e * ND + d) * F + k, E * ND * F, 0x302) ? __ldg(&Y[(e * ND + d) * F + k])
                                                                                : make_float2(0.f, 0.f);
          acc.x = fmaf(yv.x, H.x, fmaf(yv.y, H.y, acc.x));
          acc.y = fmaf(yv.y, H.x, fmaf(-yv.x, H.y, acc.y));
          const float yk = fmaf(H.x, H.x, H.y * H.y) - hcmp;
          const float tk = hs + yk;
          hcmp = (tk - hs) - yk;
          hs = tk;
        }
      }
      cb[k] = make_float2(acc.x * two_over_N, acc.y * two_over_N);
    }
    __syncthreads();
    float mx = -INFINITY, sm = 0.f;
    for (int r0 = 0; r0 < u; r0 += Gm::G) {
      const uint32_t r = (uint32_t)(r0 + g);
      const float2 cr = expm2pi(-(float)r * inv_2u);         // e^{i pi r/u}
      // first inverse pass (radix RL, Ns = 1), reading the packed transform from c_k: a
      // thread owns butterflies p and NB - p, which hold both members of every pair
      // (m, n - m), so each pair's phase ramp and packing are computed once
#pragma unroll
      for (int s2 = 0; s2 < PL::SLOTS; ++s2) {
        const int pp = t + s2 * TPR;
        const int jA = pp, jB = pp ? NB - pp : NB / 2;
        float2 vA[RL], vB[RL];
        if (pp != 0) {
#pragma unroll
          for (int q = 0; q < RL; ++q)
            tm_pair<LOGN>(cb, jA + NB * q, r, numask, inv_nu, cr, vA[q], vB[RL - 1 - q]);
        } else {
          // butterfly 0 holds Z_0 (zero: c_0 = c_n = 0), the pairs (NB q, NB (RL - q)) and
          // Z_{n/2}; butterfly NB/2 holds the pairs (NB/2 + NB q, NB/2 + NB (RL - 1 - q))
          vA[0] = make_float2(0.f, 0.f);
#pragma unroll
          for (int q = 1; q < RL; ++q) {
            if (q < RL - q) tm_pair<LOGN>(cb, NB * q, r, numask, inv_nu, cr, vA[q], vA[RL - q]);
          }
          if (RL > 1) {
            float2 zh, unused;
            tm_pair<LOGN>(cb, n / 2, r, numask, inv_nu, cr, zh, unused);
            vA[RL / 2] = zh;
          }
#pragma unroll
          for (int q = 0; q < RL / 2; ++q)
            tm_pair<LOGN>(cb, NB / 2 + NB * q, r, numask, inv_nu, cr, vB[q], vB[RL - 1 - q]);
        }
        dftR<RL, true, false>(vA);
        dftR<RL, true, false>(vB);
        store_pass<RL, 1>(bufA, jA, vA);
        store_pass<RL, 1>(bufA, jB, vB);
      }
      __syncthreads();
      const uint32_t xl = InvMiddlePP<LOGN, 1, P - 2, RL>::run(bufA, bufB, t);
      // last inverse pass (radix 8, Ns = n/8); its outputs are the grid's Re z values
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const int jj = t + i * TPR;
        float2 v[8];
        load_strided<8, n / 8>(xl, jj, v);
        float2 w[8];
        pass_twiddles<8, n / 8, true>(jj, w);
#pragma unroll
        for (int q = 1; q < 8; ++q) v[q] = cmul(v[q], w[q]);
        dft8<true, false>(v);
        if ((int)r < u) {
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const int mp = jj + q * (n / 8);
            if (2 * mp < n_tc) lse_add(mx, sm, v[q].x);
            if (2 * mp + 1 < n_tc) lse_add(mx, sm, v[q].y);
          }
        }
      }
      __syncthreads();                                        // the next round's first pass rewrites bufA
    }
    // block reductions: (max, sum) and sum |H|^2 (FP64 across threads)
    double hh = (double)hs - (double)hcmp;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      lse_merge(mx, sm, __shfl_xor_sync(0xffffffffu, mx, o), __shfl_xor_sync(0xffffffffu, sm, o));
      hh += __shfl_xor_sync(0xffffffffu, hh, o);
    }
    if (lane == 0) {
      red_m[wid] = mx;
      red_s[wid] = sm;
      red_h[wid] = hh;
    }
    __syncthreads();
    if (tid == 0) {
      float M = red_m[0], Sm = red_s[0];
      double H2 = red_h[0];
      for (int w = 1; w < NW; ++w) {
        lse_merge(M, Sm, red_m[w], red_s[w]);
        H2 += red_h[w];
      }
      double yy = 0.0;
#pragma unroll
      for (int c = 0; c < YY_CHUNKS; ++c) yy += yy_part[e * YY_CHUNKS + c];
      if (GWX_IDX_OK(base + j, S, 0x303)) lnl[base + j] = -(yy + H2) * invN + (double)M + log((double)Sm) - log_J;
    }
    __syncthreads();                                          // c_k and the reduction slots are reused
  }
}

cudaError_t launch_loglike_tmarg(const float* ydata, const float2* Ydata, const float* W, const double* theta,
                                 double df, double fs, const DetParams& dp, double gmst, double tc_lo, int n_tc,
                                 int u, const int64_t* ev_off, double* yy_part, int64_t E, int D, int64_t N,
                                 int k_lo, int64_t S, double* lnl, cudaStream_t s) {
  const int64_t F = N / 2 + 1;
  const int n = (int)(N / 2);
  if (E > 0) {
    k_event_norm<<<dim3((unsigned)E, YY_CHUNKS), 256, 0, s>>>(ydata, Ydata, D, F, k_lo, n, yy_part);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
  }
  if (S <= 0) return cudaSuccess;
  const unsigned grid = (unsigned)((S + TM_SAMPLES - 1) / TM_SAMPLES);
  const double invN = 1.0 / (double)N;
  const double log_J = log((double)u * (double)n_tc);
  const SetupConsts kc = make_setup_consts(df);
  return dispatch_log<7, 13>(ilog2_exact(n), [&](auto lg) -> cudaError_t {
    constexpr int LG = decltype(lg)::value;
    using Gm = TmGeom<LG>;
    auto run = [&](auto kern) -> cudaError_t {
      cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Gm::SMEM);
      if (e != cudaSuccess) return e;
      kern<<<grid, Gm::THREADS, Gm::SMEM, s>>>(theta, kc, fs, dp, gmst, tc_lo, Ydata, W, ev_off, yy_part, E, k_lo,
                                               n_tc, u, S, invN, log_J, lnl);
      return cudaGetLastError();
    };
    switch (D) {
      case 1: return run(k_loglike_tmarg<1, LG>);
      case 2: return run(k_loglike_tmarg<2, LG>);
      case 3: return run(k_loglike_tmarg<3, LG>);
      case 4: return run(k_loglike_tmarg<4, LG>);
      default: return cudaErrorInvalidValue;
    }
  });
}

}  // namespace gwx
