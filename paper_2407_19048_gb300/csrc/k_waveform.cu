// k_waveform.cu -- per-draw set-up, TaylorF2 waveforms (A2), projection (A3) and
// the whitened log-likelihood (A8).
#include "fft16r.cuh"
#include "waveform.cuh"

namespace gwx {

static cudaError_t fill_tmtw_for_this_tu();
cudaError_t init_tables_waveform() {
  const cudaError_t e = fill_tables_for_this_tu();
  return e == cudaSuccess ? fill_tmtw_for_this_tu() : e;
}
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
//   ln L(tc_lo + (u m + r) / (u fs)) = -(|Y|^2 + |H|^2)/N + Re sum_k c_k e^{2 pi i k (u m + r)/(N u)},
// i.e. for each sub-grid offset r < u the real inverse transform of N points of c_k a^k,
// a = e^{2 pi i r/(N u)}, of which the outputs m < n_tc are used.
//
// Each is computed as a complex inverse transform of n = N/2 points of the packed
// sequence Z_j = a^j (P_j + e^{-i pi r/u} Q_j), j < n, whose output p holds the real
// outputs 2p and 2p + 1, with the per-sample tables (w = e^{-2 pi i/N})
//   P_j = c_j (1 + i conj(w^j))/2,   Q_j = conj(c_{n-j}) (1 - i conj(w^j))/2,
// which do not depend on r: the usual pairing of bins j and n - j of a real inverse
// transform, with the ramp of bin n - j written as e^{i pi r/u} conj(a^j).  The ramp a^j
// itself is never applied element by element.  A Stockham pass of radix R and stride Ns
// consumes the digit of j of weight n/(R Ns), so the ramp enters as the factor
// a^{n/(R Ns)} on that pass's twiddle base e^{2 pi i (j mod Ns)/(R Ns)} (every twiddle
// taken at the fractional output shift r/(2u)); the first pass (Ns = 1) multiplies its
// inputs by (a^{n/16})^q.  Passes: radix 16 (the first, reading the tables), radix-16
// middle passes, and a last pass of radix RS = 2^(log2 n mod 4) (16 when that is 0).
// Its output q of butterfly j holds the grid values 2 (j + q n/RS) and that + 1, so only
// the q with 2 q n/RS < n_tc are needed; when that is q = 0 alone and RS = 4 (n = 1024
// with the window at most a quarter of N: the two-detector workload), the output is
// evaluated by Horner's rule in e^{2 pi i (j + r/(2u))/n}, otherwise the butterfly runs in
// full.
//
// A block takes 32 consecutive samples: its first warp does their FP64 set-up (one lane
// per sample); per sample all threads build P and Q in shared memory, then G groups of
// n/16 threads (16 values each) run the u transforms G at a time, each group on its own
// barrier (in-place passes where that fits more blocks on an SM, two buffers otherwise).
// The last pass folds each thread's grid values of a round into its running maximum and
// sum of exponentials at once; per sample the warps reduce theirs, and one warp finishes
// all 32 samples (warp partials merged, norms added) at the end of the block.
constexpr int TM_SAMPLES = 32;

// Twiddle powers l of a pass are products of two rounded factors at most: the powers
// l in {1, 2, 3, 4, 8, 12} are (table entry) x (ramp power), each rounded once from FP64,
// and l = 4a + b (b = 1 .. 3) is w^{4a} w^b.  (Powers formed by repeated squaring from one
// base carry ~20 ulp at l = 15 and made the grid values of loud templates ~10x less
// accurate.)
constexpr int TM_NL = 6;
__host__ __device__ constexpr int tm_l(int i) { return i < 4 ? i + 1 : 4 * (i - 2); }   // 1 2 3 4 8 12
// middle-pass twiddles e^{2 pi i l jm/(16 Ns)} for Ns = 16, 256, laid out [Ns][l][jm]
constexpr int TMTW_TOTAL = TM_NL * (16 + 256);
__host__ __device__ constexpr int tmtw_offset(int Ns) { return Ns == 16 ? 0 : TM_NL * 16; }
// last-pass twiddles e^{2 pi i l j/n} for the powers l = tm_l(i) < RS of each n = 2^LOGN,
// LOGN = 7 .. 13, laid out [LOGN][i][j], j < n/RS
__host__ __device__ constexpr int tm_rs(int logn) { return (logn % 4) ? (1 << (logn % 4)) : 16; }
__host__ __device__ constexpr int tm_nl(int rs) { return rs >= 16 ? 6 : (rs >= 8 ? 4 : (rs >= 4 ? 3 : 1)); }
__host__ __device__ constexpr int tmlast_offset(int logn) {
  return logn <= 7 ? 0 : tmlast_offset(logn - 1) + tm_nl(tm_rs(logn - 1)) * ((1 << (logn - 1)) / tm_rs(logn - 1));
}
constexpr int TMLAST_TOTAL = tmlast_offset(14);
namespace {
__device__ float2 g_tmtw[TMTW_TOTAL];
__device__ float2 g_tmlast[TMLAST_TOTAL];
}
static cudaError_t fill_tmtw_for_this_tu() {
  static float2 tw[TMTW_TOTAL];
  const double two_pi = 6.283185307179586476925286766559;
  for (int Ns = 16; Ns <= 256; Ns *= 16)
    for (int i = 0; i < TM_NL; ++i)
        for (int jm = 0; jm < Ns; ++jm) {
          const float2 w = unit_twiddle(two_pi * (double)(tm_l(i) * jm) / (16.0 * Ns));   // e^{-i angle}
          tw[tmtw_offset(Ns) + i * Ns + jm] = make_float2(w.x, -w.y);
        }
  cudaError_t e = cudaMemcpyToSymbol(g_tmtw, tw, sizeof(tw));
  if (e != cudaSuccess) return e;
  static float2 tl[TMLAST_TOTAL];
  for (int lg = 7; lg <= 13; ++lg) {
    const int n = 1 << lg, nb = n / tm_rs(lg);
    for (int i = 0; i < tm_nl(tm_rs(lg)); ++i)
      for (int j = 0; j < nb; ++j) {
        const float2 w = unit_twiddle(two_pi * (double)(tm_l(i) * j) / (double)n);
        tl[tmlast_offset(lg) + i * nb + j] = make_float2(w.x, -w.y);
      }
  }
  return cudaMemcpyToSymbol(g_tmlast, tl, sizeof(tl));
}

// Per offset r (FP64-rounded once per block), entries e^{2 pi i m/(N u)}: [0, 16) the first
// pass's twiddles (a^{n/16})^q; 16: e^{-i pi r/u}; [17, 23) and [23, 29): (a^W)^l of the
// middle passes Ns = 16 and 256 (W = n/(16 Ns)), l = tm_l(i); [29, 35): a^l of the last pass.
constexpr int TM_ROW = 36;
constexpr int TM_ROW_MID = 17, TM_ROW_LAST = 29;
constexpr int TM_U_MAX = 64;

size_t tm_rows_bytes() { return (size_t)TM_U_MAX * TM_ROW * sizeof(float2); }

// The u rows (one block, before the likelihood kernel; the blocks of that kernel copy them
// into shared memory).
__global__ void k_tm_rows(int n, int u, float2* __restrict__ rows) {
  const int64_t Nu = 2LL * n * u;
  for (int i = threadIdx.x; i < u * TM_ROW; i += blockDim.x) {
    const int r = i / TM_ROW, k = i - r * TM_ROW;
    int64_t m = 0;                                            // the entry is e^{2 pi i m/(N u)}
    if (k < 16) m = (int64_t)k * (n / 16) * r;
    else if (k == 16) m = -(int64_t)n * r;
    else if (k < TM_ROW_LAST) m = (int64_t)(n >> (4 * ((k - TM_ROW_MID) / TM_NL + 2))) * tm_l((k - TM_ROW_MID) % TM_NL) * r;
    else if (k < TM_ROW_LAST + TM_NL) m = (int64_t)tm_l(k - TM_ROW_LAST) * r;
    m %= Nu;
    if (m < 0) m += Nu;
    double sn, cs;
    sincospi(2.0 * (double)m / (double)Nu, &sn, &cs);
    rows[i] = make_float2((float)cs, (float)sn);
  }
}

template <int LOGN>
struct TmPlan {
  static constexpr int n = 1 << LOGN;
  static constexpr int TPR = n / 16;                                  // threads per transform
  static constexpr int G = TPR >= 256 ? 1 : 256 / TPR;               // transforms in flight per block
  static constexpr int THREADS = TPR * G;
  static constexpr int RS = (LOGN % 4) ? (1 << (LOGN % 4)) : 16;      // radix of the last pass
  static constexpr int NMID = LOGN / 4 - ((LOGN % 4) ? 1 : 2);       // radix-16 middle passes
  // Two buffers per transform (one barrier per pass) only where in-place passes would not
  // raise the blocks per SM: n <= 1024 in place fits three 256-thread blocks (80 registers,
  // ~62 KB of shared memory each), n = 2048 two blocks either way, n >= 4096 only in place.
  static constexpr bool PP = LOGN == 11;
  static constexpr int MIN_BLOCKS = LOGN <= 10 ? 3 : (THREADS <= 256 ? 2 : 1);
  static constexpr int HQ = RS == 4 ? 1 : 0;  // Horner's rule (three steps) when only output 0 of radix 4 is needed
  static constexpr size_t smem(int u) {
    return (size_t)n * sizeof(float4) + (size_t)G * (PP ? 2 : 1) * n * sizeof(float2) +
           (size_t)u * TM_ROW * sizeof(float2);
  }
};

// Running log-sum-exp state (max m, sum s of exp(v - m)): merge of two states.
__device__ __forceinline__ void lse_merge(float& m, float& s, float m2, float s2) {
  const float M = fmaxf(m, m2);
  if (M == -INFINITY) return;
  s = s * __expf(m - M) + s2 * __expf(m2 - M);
  m = M;
}

// Barrier of the TPR threads of transform group g (named barrier 1 + g; within a warp,
// the group's lanes).
template <int TPR>
__device__ __forceinline__ void tm_group_sync(int g) {
  if constexpr (TPR > 32) {
    asm volatile("bar.sync %0, %1;" ::"r"(1 + g), "r"(TPR) : "memory");
  } else if constexpr (TPR == 32) {
    __syncwarp();
  } else {
    __syncwarp(((1u << TPR) - 1u) << ((threadIdx.x & 31) & ~(TPR - 1)));
  }
}

// w[4a + b] = w[4a] w[b] for b = 1 .. 3 and 4a < R, from the powers tm_l(i) < R.
template <int R>
__device__ __forceinline__ void tm_fill_powers(float2* w) {
#pragma unroll
  for (int a4 = 4; a4 < R; a4 += 4) {
#pragma unroll
    for (int b = 1; b < 4; ++b) w[a4 + b] = cmul_rn(w[a4], w[b]);
  }
}

// c_k = (2/N) sum_d Y_d,k conj(H_d,k) of bin k (zero outside [k_lo, kend]); |H_d,k|^2 is
// added to the Kahan sum (hs, hcmp).
template <int ND>
__device__ __forceinline__ float2 tm_band_product(const DrawCoef& c, int k, int k_lo, int kend, int64_t F,
                                                  const float* __restrict__ W, const float2* __restrict__ Y,
                                                  int64_t e, int64_t E, float two_over_N, float& hs, float& hcmp) {
  float2 acc = make_float2(0.f, 0.f);
  if (k >= k_lo && k <= kend) {
    float k76;
    const float tt = waveform_turns(c, k, k76);
#pragma unroll
    for (int d = 0; d < ND; ++d) {
      const float x = GWX_IDX_OK((int64_t)d * F + k, (int64_t)ND * F, 0x301) ? k76 * __ldg(&W[(int64_t)d * F + k]) : 0.f;
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
  return make_float2(acc.x * two_over_N, acc.y * two_over_N);
}

// First pass (radix 16, Ns = 1): butterfly t reads Z_{t + q n/16} from the tables (without
// the factor a^t, which the later passes carry) and writes buffer dst.
template <int LOGN>
__device__ __forceinline__ void tm_first_pass(uint32_t pq, uint32_t row, uint32_t dst, int t) {
  constexpr int T = (1 << LOGN) / 16;
  const float2 crb = lds2(row + 8u * 16u);   // e^{-i pi r/u}
  float2 v[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    const float4 e = lds4(pq + 16u * (uint32_t)(t + q * T));
    const float2 z = make_float2(fmaf(crb.x, e.z, fmaf(-crb.y, e.w, e.x)), fmaf(crb.x, e.w, fmaf(crb.y, e.z, e.y)));
    v[q] = q ? cmul(z, lds2(row + 8u * (uint32_t)q)) : z;
  }
  dft16<true>(v);
  store_pass16<16, 1>(dst, t, v);
}

// Middle pass of radix 16 and stride Ns: twiddles (e^{2 pi i (t mod Ns)/(16 Ns)} a^W)^l,
// the ramp powers (a^W)^l at shared-memory address arow.
template <int LOGN, int Ns, bool PP, int TPR>
__device__ __forceinline__ void tm_mid_pass(uint32_t src, uint32_t dst, int t, int g, uint32_t arow) {
  constexpr int nR = (1 << LOGN) / 16;
  float2 v[16];
  load_strided16<16, nR>(src, t, v);
  float2 w[16];
  const float2* tw = g_tmtw + tmtw_offset(Ns) + (t & (Ns - 1));
#pragma unroll
  for (int i = 0; i < TM_NL; ++i) w[tm_l(i)] = cmul_rn(__ldg(tw + i * Ns), lds2(arow + 8u * (uint32_t)i));
  tm_fill_powers<16>(w);
#pragma unroll
  for (int l = 1; l < 16; ++l) v[l] = cmul(v[l], w[l]);
  dft16<true>(v);
  if constexpr (!PP) tm_group_sync<TPR>(g);
  store_pass16<16, Ns>(dst, t, v);
  tm_group_sync<TPR>(g);
}

// The middle passes p = 0 .. NMID-1 (Ns = 16^(p+1)); returns the buffer holding the result.
template <int LOGN, int p>
struct TmMid {
  static __device__ __forceinline__ uint32_t run(uint32_t a, uint32_t b, uint32_t row, int t, int g) {
    using PL = TmPlan<LOGN>;
    if constexpr (p < PL::NMID) {
      tm_mid_pass<LOGN, (1 << (4 * (p + 1))), PL::PP, PL::TPR>(a, PL::PP ? b : a, t, g,
                                                                row + 8u * (uint32_t)(TM_ROW_MID + TM_NL * p));
      return TmMid<LOGN, p + 1>::run(PL::PP ? b : a, PL::PP ? a : b, row, t, g);
    } else {
      return a;
    }
  }
};

// Folds a batch of K grid values into the running log-sum-exp (m, s) with one rescale;
// values outside the window are -inf (they add nothing).
template <int K>
__device__ __forceinline__ void lse_add_batch(float& m, float& s, const float* v) {
  float mb = v[0];
#pragma unroll
  for (int i = 1; i < K; ++i) mb = fmaxf(mb, v[i]);
  const float M = fmaxf(m, mb);
  if (M == -INFINITY) return;
  float acc = s * __expf(m - M);
#pragma unroll
  for (int i = 0; i < K; ++i) acc += __expf(v[i] - M);
  s = acc;
  m = M;
}

// Last pass (radix RS, stride n/RS): the needed outputs of the butterflies t + i n/16
// enter the running log-sum-exp (mx, sm); nq = the number of needed q.
template <int LOGN>
__device__ __forceinline__ void tm_last_pass(uint32_t src, int t, uint32_t row, int n_tc, int nq, float& mx, float& sm) {
  using PL = TmPlan<LOGN>;
  constexpr int n = 1 << LOGN, RS = PL::RS, NB = n / RS, T = n / 16;
  const uint32_t arow = row + 8u * (uint32_t)TM_ROW_LAST;
  if (nq <= PL::HQ) {
    // one output (q = 0) per butterfly, by Horner's rule; the thread's 2 x 16/RS grid
    // values enter the log-sum-exp together
    float vals[2 * (16 / RS)];
#pragma unroll
    for (int i = 0; i < 16 / RS; ++i) {
      const int j = t + i * T;
      float2 v[RS];
      load_strided16<RS, NB>(src, j, v);
      const float2 b = cmul_rn(__ldg(g_tmlast + tmlast_offset(LOGN) + j), lds2(arow));   // e^{2 pi i (j + r/(2u))/n}
      float2 acc = v[RS - 1];
#pragma unroll
      for (int l = RS - 2; l >= 0; --l)
        acc = make_float2(fmaf(acc.x, b.x, fmaf(-acc.y, b.y, v[l].x)), fmaf(acc.x, b.y, fmaf(acc.y, b.x, v[l].y)));
      vals[2 * i] = 2 * j < n_tc ? acc.x : -INFINITY;
      vals[2 * i + 1] = 2 * j + 1 < n_tc ? acc.y : -INFINITY;
    }
    lse_add_batch<2 * (16 / RS)>(mx, sm, vals);
    return;
  }
#pragma unroll
  for (int i = 0; i < 16 / RS; ++i) {
    const int j = t + i * T;
    float2 v[RS];
    load_strided16<RS, NB>(src, j, v);
    const float2* tl = g_tmlast + tmlast_offset(LOGN) + j;
    // twiddles (e^{2 pi i j/n} a)^l
    float2 w[RS];
#pragma unroll
    for (int k = 0; k < TM_NL; ++k) {
      if (tm_l(k) < RS) w[tm_l(k)] = cmul_rn(__ldg(tl + k * NB), lds2(arow + 8u * (uint32_t)k));
    }
    tm_fill_powers<RS>(w);
#pragma unroll
    for (int l = 1; l < RS; ++l) v[l] = cmul(v[l], w[l]);
    if constexpr (RS == 16) dft16<true>(v);
    else dftR<RS, true, false>(v);
    // the butterfly's 2 RS grid values (those inside the window) in one update
    float vals[2 * RS];
#pragma unroll
    for (int q = 0; q < RS; ++q) {
      const int mp = j + q * NB;
      vals[2 * q] = 2 * mp < n_tc ? v[q].x : -INFINITY;
      vals[2 * q + 1] = 2 * mp + 1 < n_tc ? v[q].y : -INFINITY;
    }
    lse_add_batch<2 * RS>(mx, sm, vals);
  }
}

template <int ND, int LOGN>
__global__ void __launch_bounds__(TmPlan<LOGN>::THREADS, TmPlan<LOGN>::MIN_BLOCKS)
k_loglike_tmarg(const double* __restrict__ theta, SetupConsts kc, double fs, DetParams dp, double gmst, double tc_lo,
                const float2* __restrict__ Y, const float* __restrict__ W, const int64_t* __restrict__ ev_off,
                const double* __restrict__ yy_part, const float2* __restrict__ g_rows, int64_t E, int k_lo, int n_tc,
                int u, int nq, int64_t S, double invN, double log_J, double* __restrict__ lnl) {
  using PL = TmPlan<LOGN>;
  constexpr int n = PL::n;
  constexpr int F = n + 1;
  constexpr int NT = PL::THREADS;
  constexpr int NW = NT / 32;
  constexpr int TPR = PL::TPR;
  constexpr int NBUF = PL::PP ? 2 : 1;
  extern __shared__ __align__(16) unsigned char tm_smem[];
  __shared__ DrawCoef sc[TM_SAMPLES];
  __shared__ int se[TM_SAMPLES];
  __shared__ float red_m[TM_SAMPLES][NW], red_s[TM_SAMPLES][NW];   // per sample and warp
  __shared__ double red_h[TM_SAMPLES][NW];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int g = tid / TPR, t = tid % TPR;
  // dynamic shared memory: P_j, Q_j as float4 [n]; G x NBUF buffers of n float2; u rows
  const uint32_t pq = smem_addr(tm_smem);
  const uint32_t buf0 = pq + 16u * n + 8u * (uint32_t)(g * NBUF * n);
  const uint32_t buf1 = buf0 + 8u * n;
  const uint32_t rows = pq + 16u * n + 8u * (uint32_t)(PL::G * NBUF * n);
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
  for (int i = tid; i < u * TM_ROW; i += NT) sts2(rows + 8u * (uint32_t)i, __ldg(&g_rows[i]));
  __syncthreads();
  const float two_over_N = (float)(2.0 * invN);               // a power of two: exact
  for (int j = 0; j < cnt; ++j) {
    const int64_t e = se[j];
    const int kend = min(sc[j].kcut, n - 1);
    // P, Q of the pair (k, n - k) and this thread's part of sum |H|^2 (Kahan); item 0 also
    // takes the middle bin n/2 (its own pair), so the n/2 items split evenly
    float hs = 0.f, hcmp = 0.f;
    for (int k = tid; k < n / 2; k += NT) {
#pragma unroll 1
      for (int h = 0; h < (k == 0 ? 2 : 1); ++h) {
        const int kk = h ? n / 2 : k;
        const float2 ck = tm_band_product<ND>(sc[j], kk, k_lo, kend, F, W, Y, e, E, two_over_N, hs, hcmp);
        const float2 cn =
            h ? ck : tm_band_product<ND>(sc[j], n - kk, k_lo, kend, F, W, Y, e, E, two_over_N, hs, hcmp);
        const float2 w = pack_twiddle(kk, LOGN + 1);              // e^{-2 pi i kk/N}
        const float2 h1 = make_float2(0.5f * (1.f + w.y), 0.5f * w.x);   // (1 + i conj w)/2
        const float2 h2 = make_float2(0.5f * (1.f - w.y), -0.5f * w.x);  // (1 - i conj w)/2
        const float2 Pk = cmul(ck, h1), Qk = cmul(cconj(cn), h2);
        sts4(pq + 16u * (uint32_t)kk, make_float4(Pk.x, Pk.y, Qk.x, Qk.y));
        if (kk != 0 && kk != n / 2) {
          // P_{n-k} = c_{n-k} (1 - i w)/2, Q_{n-k} = conj(c_k) (1 + i w)/2
          const float2 Pn = cmul(cn, cconj(h1)), Qn = cmul(cconj(ck), cconj(h2));
          sts4(pq + 16u * (uint32_t)(n - kk), make_float4(Pn.x, Pn.y, Qn.x, Qn.y));
        }
      }
    }
    __syncthreads();
    float mx = -INFINITY, sm = 0.f;
    for (int r0 = 0; r0 < u; r0 += PL::G) {
      const int r = r0 + g;
      if (r < u) {                                            // uniform over the group
        const uint32_t row = rows + 8u * (uint32_t)(r * TM_ROW);
        tm_first_pass<LOGN>(pq, row, buf0, t);
        tm_group_sync<TPR>(g);
        const uint32_t xl = TmMid<LOGN, 0>::run(buf0, buf1, row, t, g);
        tm_last_pass<LOGN>(xl, t, row, n_tc, nq, mx, sm);
        // the next first pass rewrites buf0, which the last pass read in these two cases
        if constexpr (!PL::PP || PL::NMID % 2 == 0) tm_group_sync<TPR>(g);
      }
    }
    // per-warp reductions of (max, sum) and sum |H|^2; the warps' partials are merged, and
    // the norms added, for all samples at once at the end
    double hh = (double)hs - (double)hcmp;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      lse_merge(mx, sm, __shfl_xor_sync(0xffffffffu, mx, o), __shfl_xor_sync(0xffffffffu, sm, o));
      hh += __shfl_xor_sync(0xffffffffu, hh, o);
    }
    if (lane == 0) {
      red_m[j][wid] = mx;
      red_s[j][wid] = sm;
      red_h[j][wid] = hh;
    }
    __syncthreads();                                          // the tables are rewritten for the next sample
  }
  if (wid == 0 && lane < cnt) {
    const int j = lane;
    float M = red_m[j][0], Sm = red_s[j][0];
    double H2 = red_h[j][0];
    for (int w = 1; w < NW; ++w) {
      lse_merge(M, Sm, red_m[j][w], red_s[j][w]);
      H2 += red_h[j][w];
    }
    const int64_t e = se[j];
    double yy = 0.0;
#pragma unroll
    for (int c = 0; c < YY_CHUNKS; ++c) yy += yy_part[e * YY_CHUNKS + c];
    if (GWX_IDX_OK(base + j, S, 0x303)) lnl[base + j] = -(yy + H2) * invN + (double)M + log((double)Sm) - log_J;
  }
}

cudaError_t launch_loglike_tmarg(const float* ydata, const float2* Ydata, const float* W, const double* theta,
                                 double df, double fs, const DetParams& dp, double gmst, double tc_lo, int n_tc,
                                 int u, const int64_t* ev_off, double* yy_part, float2* rows, int64_t E, int D,
                                 int64_t N, int k_lo, int64_t S, double* lnl, cudaStream_t s) {
  const int64_t F = N / 2 + 1;
  const int n = (int)(N / 2);
  if (E > 0) {
    k_event_norm<<<dim3((unsigned)E, YY_CHUNKS), 256, 0, s>>>(ydata, Ydata, D, F, k_lo, n, yy_part);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
  }
  if (S <= 0) return cudaSuccess;
  if (u < 1 || u > TM_U_MAX || n_tc < 1) return cudaErrorInvalidValue;
  k_tm_rows<<<1, 256, 0, s>>>(n, u, rows);
  {
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
  }
  const unsigned grid = (unsigned)((S + TM_SAMPLES - 1) / TM_SAMPLES);
  const double invN = 1.0 / (double)N;
  const double log_J = log((double)u * (double)n_tc);
  const SetupConsts kc = make_setup_consts(df);
  return dispatch_log<7, 13>(ilog2_exact(n), [&](auto lg) -> cudaError_t {
    constexpr int LG = decltype(lg)::value;
    using PL = TmPlan<LG>;
    constexpr int NB = PL::n / PL::RS;
    const int nq = min(PL::RS, (n_tc + 2 * NB - 1) / (2 * NB));   // outputs q of the last pass with 2 q NB < n_tc
    const size_t smem = PL::smem(u);
    auto run = [&](auto kern) -> cudaError_t {
      cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PL::smem(TM_U_MAX));
      if (e != cudaSuccess) return e;
      kern<<<grid, PL::THREADS, smem, s>>>(theta, kc, fs, dp, gmst, tc_lo, Ydata, W, ev_off, yy_part, rows, E, k_lo,
                                           n_tc, u, nq, S, invN, log_J, lnl);
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
