// k_fused.cu -- the per-batch pass of Sec. 3.2 fused per draw: for each draw b and
// detector d,
//   y[b][d] = irfft( (rfft(noise[d][off_b : off_b + N]) + fs h_d(theta_b)) W_d )
// which equals whiten(inject(...)) because the injection is linear.  One block per
// draw (persistent over draws): the D windows live in shared memory as n = N/2
// complex points each; the waveform of a bin is evaluated once and projected onto
// all D detectors, so the frequency-domain stage costs one phase/amplitude
// evaluation per bin plus one complex exponential per detector.
#include <map>
#include <mutex>
#include <utility>

#include "fft16.cuh"
#include "waveform.cuh"

namespace gwx {

cudaError_t init_tables_fused() { return fill_tables_for_this_tu(); }
cudaError_t debug_take_fused(unsigned long long* v) { return dbg_take_this_tu(v); }

// Frequency-domain step of one real-FFT bin pair (k, nk = n - k), 0 < k < n, k != n/2,
// done on the half-length transform Z directly.  Whitening (s = W/n) in that domain is
//   Z'_k = alpha_k Z_k + i beta_k conj(Z_nk)   (packed filter table Wp = (alpha, beta));
// the injected strain H (continuous FT times fs) adds
//   Z'_k += p s_k H_k + q s_nk conj(H_nk),  p = (1 + i conj w)/2, q = (1 - i conj w)/2,
// w = e^{-2 pi i k/N}, and the mirrored terms with w_nk = -conj(w) for Z'_nk.
// (tk, ak), (tnk, ank): waveform phase in turns and amplitude factor k^-7/6 of the two
// bins (ak = 0 outside the support).
template <int LOGN>
__device__ __forceinline__ void fd_pair(float2& zk, float2& znk, int k, float tk, float ak, float tnk, float ank,
                                        float2 gd, unsigned long long nu, const float* __restrict__ Wd,
                                        const float2* __restrict__ Wpd, float inv_n) {
  constexpr int n = 1 << LOGN;
  const int nk = n - k;
  const float2 fk = __ldg(&Wpd[k]), fnk = __ldg(&Wpd[nk]);
  const float2 a = zk, b = znk;
  zk = make_float2(fmaf(fk.x, a.x, fk.y * b.y), fmaf(fk.x, a.y, fk.y * b.x));
  znk = make_float2(fmaf(fnk.x, b.x, fnk.y * a.y), fmaf(fnk.x, b.y, fnk.y * a.x));
  if (ak != 0.f || ank != 0.f) {
    float2 hk = make_float2(0.f, 0.f), hnk = hk;
    if (ak != 0.f) hk = cscale(cmul(gd, expm2pi(tk + lin_turns(nu, k))), ak * __ldg(&Wd[k]) * inv_n);
    if (ank != 0.f) hnk = cscale(cmul(gd, expm2pi(tnk + lin_turns(nu, nk))), ank * __ldg(&Wd[nk]) * inv_n);
    // hk, hnk now carry s_k and s_nk
    const float2 w = pack_twiddle(k, LOGN + 1);
    const float pr = 0.5f * (1.0f + w.y), qr = 0.5f * (1.0f - w.y), wi = 0.5f * w.x;
    // Z'_k += p hk + q conj(hnk), p = (pr, wi), q = (qr, -wi)
    zk.x += pr * hk.x - wi * hk.y + qr * hnk.x - wi * hnk.y;
    zk.y += pr * hk.y + wi * hk.x - qr * hnk.y - wi * hnk.x;
    // Z'_nk += p' hnk + q' conj(hk), p' = (pr, -wi), q' = (qr, wi)
    znk.x += pr * hnk.x + wi * hnk.y + qr * hk.x + wi * hk.y;
    znk.y += pr * hnk.y - wi * hnk.x - qr * hk.y + wi * hk.x;
  }
}

// The bin k = n/2, which pairs with itself (w = -i, so p = 0 and q = 1).
template <int LOGN>
__device__ __forceinline__ void fd_half(float2& z, float t, float a, float2 gd, unsigned long long nu,
                                        const float* __restrict__ Wd, const float2* __restrict__ Wpd, float inv_n) {
  constexpr int h = (1 << LOGN) / 2;
  const float2 f = __ldg(&Wpd[h]);
  const float2 v = z;
  z = make_float2(fmaf(f.x, v.x, f.y * v.y), fmaf(f.x, v.y, f.y * v.x));
  if (a != 0.f) {
    const float2 hh = cscale(cmul(gd, expm2pi(t + lin_turns(nu, h))), a * __ldg(&Wd[h]) * inv_n);
    z.x += hh.x;
    z.y -= hh.y;
  }
}

// DC and Nyquist (carried together in element 0); the waveform is zero there.
__device__ __forceinline__ void fd_dc(float2& z0, const float2* __restrict__ Wpd) {
  const float2 f = __ldg(&Wpd[0]);
  const float2 v = z0;
  z0 = make_float2(fmaf(f.x, v.x, f.y * v.y), fmaf(f.y, v.x, f.x * v.y));
}

// Waveform phase (turns) and amplitude factor of bin k; amplitude 0 outside the support.
__device__ __forceinline__ void wave_bin(const DrawCoef& c, int k, int k_lo, float& t, float& a) {
  t = 0.f;
  a = 0.f;
  if (k >= k_lo && k <= c.kcut) t = waveform_turns(c, k, a);
}

// One block per draw (persistent over draws), n/16 threads.  The D windows go
// through the shared window buffer in turn; the waveform values of the bins a
// thread owns are computed once per draw and shared by the detectors.
// PP: the Stockham passes alternate between two n-point buffers (one barrier per pass)
// instead of running in place in one (two barriers per pass, half the shared memory);
// both forms do the same arithmetic, so their outputs agree bit for bit.
// VEC: the background rows are 8-byte aligned (aligned base, even L), so the crop is
// read as float pairs; otherwise it is read one float at a time.
template <int LOGN, bool VEC, bool PP>
__global__ void __launch_bounds__((1 << LOGN) / 16, LOGN >= 13 ? 1 : 2)
    k_simulate(const DrawCoef* __restrict__ coef, const float* __restrict__ noise, int64_t L,
               const int64_t* __restrict__ offsets, const float* __restrict__ W, const float2* __restrict__ Wp,
               int k_lo, int D, int64_t B, float* __restrict__ y) {
  using PL = Plan16<LOGN>;
  constexpr int n = PL::n, T = PL::T, RL = PL::RL, NB = PL::NB, SLOTS = PL::SLOTS, P = PL::P;
  constexpr int64_t N = 2 * n;
  constexpr int64_t F = n + 1;
  extern __shared__ float2 sm[];
  __shared__ DrawCoef sc;
  float2 (*wv)[T] = reinterpret_cast<float2 (*)[T]>(sm + (PP ? 2 : 1) * n);   // 16 x T waveform values
#define WIDX(s, h, r) (((s) * 2 + (h)) * RL + (r))
  const int t = threadIdx.x;
  const int lane = t & 31;
  const uint32_t x = smem_addr(sm), x2 = x + 8u * (uint32_t)n;
  const float inv_n = 1.0f / (float)n;
  for (int64_t b = blockIdx.x; b < B; b += gridDim.x) {
    for (int i = t; i < (int)(sizeof(DrawCoef) / 16); i += T)
      reinterpret_cast<int4*>(&sc)[i] = __ldg(reinterpret_cast<const int4*>(coef + b) + i);
    int64_t off = __ldg(&offsets[b]);
    off = off < 0 ? 0 : (off > L - N ? L - N : off);   // keep a bad offset inside the stretch
    const int64_t a0 = off & ~(int64_t)1;
    const bool odd = (off & 1) != 0;
    __syncthreads();
    const DrawCoef& c = sc;

    // waveform values (turns, amplitude factor) of the 16 bins this thread owns in the
    // short-radix pass, kept in shared memory as wv[v][t] for the D detectors
#pragma unroll
    for (int s = 0; s < SLOTS; ++s) {
      const int p = t + s * T;
      const int jA = p, jB = p ? NB - p : NB / 2;
#pragma unroll
      for (int r = 0; r < RL; ++r) {
        float tt, aa;
        wave_bin(c, jA + NB * r, k_lo, tt, aa);
        wv[WIDX(s, 0, r)][t] = make_float2(tt, aa);
        wave_bin(c, jB + NB * r, k_lo, tt, aa);
        wv[WIDX(s, 1, r)][t] = make_float2(tt, aa);
      }
    }

    for (int d = 0; d < D; ++d) {
      // forward pass 1 (radix 8, Ns = 1), input straight from the background crop
      {
        const float* row = noise + (int64_t)d * L + a0;
        const float2* row2 = reinterpret_cast<const float2*>(row);
#pragma unroll
        for (int i = 0; i < 2; ++i) {
          const int j = t + i * T;
          float2 v[8];
#pragma unroll
          for (int r = 0; r < 8; ++r) {
            const int m = j + r * (n / 8);
            const int64_t at = (int64_t)d * L + a0 + 2 * m;   // index of row[2 m] in the background
            if constexpr (!VEC) {
              const int o = odd ? 1 : 0;
              v[r] = GWX_IDX_OK(at + o + 1, (int64_t)D * L, 0x101)
                         ? make_float2(__ldg(&row[o + 2 * m]), __ldg(&row[o + 2 * m + 1]))
                         : make_float2(0.f, 0.f);
            } else {
              const float2 q = GWX_IDX_OK(at + 1, (int64_t)D * L, 0x102) ? __ldg(&row2[m]) : make_float2(0.f, 0.f);
              v[r] = q;
              if (odd) {   // the window starts at an odd sample: pair (own .y, next pair's .x)
                float nx;
                if constexpr (T >= 32) {
                  nx = __shfl_down_sync(0xffffffffu, q.x, 1);
                  if (lane == 31) nx = GWX_IDX_OK(at + 2, (int64_t)D * L, 0x103) ? __ldg(&row[2 * m + 2]) : 0.f;
                } else {
                  nx = GWX_IDX_OK(at + 2, (int64_t)D * L, 0x103) ? __ldg(&row[2 * m + 2]) : 0.f;
                }
                v[r] = make_float2(q.y, nx);
              }
            }
          }
          dft8<false, false>(v);
          store_pass<8, 1>(x, j, v);
        }
      }
      __syncthreads();
      uint32_t xf = x;
      if constexpr (PP) {
        xf = FwdMiddlePP<LOGN, 1, P - 2>::run(x, x2, t);
      } else {
        FwdMiddle<LOGN, 1, P - 2>::run(x, t);
      }
      const uint32_t xi = PP ? (xf == x ? x2 : x) : x;

      // last forward pass (radix RL, Ns = NB) on butterfly pairs, frequency-domain
      // step and first inverse pass, all in registers
      const float2 gd = make_float2(c.g[d].x, c.g[d].z);
      const unsigned long long nu = c.nu[d];
      const float* Wd = W + (int64_t)d * F;
      const float2* Wpd = Wp + (int64_t)d * n;
      float2 vA[SLOTS][RL], vB[SLOTS][RL];
#pragma unroll
      for (int s = 0; s < SLOTS; ++s) {
        const int p = t + s * T;
        const int jA = p, jB = p ? NB - p : NB / 2;
        load_strided<RL, NB>(xf, jA, vA[s]);
        load_strided<RL, NB>(xf, jB, vB[s]);
        if constexpr (NB > 1) {
          float2 w[RL];
          pass_twiddles<RL, NB, false>(jA, w);
#pragma unroll
          for (int r = 1; r < RL; ++r) vA[s][r] = cmul(vA[s][r], w[r]);
          pass_twiddles<RL, NB, false>(jB, w);
#pragma unroll
          for (int r = 1; r < RL; ++r) vB[s][r] = cmul(vB[s][r], w[r]);
        }
        dftR<RL, false, false>(vA[s]);
        dftR<RL, false, false>(vB[s]);
        // now vA[s][r] = Z[jA + NB r], vB[s][r] = Z[jB + NB r]
        if (p != 0) {
#pragma unroll
          for (int r = 0; r < RL; ++r) {
            const float2 ea = wv[WIDX(s, 0, r)][t], eb = wv[WIDX(s, 1, RL - 1 - r)][t];
            fd_pair<LOGN>(vA[s][r], vB[s][RL - 1 - r], jA + NB * r, ea.x, ea.y, eb.x, eb.y, gd, nu, Wd, Wpd, inv_n);
          }
        } else {
          fd_dc(vA[s][0], Wpd);
          const float2 eh = wv[WIDX(s, 0, RL / 2)][t];
          fd_half<LOGN>(vA[s][RL / 2], eh.x, eh.y, gd, nu, Wd, Wpd, inv_n);
#pragma unroll
          for (int r = 1; r < RL / 2; ++r) {
            const float2 ea = wv[WIDX(s, 0, r)][t], eb = wv[WIDX(s, 0, RL - r)][t];
            fd_pair<LOGN>(vA[s][r], vA[s][RL - r], NB * r, ea.x, ea.y, eb.x, eb.y, gd, nu, Wd, Wpd, inv_n);
          }
#pragma unroll
          for (int r = 0; r < RL / 2; ++r) {
            const float2 ea = wv[WIDX(s, 1, r)][t], eb = wv[WIDX(s, 1, RL - 1 - r)][t];
            fd_pair<LOGN>(vB[s][r], vB[s][RL - 1 - r], NB / 2 + NB * r, ea.x, ea.y, eb.x, eb.y, gd, nu, Wd, Wpd, inv_n);
          }
        }
        dftR<RL, true, false>(vA[s]);
        dftR<RL, true, false>(vB[s]);
      }
      // in place, every read of the last forward pass must precede the writes below; with
      // two buffers the first inverse pass writes the other one
      if constexpr (!PP) __syncthreads();
#pragma unroll
      for (int s = 0; s < SLOTS; ++s) {
        const int p = t + s * T;
        store_pass<RL, 1>(xi, p, vA[s]);
        store_pass<RL, 1>(xi, p ? NB - p : NB / 2, vB[s]);
      }
      __syncthreads();
      uint32_t xl = x;
      if constexpr (PP) {
        xl = InvMiddlePP<LOGN, 1, P - 2, RL>::run(xi, xf, t);
      } else {
        InvMiddle<LOGN, 1, P - 2, RL>::run(x, t);
      }

      // last inverse pass (radix 8, Ns = n/8), output straight to the whitened batch
      float2* out = reinterpret_cast<float2*>(y + (b * D + d) * N);
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const int j = t + i * T;
        float2 v[8];
        load_strided<8, n / 8>(xl, j, v);
        float2 w[8];
        pass_twiddles<8, n / 8, true>(j, w);
#pragma unroll
        for (int r = 1; r < 8; ++r) v[r] = cmul(v[r], w[r]);
        dft8<true, false>(v);
#pragma unroll
        for (int r = 0; r < 8; ++r)
          if (GWX_IDX_OK((b * D + d) * N + 2 * (j + r * (n / 8)) + 1, B * D * N, 0x104))
            __stcs(&out[j + r * (n / 8)], v[r]);
      }
      __syncthreads();
    }
  }
#undef WIDX
}

// Launch shapes of the fused pass (all give the same output bit for bit): bit 0 selects
// the two-buffer passes, bits 1-2 the resident blocks per SM (1 .. the occupancy limit,
// 0 = the limit).  The autotuner times them per (N, D) and records its choice here.
std::mutex g_sim_tune_mu;
std::map<std::pair<int64_t, int>, int> g_sim_tune;

int sim_default_shape(int64_t N) { return N >= 16384 ? 1 : 0; }

int sim_shape_for(int64_t N, int D) {
  std::lock_guard<std::mutex> lk(g_sim_tune_mu);
  auto it = g_sim_tune.find({N, D});
  return it == g_sim_tune.end() ? sim_default_shape(N) : it->second;
}

void sim_shape_set(int64_t N, int D, int shape) {
  std::lock_guard<std::mutex> lk(g_sim_tune_mu);
  if (shape < 0)
    g_sim_tune.erase({N, D});
  else
    g_sim_tune[{N, D}] = shape;
}

template <int LG, bool VEC, bool PP>
static cudaError_t launch_simulate_lg(const DrawCoef* coef, const float* noise, int64_t L, const int64_t* offsets,
                                      const float* W, const float2* Wp, int k_lo, int D, int64_t B, float* y,
                                      int per_sm_want, cudaStream_t s) {
  constexpr int NT = Plan16<LG>::T;
  // one (or two, PP) window buffers plus 16 waveform values per thread
  const size_t smem = (size_t)(PP ? 2 : 1) * (1 << LG) * sizeof(float2) + (size_t)16 * NT * sizeof(float2);
  cudaError_t e = cudaFuncSetAttribute(k_simulate<LG, VEC, PP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per_sm = 0;
  e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_simulate<LG, VEC, PP>, NT, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  if (per_sm_want > 0 && per_sm_want < per_sm) per_sm = per_sm_want;
  int64_t grid = (int64_t)sms * per_sm;
  if (grid > B) grid = B;
  k_simulate<LG, VEC, PP><<<(unsigned)grid, NT, smem, s>>>(coef, noise, L, offsets, W, Wp, k_lo, D, B, y);
  return cudaGetLastError();
}

cudaError_t launch_simulate_fused(const DrawCoef* coef, const float* noise, int64_t L, const int64_t* offsets,
                                  const float* W, const float2* Wp, int k_lo, int D, int64_t B, int64_t N, double fs,
                                  float* y, cudaStream_t s, int shape) {
  if (B <= 0) return cudaSuccess;
  if (shape < 0) shape = sim_shape_for(N, D);
  const bool pp = (shape & 1) != 0;
  const int per_sm = (shape >> 1) & 3;
  const bool vec = ((uintptr_t)noise % 8 == 0) && (L % 2 == 0);
  return dispatch_log<7, 13>(ilog2_exact(N / 2), [&](auto cst) {
    constexpr int LG = decltype(cst)::value;
    if (pp)
      return vec ? launch_simulate_lg<LG, true, true>(coef, noise, L, offsets, W, Wp, k_lo, D, B, y, per_sm, s)
                 : launch_simulate_lg<LG, false, true>(coef, noise, L, offsets, W, Wp, k_lo, D, B, y, per_sm, s);
    return vec ? launch_simulate_lg<LG, true, false>(coef, noise, L, offsets, W, Wp, k_lo, D, B, y, per_sm, s)
               : launch_simulate_lg<LG, false, false>(coef, noise, L, offsets, W, Wp, k_lo, D, B, y, per_sm, s);
  });
}

}  // namespace gwx
