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
#include "fft16r.cuh"
#include "tc05.cuh"
#include "waveform.cuh"

namespace gwx {

cudaError_t init_tables_fused() {
  const cudaError_t e = fill_tables_for_this_tu();
  return e == cudaSuccess ? fill_tw16_for_this_tu() : e;
}
cudaError_t debug_take_fused(unsigned long long* v) { return dbg_take_this_tu(v); }

// Frequency-domain step of one real-FFT bin pair (k, nk = n - k), 0 < k < n, k != n/2,
// done on the half-length transform Z directly.  With s = W/n and theta = 2 pi k/N, whitening
// in that domain is
//   Z'_k = alpha_k Z_k + i beta Z*_nk,   Z'_nk = alpha_nk Z_nk + i beta Z*_k,
//   alpha_k = A - sin(theta) Dl,  alpha_nk = A + sin(theta) Dl,  beta = cos(theta) Dl,
//   A = (s_k + s_nk)/2, Dl = (s_k - s_nk)/2
// (unpack X_k, X_nk from Z_k, Z_nk, scale by s, repack); the injected strain H (continuous
// FT times fs) adds
//   Z'_k += p s_k H_k + q s_nk conj(H_nk),  p = (1 + i conj w)/2, q = (1 - i conj w)/2,
// w = e^{-i theta}, and the mirrored terms with w_nk = -conj(w) for Z'_nk.
// (tk, ak), (tnk, ank): waveform phase in turns and amplitude factor k^-7/6 of the two
// bins (ak = 0 outside the support); (cs, sn) = (cos, sin) theta.
template <int LOGN>
__device__ __forceinline__ void fd_pair(float2& zk, float2& znk, int k, float tk, float ak, float tnk, float ank,
                                        float2 gd, unsigned long long nu, float sk, float snk, float cs, float sn) {
  constexpr int n = 1 << LOGN;
  const float A = 0.5f * (sk + snk), Dl = 0.5f * (sk - snk);
  const float alk = fmaf(-sn, Dl, A), alnk = fmaf(sn, Dl, A), be = __fmul_rn(cs, Dl);
  const float2 a = zk, b = znk;
  zk = make_float2(fmaf(alk, a.x, be * b.y), fmaf(alk, a.y, be * b.x));
  znk = make_float2(fmaf(alnk, b.x, be * a.y), fmaf(alnk, b.y, be * a.x));
  if (ak != 0.f || ank != 0.f) {
    float2 hk = make_float2(0.f, 0.f), hnk = hk;
    if (ak != 0.f) hk = cscale(cmul(gd, expm2pi(tk + lin_turns(nu, k))), ak * sk);
    if (ank != 0.f) hnk = cscale(cmul(gd, expm2pi(tnk + lin_turns(nu, n - k))), ank * snk);
    // hk, hnk now carry s_k and s_nk
    const float pr = 0.5f * (1.0f - sn), qr = 0.5f * (1.0f + sn), wi = 0.5f * cs;
    // Z'_k += p hk + q conj(hnk), p = (pr, wi), q = (qr, -wi)
    zk.x += pr * hk.x - wi * hk.y + qr * hnk.x - wi * hnk.y;
    zk.y += pr * hk.y + wi * hk.x - qr * hnk.y - wi * hnk.x;
    // Z'_nk += p' hnk + q' conj(hk), p' = (pr, -wi), q' = (qr, wi)
    znk.x += pr * hnk.x + wi * hnk.y + qr * hk.x + wi * hk.y;
    znk.y += pr * hnk.y - wi * hnk.x - qr * hk.y + wi * hk.x;
  }
}

// The bin k = n/2, which pairs with itself (theta = pi/2: alpha = s_h, beta = 0, p = 0, q = 1).
template <int LOGN>
__device__ __forceinline__ void fd_half(float2& z, float t, float a, float2 gd, unsigned long long nu, float sh) {
  constexpr int h = (1 << LOGN) / 2;
  z = cscale(z, sh);
  if (a != 0.f) {
    const float2 hh = cscale(cmul(gd, expm2pi(t + lin_turns(nu, h))), a * sh);
    z.x += hh.x;
    z.y -= hh.y;
  }
}

// DC and Nyquist (carried together in element 0); the waveform is zero there.
__device__ __forceinline__ void fd_dc(float2& z0, float s0, float sn) {
  const float a = 0.5f * (s0 + sn), b = 0.5f * (s0 - sn);
  const float2 v = z0;
  z0 = make_float2(fmaf(a, v.x, b * v.y), fmaf(b, v.x, a * v.y));
}

// e^{i pi q/16} for a sixteenth-of-pi count q (folds to constants once q is known).
__device__ __forceinline__ float2 eipi16(int q) {
  constexpr float c[9] = {1.0f, 0.980785250663757324f, 0.923879504203796387f, 0.831469595432281494f,
                          0.707106769084930420f, 0.555570244789123535f, 0.382683426141738892f,
                          0.195090323686599731f, 0.0f};
  const int m = q & 31;
  const int r = m & 15;   // e^{i pi m/16} = (-1)^(m >= 16) e^{i pi r/16}
  const float2 u = r <= 8 ? make_float2(c[r], c[8 - r]) : make_float2(-c[16 - r], c[r - 8]);
  return m >= 16 ? make_float2(-u.x, -u.y) : u;
}
// u e^{i pi q/16}: quarter turns exactly, other angles by a product with the constant
// (written with explicit fused products, so that it rounds alike wherever it is inlined).
__device__ __forceinline__ float2 rot_pi16(float2 u, int q) {
  switch (q & 31) {
    case 0: return u;
    case 8: return make_float2(-u.y, u.x);
    case 16: return make_float2(-u.x, -u.y);
    case 24: return make_float2(u.y, -u.x);
    default: {
      const float2 c = eipi16(q);
      return make_float2(fmaf(u.x, c.x, -__fmul_rn(u.y, c.y)), fmaf(u.x, c.y, __fmul_rn(u.y, c.x)));
    }
  }
}

// Waveform phase (turns) and amplitude factor of bin k; amplitude 0 outside the support.
__device__ __forceinline__ void wave_bin(const DrawCoef& c, int k, int k_lo, float& t, float& a) {
  t = 0.f;
  a = 0.f;
  if (k >= k_lo && k <= c.kcut) t = waveform_turns(c, k, a);
}

// x e^{-2 pi i e/8} for an eighth-turn count e (folds to a few additions once e is known).
__device__ __forceinline__ float2 rot_turns8(float2 x, int e) {
  constexpr float h = 0.707106769084930419921875f;   // nearest float to sqrt(1/2)
  switch (e & 7) {
    case 0: return x;
    case 1: return make_float2(h * (x.x + x.y), h * (x.y - x.x));
    case 2: return mul_mi<false>(x);
    case 3: return make_float2(h * (x.y - x.x), -h * (x.x + x.y));
    case 4: return make_float2(-x.x, -x.y);
    case 5: return make_float2(-h * (x.x + x.y), h * (x.x - x.y));
    case 6: return mul_mi<true>(x);
    default: return make_float2(h * (x.x - x.y), h * (x.x + x.y));
  }
}

// Pass plan of the fused kernel for n = 2^LOGN complex points, 16 values per thread.
// R16: radix-16 passes (one butterfly per thread, swizzle sw16) when log2 n is not a
// multiple of 4, else radix-8 passes (two butterflies per thread, swizzle sw).  Either
// way the forward transform ends with the short radix RL and the inverse starts with it.
template <int LOGN>
struct SimPlan {
  static constexpr bool R16 = (LOGN % 4) != 0;
  static constexpr int n = 1 << LOGN;
  static constexpr int T = n / 16;
  static constexpr int RL = R16 ? (1 << (LOGN % 4)) : Plan16<LOGN>::RL;
  static constexpr int NB = n / RL;
  static constexpr int SLOTS = 8 / RL;
  static constexpr int MID = R16 ? LOGN / 4 - 1 : Plan16<LOGN>::P - 2;   // middle passes per direction
};

template <bool R16, int R, int nR>
__device__ __forceinline__ void sim_load(uint32_t x, int j, float2* v) {
  if constexpr (R16) load_strided16<R, nR>(x, j, v);
  else load_strided<R, nR>(x, j, v);
}
template <bool R16, int R, int Ns>
__device__ __forceinline__ void sim_store(uint32_t x, int j, const float2* v) {
  if constexpr (R16) store_pass16<R, Ns>(x, j, v);
  else store_pass<R, Ns>(x, j, v);
}

// One crop value pair of the background: the complex point m (samples 2m, 2m + 1 of the
// window) of detector row d.  at = index of row[2 m] in the background, D L its size.
template <bool VEC, int T>
__device__ __forceinline__ float2 crop_point(const float* row, int m, bool odd, int lane, int64_t at, int64_t DL) {
  if constexpr (!VEC) {
    const int o = odd ? 1 : 0;
    return GWX_IDX_OK(at + o + 1, DL, 0x101) ? make_float2(__ldg(&row[o + 2 * m]), __ldg(&row[o + 2 * m + 1]))
                                            : make_float2(0.f, 0.f);
  } else {
    const float2* row2 = reinterpret_cast<const float2*>(row);
    const float2 q = GWX_IDX_OK(at + 1, DL, 0x102) ? __ldg(&row2[m]) : make_float2(0.f, 0.f);
    if (!odd) return q;
    // the window starts at an odd sample: pair (own .y, next pair's .x)
    float nx;
    if constexpr (T >= 32) {
      nx = __shfl_down_sync(0xffffffffu, q.x, 1);
      if (lane == 31) nx = GWX_IDX_OK(at + 2, DL, 0x103) ? __ldg(&row[2 * m + 2]) : 0.f;
    } else {
      nx = GWX_IDX_OK(at + 2, DL, 0x103) ? __ldg(&row[2 * m + 2]) : 0.f;
    }
    return make_float2(q.y, nx);
  }
}

// ---------------------------------------------------------------- staging
// Bulk asynchronous copies (global -> shared) of the next window's background crop and
// the next detector's whitening filter, each completing on an mbarrier.
__device__ int g_sim_status;                 // a block gave up waiting for its own copies
constexpr uint32_t kStagePolls = 1u << 20;   // polls of a staging barrier before giving up

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}
__device__ __forceinline__ void proxy_fence_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Crop of window (b, d) for the staged form: the 16-byte aligned start of the copy, its size
// and the float offset o of the window's first sample within it.
struct CropCopy {
  int64_t src;   // first float copied
  uint32_t bytes;
  int o;
};
__device__ __forceinline__ CropCopy crop_copy(const int64_t* offsets, int64_t b, int d, int64_t L, int64_t N,
                                              int64_t DL) {
  int64_t off = __ldg(&offsets[b]);
  off = off < 0 ? 0 : (off > L - N ? L - N : off);   // keep a bad offset inside the stretch
  const int64_t first = (int64_t)d * L + off;
  CropCopy c;
  c.src = first & ~(int64_t)3;
  c.o = (int)(first - c.src);
  const int64_t cnt = (N + 4 < DL - c.src) ? N + 4 : DL - c.src;   // L % 4 == 0: a multiple of 4
  c.bytes = (uint32_t)(4 * cnt);
  return c;
}

// One block per draw (persistent over draws), n/16 threads.  The D windows go
// through the shared window buffer in turn; the waveform values of the bins a
// thread owns are computed once per draw and shared by the detectors.
// PP: the Stockham passes alternate between two n-point buffers (one barrier per pass)
// instead of running in place in one (two barriers per pass, half the shared memory);
// both forms do the same arithmetic, so their outputs agree bit for bit.
// VEC: the background rows are 8-byte aligned (aligned base, even L), so the crop is
// read as float pairs; otherwise it is read one float at a time.
// ST (in place only; 16-byte aligned background and filter, L % 4 == 0): the next window's
// crop and the next detector's filter arrive in shared staging buffers by bulk asynchronous
// copies issued one window ahead, so no pass waits on a global load; same arithmetic again.
// Wcap: floats of the filter allocation W (the staged copies may read up to it).
template <int LOGN, bool VEC, bool PP, bool ST>
__global__ void __launch_bounds__((1 << LOGN) / 16, LOGN >= 13 ? 1 : 2)
    k_simulate(const DrawCoef* __restrict__ coef, const float* __restrict__ noise, int64_t L,
               const int64_t* __restrict__ offsets, const float* __restrict__ W, int64_t Wcap, int k_lo, int D,
               int64_t B, float* __restrict__ y) {
  static_assert(!(ST && PP), "staging uses the in-place passes");
  using PL = SimPlan<LOGN>;
  constexpr bool R16 = PL::R16;
  constexpr int n = PL::n, T = PL::T, RL = PL::RL, NB = PL::NB, SLOTS = PL::SLOTS, MID = PL::MID;
  constexpr int64_t N = 2 * n;
  constexpr int64_t F = n + 1;
  extern __shared__ float2 sm[];
  __shared__ DrawCoef sc;
  __shared__ __align__(8) uint64_t bars[2];   // staging barriers: crop, filter
  __shared__ int s_o[2];                      // offsets within the staged crop and filter
  float2 (*wv)[T] = reinterpret_cast<float2 (*)[T]>(sm + (PP ? 2 : 1) * n);   // 16 x T waveform values
  float* crop_s = reinterpret_cast<float*>(sm + 2 * n);                        // ST: N + 4 floats
  float* w_s = crop_s + N + 4;                                                  // ST: n + 4 floats
#define WIDX(s, h, r) (((s) * 2 + (h)) * RL + (r))
  const int t = threadIdx.x;
  const int lane = t & 31;
  const uint32_t x = smem_addr(sm), x2 = x + 8u * (uint32_t)n;
  const float inv_n = 1.0f / (float)n;
  const int64_t DL = (int64_t)D * L;
  const uint32_t bar_c = smem_addr(&bars[0]), bar_w = smem_addr(&bars[1]);
  uint32_t ph_c = 0, ph_w = 0;   // parity of the staging barriers' next phase

  // e^{i pi t/n}: the pair pass's twiddles and the packing angles of this thread's bins
  // follow from it by fixed rotations
  const float2 bt = cconj(__ldg(&g_tw[t << (13 - LOGN)]));

  if constexpr (ST) {
    if (t == 0) {
      tc::mbar_init(bar_c, 1);
      tc::mbar_init(bar_w, 1);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
      if (blockIdx.x < B) {
        const CropCopy cc = crop_copy(offsets, blockIdx.x, 0, L, N, DL);
        s_o[0] = cc.o;
        tc::mbar_expect_tx(bar_c, cc.bytes);
        bulk_g2s(smem_addr(crop_s), noise + cc.src, cc.bytes, bar_c);
        const int64_t wsrc = 0;
        s_o[1] = 0;
        const uint32_t wb = (uint32_t)(4 * ((int64_t)n + 4 < Wcap - wsrc ? (int64_t)n + 4 : Wcap - wsrc));
        tc::mbar_expect_tx(bar_w, wb);
        bulk_g2s(smem_addr(w_s), W + wsrc, wb, bar_w);
      }
    }
    __syncthreads();
  }

  for (int64_t b = blockIdx.x; b < B; b += gridDim.x) {
    for (int i = t; i < (int)(sizeof(DrawCoef) / 16); i += T)
      reinterpret_cast<int4*>(&sc)[i] = __ldg(reinterpret_cast<const int4*>(coef + b) + i);
    int64_t off = 0;
    if constexpr (!ST) {
      off = __ldg(&offsets[b]);
      off = off < 0 ? 0 : (off > L - N ? L - N : off);   // keep a bad offset inside the stretch
    }
    const int64_t a0 = off & ~(int64_t)1;
    const bool odd = (off & 1) != 0;
    __syncthreads();
    const DrawCoef& c = sc;

    // waveform values (turns, amplitude factor) of the 16 bins this thread owns in the
    // short-radix pass, kept in shared memory as wv[v][t] for the D detectors (a rolled
    // loop: the evaluation is long, and 32 inlined copies crowd the instruction cache)
#pragma unroll 1
    for (int s = 0; s < SLOTS; ++s) {
      const int p = t + s * T;
      const int jA = p, jB = p ? NB - p : NB / 2;
#pragma unroll 1
      for (int r = 0; r < RL; ++r) {
        float tt, aa;
        wave_bin(c, jA + NB * r, k_lo, tt, aa);
        wv[WIDX(s, 0, r)][t] = make_float2(tt, aa);
        wave_bin(c, jB + NB * r, k_lo, tt, aa);
        wv[WIDX(s, 1, r)][t] = make_float2(tt, aa);
      }
    }

    for (int d = 0; d < D; ++d) {
      // the window after this one: (b, d + 1), else the block's next draw
      const bool more = d + 1 < D || b + gridDim.x < B;
      const int64_t b_next = d + 1 < D ? b : b + gridDim.x;
      const int d_next = d + 1 < D ? d + 1 : 0;

      // first forward pass (Ns = 1), input straight from the background crop
      bool ok = true;
      if constexpr (ST) {
        ok = tc::mbar_wait(bar_c, ph_c, kStagePolls);
        ph_c ^= 1u;
        const int o = s_o[0];
        const uint32_t cs0 = smem_addr(crop_s);
        // complex point m = (crop[o + 2m], crop[o + 2m + 1])
        auto staged = [&](int m) -> float2 {
          if (!(o & 1)) return lds2(cs0 + 4u * (uint32_t)(o + 2 * m));
          if constexpr (T < 32) {
            return make_float2(crop_s[o + 2 * m], crop_s[o + 2 * m + 1]);
          } else {
            // odd start: (own pair's .y, the next lane's .x)
            const float2 q = lds2(cs0 + 4u * (uint32_t)(o - 1 + 2 * m));
            float nx = __shfl_down_sync(0xffffffffu, q.x, 1);
            if (lane == 31) nx = crop_s[o + 2 * m + 1];
            return make_float2(q.y, nx);
          }
        };
        if constexpr (R16) {
          float2 v[16];
#pragma unroll
          for (int r = 0; r < 16; ++r) v[r] = staged(t + r * (n / 16));
          dft16<false>(v);
          store_pass16<16, 1>(x, t, v);
        } else {
#pragma unroll
          for (int i = 0; i < 2; ++i) {
            const int j = t + i * T;
            float2 v[8];
#pragma unroll
            for (int r = 0; r < 8; ++r) v[r] = staged(j + r * (n / 8));
            dft8<false, false>(v);
            store_pass<8, 1>(x, j, v);
          }
        }
      } else {
        const float* row = noise + (int64_t)d * L + a0;
        const int64_t at0 = (int64_t)d * L + a0;
        if constexpr (R16) {
          float2 v[16];
#pragma unroll
          for (int r = 0; r < 16; ++r) {
            const int m = t + r * (n / 16);
            v[r] = crop_point<VEC, T>(row, m, odd, lane, at0 + 2 * m, DL);
          }
          dft16<false>(v);
          store_pass16<16, 1>(x, t, v);
        } else {
#pragma unroll
          for (int i = 0; i < 2; ++i) {
            const int j = t + i * T;
            float2 v[8];
#pragma unroll
            for (int r = 0; r < 8; ++r) {
              const int m = j + r * (n / 8);
              v[r] = crop_point<VEC, T>(row, m, odd, lane, at0 + 2 * m, DL);
            }
            dft8<false, false>(v);
            store_pass<8, 1>(x, j, v);
          }
        }
      }
      if constexpr (ST) {
        if (__syncthreads_or(!ok)) {
          // the crop never landed: record it, let this block's copies finish, stop
          if (t == 0) {
            atomicExch(&g_sim_status, 1);
            tc::mbar_wait(bar_c, ph_c ^ 1u, kStagePolls);
            tc::mbar_wait(bar_w, ph_w, kStagePolls);
          }
          return;
        }
        // every read of the staged crop is done: fetch the next window's
        if (t == 0 && more) {
          const CropCopy cc = crop_copy(offsets, b_next, d_next, L, N, DL);
          s_o[0] = cc.o;
          proxy_fence_async();
          tc::mbar_expect_tx(bar_c, cc.bytes);
          bulk_g2s(smem_addr(crop_s), noise + cc.src, cc.bytes, bar_c);
        }
      } else {
        __syncthreads();
      }
      uint32_t xf = x;
      if constexpr (R16) {
        xf = FwdMiddle16<LOGN, 1, MID, PP>::run(x, x2, t);
      } else if constexpr (PP) {
        xf = FwdMiddlePP<LOGN, 1, MID>::run(x, x2, t);
      } else {
        FwdMiddle<LOGN, 1, MID>::run(x, t);
      }
      const uint32_t xi = PP ? (xf == x ? x2 : x) : x;

      // last forward pass (radix RL, Ns = NB) on butterfly pairs, frequency-domain
      // step and first inverse pass, all in registers
      const float2 gd = make_float2(c.g[d].x, c.g[d].z);
      const unsigned long long nu = c.nu[d];
      const float* Wd = W + (int64_t)d * F;
      int ow = 0;
      if constexpr (ST) {
        ok = tc::mbar_wait(bar_w, ph_w, kStagePolls);
        ph_w ^= 1u;
        ow = s_o[1];
      }
      // s_k = W_k / n for bin k of this detector, rounded on its own (an explicit product
      // cannot be fused into a later addition, so every launch shape rounds alike)
      auto s_of = [&](int k) -> float { return __fmul_rn(ST ? w_s[ow + k] : __ldg(&Wd[k]), inv_n); };
      float2 vA[SLOTS][RL], vB[SLOTS][RL];
#pragma unroll
      for (int s = 0; s < SLOTS; ++s) {
        const int p = t + s * T;
        const int jA = p, jB = p ? NB - p : NB / 2;
        // u = e^{i pi jA/n}: angle of bin jA; the pass twiddle of butterfly jA is conj(u)^2
        const float2 u = rot_pi16(bt, s);
        sim_load<R16, RL, NB>(xf, jA, vA[s]);
        sim_load<R16, RL, NB>(xf, jB, vB[s]);
        if constexpr (NB > 1) {
          float2 w[RL];
          if constexpr (!R16 && RL == 8) {
            pass_twiddles<RL, NB, false>(jA, w);
          } else {
            w[1] = cconj(make_float2(fmaf(u.x, u.x, -__fmul_rn(u.y, u.y)), __fmul_rn(2.f * u.x, u.y)));
            if constexpr (RL >= 4) {
              w[2] = make_float2(fmaf(w[1].x, w[1].x, -w[1].y * w[1].y), 2.f * w[1].x * w[1].y);
              w[3] = cmul(w[1], w[2]);
            }
            if constexpr (RL == 8) {
              w[4] = make_float2(fmaf(w[2].x, w[2].x, -w[2].y * w[2].y), 2.f * w[2].x * w[2].y);
#pragma unroll
              for (int r = 5; r < 8; ++r) w[r] = cmul(w[4], w[r - 4]);
            }
          }
#pragma unroll
          for (int r = 1; r < RL; ++r) vA[s][r] = cmul(vA[s][r], w[r]);
          // butterfly NB - p: e^{-2 pi i (NB - p) r/n} = e^{-2 pi i r/RL} conj(w_p^r); for
          // p = 0 the partner is NB/2, with e^{-2 pi i r/(2 RL)}.  (The radix-8 plan's
          // radix-8 pair pass, with no registers to spare, reads the table instead.)
          if constexpr (!R16 && RL == 8) {
            pass_twiddles<RL, NB, false>(jB, w);
#pragma unroll
            for (int r = 1; r < RL; ++r) vB[s][r] = cmul(vB[s][r], w[r]);
          } else {
#pragma unroll
            for (int r = 1; r < RL; ++r) {
              const float2 wb = p != 0 ? rot_turns8(cconj(w[r]), r * (8 / RL))
                                       : cconj(eipi16(r * (16 / RL)));   // e^{-i pi r/RL}
              vB[s][r] = cmul(vB[s][r], wb);
            }
          }
        }
        dftR<RL, false, false>(vA[s]);
        dftR<RL, false, false>(vB[s]);
        // now vA[s][r] = Z[jA + NB r], vB[s][r] = Z[jB + NB r]
        if (p != 0) {
#pragma unroll
          for (int r = 0; r < RL; ++r) {
            const float2 ea = wv[WIDX(s, 0, r)][t], eb = wv[WIDX(s, 1, RL - 1 - r)][t];
            const int k = jA + NB * r;
            const float2 e = rot_pi16(u, r * (16 / RL));   // e^{i pi k/n}
            fd_pair<LOGN>(vA[s][r], vB[s][RL - 1 - r], k, ea.x, ea.y, eb.x, eb.y, gd, nu, s_of(k), s_of(n - k), e.x,
                          e.y);
          }
        } else {
          fd_dc(vA[s][0], s_of(0), s_of(n));
          const float2 eh = wv[WIDX(s, 0, RL / 2)][t];
          fd_half<LOGN>(vA[s][RL / 2], eh.x, eh.y, gd, nu, s_of(n / 2));
#pragma unroll
          for (int r = 1; r < RL / 2; ++r) {
            const float2 ea = wv[WIDX(s, 0, r)][t], eb = wv[WIDX(s, 0, RL - r)][t];
            const int k = NB * r;
            const float2 e = eipi16(r * (16 / RL));
            fd_pair<LOGN>(vA[s][r], vA[s][RL - r], k, ea.x, ea.y, eb.x, eb.y, gd, nu, s_of(k), s_of(n - k), e.x, e.y);
          }
#pragma unroll
          for (int r = 0; r < RL / 2; ++r) {
            const float2 ea = wv[WIDX(s, 1, r)][t], eb = wv[WIDX(s, 1, RL - 1 - r)][t];
            const int k = NB / 2 + NB * r;
            const float2 e = eipi16(8 / RL + r * (16 / RL));
            fd_pair<LOGN>(vB[s][r], vB[s][RL - 1 - r], k, ea.x, ea.y, eb.x, eb.y, gd, nu, s_of(k), s_of(n - k), e.x,
                          e.y);
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
        sim_store<R16, RL, 1>(xi, p, vA[s]);
        sim_store<R16, RL, 1>(xi, p ? NB - p : NB / 2, vB[s]);
      }
      if constexpr (ST) {
        if (__syncthreads_or(!ok)) {
          if (t == 0) {
            atomicExch(&g_sim_status, 1);
            tc::mbar_wait(bar_w, ph_w ^ 1u, kStagePolls);
            if (more) tc::mbar_wait(bar_c, ph_c, kStagePolls);
          }
          return;
        }
        // every read of the staged filter is done: fetch the next window's detector
        if (t == 0 && more) {
          const int64_t first = (int64_t)d_next * F;
          const int64_t wsrc = first & ~(int64_t)3;
          s_o[1] = (int)(first - wsrc);
          const uint32_t wb = (uint32_t)(4 * ((int64_t)n + 4 < Wcap - wsrc ? (int64_t)n + 4 : Wcap - wsrc));
          proxy_fence_async();
          tc::mbar_expect_tx(bar_w, wb);
          bulk_g2s(smem_addr(w_s), W + wsrc, wb, bar_w);
        }
      } else {
        __syncthreads();
      }
      uint32_t xl = x;
      if constexpr (R16) {
        xl = InvMiddle16<LOGN, 1, MID, RL, PP>::run(xi, xf, t);
      } else if constexpr (PP) {
        xl = InvMiddlePP<LOGN, 1, MID, RL>::run(xi, xf, t);
      } else {
        InvMiddle<LOGN, 1, MID, RL>::run(x, t);
      }

      // last inverse pass (Ns = n/R), output straight to the whitened batch
      float2* out = reinterpret_cast<float2*>(y + (b * D + d) * N);
      if constexpr (R16) {
        float2 v[16];
        load_strided16<16, n / 16>(xl, t, v);
        float2 w[16];
        tw16<n / 16, true>(t, w);
#pragma unroll
        for (int r = 1; r < 16; ++r) v[r] = cmul(v[r], w[r]);
        dft16<true>(v);
#pragma unroll
        for (int r = 0; r < 16; ++r)
          if (GWX_IDX_OK((b * D + d) * N + 2 * (t + r * (n / 16)) + 1, B * D * N, 0x104))
            __stcs(&out[t + r * (n / 16)], v[r]);
      } else {
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
      }
      __syncthreads();
    }
  }
#undef WIDX
}

// Launch shapes of the fused pass (all give the same output bit for bit): bit 0 selects
// the two-buffer passes, bits 1-2 the resident blocks per SM (1 .. the occupancy limit,
// 0 = the limit), bit 3 the staged crop and filter (in place; ignored when the background,
// its row length or the filter are not aligned for bulk copies).  The autotuner times them
// per (N, D) and records its choice here.
std::mutex g_sim_tune_mu;
std::map<std::pair<int64_t, int>, int> g_sim_tune;

int sim_default_shape(int64_t N) { return N >= 8192 ? 8 : 0; }

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

bool sim_can_stage(const float* noise, int64_t L, const float* W, int64_t N) {
  // one in-place window, the waveform values and both staging buffers in one block
  const size_t smem = (size_t)14 * (size_t)N + 32;   // 28 n + 32 bytes
  return (uintptr_t)noise % 16 == 0 && L % 4 == 0 && (uintptr_t)W % 16 == 0 && smem <= (size_t)227 * 1024;
}

template <int LG, bool VEC, bool PP, bool ST>
static cudaError_t launch_simulate_lg(const DrawCoef* coef, const float* noise, int64_t L, const int64_t* offsets,
                                      const float* W, int64_t Wcap, int k_lo, int D, int64_t B, float* y,
                                      int per_sm_want, cudaStream_t s) {
  constexpr int NT = Plan16<LG>::T;
  constexpr size_t n = (size_t)1 << LG;
  // one (or two, PP) window buffers plus 16 waveform values per thread; staged: the crop
  // (N + 4 floats) and the filter (n + 4 floats) after them
  const size_t smem = (PP ? 2 : 1) * n * sizeof(float2) + (size_t)16 * NT * sizeof(float2) +
                      (ST ? (2 * n + 4 + n + 4) * sizeof(float) : 0);
  auto kern = k_simulate<LG, VEC, PP, ST>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per_sm = 0;
  e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  if (per_sm_want > 0 && per_sm_want < per_sm) per_sm = per_sm_want;
  int64_t grid = (int64_t)sms * per_sm;
  if (grid > B) grid = B;
  kern<<<(unsigned)grid, NT, smem, s>>>(coef, noise, L, offsets, W, Wcap, k_lo, D, B, y);
  return cudaGetLastError();
}

cudaError_t launch_simulate_fused(const DrawCoef* coef, const float* noise, int64_t L, const int64_t* offsets,
                                  const float* W, int64_t Wcap, int k_lo, int D, int64_t B, int64_t N, double fs,
                                  float* y, cudaStream_t s, int shape) {
  (void)fs;
  if (B <= 0) return cudaSuccess;
  if (shape < 0) shape = sim_shape_for(N, D);
  const bool st = (shape & 8) != 0 && sim_can_stage(noise, L, W, N);
  const bool pp = !st && (shape & 1) != 0;
  const int per_sm = (shape >> 1) & 3;
  const bool vec = ((uintptr_t)noise % 8 == 0) && (L % 2 == 0);
  return dispatch_log<7, 13>(ilog2_exact(N / 2), [&](auto cst) {
    constexpr int LG = decltype(cst)::value;
    if (st) return launch_simulate_lg<LG, true, false, true>(coef, noise, L, offsets, W, Wcap, k_lo, D, B, y, per_sm, s);
    if (pp)
      return vec ? launch_simulate_lg<LG, true, true, false>(coef, noise, L, offsets, W, Wcap, k_lo, D, B, y, per_sm, s)
                 : launch_simulate_lg<LG, false, true, false>(coef, noise, L, offsets, W, Wcap, k_lo, D, B, y, per_sm, s);
    return vec ? launch_simulate_lg<LG, true, false, false>(coef, noise, L, offsets, W, Wcap, k_lo, D, B, y, per_sm, s)
               : launch_simulate_lg<LG, false, false, false>(coef, noise, L, offsets, W, Wcap, k_lo, D, B, y, per_sm, s);
  });
}

cudaError_t sim_status(int* status) {
  const int zero = 0;
  cudaError_t e = cudaMemcpyFromSymbol(status, g_sim_status, sizeof(int));
  if (e == cudaSuccess && *status != 0) e = cudaMemcpyToSymbol(g_sim_status, &zero, sizeof(int));
  return e;
}

}  // namespace gwx
