// k_weights.cu -- per-event importance weights, Kish effective sample size and
// importance-sampling evidence for samples scored by the likelihood (A8 downstream):
//   ln w_s = ln L_s + log_ratio_s,   weight_s = w_s / sum_e w,
//   ess_e = (sum w)^2 / sum w^2,   efficiency_e = ess_e / S_e,   ln Z_e = ln((1/S_e) sum w).
// Two launches over an E x IW_CHUNKS grid: per chunk the largest ln w and the sums of
// exp(ln w - max) and its square; then every block merges its event's chunk partials
// and writes its chunk's weights (chunk 0 also writes the event's ess, efficiency, ln Z).
// exp is evaluated in FP32 on ln w - max split into a float and its float remainder,
// exp(hi + lo) = exp(hi) (1 + lo) (relative error ~2e-7); sums and merges are FP64.
#include <math.h>

#include "gwx_internal.h"

namespace gwx {

constexpr int IW_THREADS = 256;

struct IwPartial {
  double m, s1, s2;
};

__device__ __forceinline__ double iw_lnw(const double* lnl, const double* ratio, int64_t s) {
  return ratio ? lnl[s] + ratio[s] : lnl[s];
}

// exp(d) for d <= 0 (or -inf), relative error ~2e-7.
__device__ __forceinline__ float iw_exp(double d) {
  if (!(d > -200.0)) return d != d ? __int_as_float(0x7fc00000) : 0.f;
  const float hi = (float)d;
  const float lo = (float)(d - (double)hi);
  const float e = expf(hi);
  return fmaf(e, lo, e);
}

// Chunk [a, b) of event e: the clamped event range split into `chunks` pieces.
__device__ __forceinline__ void iw_chunk(const int64_t* off, int64_t S, int e, int c, int chunks, int64_t& a,
                                         int64_t& b, int64_t& n) {
  int64_t lo = off[e], hi = off[e + 1];
  lo = lo < 0 ? 0 : (lo > S ? S : lo);
  hi = hi < lo ? lo : (hi > S ? S : hi);
  n = hi - lo;
  a = lo + n * c / chunks;
  b = lo + n * (c + 1) / chunks;
}

template <typename T, typename Op>
__device__ T block_reduce(T v, Op op, T* sh) {
  for (int o = 16; o > 0; o >>= 1) v = op(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[w] = v;
  __syncthreads();
  v = sh[0];
  for (int i = 1; i < nw; ++i) v = op(v, sh[i]);
  return v;
}

struct MaxOp {
  __device__ double operator()(double a, double b) const { return fmax(a, b); }
};
struct AddOp {
  __device__ double operator()(double a, double b) const { return a + b; }
};

__global__ void __launch_bounds__(IW_THREADS) k_iw_partial(const double* __restrict__ lnl,
                                                           const double* __restrict__ ratio,
                                                           const int64_t* __restrict__ off, int64_t S, int chunks,
                                                           IwPartial* __restrict__ part) {
  __shared__ double sh[IW_THREADS / 32];
  const int e = blockIdx.x, c = blockIdx.y;
  int64_t a, b, n;
  iw_chunk(off, S, e, c, chunks, a, b, n);
  double m = -INFINITY;
  for (int64_t s = a + threadIdx.x; s < b; s += blockDim.x) m = fmax(m, iw_lnw(lnl, ratio, s));
  m = block_reduce(m, MaxOp(), sh);
  double s1 = 0.0, s2 = 0.0;
  if (m > -INFINITY) {
    for (int64_t s = a + threadIdx.x; s < b; s += blockDim.x) {
      const double w = (double)iw_exp(iw_lnw(lnl, ratio, s) - m);
      s1 += w;
      s2 = fma(w, w, s2);
    }
  }
  s1 = block_reduce(s1, AddOp(), sh);
  s2 = block_reduce(s2, AddOp(), sh);
  if (threadIdx.x == 0) part[(int64_t)e * chunks + c] = IwPartial{m, s1, s2};
}

__global__ void __launch_bounds__(IW_THREADS) k_iw_finish(const double* __restrict__ lnl,
                                                          const double* __restrict__ ratio,
                                                          const int64_t* __restrict__ off, int64_t S, int chunks,
                                                          const IwPartial* __restrict__ part,
                                                          double* __restrict__ weights, double* __restrict__ ess,
                                                          double* __restrict__ eff, double* __restrict__ lnz) {
  __shared__ double sh[IW_THREADS / 32];
  const int e = blockIdx.x, c = blockIdx.y;
  int64_t a, b, n;
  iw_chunk(off, S, e, c, chunks, a, b, n);
  const IwPartial* pe = part + (int64_t)e * chunks;
  // merge the chunk partials (chunks <= blockDim.x): rescale each to the event maximum
  double m = threadIdx.x < chunks ? pe[threadIdx.x].m : -INFINITY;
  const double M = block_reduce(m, MaxOp(), sh);
  double s1 = 0.0, s2 = 0.0;
  if (threadIdx.x < chunks && M > -INFINITY && m > -INFINITY) {
    const double r = exp(m - M);
    s1 = pe[threadIdx.x].s1 * r;
    s2 = pe[threadIdx.x].s2 * r * r;
  }
  const double S1 = block_reduce(s1, AddOp(), sh);
  const double S2 = block_reduce(s2, AddOp(), sh);
  const bool any = M > -INFINITY && S1 > 0.0;
  if (c == 0 && threadIdx.x == 0) {
    const double q = any ? S1 * S1 / S2 : 0.0;
    if (ess) ess[e] = q;
    if (eff) eff[e] = n > 0 ? q / (double)n : 0.0;
    if (lnz) lnz[e] = any ? M + log(S1) - log((double)n) : -INFINITY;
  }
  if (!weights) return;
  const double inv = any ? 1.0 / S1 : 0.0;
  for (int64_t s = a + threadIdx.x; s < b; s += blockDim.x)
    weights[s] = any ? (double)iw_exp(iw_lnw(lnl, ratio, s) - M) * inv : 0.0;
}

int iw_chunks(int64_t E) {
  if (E <= 0) return 1;
  const int64_t c = 1024 / E;
  return (int)(c < 1 ? 1 : (c > 64 ? 64 : c));
}

size_t iw_workspace_bytes(int64_t E) { return (size_t)(E > 0 ? E : 0) * iw_chunks(E) * sizeof(IwPartial); }

cudaError_t launch_importance_weights(const double* lnl, const double* ratio, const int64_t* off, int64_t E,
                                      int64_t S, double* weights, double* ess, double* eff, double* lnz, void* ws,
                                      cudaStream_t s) {
  if (E <= 0) return cudaSuccess;
  const int C = iw_chunks(E);
  IwPartial* part = reinterpret_cast<IwPartial*>(ws);
  const dim3 grid((unsigned)E, (unsigned)C);
  k_iw_partial<<<grid, IW_THREADS, 0, s>>>(lnl, ratio, off, S, C, part);
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  k_iw_finish<<<grid, IW_THREADS, 0, s>>>(lnl, ratio, off, S, C, part, weights, ess, eff, lnz);
  return cudaGetLastError();
}

}  // namespace gwx
