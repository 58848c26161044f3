// k_vicreg.cu -- self-supervised pre-training of the data summary (Sec. 4.1): the VICReg
// loss of two views' expanded representations and its gradient, and the second view's
// parameters (the same source with a new merger time).
//
// k_vicreg runs in one block: per view the column means and the d x d sample covariance
// (FP64 sums over the batch staged through shared memory), then the three terms
//   inv = sum (x - x')^2 / (B d),  v = sum_j max(0, gamma - sqrt(Var_j + eps)) / d,
//   c = sum_{i != j} C_ij^2 / d,
// the weighted loss, and dL/dx, dL/dx' element by element.
#include "common.cuh"

namespace gwx {

namespace {

constexpr int VT = 1024;          // threads of the single block
constexpr int VD = 32;            // largest representation width
constexpr int VROWS = 64;         // rows staged per chunk
constexpr double V_GAMMA = 1.0, V_EPS = 1e-4;
constexpr uint32_t TAG_RETIME = 5u;

__global__ void __launch_bounds__(VT) k_vicreg(const float* __restrict__ x, const float* __restrict__ xp, int B, int d,
                                               double l1, double l2, double l3, double* __restrict__ loss,
                                               double* __restrict__ terms, float* __restrict__ gx,
                                               float* __restrict__ gxp) {
  __shared__ float tile[2][VROWS][VD];
  __shared__ double mean[2][VD], cov[2][VD][VD + 1];
  __shared__ double red[VT / 32];
  const int tid = threadIdx.x;
  const float* src[2] = {x, xp};
  // column means
  double acc = 0.0;
  const int mv = tid / VD, mj = tid % VD;           // threads 0 .. 2 VD - 1
  for (int r0 = 0; r0 < B; r0 += VROWS) {
    const int rows = min(VROWS, B - r0);
    for (int e = tid; e < 2 * rows * d; e += VT) {
      const int v = e / (rows * d), rem = e % (rows * d);
      tile[v][rem / d][rem % d] = src[v][(int64_t)(r0 + rem / d) * d + rem % d];
    }
    __syncthreads();
    if (tid < 2 * VD && mj < d)
      for (int r = 0; r < rows; ++r) acc += (double)tile[mv][r][mj];
    __syncthreads();
  }
  if (tid < 2 * VD && mj < d) mean[mv][mj] = acc / B;
  __syncthreads();
  // covariance C[v][i][j], one entry per thread and view
  const int ci = tid / VD, cj = tid % VD;
  double c0 = 0.0, c1 = 0.0;
  for (int r0 = 0; r0 < B; r0 += VROWS) {
    const int rows = min(VROWS, B - r0);
    for (int e = tid; e < 2 * rows * d; e += VT) {
      const int v = e / (rows * d), rem = e % (rows * d);
      tile[v][rem / d][rem % d] = src[v][(int64_t)(r0 + rem / d) * d + rem % d];
    }
    __syncthreads();
    if (ci < d && cj < d)
      for (int r = 0; r < rows; ++r) {
        c0 += ((double)tile[0][r][ci] - mean[0][ci]) * ((double)tile[0][r][cj] - mean[0][cj]);
        c1 += ((double)tile[1][r][ci] - mean[1][ci]) * ((double)tile[1][r][cj] - mean[1][cj]);
      }
    __syncthreads();
  }
  if (ci < d && cj < d) {
    cov[0][ci][cj] = c0 / (B - 1);
    cov[1][ci][cj] = c1 / (B - 1);
  }
  __syncthreads();
  // terms: invariance over all elements, variance hinge and off-diagonal covariance
  double inv = 0.0;
  for (int64_t e = tid; e < (int64_t)B * d; e += VT) {
    const double df = (double)x[e] - (double)xp[e];
    inv += df * df;
  }
  for (int o = 16; o > 0; o >>= 1) inv += __shfl_down_sync(0xffffffffu, inv, o);
  if ((tid & 31) == 0) red[tid >> 5] = inv;
  __syncthreads();
  if (tid == 0) {
    double t[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int w = 0; w < VT / 32; ++w) t[0] += red[w];
    t[0] /= (double)B * d;
    for (int v = 0; v < 2; ++v)
      for (int i = 0; i < d; ++i) {
        t[1 + v] += fmax(0.0, V_GAMMA - sqrt(cov[v][i][i] + V_EPS)) / d;
        for (int j = 0; j < d; ++j)
          if (j != i) t[3 + v] += cov[v][i][j] * cov[v][i][j] / d;
      }
    *loss = l1 * t[0] + l2 * (t[1] + t[2]) + l3 * (t[3] + t[4]);
    if (terms)
      for (int k = 0; k < 5; ++k) terms[k] = t[k];
  }
  // gradients
  const double ginv = 2.0 * l1 / ((double)B * d), gc = 4.0 * l3 / ((double)d * (B - 1));
  for (int64_t e = tid; e < (int64_t)B * d; e += VT) {
    const int b = (int)(e / d), k = (int)(e % d);
    for (int v = 0; v < 2; ++v) {
      const float* z = src[v];
      const double zc = (double)z[e] - mean[v][k];
      const double S = sqrt(cov[v][k][k] + V_EPS);
      double g = ginv * ((double)z[e] - (double)src[1 - v][e]);
      if (S < V_GAMMA) g -= l2 * zc / ((double)(B - 1) * S * d);
      double dot = 0.0;
      for (int j = 0; j < d; ++j)
        if (j != k) dot += cov[v][k][j] * ((double)z[(int64_t)b * d + j] - mean[v][j]);
      g += gc * dot;
      (v == 0 ? gx : gxp)[e] = (float)g;
    }
  }
}

// theta_out = theta_in with the merger time redrawn uniformly in [tc_lo, tc_hi]:
// u = uniform52 of Philox words 0, 1 with counter (b, 0, TAG_RETIME, counter).
__global__ void k_retime(const double* __restrict__ in, double* __restrict__ out, int64_t B, double tc_lo,
                         double tc_hi, uint32_t k0, uint32_t k1, uint32_t counter) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 11 * B) return;
  const int64_t p = i / B, b = i - p * B;
  if (p == 5) {
    const u32x4 w = philox4x32_10((uint32_t)b, 0u, TAG_RETIME, counter, k0, k1);
    out[i] = tc_lo + (tc_hi - tc_lo) * uniform52(w.x, w.y);
  } else {
    out[i] = in[i];
  }
}

}  // namespace

bool vicreg_supported(int B, int d) { return B >= 2 && d >= 1 && d <= VD; }

cudaError_t launch_vicreg(const float* x, const float* xp, int B, int d, double l1, double l2, double l3,
                          double* loss, double* terms, float* gx, float* gxp, cudaStream_t s) {
  k_vicreg<<<1, VT, 0, s>>>(x, xp, B, d, l1, l2, l3, loss, terms, gx, gxp);
  return cudaGetLastError();
}

cudaError_t launch_retime(const double* in, double* out, int64_t B, double tc_lo, double tc_hi, uint64_t seed,
                          uint32_t counter, cudaStream_t s) {
  if (B == 0) return cudaSuccess;
  k_retime<<<(unsigned)((11 * B + 255) / 256), 256, 0, s>>>(in, out, B, tc_lo, tc_hi, (uint32_t)(seed & 0xffffffffu),
                                                            (uint32_t)(seed >> 32), counter);
  return cudaGetLastError();
}

}  // namespace gwx
