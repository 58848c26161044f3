// k_dense.cu -- backward pass of the dense layer Y = act(X W^T + b) of the learned part
// (the embedding network of Sec. 4 and the flow of Sec. 5), by the chain rule:
//   dZ = dY * act'(Z),  dX = dZ W,  dW = dZ^T X,  db = sum over rows of dZ,
// with both products on the tensor cores (the tcgen05 GEMM, K-major operands): dX takes
// dZ [M][N] and W^T [K][N], dW takes dZ^T [N][M] and X^T [K][M] (split along M when its
// N x K output has few tiles: M is the batch and can be long).  This file holds the
// elementwise and layout kernels around them: the activation derivative with the
// bfloat16 dZ, its transpose and per-tile column sums in one pass, bfloat16 transposes,
// and the final column-sum reduction.
#include <cuda_bf16.h>

#include <algorithm>

#include "gwx_internal.h"

namespace gwx {

namespace {

constexpr int TT = 32;   // transpose tile

__device__ __forceinline__ float act_grad(float z, int act) {
  if (act == GWX_ACT_RELU) return z > 0.f ? 1.f : 0.f;
  if (act == GWX_ACT_GELU)   // Phi(z) + z phi(z)
    return 0.5f * erfcf(-0.70710678118654752f * z) + z * 0.39894228040143268f * expf(-0.5f * z * z);
  return 1.f;
}

// One 32 x 32 tile per block (32 x 8 threads): dz = dY act'(Z) in FP32; dZ and dZ^T in
// bfloat16 (round to nearest even); the tile's column sums of the FP32 dz into
// part[blockIdx.y][n].  With Y (the layer's bfloat16 output, ReLU only) the mask is Y > 0,
// which is Z > 0 (a positive float never rounds to a bfloat16 zero short of 1e-40), and Z
// is not read.
__global__ void __launch_bounds__(256) k_act_backward(const float* __restrict__ Z, const __nv_bfloat16* __restrict__ Y,
                                                      const float* __restrict__ dY, int act, int M, int N,
                                                      __nv_bfloat16* __restrict__ dZ, __nv_bfloat16* __restrict__ dZt,
                                                      float* __restrict__ part) {
  __shared__ float tile[TT][TT + 1];
  const int n0 = blockIdx.x * TT, m0 = blockIdx.y * TT;
  const int tx = threadIdx.x, ty = threadIdx.y;
#pragma unroll
  for (int i = 0; i < TT; i += 8) {
    const int m = m0 + ty + i, n = n0 + tx;
    float v = 0.f;
    if (m < M && n < N) {
      const int64_t at = (int64_t)m * N + n;
      v = __ldg(&dY[at]);
      if (Y != nullptr) v = __bfloat162float(Y[at]) > 0.f ? v : 0.f;
      else if (act != GWX_ACT_NONE) v *= act_grad(__ldg(&Z[at]), act);
      dZ[at] = __float2bfloat16_rn(v);
    }
    tile[ty + i][tx] = v;
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < TT; i += 8) {
    const int n = n0 + ty + i, m = m0 + tx;
    if (n < N && m < M) dZt[(int64_t)n * M + m] = __float2bfloat16_rn(tile[tx][ty + i]);
  }
  if (ty == 0 && n0 + tx < N) {
    float sum = 0.f;
#pragma unroll 8
    for (int r = 0; r < TT; ++r) sum += tile[r][tx];
    part[(int64_t)blockIdx.y * N + n0 + tx] = sum;
  }
}

// out[c][r] = in[r][c] for bfloat16 [R][C] matrices, two in one launch (blockIdx.z picks
// the matrix; a block past its matrix's extent returns at once, before any barrier).
struct Transpose {
  const __nv_bfloat16* in;
  int R, C;
  __nv_bfloat16* out;
};
__global__ void __launch_bounds__(256) k_transpose2_bf16(Transpose a, Transpose b) {
  const Transpose p = blockIdx.z ? b : a;
  const int c0 = blockIdx.x * TT, r0 = blockIdx.y * TT;
  if (c0 >= p.C || r0 >= p.R) return;
  __shared__ __nv_bfloat16 tile[TT][TT + 2];
  const int tx = threadIdx.x, ty = threadIdx.y;
#pragma unroll
  for (int i = 0; i < TT; i += 8) {
    const int r = r0 + ty + i, c = c0 + tx;
    if (r < p.R && c < p.C) tile[ty + i][tx] = p.in[(int64_t)r * p.C + c];
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < TT; i += 8) {
    const int c = c0 + ty + i, r = r0 + tx;
    if (c < p.C && r < p.R) p.out[(int64_t)c * p.R + r] = tile[tx][ty + i];
  }
}

// db[n] = sum_p part[p][n] (FP64 accumulation of the FP32 tile sums), in two
// deterministic passes: block (32 columns, slice y of the partials) has row lane ty sum
// partials ty, ty + 32, ... of its slice, the 32 lanes in order into part2[y][n]; then
// k_colsum_finish adds the slices in order.  With one slice the first pass writes db itself
// (db non-null): the same FP64 sum, rounded once.
constexpr int CS_MAX_SLICES = 64;

int colsum_slices(int64_t P) { return (int)std::min<int64_t>(CS_MAX_SLICES, std::max<int64_t>(1, (P + 255) / 256)); }

__global__ void __launch_bounds__(1024) k_colsum(const float* __restrict__ part, int P, int N,
                                                 double* __restrict__ part2, float* __restrict__ db) {
  __shared__ double red[TT][TT + 1];
  const int n = blockIdx.x * TT + threadIdx.x;
  const int per = (P + gridDim.y - 1) / gridDim.y, p0 = blockIdx.y * per, p1 = min(P, p0 + per);
  double s = 0.0;
  if (n < N)
    for (int p = p0 + threadIdx.y; p < p1; p += TT) s += (double)__ldg(&part[(int64_t)p * N + n]);
  red[threadIdx.y][threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.y == 0 && n < N) {
    double t = 0.0;
    for (int y = 0; y < TT; ++y) t += red[y][threadIdx.x];
    if (db) db[n] = (float)t;
    else part2[(int64_t)blockIdx.y * N + n] = t;
  }
}

__global__ void k_colsum_finish(const double* __restrict__ part2, int slices, int N, float* __restrict__ db) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  double t = 0.0;
  for (int y = 0; y < slices; ++y) t += part2[(int64_t)y * N + n];
  db[n] = (float)t;
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace

size_t dense_backward_ws(int64_t M, int64_t N, int64_t K) {
  const int64_t P = (M + TT - 1) / TT;
  return align256((size_t)M * N * 4)            // Z (FP32)
         + align256((size_t)M * N * 2) * 2      // dZ, dZ^T
         + align256((size_t)K * M * 2)          // X^T
         + align256((size_t)K * N * 2)          // W^T
         + align256((size_t)P * N * 4)          // column-sum partials
         + align256((size_t)CS_MAX_SLICES * N * 8)   // their slice sums
         + align256(gemm_splitk_ws(N, K, M));   // split-K slices of dW
}

cudaError_t launch_dense_backward(const void* X, const void* W, const float* bias, const float* dY, int64_t M,
                                  int64_t N, int64_t K, int act, float* dX, float* dW, float* db, void* ws, int group,
                                  cudaStream_t s, const void* Y) {
  char* w = reinterpret_cast<char*>(ws);
  float* Z = reinterpret_cast<float*>(w);
  w += align256((size_t)M * N * 4);
  __nv_bfloat16* dZ = reinterpret_cast<__nv_bfloat16*>(w);
  w += align256((size_t)M * N * 2);
  __nv_bfloat16* dZt = reinterpret_cast<__nv_bfloat16*>(w);
  w += align256((size_t)M * N * 2);
  __nv_bfloat16* Xt = reinterpret_cast<__nv_bfloat16*>(w);
  w += align256((size_t)K * M * 2);
  __nv_bfloat16* Wt = reinterpret_cast<__nv_bfloat16*>(w);
  w += align256((size_t)K * N * 2);
  float* part = reinterpret_cast<float*>(w);
  const int64_t P = (M + TT - 1) / TT;
  w += align256((size_t)P * N * 4);
  double* part2 = reinterpret_cast<double*>(w);
  w += align256((size_t)CS_MAX_SLICES * N * 8);
  float* kpart = reinterpret_cast<float*>(w);
  cudaError_t e = cudaSuccess;
  // pre-activation Z = X W^T + b (only the activation derivative needs it, and a ReLU
  // layer whose output Y is given takes its mask from Y instead)
  const __nv_bfloat16* Y16 = act == GWX_ACT_RELU ? reinterpret_cast<const __nv_bfloat16*>(Y) : nullptr;
  if (act != GWX_ACT_NONE && Y16 == nullptr) {
    e = launch_gemm_bf16(X, W, Z, M, N, K, false, bias, GWX_ACT_NONE, group, s);
    if (e != cudaSuccess) return e;
  }
  const dim3 tb(TT, 8);
  k_act_backward<<<dim3((unsigned)((N + TT - 1) / TT), (unsigned)P), tb, 0, s>>>(Z, Y16, dY, act, (int)M, (int)N, dZ,
                                                                                 dZt, part);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // X^T (for dW) and W^T (for dX), only those needed, in one launch
  {
    const Transpose tx{reinterpret_cast<const __nv_bfloat16*>(X), (int)M, (int)K, Xt};
    const Transpose tw{reinterpret_cast<const __nv_bfloat16*>(W), (int)N, (int)K, Wt};
    const int nz = (dW ? 1 : 0) + (dX ? 1 : 0);
    if (nz > 0) {
      const Transpose first = dW ? tx : tw;
      const int64_t rows = nz == 2 ? std::max(M, N) : first.R;
      k_transpose2_bf16<<<dim3((unsigned)((K + TT - 1) / TT), (unsigned)((rows + TT - 1) / TT), (unsigned)nz), tb, 0,
                          s>>>(first, tw);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
  }
  // dX [M][K] = dZ [M][N] . (W^T [K][N])^T ;  dW [N][K] = dZ^T [N][M] . (X^T [K][M])^T
  if (dX && (e = launch_gemm_bf16(dZ, Wt, dX, M, K, N, false, nullptr, GWX_ACT_NONE, 0, s)) != cudaSuccess) return e;
  if (dW && (e = launch_gemm_splitk(dZt, Xt, dW, N, K, M, kpart, s)) != cudaSuccess) return e;
  if (db) {
    const int slices = colsum_slices(P);
    k_colsum<<<dim3((unsigned)((N + TT - 1) / TT), (unsigned)slices), dim3(TT, TT), 0, s>>>(
        part, (int)P, (int)N, part2, slices == 1 ? db : nullptr);
    if (slices > 1) k_colsum_finish<<<(unsigned)((N + 127) / 128), 128, 0, s>>>(part2, slices, (int)N, db);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace gwx
