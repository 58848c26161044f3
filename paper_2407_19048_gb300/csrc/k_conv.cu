// k_conv.cu -- the stride-1 convolutions of the ResNet-1D data summary (Sec. 4) as
// implicit GEMMs on the tensor cores: no im2col matrix is materialised for the product
// or for the input gradient.
//   forward:        z[b][t][o]  = sum_{j,c} x[b][t + j - p][c] W[o][j C + c]
//   input gradient: dx[b][t][c] = sum_{j,o} dz[b][t - (j - p)][o] Wt[c][j O + o],
//                   Wt[c][j O + o] = W[o][j C + c]   (the same implicit form, taps mirrored)
//   weight gradient: dW[o][j C + c] = sum_{b,t} dz[b][t][o] x[b][t + j - p][c]
//                   = dZ^T [O][B T] . (colsT [k C][B T])^T, colsT written straight from x
// (p = (k - 1)/2, zero outside [0, T)); the products run in k_gemm.cu's kernel, whose A
// tiles come from a 3-D tensor map of the channels-last activations.
#include <cuda_bf16.h>

#include "gwx_internal.h"

namespace gwx {

namespace {

constexpr int CT = 32;   // transpose tile edge

// dZ [M][O] bfloat16 and its transpose dZt [O][M] from dz FP32 [M][O].
__global__ void k_conv_dz(const float* __restrict__ dz, int64_t M, int O, __nv_bfloat16* __restrict__ dZ,
                          __nv_bfloat16* __restrict__ dZt) {
  __shared__ __nv_bfloat16 tile[CT][CT + 2];
  const int64_t m0 = (int64_t)blockIdx.y * CT;
  const int o0 = blockIdx.x * CT;
  for (int i = threadIdx.y; i < CT; i += blockDim.y) {
    const int64_t m = m0 + i;
    const int o = o0 + threadIdx.x;
    if (m < M && o < O) {
      const __nv_bfloat16 v = __float2bfloat16_rn(dz[m * O + o]);
      dZ[m * O + o] = v;
      tile[i][threadIdx.x] = v;
    }
  }
  __syncthreads();
  for (int i = threadIdx.y; i < CT; i += blockDim.y) {
    const int o = o0 + i;
    const int64_t m = m0 + threadIdx.x;
    if (o < O && m < M) dZt[(int64_t)o * M + m] = tile[threadIdx.x][i];
  }
}

// Wt[c][j O + o] = W[o][j C + c]
__global__ void k_conv_wt(const __nv_bfloat16* __restrict__ W, int O, int C, int k, __nv_bfloat16* __restrict__ Wt) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t n = (int64_t)O * k * C;
  if (i >= n) return;
  const int c = (int)(i / ((int64_t)k * O));
  const int r = (int)(i - (int64_t)c * k * O);
  const int j = r / O, o = r - j * O;
  Wt[i] = W[(int64_t)o * k * C + (int64_t)j * C + c];
}

// colsT[j C + c][b T + t] = x[b][t + j - p][c] (zero outside [0, T)).  One block per
// 64-time x 64-channel tile, all k taps: the 63 + k input rows it needs are loaded once as
// 16-byte vectors into a shared tile of 33-word rows (conflict-free both ways), then every
// tap's 64 output rows are written as 16-byte vectors of 8 consecutive times.
constexpr int IT = 64;   // tile edge (times and channels)
constexpr int IW = 33;   // shared row stride in 32-bit words (32 data + 1 pad)

__global__ void __launch_bounds__(256) k_im2col_t(const __nv_bfloat16* __restrict__ x, int64_t Bn, int T, int C, int k,
                                                  __nv_bfloat16* __restrict__ colsT) {
  __shared__ uint32_t tile[(IT + 14) * IW];
  const int64_t M = Bn * T;
  const int64_t q0 = (int64_t)blockIdx.x * IT;   // first (b, t) row (T % 64 == 0)
  const int c0 = blockIdx.y * IT;
  const int p = (k - 1) / 2;
  const int64_t b = q0 / T;
  const int t0 = (int)(q0 - b * T);
  const int rows = IT + k - 1;
  const int tid = threadIdx.x;
  // load: row r = source time t0 - p + r, 8 vectors of 8 channels
  for (int e = tid; e < rows * 8; e += 256) {
    const int r = e >> 3, v = e & 7;
    const int ts = t0 - p + r;
    uint4 val = make_uint4(0u, 0u, 0u, 0u);
    if (ts >= 0 && ts < T) val = __ldg(reinterpret_cast<const uint4*>(x + (b * T + ts) * C + c0) + v);
    uint32_t* d = tile + r * IW + 4 * v;
    d[0] = val.x;
    d[1] = val.y;
    d[2] = val.z;
    d[3] = val.w;
  }
  __syncthreads();
  const unsigned short* ts16 = reinterpret_cast<const unsigned short*>(tile);
  for (int j = 0; j < k; ++j) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      // output row c, times 8 u .. 8 u + 7; a warp covers 8 channels x 4 vectors, whose
      // shared rows 8 u + const land in distinct banks
      const int c = tid >> 2, u = (tid & 3) + 4 * h;
      uint32_t w[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int r0 = 8 * u + 2 * i + j;
        const uint32_t lo = ts16[2 * (r0 * IW) + c], hi = ts16[2 * ((r0 + 1) * IW) + c];
        w[i] = lo | (hi << 16);
      }
      *reinterpret_cast<uint4*>(colsT + ((int64_t)j * C + c0 + c) * M + q0 + 8 * u) = make_uint4(w[0], w[1], w[2], w[3]);
    }
  }
}

size_t al256(size_t v) { return (v + 255) / 256 * 256; }

}  // namespace

// Workspace of conv_backward: dZ, dZt (bfloat16 [B T][O] and [O][B T]), Wt (bfloat16
// [C][k O]), colsT (bfloat16 [k C][B T]) and the split-K partial products of dW.
size_t conv_backward_ws(int64_t Bn, int64_t T, int C, int O, int k) {
  const int64_t M = Bn * T;
  return 2 * al256((size_t)M * O * 2) + al256((size_t)C * k * O * 2) + al256((size_t)k * C * M * 2) +
         al256(gemm_splitk_ws(O, (int64_t)k * C, M));
}

cudaError_t launch_conv_forward(const void* x, int64_t Bn, int64_t T, int C, int k, const void* W, int O,
                                const float* addend, float* z, cudaStream_t s) {
  return launch_conv_gemm(x, Bn, T, C, k, +1, W, O, z, addend, s);
}

// dx [B][T][C] (+ addend) and dW [O][k C] of the stride-1 convolution z = conv(x, W) given
// dz [B][T][O] (FP32).
cudaError_t launch_conv_backward(const float* dz, const void* x, const void* W, int64_t Bn, int64_t T, int C, int O,
                                 int k, const float* addend, float* dx, float* dW, void* ws, cudaStream_t s) {
  const int64_t M = Bn * T;
  char* w = reinterpret_cast<char*>(ws);
  auto* dZ = reinterpret_cast<__nv_bfloat16*>(w);
  w += al256((size_t)M * O * 2);
  auto* dZt = reinterpret_cast<__nv_bfloat16*>(w);
  w += al256((size_t)M * O * 2);
  auto* Wt = reinterpret_cast<__nv_bfloat16*>(w);
  w += al256((size_t)C * k * O * 2);
  auto* colsT = reinterpret_cast<__nv_bfloat16*>(w);
  w += al256((size_t)k * C * M * 2);
  float* part = reinterpret_cast<float*>(w);
  const dim3 tb(CT, 8);
  k_conv_dz<<<dim3((unsigned)((O + CT - 1) / CT), (unsigned)((M + CT - 1) / CT)), tb, 0, s>>>(dz, M, O, dZ, dZt);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (dx) {
    const int64_t nw = (int64_t)O * k * C;
    k_conv_wt<<<(unsigned)((nw + 255) / 256), 256, 0, s>>>(reinterpret_cast<const __nv_bfloat16*>(W), O, C, k, Wt);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // the input gradient: dz as the implicit A (channels O), taps mirrored
    if ((e = launch_conv_gemm(dZ, Bn, T, O, k, -1, Wt, C, dx, addend, s)) != cudaSuccess) return e;
  }
  if (dW) {
    k_im2col_t<<<dim3((unsigned)(M / IT), (unsigned)(C / IT)), 256, 0, s>>>(
        reinterpret_cast<const __nv_bfloat16*>(x), Bn, (int)T, C, k, colsT);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = launch_gemm_splitk(dZt, colsT, dW, O, (int64_t)k * C, M, part, s)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace gwx
