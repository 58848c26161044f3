// k_flow_fused.cu -- the coupling flow's sampling pass as one persistent tensor-core
// kernel (the draw step of Sec. 5's posterior estimator).  Each CTA takes 128 draws at a
// time through all K coupling layers without leaving the SM:
//   - warp 0 streams each layer's conditioner weights from L2 with 3-D TMA boxes into a
//     two-slot ring (part 0: V1; parts 1..H/128: pairs of V2's 64-column K-blocks; last
//     part: V3 padded to 16 rows by the box's zero fill);
//   - warp 1 issues tcgen05.mma: acc1 = X V1^T, acc2 = g1 V2^T, acc3 = g2 V3^T (FP32 in
//     tensor memory, columns 0 and 256; acc3 reuses acc1's columns).  The products are cut
//     into 128-column parts (N) and 128-column rounds of their input (K) so that the
//     row warps and the tensor core overlap: the rows drain acc1's first part while the
//     second is computed, acc2's first K round runs while the rows write the second
//     quarter-pair of g1, and so on;
//   - warps 2-9 own one draw (row) per thread, two warps per tensor-memory lane quarter:
//     the first keeps the draw's eight coordinates and its log-scale sum in registers,
//     writes the conditioning half of the conditioner input X once per layer and applies
//     the coupling step from acc3; both write the context into X once per tile and half
//     of the hidden activations g1, g2 (bias, ReLU, bfloat16) each, into shared memory in
//     the 128-byte-swizzle layout the MMA reads.
// The activations never go to global memory: per draw and layer only the weights (shared
// by all draws, L2-resident) move.  Every mbarrier wait is bounded; on expiry the CTA
// records a status, stops and frees its tensor memory.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include "gwx_internal.h"
#include "tc05.cuh"

namespace gwx {

namespace {

using namespace tc;

constexpr int FM = 128;                                  // draws per tile
constexpr int F_THREADS = 320;                           // warp 0 TMA, warp 1 MMA, warps 2-9 rows
constexpr uint32_t KB_BYTES = FM * 128;                  // one 128-row x 64-column bfloat16 K-block: 16 KiB
constexpr uint32_t X_BYTES = 2 * KB_BYTES;               // conditioner input, 8 + C <= 128 columns
constexpr uint32_t G_BYTES = 4 * KB_BYTES;               // hidden activations, H <= 256 columns
constexpr uint32_t SLOT_BYTES = 2 * 256 * 128;           // two K-blocks of a 256-row weight tile
constexpr uint32_t F_WAIT = 1u << 22;
constexpr size_t FUSED_SMEM = (size_t)X_BYTES + G_BYTES + 2 * SLOT_BYTES + 1024;
constexpr float S_MAX = 3.f;

// Split p of the eight coordinates: conditioning half a_j = A(p, j), transformed half
// b_j = Bc(p, j) (the flow's four fixed splits; compile-time so v[] stays in registers).
__host__ __device__ constexpr int A(int p, int j) {
  return p == 0 ? j : p == 1 ? 4 + j : p == 2 ? 2 * j : 2 * j + 1;
}
__host__ __device__ constexpr int Bc(int p, int j) {
  return p == 0 ? 4 + j : p == 1 ? j : p == 2 ? 2 * j + 1 : 2 * j;
}

template <int P>
__device__ __forceinline__ void pack_half(const float* v, uint32_t& w0, uint32_t& w1);
template <int P>
__device__ __forceinline__ void couple(float* v, const float* o, const float* b3, float& ss);

__device__ int g_flow_status;

struct FusedArgs {
  const float* z;                 // [n][8] base draws of this chunk
  const __nv_bfloat16* ctx;       // [E][C] per-event context
  const int64_t* off;             // [E + 1] event offsets (global rows)
  int64_t E, row0, n;
  int C, H, K;
  const float* e1;                // layer-0 biases; layer l at + l * lstride
  const float* e2;
  const float* e3;
  int64_t lstride;                // elements between consecutive layers' tensors
  float* x_out;                   // [n][8]
  float* ss_out;                  // [n]
};

// Byte offset of 16-byte chunk j of row r inside a 128-row K-block (128-byte swizzle).
__device__ __forceinline__ uint32_t swz(int r, int j) {
  return (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((j ^ (r & 7)) << 4));
}

__device__ __forceinline__ uint32_t pack2(float a, float b) {
  __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&h);
}

__device__ __forceinline__ void sts128(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d) : "memory");
}

__device__ __forceinline__ void proxy_fence() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

template <int P>
__device__ __forceinline__ void pack_half(const float* v, uint32_t& w0, uint32_t& w1) {
  w0 = pack2(v[A(P, 0)], v[A(P, 1)]);
  w1 = pack2(v[A(P, 2)], v[A(P, 3)]);
}

// v_b <- v_b e^s + mu with mu_j = o_j + b3_j, s_j = 3 tanh((o_{4+j} + b3_{4+j}) / 3);
// b3: the layer's eight output biases, in registers
template <int P>
__device__ __forceinline__ void couple(float* v, const float* o, const float* b3, float& ss) {
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const float s = S_MAX * tanhf((o[4 + j] + b3[4 + j]) / S_MAX);
    v[Bc(P, j)] = fmaf(v[Bc(P, j)], expf(s), o[j] + b3[j]);
    ss += s;
  }
}

__global__ void __launch_bounds__(F_THREADS, 1)
    k_flow_sample_fused(const __grid_constant__ CUtensorMap mv1, const __grid_constant__ CUtensorMap mv2,
                        const __grid_constant__ CUtensorMap mv3, FusedArgs a) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full[2], empty[2], xready, gready[2], acc1f[2], acc2f[2], acc3f;
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t base = (su32(smem_raw) + 1023u) & ~1023u;
  const uint32_t sx = base, sg = base + X_BYTES, sw = base + X_BYTES + G_BYTES;
  const int H = a.H, K = a.K, C = a.C;
  const int NP = 2 + H / 128;                              // weight parts per layer
  const int NR = H / 128;                                  // 128-column parts and rounds
  const int tiles = (int)((a.n + FM - 1) / FM);
  const uint32_t id_128 = idesc_bf16(FM, 128), id_16 = idesc_bf16(FM, 16);

  if (threadIdx.x == 0) {
    for (int s = 0; s < 2; ++s) {
      mbar_init(su32(&full[s]), 1);
      mbar_init(su32(&empty[s]), 1);
    }
    mbar_init(su32(&xready), 8);
    for (int r = 0; r < 2; ++r) {
      mbar_init(su32(&gready[r]), 8);
      mbar_init(su32(&acc1f[r]), 1);
      mbar_init(su32(&acc2f[r]), 1);
    }
    mbar_init(su32(&acc3f), 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_slot)),
                 "r"(512)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      uint32_t it = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < tiles && ok; t += gridDim.x)
        for (int l = 0; l < K && ok; ++l)
          for (int p = 0; p < NP; ++p, ++it) {
            const uint32_t s = it & 1u;
            if (it >= 2 && !mbar_wait(su32(&empty[s]), ((it >> 1) - 1) & 1u, F_WAIT)) {
              ok = false;
              break;
            }
            if (*(volatile int*)&abort_flag) {
              ok = false;
              break;
            }
            const uint32_t dst = sw + s * SLOT_BYTES, bar = su32(&full[s]);
            if (p == 0) {
              mbar_expect_tx(bar, (uint32_t)H * 256u);
              tma_load_3d(dst, &mv1, 0, 0, l, bar);
              tma_load_3d(dst + (uint32_t)H * 128u, &mv1, 64, 0, l, bar);
            } else if (p < NP - 1) {
              const int kb0 = 2 * (p - 1);
              mbar_expect_tx(bar, (uint32_t)H * 256u);
              tma_load_3d(dst, &mv2, 64 * kb0, 0, l, bar);
              tma_load_3d(dst + (uint32_t)H * 128u, &mv2, 64 * (kb0 + 1), 0, l, bar);
            } else {
              mbar_expect_tx(bar, (uint32_t)H * 32u);
              for (int kb = 0; kb < H / 64; ++kb) tma_load_3d(dst + 2048u * kb, &mv3, 64 * kb, 0, l, bar);
            }
          }
      if (!ok) atomicExch(&abort_flag, 1);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      uint32_t it = 0, li = 0;
      bool ok = true;
      auto take = [&](uint32_t& slot) -> bool {
        slot = it & 1u;
        if (!mbar_wait(su32(&full[slot]), (it >> 1) & 1u, F_WAIT)) return false;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        return true;
      };
      auto wait_on = [&](uint64_t* bar, uint32_t parity) -> bool {
        if (!mbar_wait(su32(bar), parity, F_WAIT)) return false;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        return true;
      };
      for (int t = blockIdx.x; t < tiles && ok; t += gridDim.x)
        for (int l = 0; l < K && ok; ++l, ++li) {
          uint32_t slot;
          // acc1 = X V1^T (two K-blocks of the input row), one 128-column part at a time
          if (!(ok = wait_on(&xready, li & 1u)) || !(ok = take(slot))) break;
          {
            const uint32_t wb = sw + slot * SLOT_BYTES;
            for (int np = 0; np < NR; ++np) {
              for (int kb = 0; kb < 2; ++kb)
#pragma unroll
                for (int kk = 0; kk < 4; ++kk)
                  mma_bf16(tmem + 128u * np, sw128_desc(sx + KB_BYTES * kb + 32u * kk),
                           sw128_desc(wb + (uint32_t)H * 128u * kb + 16384u * np + 32u * kk), id_128,
                           (kb | kk) != 0);
              mma_commit(su32(&acc1f[np]));
            }
            mma_commit(su32(&empty[slot]));
            ++it;
          }
          // acc2 = g1 V2^T: K round pr (g1 columns 128 pr .. + 127, weight part pr) once the
          // rows have written it, both 128-column output parts per round
          for (int pr = 0; pr < NR && ok; ++pr) {
            if (!(ok = wait_on(&gready[pr], 0u)) || !(ok = take(slot))) break;
            const uint32_t wb = sw + slot * SLOT_BYTES;
            for (int np = 0; np < NR; ++np) {
              for (int kb = 0; kb < 2; ++kb) {
                const int kg = 2 * pr + kb;
#pragma unroll
                for (int kk = 0; kk < 4; ++kk)
                  mma_bf16(tmem + 256u + 128u * np, sw128_desc(sg + KB_BYTES * kg + 32u * kk),
                           sw128_desc(wb + (uint32_t)H * 128u * kb + 16384u * np + 32u * kk), id_128,
                           (kg | kk) != 0);
              }
              if (pr == NR - 1) mma_commit(su32(&acc2f[np]));
            }
            mma_commit(su32(&empty[slot]));
            ++it;
          }
          if (!ok) break;
          // acc3 = g2 V3^T (16 rows, 8 of them the conditioner's outputs), K round by round
          if (!(ok = take(slot))) break;
          {
            const uint32_t wb = sw + slot * SLOT_BYTES;
            for (int r = 0; r < NR && ok; ++r) {
              if (!(ok = wait_on(&gready[r], 1u))) break;
              for (int kb = 2 * r; kb < 2 * r + 2; ++kb)
#pragma unroll
                for (int kk = 0; kk < 4; ++kk)
                  mma_bf16(tmem, sw128_desc(sg + KB_BYTES * kb + 32u * kk), sw128_desc(wb + 2048u * kb + 32u * kk),
                           id_16, (kb | kk) != 0);
            }
            if (!ok) break;
            mma_commit(su32(&empty[slot]));
            ++it;
            mma_commit(su32(&acc3f));
          }
        }
      if (!ok) atomicExch(&abort_flag, 1);
    }
  } else {
    const int q = warp & 3;
    const int h = (warp - 2) >> 2;                             // which half of the columns
    const int r = 32 * q + lane;                               // row of the tile = tensor-memory lane
    const uint32_t lane_addr = tmem + ((uint32_t)(32 * q) << 16);
    uint32_t li = 0;
    bool ok = true;
    auto arrive = [&](uint64_t* bar) {
      proxy_fence();
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(su32(bar));
    };
    auto wait_on = [&](uint64_t* bar, uint32_t parity) -> bool {
      const bool got = mbar_wait(su32(bar), parity, F_WAIT);
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      return __all_sync(0xffffffffu, got) && !*(volatile int*)&abort_flag;
    };
    // bias + ReLU of 64 accumulator columns (chunk c: two loads, one wait) into K-block c
    // of the activation tile g; round rd of a hidden layer is chunk 2 rd + h.  The chunk's
    // biases bb (loaded by load_bias before the wait for its accumulator, so that their
    // latency overlaps the products) are read from registers.
    auto load_bias = [&](const float* bias, int c, float4* bb) {
      const float4* b4 = reinterpret_cast<const float4*>(bias + 64 * c);
#pragma unroll
      for (int i = 0; i < 16; ++i) bb[i] = __ldg(b4 + i);
    };
    auto hidden = [&](uint32_t col0, const float4* bb, int c) {
      uint32_t raw[2][32];
      tmem_ld32_async(lane_addr + col0 + 64u * c, raw[0]);
      tmem_ld32_async(lane_addr + col0 + 64u * c + 32u, raw[1]);
      tmem_wait_ld();
#pragma unroll
      for (int hh = 0; hh < 2; ++hh) {
        uint32_t w[16];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const float4 b = bb[8 * hh + i];
          w[2 * i] = pack2(fmaxf(__uint_as_float(raw[hh][4 * i]) + b.x, 0.f),
                           fmaxf(__uint_as_float(raw[hh][4 * i + 1]) + b.y, 0.f));
          w[2 * i + 1] = pack2(fmaxf(__uint_as_float(raw[hh][4 * i + 2]) + b.z, 0.f),
                               fmaxf(__uint_as_float(raw[hh][4 * i + 3]) + b.w, 0.f));
        }
#pragma unroll
        for (int t4 = 0; t4 < 4; ++t4) {
          const int col = 64 * c + 32 * hh + 8 * t4;
          sts128(sg + KB_BYTES * (col >> 6) + swz(r, (col & 63) >> 3), w[4 * t4], w[4 * t4 + 1], w[4 * t4 + 2],
                 w[4 * t4 + 3]);
        }
      }
    };
    for (int t = blockIdx.x; t < tiles && ok; t += gridDim.x) {
      const int64_t row = (int64_t)t * FM + r;
      const bool valid = row < a.n;
      float v[8], ss = 0.f;
      if (valid && h == 0) {
        const float4 z0 = reinterpret_cast<const float4*>(a.z + row * 8)[0];
        const float4 z1 = reinterpret_cast<const float4*>(a.z + row * 8)[1];
        v[0] = z0.x; v[1] = z0.y; v[2] = z0.z; v[3] = z0.w; v[4] = z1.x; v[5] = z1.y; v[6] = z1.z; v[7] = z1.w;
      } else {
#pragma unroll
        for (int i = 0; i < 8; ++i) v[i] = 0.f;
      }
      // context: columns 8 .. 8 + C - 1 of the input row, zeros up to 128
      int64_t e = 0;
      if (valid) {
        int64_t lo = 0, hi = a.E, s = a.row0 + row;
        while (hi - lo > 1) {
          const int64_t mid = (lo + hi) >> 1;
          if (__ldg(&a.off[mid]) <= s) lo = mid; else hi = mid;
        }
        e = lo;
      }
      const uint4* crow = reinterpret_cast<const uint4*>(a.ctx + e * C);
      for (int g = h == 0 ? 1 : 8; g < (h == 0 ? 8 : 16); ++g) {
        uint4 d = make_uint4(0u, 0u, 0u, 0u);
        if (valid && g <= C / 8) d = __ldg(crow + (g - 1));
        sts128(sx + KB_BYTES * (g >> 3) + swz(r, g & 7), d.x, d.y, d.z, d.w);
      }
      for (int l = 0; l < K; ++l, ++li) {
        const int p = l & 3;
        if (h == 0) {
          uint32_t w0, w1;
          switch (p) {
            case 0: pack_half<0>(v, w0, w1); break;
            case 1: pack_half<1>(v, w0, w1); break;
            case 2: pack_half<2>(v, w0, w1); break;
            default: pack_half<3>(v, w0, w1); break;
          }
          sts128(sx + swz(r, 0), w0, w1, 0u, 0u);
        }
        arrive(&xready);
        for (int rd = 0; rd < NR && ok; ++rd) {
          float4 bb[16];
          load_bias(a.e1 + l * a.lstride, 2 * rd + h, bb);
          if (!(ok = wait_on(&acc1f[rd], li & 1u))) break;
          hidden(0u, bb, 2 * rd + h);
          arrive(&gready[rd]);
        }
        for (int rd = 0; rd < NR && ok; ++rd) {
          float4 bb[16];
          load_bias(a.e2 + l * a.lstride, 2 * rd + h, bb);
          if (!(ok = wait_on(&acc2f[rd], li & 1u))) break;
          hidden(256u, bb, 2 * rd + h);
          arrive(&gready[rd]);
        }
        if (!ok) break;
        if (h != 0) continue;                                  // the coupling step is the first warp's
        float b3[8];
        {
          const float4* b4 = reinterpret_cast<const float4*>(a.e3 + l * a.lstride);
          const float4 lo4 = __ldg(b4), hi4 = __ldg(b4 + 1);
          b3[0] = lo4.x; b3[1] = lo4.y; b3[2] = lo4.z; b3[3] = lo4.w;
          b3[4] = hi4.x; b3[5] = hi4.y; b3[6] = hi4.z; b3[7] = hi4.w;
        }
        if (!(ok = wait_on(&acc3f, li & 1u))) break;
        float o[16];
        tmem_ld16(lane_addr, o);
        switch (p) {
          case 0: couple<0>(v, o, b3, ss); break;
          case 1: couple<1>(v, o, b3, ss); break;
          case 2: couple<2>(v, o, b3, ss); break;
          default: couple<3>(v, o, b3, ss); break;
        }
      }
      if (!ok) break;
      if (valid && h == 0) {
        reinterpret_cast<float4*>(a.x_out + row * 8)[0] = make_float4(v[0], v[1], v[2], v[3]);
        reinterpret_cast<float4*>(a.x_out + row * 8)[1] = make_float4(v[4], v[5], v[6], v[7]);
        a.ss_out[row] = ss;
      }
    }
    if (!ok && lane == 0) atomicExch(&abort_flag, 1);
  }
  __syncwarp();
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (threadIdx.x == 0 && *(volatile int*)&abort_flag) atomicExch(&g_flow_status, 1);
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
}

PFN_cuTensorMapEncodeTiled_v12000 encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// bfloat16 weights of every layer as a 3-D tensor [layers][rows][cols] with the layers
// lstride elements apart; boxes of 64 columns x box_rows rows x one layer.
bool layer_map(CUtensorMap* map, const void* base, int64_t cols, int64_t rows, int64_t layers, int64_t lstride,
               uint32_t box_rows) {
  auto enc = encoder();
  if (!enc) return false;
  cuuint64_t dims[3] = {(cuuint64_t)cols, (cuuint64_t)rows, (cuuint64_t)layers};
  cuuint64_t strides[2] = {(cuuint64_t)cols * 2, (cuuint64_t)lstride * 2};
  cuuint32_t box[3] = {64, box_rows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

bool flow_fused_supported(int C, int H, int K) {
  return (H == 128 || H == 256) && C >= 8 && C % 8 == 0 && 8 + C <= 128 && K >= 1;
}

cudaError_t launch_flow_sample_fused(const void* params_bf16, const float* params, const int64_t* off_t, int C, int H,
                                     int K, const float* z, const void* ctx, const int64_t* ev_off, int64_t E,
                                     int64_t row0, int64_t n, float* x_out, float* ss_out, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const __nv_bfloat16* p16 = reinterpret_cast<const __nv_bfloat16*>(params_bf16);
  // one layer's tensors repeat every lstride elements (a multiple of 64, so 128 bytes)
  const int64_t lstride = K > 1 ? off_t[12] - off_t[6] : 64;
  CUtensorMap m1, m2, m3;
  if (!layer_map(&m1, p16 + off_t[6], 8 + C, H, K, lstride, (uint32_t)H) ||
      !layer_map(&m2, p16 + off_t[8], H, H, K, lstride, (uint32_t)H) ||
      !layer_map(&m3, p16 + off_t[10], H, 8, K, lstride, 16u))
    return cudaErrorInvalidValue;
  FusedArgs a;
  a.z = z;
  a.ctx = reinterpret_cast<const __nv_bfloat16*>(ctx);
  a.off = ev_off;
  a.E = E;
  a.row0 = row0;
  a.n = n;
  a.C = C;
  a.H = H;
  a.K = K;
  a.e1 = params + off_t[7];
  a.e2 = params + off_t[9];
  a.e3 = params + off_t[11];
  a.lstride = lstride;
  a.x_out = x_out;
  a.ss_out = ss_out;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int64_t tiles = (n + FM - 1) / FM;
  const unsigned grid = (unsigned)(tiles < sms ? tiles : sms);
  e = cudaFuncSetAttribute(k_flow_sample_fused, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FUSED_SMEM);
  if (e != cudaSuccess) return e;
  k_flow_sample_fused<<<grid, F_THREADS, FUSED_SMEM, s>>>(m1, m2, m3, a);
  return cudaGetLastError();
}

cudaError_t flow_fused_status(int* status) {
  int zero = 0;
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpyFromSymbol(status, g_flow_status, sizeof(int));
  if (e == cudaSuccess && *status != 0) e = cudaMemcpyToSymbol(g_flow_status, &zero, sizeof(int));
  return e;
}

}  // namespace gwx
