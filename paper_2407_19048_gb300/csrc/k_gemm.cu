// k_gemm.cu -- C = A B^T with bfloat16 operands and FP32 accumulation on the fifth-
// generation tensor cores: the dense layers of the learned part (the embedding network
// of Sec. 4 and the normalizing flow of Sec. 5) are products of this form.
//
// Persistent CTAs (one per SM) walk the 128 x 256 tiles of C; per CTA:
// - warp 0 streams 128 x 64 (A) and 256 x 64 (B) bfloat16 tiles into shared memory with
//   TMA (cp.async.bulk.tensor, 128-byte swizzle), four stages deep, each stage completing
//   on a "full" mbarrier;
// - warp 1 allocates 512 tensor-memory columns and issues tcgen05.mma (M 128, N 256,
//   K 16; four per stage) into one of two 256-column FP32 accumulators, committing each
//   stage to an "empty" mbarrier (the stage goes back to the producer) and each tile to a
//   "tfull" mbarrier;
// - warps 2-9 drain the accumulator of the previous tile with tcgen05.ld (lane quarter
//   warp % 4 = rows 32 q .. 32 q + 31; two warps per quarter, 128 columns each) and
//   store C, while the next tile accumulates.  Eight draining warps keep the fused
//   epilogue (bias, activation, conversion, stores) off the critical path of products
//   with a short K, where it, not the MMA, sets the time per tile.
// Every mbarrier wait is bounded: on expiry the CTA records a status, stops storing,
// frees its tensor memory and returns.
//
// Wide tiles (MW = 2, large products): a CTA computes a 256 x 256 tile of C as two
// M 128 x N 256 products that share each B tile, from three 64 KiB stages (A 256 x 64 in
// one TMA box, B 256 x 64).  Per flop this moves a third less operand data from L2 into
// shared memory than the 128 x 256 tile (the 128 x 256 kernel's operand stream, ~84 B per
// cycle and SM at full tensor rate, is what holds its tensor pipe near 70 %).  The two
// accumulators fill the 512 tensor-memory columns, so a tile's epilogue no longer overlaps
// the next tile's products (~2 % at K = 8192); the eight draining warps take one
// accumulator half each.
//
// Split K: a product with few tiles and a long K (the weight gradients dW = dZ^T X, whose
// K is the batch) would run on a handful of SMs.  There the work list is (tile, K slice)
// pairs: slice s covers K blocks [s kbs, (s + 1) kbs) and stores its FP32 partial product
// at C + s M N; a second kernel sums the slices in a fixed order (deterministic).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include "gwx_internal.h"
#include "tc05.cuh"

namespace gwx {

namespace {

using namespace tc;

constexpr int GM = 128, GN = 256, GK = 64, STAGES = 4;   // GN: the dense products' tile width
constexpr int EPI_WARPS = 8;                            // two per tensor-memory lane quarter
constexpr int GEMM_THREADS = 64 + 32 * EPI_WARPS;
constexpr uint32_t WAIT_POLLS = 1u << 22;
constexpr uint32_t EPI_BUF_BYTES = 32 * 32 * 4;         // per epilogue warp: a 32 x 32 FP32 transpose tile

// Per tile width TN_ (64, 128 or 256 columns of C) and M-tiles per CTA MW (1, or 2 with
// TN_ = 256): B tile, stage and accumulator sizes.  MW = 1: two accumulators of TN_
// columns alternate between tiles; MW = 2: one pair (rows 0-127, 128-255) per tile.
template <int TN_, int MW = 1>
struct Tile {
  static_assert(MW == 1 || (MW == 2 && TN_ == 256), "wide tiles are 256 x 256");
  static constexpr int ROWS = GM * MW;                     // rows of C per tile
  static constexpr uint32_t A_TILE = (uint32_t)ROWS * GK * 2;
  static constexpr uint32_t B_BYTES = TN_ * GK * 2;
  static constexpr uint32_t STAGE_BYTES = A_TILE + B_BYTES;
  static constexpr int NSTAGE = MW == 1 ? STAGES : 3;
  static constexpr int NACC = MW == 1 ? 2 : 1;             // accumulator sets in tensor memory
  static constexpr uint32_t TMEM_COLS = TN_;              // FP32 columns of one accumulator
  static constexpr uint32_t IDESC = idesc_bf16(GM, TN_);
  static constexpr size_t SMEM = (size_t)NSTAGE * STAGE_BYTES + (size_t)EPI_WARPS * EPI_BUF_BYTES + 1024;
};

// Implicit-GEMM convolution geometry (conv mode): A is the channels-last activation
// x [B][T][Cin] as a 3-D tensor map; M tile tm covers times 128 (tm mod T/128) ..
// + 127 of sample tm div (T/128), and K block kb covers tap kb div KC, channels
// 64 (kb mod KC) .. + 63, read at time t + dir (tap - pad) (zero outside [0, T)).
struct ConvGeo {
  int T;     // time steps per sample (a multiple of 128)
  int KC;    // Cin / 64
  int pad;   // (k - 1) / 2
  int dir;   // +1: convolution; -1: its input gradient (taps mirrored)
};

__device__ int g_gemm_status;

// Fused epilogue of a dense layer on 32 accumulator columns starting at col0:
// z = acc + bias[col], then the activation (0 identity, 1 ReLU, 2 GELU z Phi(z)).
__device__ __forceinline__ void epilogue_ops(float* v, const float* __restrict__ bias, int act, int col0, int N) {
  if (bias) {
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] += (col0 + i < N) ? __ldg(&bias[col0 + i]) : 0.f;
  }
  if (act == 1) {
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = fmaxf(v[i], 0.f);
  } else if (act == 2) {
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = 0.5f * v[i] * erfcf(-0.70710678118654752f * v[i]);
  }
}

// Tile t of a persistent CTA -> (tm, tn): bands of `group` tile-rows, columns fastest
// within a band, so the CTAs working at the same time share a few A and B panels in L2.
constexpr int DEFAULT_GROUP = 16;
__device__ __forceinline__ void tile_coords(int t, int TM, int TN, int group, int& tm, int& tn) {
  const int band = t / (group * TN);
  const int r = t - band * group * TN;
  const int rows = min(group, TM - band * group);
  tm = band * group + r % rows;
  tn = r / rows;
}

// Persistent, warp-specialised: warp 0 lane 0 produces (TMA), warp 1 allocates tensor
// memory and its lane 0 issues the MMAs, warps 2-9 drain accumulators.  MW = 1: two
// TN_-column accumulators alternate between tiles, so a tile's epilogue overlaps the next
// tile's main loop; MW = 2 (256 x 256 tiles): the two accumulators are the tile's two
// 128-row halves and the next tile waits for both to drain.  "tfull" (MMA commit) and
// "tempty" (one arrival per epilogue warp) hand them over.
// TN_: tile width; CONV: A is loaded as an implicit im2col tile (ConvGeo).  addend
// (optional; N % 32 == 0, 16-byte aligned): C = (A B^T + addend), then bias and activation.
template <bool OUT_BF16, int TN_, bool CONV, int MW = 1>
__global__ void __launch_bounds__(GEMM_THREADS, 1)
    k_gemm_bf16(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb, void* __restrict__ C,
                const float* __restrict__ bias, int act, int group, int M, int N, int K, int kbs, int splits,
                const float* __restrict__ addend, ConvGeo geo) {
  static_assert(MW == 1 || !CONV, "wide tiles are for plain products");
  constexpr int GN = TN_;
  using TL = Tile<TN_, MW>;
  constexpr int GMT = TL::ROWS;
  constexpr int STAGES = TL::NSTAGE;
  constexpr int NACC = TL::NACC;
  constexpr uint32_t A_BYTES = TL::A_TILE;
  constexpr uint32_t STAGE_BYTES = TL::STAGE_BYTES;
  constexpr uint32_t TMEM_COLS = TL::TMEM_COLS;
  constexpr uint32_t IDESC = TL::IDESC;
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full[STAGES], empty[STAGES], tfull[2], tempty[2];
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t base = (su32(smem_raw) + 1023u) & ~1023u;   // 1024-byte aligned stages
  const int KB = (K + GK - 1) / GK;
  const int TM = (M + GMT - 1) / GMT, TN = (N + GN - 1) / GN;
  const int tiles = TM * TN;
  const int work = tiles * splits;   // (tile, K slice) pairs, tile fastest

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(su32(&full[s]), 1);
      mbar_init(su32(&empty[s]), 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(su32(&tfull[a]), 1);
      mbar_init(su32(&tempty[a]), EPI_WARPS);
    }
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_slot)),
                 "r"(2 * TMEM_COLS)
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
      for (int w = blockIdx.x; w < work && !*(volatile int*)&abort_flag; w += gridDim.x) {
        int tm, tn;
        tile_coords(w % tiles, TM, TN, group, tm, tn);
        const int kb0 = (w / tiles) * kbs, kb1 = min(KB, kb0 + kbs);
        for (int kb = kb0; kb < kb1; ++kb, ++it) {
          const uint32_t s = it % STAGES;
          if (it >= STAGES && !mbar_wait(su32(&empty[s]), ((it / STAGES) - 1) & 1u, WAIT_POLLS)) {
            atomicExch(&abort_flag, 1);
            break;
          }
          const uint32_t sa = base + s * STAGE_BYTES, sb = sa + A_BYTES;
          mbar_expect_tx(su32(&full[s]), STAGE_BYTES);
          if constexpr (CONV) {
            const int tpb = geo.T / GM;   // M tiles per sample
            const int tap = kb / geo.KC, cb = kb - tap * geo.KC;
            tma_load_3d(sa, &ta, cb * GK, (tm % tpb) * GM + geo.dir * (tap - geo.pad), tm / tpb, su32(&full[s]));
          } else {
            tma_load_2d(sa, &ta, kb * GK, tm * GMT, su32(&full[s]));   // one box of GMT rows
          }
          tma_load_2d(sb, &tb, kb * GK, tn * GN, su32(&full[s]));
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      uint32_t it = 0, tl = 0;
      for (int w = blockIdx.x; w < work && !*(volatile int*)&abort_flag; w += gridDim.x, ++tl) {
        const uint32_t acc = tl % NACC;
        const int kb0 = (w / tiles) * kbs, kb1 = min(KB, kb0 + kbs);
        if (tl >= NACC && !mbar_wait(su32(&tempty[acc]), ((tl / NACC) - 1) & 1u, WAIT_POLLS)) {
          atomicExch(&abort_flag, 1);
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t d = tmem + acc * TMEM_COLS;
        bool ok = true;
        for (int kb = kb0; kb < kb1; ++kb, ++it) {
          const uint32_t s = it % STAGES;
          if (!mbar_wait(su32(&full[s]), (it / STAGES) & 1u, WAIT_POLLS)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t sa = base + s * STAGE_BYTES, sb = sa + A_BYTES;
#pragma unroll
          for (int kk = 0; kk < GK / 16; ++kk) {   // 16 bfloat16 = 32 bytes along K per instruction
            // M-tile m: rows 128 m .. of the A box (16 KiB apart), accumulator columns m TN_ ..
#pragma unroll
            for (int m = 0; m < MW; ++m)
              mma_bf16(d + (uint32_t)m * TMEM_COLS, sw128_desc(sa + (uint32_t)m * (GM * GK * 2) + 32u * kk),
                       sw128_desc(sb + 32u * kk), IDESC, kb != kb0 || kk != 0);
          }
          mma_commit(su32(&empty[s]));
        }
        if (!ok) atomicExch(&abort_flag, 1);
        mma_commit(su32(&tfull[acc]));   // arrives once the tile's MMAs have completed
        if (!ok) break;
      }
    }
  } else {
    // epilogue warps 2-9; tensor-memory lane quarter (warp % 4) = tile rows 32 q .. 32 q + 31;
    // (warp - 2) / 4 picks the column half (MW = 1) or the M-tile (MW = 2, all columns)
    const int q = warp & 3;
    const int hsel = (warp - 2) >> 2;
    const int c_lo = MW == 1 ? hsel * (GN / 64) : 0, c_hi = MW == 1 ? c_lo + GN / 64 : GN / 32;
    const int msel = MW == 1 ? 0 : hsel;
    float* ebuf = reinterpret_cast<float*>(smem_raw + (base - su32(smem_raw)) + STAGES * STAGE_BYTES +
                                           (warp - 2) * EPI_BUF_BYTES);
    uint32_t tl = 0;
    for (int w = blockIdx.x; w < work; w += gridDim.x, ++tl) {
      int tm, tn;
      tile_coords(w % tiles, TM, TN, group, tm, tn);
      const size_t slice = (size_t)(w / tiles) * (size_t)M * (size_t)N;   // 0 unless split
      const uint32_t acc = tl % NACC;
      const bool have = mbar_wait(su32(&tfull[acc]), (tl / NACC) & 1u, WAIT_POLLS);
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (__any_sync(0xffffffffu, !have || *(volatile int*)&abort_flag != 0)) {
        if (lane == 0) atomicExch(&abort_flag, 1);
        break;
      }
      // Each warp stages its 32 rows x 32 columns through a swizzled shared tile (word j of
      // row r at r * 32 + (j ^ r): conflict-free both ways), then stores whole row segments:
      // FP32 one 128-byte row per instruction, bfloat16 two 64-byte rows per instruction.
      const int row0 = tm * GMT + GM * msel + 32 * q;
#pragma unroll 1
      for (int c = c_lo; c < c_hi; ++c) {
        float v[32];
        const int col0 = tn * GN + 32 * c;
        // addend row segment of this lane's row (columns col0 .. col0 + 31; N % 32 == 0 and a
        // 16-byte aligned addend when one is given), fetched before the accumulator so that
        // its latency overlaps the tensor-memory load
        float4 ad[8];
        if (addend != nullptr) {
          const bool in = row0 + lane < M && col0 < N;
          const float4* ap = reinterpret_cast<const float4*>(addend + (int64_t)(row0 + lane) * N + col0);
#pragma unroll
          for (int j = 0; j < 8; ++j) ad[j] = in ? __ldg(ap + j) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (acc + (uint32_t)msel) * TMEM_COLS + (uint32_t)(32 * c), v);
        if (row0 >= M || col0 >= N) continue;   // warp-uniform
        if (addend != nullptr) {
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            v[4 * j] += ad[j].x;
            v[4 * j + 1] += ad[j].y;
            v[4 * j + 2] += ad[j].z;
            v[4 * j + 3] += ad[j].w;
          }
        }
        epilogue_ops(v, bias, act, col0, N);
#pragma unroll
        for (int j = 0; j < 32; ++j) ebuf[lane * 32 + (j ^ lane)] = v[j];
        __syncwarp();
        if constexpr (OUT_BF16) {
          __nv_bfloat16* out = reinterpret_cast<__nv_bfloat16*>(C) + slice;
          const int w = lane & 15, col = col0 + 2 * w;
#pragma unroll 4
          for (int r2 = 0; r2 < 16; ++r2) {
            const int r = 2 * r2 + (lane >> 4);
            const int grow = row0 + r;
            const float a = ebuf[r * 32 + ((2 * w) ^ r)], b = ebuf[r * 32 + ((2 * w + 1) ^ r)];
            if (grow < M) {
              __nv_bfloat16* o = out + (int64_t)grow * N + col;
              if (col + 1 < N && (N % 2) == 0) {
                *reinterpret_cast<__nv_bfloat162*>(o) = __floats2bfloat162_rn(a, b);
              } else {
                if (col < N) o[0] = __float2bfloat16_rn(a);
                if (col + 1 < N) o[1] = __float2bfloat16_rn(b);
              }
            }
          }
        } else {
          float* out = reinterpret_cast<float*>(C) + slice;
          const int col = col0 + lane;
#pragma unroll 4
          for (int r = 0; r < 32; ++r) {
            const float a = ebuf[r * 32 + (lane ^ r)];
            if (row0 + r < M && col < N) out[(int64_t)(row0 + r) * N + col] = a;
          }
        }
        __syncwarp();
      }
      // the accumulator is drained: hand it back to the MMA issuer
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(su32(&tempty[acc]));
    }
  }
  __syncwarp();
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (threadIdx.x == 0 && *(volatile int*)&abort_flag) atomicExch(&g_gemm_status, 1);
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * TMEM_COLS) : "memory");
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
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

// Row-major bfloat16 [rows][K] as a 2-D tensor map with boxes of box_rows x 64.
bool make_map(CUtensorMap* map, const void* ptr, int64_t rows, int64_t K, uint32_t box_rows) {
  auto enc = encode_fn();
  if (!enc) return false;
  cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)K * 2};
  cuuint32_t box[2] = {(cuuint32_t)GK, box_rows};
  cuuint32_t estr[2] = {1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// out[i] = sum over s of part[s][i] for i < n (slices in order: deterministic).
__global__ void k_split_reduce(const float* __restrict__ part, int splits, int64_t n, float* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float acc = 0.f;
  for (int s = 0; s < splits; ++s) acc += __ldg(&part[(int64_t)s * n + i]);
  out[i] = acc;
}

template <int TN_, int MW = 1>
cudaError_t launch_gemm_tn(const CUtensorMap& ta, const CUtensorMap& tb, void* C, int64_t M, int64_t N, int64_t K,
                           bool out_bf16, const float* bias, int act, int group, int splits, int sms,
                           cudaStream_t s) {
  const int KB = (int)((K + GK - 1) / GK);
  const int kbs = (KB + splits - 1) / splits;   // every slice has at least one K block
  splits = (KB + kbs - 1) / kbs;
  const int64_t work = ((M + Tile<TN_, MW>::ROWS - 1) / Tile<TN_, MW>::ROWS) * ((N + TN_ - 1) / TN_) * splits;
  const unsigned grid = (unsigned)(work < sms ? work : sms);   // persistent: one CTA per SM
  constexpr size_t smem = Tile<TN_, MW>::SMEM;
  const ConvGeo none{0, 0, 0, 0};
  cudaError_t e;
  if (out_bf16) {
    e = cudaFuncSetAttribute(k_gemm_bf16<true, TN_, false, MW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) return e;
    k_gemm_bf16<true, TN_, false, MW><<<grid, GEMM_THREADS, smem, s>>>(ta, tb, C, bias, act, group, (int)M, (int)N,
                                                                       (int)K, kbs, splits, nullptr, none);
  } else {
    e = cudaFuncSetAttribute(k_gemm_bf16<false, TN_, false, MW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) return e;
    k_gemm_bf16<false, TN_, false, MW><<<grid, GEMM_THREADS, smem, s>>>(ta, tb, C, bias, act, group, (int)M, (int)N,
                                                                        (int)K, kbs, splits, nullptr, none);
  }
  return cudaGetLastError();
}

// Tile width of a product: 256 columns unless the 128 x 256 tiles would leave more than half
// of the SMs idle (the flow's conditioner products on a few hundred to a few thousand rows),
// then 128 or 64, so that more CTAs share the work.  Split-K products keep 256.
int gemm_tile_width(int64_t M, int64_t N, int splits, int sms) {
  if (splits > 1) return GN;
  const int64_t tm = (M + GM - 1) / GM;
  for (int tn : {256, 128})
    if (tm * ((N + tn - 1) / tn) * 2 >= sms) return tn;
  return 64;
}

// Wide 256 x 256 tiles for large products: no split K, a K long enough that the epilogue
// (no longer overlapped) is a small part of a tile, at least one full wave of them, and no
// GELU (its erfc epilogue, unoverlapped, cost more than the wide tiles gained: 0.77 vs
// 0.73 ms for an 8192^3 dense layer).
bool gemm_wide(int64_t M, int64_t N, int64_t K, int splits, int act, int sms) {
  return splits == 1 && K >= 1024 && act != GWX_ACT_GELU && ((M + 255) / 256) * ((N + 255) / 256) >= sms;
}

cudaError_t launch_gemm(const void* A, const void* B, void* C, int64_t M, int64_t N, int64_t K, bool out_bf16,
                        const float* bias, int act, int group, int splits, cudaStream_t s) {
  if (group < 1) group = DEFAULT_GROUP;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  CUtensorMap ta, tb;
  if (gemm_wide(M, N, K, splits, act, sms)) {
    if (!make_map(&ta, A, M, K, 2 * GM) || !make_map(&tb, B, N, K, 256)) return cudaErrorInvalidValue;
    return launch_gemm_tn<256, 2>(ta, tb, C, M, N, K, out_bf16, bias, act, group, splits, sms, s);
  }
  const int tn = gemm_tile_width(M, N, splits, sms);
  if (!make_map(&ta, A, M, K, GM) || !make_map(&tb, B, N, K, (uint32_t)tn)) return cudaErrorInvalidValue;
  if (tn == 64) return launch_gemm_tn<64>(ta, tb, C, M, N, K, out_bf16, bias, act, group, splits, sms, s);
  if (tn == 128) return launch_gemm_tn<128>(ta, tb, C, M, N, K, out_bf16, bias, act, group, splits, sms, s);
  return launch_gemm_tn<256>(ta, tb, C, M, N, K, out_bf16, bias, act, group, splits, sms, s);
}

// Channels-last bfloat16 x [Bn][T][C] as a 3-D tensor map with boxes of 64 channels x 128 times.
bool make_map_3d(CUtensorMap* map, const void* ptr, int64_t Bn, int64_t T, int64_t C) {
  auto enc = encode_fn();
  if (!enc) return false;
  cuuint64_t dims[3] = {(cuuint64_t)C, (cuuint64_t)T, (cuuint64_t)Bn};
  cuuint64_t strides[2] = {(cuuint64_t)C * 2, (cuuint64_t)T * C * 2};
  cuuint32_t box[3] = {(cuuint32_t)GK, (cuuint32_t)GM, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(ptr), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int TN_>
cudaError_t launch_conv_tn(const CUtensorMap& ta, const CUtensorMap& tb, float* out, const float* addend, int M, int N,
                           int K, ConvGeo geo, cudaStream_t s) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int KB = K / GK;
  const int64_t work = (int64_t)(M / GM) * ((N + TN_ - 1) / TN_);
  const unsigned grid = (unsigned)(work < sms ? work : sms);
  constexpr size_t smem = Tile<TN_>::SMEM;
  e = cudaFuncSetAttribute(k_gemm_bf16<false, TN_, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_gemm_bf16<false, TN_, true><<<grid, GEMM_THREADS, smem, s>>>(ta, tb, out, nullptr, GWX_ACT_NONE, DEFAULT_GROUP, M,
                                                                 N, K, KB, 1, addend, geo);
  return cudaGetLastError();
}

}  // namespace

// Implicit-GEMM 1-D convolution, stride 1, "same" zero padding: out [Bn][T][N] (FP32) =
// sum over taps j < k and channels c of x[b][t + dir (j - (k-1)/2)][c] W[o][j C + c], plus
// addend if given.  Tile width 64 / 128 / 256 by N.  Shapes checked by the caller.
cudaError_t launch_conv_gemm(const void* x, int64_t Bn, int64_t T, int64_t C, int k, int dir, const void* W, int64_t N,
                             float* out, const float* addend, cudaStream_t s) {
  CUtensorMap ta, tb;
  const int64_t K = (int64_t)k * C;
  const int tn = N <= 64 ? 64 : (N <= 128 ? 128 : 256);
  if (!make_map_3d(&ta, x, Bn, T, C) || !make_map(&tb, W, N, K, (uint32_t)tn)) return cudaErrorInvalidValue;
  const ConvGeo geo{(int)T, (int)(C / GK), (k - 1) / 2, dir};
  const int M = (int)(Bn * T);
  if (tn == 64) return launch_conv_tn<64>(ta, tb, out, addend, M, (int)N, (int)K, geo, s);
  if (tn == 128) return launch_conv_tn<128>(ta, tb, out, addend, M, (int)N, (int)K, geo, s);
  return launch_conv_tn<256>(ta, tb, out, addend, M, (int)N, (int)K, geo, s);
}

cudaError_t launch_gemm_bf16(const void* A, const void* B, void* C, int64_t M, int64_t N, int64_t K, bool out_bf16,
                             const float* bias, int act, int group, cudaStream_t s) {
  return launch_gemm(A, B, C, M, N, K, out_bf16, bias, act, group, 1, s);
}

int gemm_splits(int64_t M, int64_t N, int64_t K) {
  const int64_t tiles = ((M + GM - 1) / GM) * ((N + GN - 1) / GN);
  const int64_t KB = (K + GK - 1) / GK;
  if (tiles >= 64) return 1;
  int64_t sp = std::min<int64_t>(128 / tiles, KB / 4);   // ~128 work items, >= 4 K blocks per slice
  if (sp <= 1) return 1;
  const int64_t kbs = (KB + sp - 1) / sp;
  return (int)((KB + kbs - 1) / kbs);
}

size_t gemm_splitk_ws(int64_t M, int64_t N, int64_t K) {
  const int sp = gemm_splits(M, N, K);
  return sp > 1 ? (size_t)sp * (size_t)M * (size_t)N * 4 : 0;
}

cudaError_t launch_gemm_splitk(const void* A, const void* B, float* C, int64_t M, int64_t N, int64_t K, float* part,
                               cudaStream_t s) {
  const int sp = gemm_splits(M, N, K);
  if (sp <= 1) return launch_gemm(A, B, C, M, N, K, false, nullptr, GWX_ACT_NONE, 0, 1, s);
  cudaError_t e = launch_gemm(A, B, part, M, N, K, false, nullptr, GWX_ACT_NONE, 0, sp, s);
  if (e != cudaSuccess) return e;
  const int64_t n = M * N;
  k_split_reduce<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(part, sp, n, C);
  return cudaGetLastError();
}

// Self-test of the bounded waits: one thread waits on an mbarrier that nothing arrives at,
// gives up after `polls` polls and records the expiry in the status flag the tensor-core
// kernels use, as they do when their own copies never land.
__global__ void k_selftest_wait(uint32_t polls) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(su32(&bar), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0 && !mbar_wait(su32(&bar), 0u, polls)) atomicExch(&g_gemm_status, 1);
}

cudaError_t launch_selftest_wait(uint32_t polls, cudaStream_t s) {
  k_selftest_wait<<<1, 32, 0, s>>>(polls);
  return cudaGetLastError();
}

cudaError_t gemm_status(int* status) {
  int zero = 0;
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpyFromSymbol(status, g_gemm_status, sizeof(int));
  if (e == cudaSuccess && *status != 0) e = cudaMemcpyToSymbol(g_gemm_status, &zero, sizeof(int));
  return e;
}

}  // namespace gwx
