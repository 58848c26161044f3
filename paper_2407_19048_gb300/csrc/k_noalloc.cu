// k_noalloc.cu -- whitening for callers that cannot allocate device memory.
//
// gwx_whiten needs scratch for its whitening filter (D x (N/2+1) floats), which
// the caller normally passes in as a workspace.  Some callers cannot provide one:
// a plug-in whose host application owns every device allocation, a serving loop
// that runs under a fixed, pre-reserved memory budget where no allocation or pool
// growth may happen, or a binding from a language that can only pass the data
// pointers.  gwx_whiten_static serves them: its scratch is a file-scope device
// array of fixed size that is part of the loaded library, so the call itself
// allocates nothing (no cudaMalloc, no cudaFree, no allocating library routine).
//
// The array is reached from host code only through the address returned by
// cudaGetSymbolAddress; in host code the array's name is a host-side stand-in,
// not a device address.  That address is looked up once per device, with the
// device current, on the first call on that device.
#include <math.h>

#include <mutex>

#include "gwx_internal.h"

namespace gwx {
namespace {

// Largest filter the array holds: GWX_MAX_DET detectors x (16384/2 + 1) bins.
constexpr size_t kStaticFilterFloats = (size_t)GWX_MAX_DET * (16384 / 2 + 1);

// Every GPU that loads the library holds this array (about 128 KiB) until exit.
static __device__ __align__(256) float g_static_filter[kStaticFilterFloats];

std::mutex g_addr_mu;
float* g_addr[256] = {nullptr};

// Device address of g_static_filter on the current device (looked up once per device).
cudaError_t static_filter_address(float** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 256) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_addr_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_filter);
    if (e != cudaSuccess) return e;
    g_addr[dev] = static_cast<float*>(p);
  }
  *out = g_addr[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace gwx

extern "C" {

int gwx_whiten_static(const float* d, const double* psd, int64_t seg_len, double fs, double f_lo, int64_t B, int D,
                      int64_t N, float* y, void* stream) {
  using namespace gwx;
  auto fail = [](int st, const char* msg) { return set_last_error(st, msg); };
  if (N < 256 || N > 16384 || (N & (N - 1)) != 0)
    return fail(GWX_ESHAPE, "gwx_whiten_static: N must be a power of two in [256, 16384]");
  if (D < 1 || D > GWX_MAX_DET) return fail(GWX_ESHAPE, "gwx_whiten_static: D must be in [1, GWX_MAX_DET]");
  if ((size_t)D * (size_t)(N / 2 + 1) > kStaticFilterFloats)
    return fail(GWX_ESHAPE, "gwx_whiten_static: D x (N/2+1) exceeds the static scratch of 4 x 8193 floats");
  if (seg_len < 16 || seg_len > 16384 || (seg_len & (seg_len - 1)) != 0)
    return fail(GWX_ESHAPE, "gwx_whiten_static: seg_len must be a power of two in [16, 16384]");
  if (B < 0 || B * D > 0x7fffffffLL) return fail(GWX_ESHAPE, "gwx_whiten_static: bad B");
  if (!(fs > 0.0) || !(f_lo > 0.0)) return fail(GWX_EINVAL, "gwx_whiten_static: fs and f_lo must be positive");
  const double k = ceil(f_lo / (fs / (double)N));
  if (k >= (double)(N / 2)) return fail(GWX_ESHAPE, "gwx_whiten_static: f_lo is above the last usable bin");
  if (B == 0) return GWX_OK;
  if (!d || !psd || !y) return fail(GWX_EINVAL, "gwx_whiten_static: NULL array");
  if ((((uintptr_t)d) | ((uintptr_t)psd) | ((uintptr_t)y)) & 7u)
    return fail(GWX_EINVAL, "gwx_whiten_static: d, psd and y must be 8-byte aligned");
  int st = gwx_init();
  if (st != GWX_OK) return fail(st, "gwx_whiten_static: device set-up failed");
  float* W = nullptr;
  cudaError_t e = static_filter_address(&W);
  if (e != cudaSuccess) return fail(GWX_ECUDA, "gwx_whiten_static: cudaGetSymbolAddress failed");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  // every filter entry the rows read is written first, so no clearing is needed
  e = launch_whiten_filter(psd, D, seg_len, fs, (int)k, N, W, s);
  if (e == cudaSuccess) e = launch_whiten_rows(d, W, B * D, D, N, y, s);
  if (e != cudaSuccess) return fail(GWX_ECUDA, "gwx_whiten_static: kernel launch failed");
  return GWX_OK;
}

}  // extern "C"
