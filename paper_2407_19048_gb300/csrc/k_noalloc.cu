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
#include <mutex>

#include "gwx_internal.h"

namespace gwx {
namespace {

// Largest filter the array holds: GWX_MAX_DET detectors x (16384/2 + 1) bins.  The
// window check (N a power of two in [256, 16384]) and D <= GWX_MAX_DET keep every
// accepted request inside it.
constexpr size_t kStaticFilterFloats = (size_t)GWX_MAX_DET * (16384 / 2 + 1);
static_assert((size_t)GWX_MAX_DET * (16384 / 2 + 1) <= kStaticFilterFloats,
              "the largest accepted D x (N/2 + 1) must fit in the static filter");

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
  // the same checks, statuses and messages as gwx_whiten (no workspace to check)
  int k_lo = 0;
  int st = whiten_check_args(d, psd, seg_len, fs, f_lo, B, D, N, y, &k_lo);
  if (st != GWX_OK || B == 0) return st;
  st = init_device();                 // keeps the message of the step that failed
  if (st != GWX_OK) return st;
  float* W = nullptr;
  st = launch_status(static_filter_address(&W), "gwx_whiten_static: cudaGetSymbolAddress");
  if (st != GWX_OK) return st;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  // every filter entry the rows read is written first, so no clearing is needed
  st = launch_status(launch_whiten_filter(psd, D, seg_len, fs, k_lo, N, W, s), "gwx_whiten_static: whiten filter");
  if (st != GWX_OK) return st;
  return launch_status(launch_whiten_rows(d, W, B * D, D, N, y, s), "gwx_whiten_static: whiten");
}

}  // extern "C"
