// capi.cu -- the extern "C" entry points of libgwx: argument validation, the
// detector site table, per-device table set-up, workspace layout and dispatch to
// the kernel launchers.  Nothing here allocates device memory.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>

#include "gwx_internal.h"

using namespace gwx;

namespace {

thread_local char g_err[512] = "";

int fail(int status, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return status;
}

int cuda_fail(cudaError_t e, const char* where) {
  return fail(GWX_ECUDA, "%s: %s (%s)", where, cudaGetErrorName(e), cudaGetErrorString(e));
}

bool is_pow2(int64_t v) { return v > 0 && (v & (v - 1)) == 0; }

// ---------------------------------------------------------------- detector sites
// Vertex geodetic latitude and longitude [deg], elevation [m], x- and y-arm
// azimuths [deg clockwise from North] (approximate published values for the LIGO
// Hanford, LIGO Livingston and Virgo vertices; arm tilts neglected).
struct Site { double lat, lon, h, xaz, yaz; };
const Site kSites[3] = {
    {46.455147, -119.407657, 142.554, 324.0000, 234.0000},  // H1
    {30.562894, -90.774240, -6.574, 252.2835, 162.2835},    // L1
    {43.631415, 10.504497, 51.884, 19.4326, 289.4326},      // V1
};

void site_geometry(int det, double* T, double* r) {
  const double deg = 3.141592653589793238462643383279502884 / 180.0;
  const Site& s = kSites[det];
  const double phi = s.lat * deg, lam = s.lon * deg;
  const double north[3] = {-sin(phi) * cos(lam), -sin(phi) * sin(lam), cos(phi)};
  const double east[3] = {-sin(lam), cos(lam), 0.0};
  double x[3], y[3];
  for (int i = 0; i < 3; ++i) {
    x[i] = cos(s.xaz * deg) * north[i] + sin(s.xaz * deg) * east[i];
    y[i] = cos(s.yaz * deg) * north[i] + sin(s.yaz * deg) * east[i];
  }
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) T[3 * i + j] = 0.5 * (x[i] * x[j] - y[i] * y[j]);
  const double a = 6378137.0, f = 1.0 / 298.257223563, e2 = f * (2.0 - f);
  const double Nphi = a / sqrt(1.0 - e2 * sin(phi) * sin(phi));
  r[0] = (Nphi + s.h) * cos(phi) * cos(lam);
  r[1] = (Nphi + s.h) * cos(phi) * sin(lam);
  r[2] = (Nphi * (1.0 - e2) + s.h) * sin(phi);
}

int make_detparams(const int32_t* det_ids, int D, DetParams& dp) {
  if (D < 1 || D > GWX_MAX_DET) return fail(GWX_ESHAPE, "D=%d outside [1, %d]", D, GWX_MAX_DET);
  if (!det_ids) return fail(GWX_EINVAL, "det_ids is NULL");
  memset(&dp, 0, sizeof(dp));
  dp.D = D;
  for (int d = 0; d < D; ++d) {
    if (det_ids[d] < 0 || det_ids[d] > 2) return fail(GWX_EINVAL, "unknown detector id %d", det_ids[d]);
    site_geometry(det_ids[d], dp.tensor[d], dp.pos[d]);
  }
  return GWX_OK;
}

// ---------------------------------------------------------------- per-device set-up
std::mutex g_init_mu;
bool g_init_done[256] = {false};

int ensure_init() {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= 256) return fail(GWX_EUNSUPPORTED, "device ordinal %d", dev);
  std::lock_guard<std::mutex> lk(g_init_mu);
  if (g_init_done[dev]) return GWX_OK;
  if ((e = init_tables_random()) != cudaSuccess) return cuda_fail(e, "table set-up");
  if ((e = init_tables_spectral()) != cudaSuccess) return cuda_fail(e, "table set-up");
  if ((e = init_tables_waveform()) != cudaSuccess) return cuda_fail(e, "table set-up");
  if ((e = init_tables_fused()) != cudaSuccess) return cuda_fail(e, "table set-up");
  g_init_done[dev] = true;
  return GWX_OK;
}

cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

int launched(cudaError_t e, const char* what) { return e == cudaSuccess ? GWX_OK : cuda_fail(e, what); }

// ---------------------------------------------------------------- validation helpers
int check_window(int64_t N) {
  if (!is_pow2(N) || N < 256 || N > 16384)
    return fail(GWX_ESHAPE, "window length N=%lld must be a power of two in [256, 16384]", (long long)N);
  return GWX_OK;
}

int band_start(double f_lo, double df, int64_t limit, int* k_lo) {
  if (!(f_lo > 0.0) || !(df > 0.0) || !isfinite(f_lo) || !isfinite(df))
    return fail(GWX_EINVAL, "f_lo=%g and df=%g must be positive", f_lo, df);
  const double k = ceil(f_lo / df);
  if (k >= (double)limit) return fail(GWX_ESHAPE, "f_lo=%g is above the last usable bin", f_lo);
  *k_lo = (int)k;
  return GWX_OK;
}

constexpr size_t kAlign = 256;
size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

size_t whiten_ws_bytes(int D, int64_t N) { return align_up((size_t)D * (size_t)(N / 2 + 1) * sizeof(float)); }
size_t coef_bytes(int64_t B) { return align_up((size_t)B * sizeof(DrawCoef)); }

int check_ws(void* ws, size_t have, size_t need) {
  if (need == 0) return GWX_OK;
  if (!ws) return fail(GWX_EINVAL, "workspace is NULL (need %zu bytes)", need);
  if (have < need) return fail(GWX_ENOMEM, "workspace of %zu bytes is smaller than the %zu required", have, need);
  if (reinterpret_cast<uintptr_t>(ws) % kAlign) return fail(GWX_EINVAL, "workspace must be %zu-byte aligned", kAlign);
  return GWX_OK;
}

#define GWX_TRY(expr)          \
  do {                         \
    int _st = (expr);          \
    if (_st != GWX_OK) return _st; \
  } while (0)

// Arrays the kernels read or write with 64-bit accesses (complex values, pairs of
// floats, doubles, int64) must be 8-byte aligned; a misaligned pointer is rejected here
// instead of faulting on the device.
#define GWX_ALIGN16(p)                                                                     \
  do {                                                                                     \
    if (((uintptr_t)(const void*)(p)) & 15u) return fail(GWX_EINVAL, "%s is not 16-byte aligned", #p); \
  } while (0)

#define GWX_ALIGN8(p)                                                                     \
  do {                                                                                    \
    if (((uintptr_t)(const void*)(p)) & 7u) return fail(GWX_EINVAL, "%s is not 8-byte aligned", #p); \
  } while (0)

}  // namespace

namespace {
int check_psd_args(int64_t seg_len, int64_t N) {
  if (!is_pow2(seg_len) || seg_len < 16 || seg_len > 16384)
    return fail(GWX_ESHAPE, "seg_len=%lld must be a power of two in [16, 16384]", (long long)seg_len);
  (void)N;
  return GWX_OK;
}

int check_sim_shapes(int D, int64_t L, int64_t B, int64_t N, double fs, double f_lo, int* k_lo) {
  GWX_TRY(check_window(N));
  if (D < 1 || D > GWX_MAX_DET) return fail(GWX_ESHAPE, "D=%d outside [1, %d]", D, GWX_MAX_DET);
  if ((size_t)D * (size_t)(N / 2) * sizeof(float2) > 200 * 1024)
    return fail(GWX_EUNSUPPORTED, "D=%d windows of N=%lld do not fit in shared memory", D, (long long)N);
  if (L < N || L - N + 1 > 0xffffffffLL) return fail(GWX_ESHAPE, "need N <= L, L-N < 2^32");
  if (B < 0 || B > 0x7fffffffLL) return fail(GWX_ESHAPE, "B=%lld", (long long)B);
  if (!(fs > 0.0)) return fail(GWX_EINVAL, "fs must be positive");
  return band_start(f_lo, fs / (double)N, N / 2, k_lo);
}

// simulate workspace: [W: D x (N/2+1) floats | Wp: D x N/2 float2 | per-draw coefficients]
// floats of the filter region at the start of a simulation workspace (a multiple of 64)
int64_t sim_filter_floats(int D, int64_t N) { return (int64_t)(whiten_ws_bytes(D, N) / sizeof(float)); }
DrawCoef* sim_coef(void* ws, int D, int64_t N) {
  return reinterpret_cast<DrawCoef*>(reinterpret_cast<char*>(ws) + whiten_ws_bytes(D, N));
}
}  // namespace

int gwx::set_last_error(int status, const char* msg) { return fail(status, "%s", msg); }

// Argument checks shared by gwx_whiten, gwx_unwhiten and gwx_whiten_static (everything
// but the workspace); *k_lo receives the first band bin.  B == 0 passes with the
// arrays unchecked.
int gwx::whiten_check_args(const float* d, const double* psd, int64_t seg_len, double fs, double f_lo, int64_t B,
                           int D, int64_t N, const float* y, int* k_lo) {
  GWX_TRY(check_window(N));
  GWX_TRY(check_psd_args(seg_len, N));
  if (D < 1 || D > GWX_MAX_DET) return fail(GWX_ESHAPE, "D=%d", D);
  if (B < 0 || B * D > 0x7fffffffLL) return fail(GWX_ESHAPE, "B=%lld", (long long)B);
  if (!(fs > 0.0)) return fail(GWX_EINVAL, "fs must be positive");
  GWX_TRY(band_start(f_lo, fs / (double)N, N / 2, k_lo));
  if (B == 0) return GWX_OK;
  if (!d || !psd || !y) return fail(GWX_EINVAL, "NULL array");
  GWX_ALIGN8(d);
  GWX_ALIGN8(psd);
  GWX_ALIGN8(y);
  return GWX_OK;
}

int gwx::init_device() { return ensure_init(); }

int gwx::launch_status(cudaError_t e, const char* what) { return launched(e, what); }


namespace {
// Guard bytes after a workspace: byte i holds (0xA5 ^ (i * 131)) & 0xFF.
__device__ int g_guard_bad;
__global__ void k_guard_fill(uint8_t* p, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    p[i] = (uint8_t)(0xA5u ^ (unsigned)(i * 131u));
}
__global__ void k_guard_check(const uint8_t* p, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    if (p[i] != (uint8_t)(0xA5u ^ (unsigned)(i * 131u))) atomicExch(&g_guard_bad, 1);
}
}  // namespace

namespace gwx {
// defined in k_gemm.cu, next to the status flag it sets
cudaError_t launch_selftest_wait(uint32_t polls, cudaStream_t s);
}  // namespace gwx

extern "C" {

int gwx_version(void) { return 100; }

const char* gwx_status_string(int status) {
  switch (status) {
    case GWX_OK: return "ok";
    case GWX_EINVAL: return "invalid argument";
    case GWX_ESHAPE: return "unsupported or inconsistent sizes";
    case GWX_ECUDA: return "CUDA runtime error";
    case GWX_ENOMEM: return "workspace too small";
    case GWX_ETIMEOUT: return "device wait timed out";
    case GWX_EUNSUPPORTED: return "unsupported";
    default: return "unknown status";
  }
}

const char* gwx_last_error(void) { return g_err; }

int gwx_init(void) { return ensure_init(); }

int gwx_detector_geometry(int det, double* tensor9, double* position3) {
  if (det < 0 || det > 2) return fail(GWX_EINVAL, "unknown detector id %d", det);
  if (!tensor9 || !position3) return fail(GWX_EINVAL, "NULL output");
  site_geometry(det, tensor9, position3);
  return GWX_OK;
}

int gwx_sample_prior(const gwx_prior* prior, uint64_t seed, uint32_t step, int64_t B, int64_t L, int64_t N,
                     double* theta, int64_t* offsets, void* stream) {
  if (!prior) return fail(GWX_EINVAL, "prior is NULL");
  if (B < 0 || B > 0x7fffffffLL) return fail(GWX_ESHAPE, "B=%lld", (long long)B);
  if (N < 1 || L < N || L - N + 1 > 0xffffffffLL) return fail(GWX_ESHAPE, "need 1 <= N <= L, L-N < 2^32");
  if (B == 0) return GWX_OK;
  if (!theta || !offsets) return fail(GWX_EINVAL, "NULL output");
  GWX_ALIGN8(theta);
  GWX_ALIGN8(offsets);
  GWX_TRY(ensure_init());
  return launched(launch_sample_prior(*prior, seed, step, B, L, N, theta, offsets, as_stream(stream)),
                  "sample_prior");
}

int gwx_generate_waveforms(int approximant, const double* theta, int64_t B, double f_lo, double df, int64_t F,
                           float* hp, float* hc, void* stream) {
  if (approximant == GWX_IMRPHENOMD)
    return fail(GWX_EUNSUPPORTED, "IMRPhenomD is not available: its fitted coefficient tables are not in this build");
  if (approximant != GWX_TAYLORF2) return fail(GWX_EINVAL, "unknown approximant %d", approximant);
  if (B < 0 || B > 0x7fffffffLL) return fail(GWX_ESHAPE, "B=%lld", (long long)B);
  if (F < 2 || F - 1 > 16384) return fail(GWX_ESHAPE, "F=%lld outside [2, 16385]", (long long)F);
  int k_lo = 0;
  GWX_TRY(band_start(f_lo, df, F, &k_lo));
  if (B == 0) return GWX_OK;
  if (!theta || !hp || !hc) return fail(GWX_EINVAL, "NULL array");
  GWX_ALIGN8(theta);
  GWX_ALIGN8(hp);
  GWX_ALIGN8(hc);
  GWX_TRY(ensure_init());
  return launched(launch_generate_waveforms(theta, B, k_lo, df, F, reinterpret_cast<float2*>(hp),
                                            reinterpret_cast<float2*>(hc), as_stream(stream)),
                  "generate_waveforms");
}

int gwx_project(const float* hp, const float* hc, const double* theta, int64_t B, const int32_t* det_ids, int D,
                double gmst, double df, int64_t F, float* h_det, void* stream) {
  DetParams dp;
  GWX_TRY(make_detparams(det_ids, D, dp));
  if (B < 0 || B > 0x7fffffffLL) return fail(GWX_ESHAPE, "B=%lld", (long long)B);
  if (F < 1 || !(df > 0.0) || !isfinite(gmst)) return fail(GWX_EINVAL, "bad F, df or gmst");
  if (B == 0) return GWX_OK;
  if (!hp || !hc || !theta || !h_det) return fail(GWX_EINVAL, "NULL array");
  GWX_ALIGN8(hp);
  GWX_ALIGN8(hc);
  GWX_ALIGN8(theta);
  GWX_ALIGN8(h_det);
  GWX_TRY(ensure_init());
  return launched(launch_project(reinterpret_cast<const float2*>(hp), reinterpret_cast<const float2*>(hc), theta, B,
                                 dp, gmst, df, F, reinterpret_cast<float2*>(h_det), as_stream(stream)),
                  "project");
}

size_t gwx_colored_noise_workspace(int D, int64_t L) {
  if (D < 1 || L < 2) return 0;
  return align_up(colored_noise_ws(D, L));
}

int gwx_colored_noise(uint64_t seed, uint32_t step, int D, int64_t L, double fs, double f_lo, float* noise,
                      void* workspace, size_t workspace_bytes, void* stream) {
  if (D < 1 || D > GWX_MAX_DET) return fail(GWX_ESHAPE, "D=%d", D);
  if (!is_pow2(L) || L < 1024 || L > ((int64_t)1 << 24))
    return fail(GWX_ESHAPE, "L=%lld must be a power of two in [1024, 2^24]", (long long)L);
  if (!(fs > 0.0) || !(f_lo > 0.0)) return fail(GWX_EINVAL, "fs and f_lo must be positive");
  if (!noise) return fail(GWX_EINVAL, "noise is NULL");
  GWX_ALIGN8(noise);
  GWX_TRY(check_ws(workspace, workspace_bytes, gwx_colored_noise_workspace(D, L)));
  GWX_TRY(ensure_init());
  return launched(launch_colored_noise(seed, step, D, L, fs, f_lo, noise, workspace, as_stream(stream)),
                  "colored_noise");
}

size_t gwx_welch_psd_workspace(int D, int64_t L, int64_t seg_len, int64_t stride) {
  if (D < 1 || seg_len < 2 || stride < 1 || L < seg_len) return 0;
  return align_up(welch_ws(D, L, seg_len, stride));
}

int gwx_welch_psd(const float* x, int D, int64_t L, double fs, int64_t seg_len, int64_t stride, double* psd,
                  void* workspace, size_t workspace_bytes, void* stream) {
  if (D < 1 || D > GWX_MAX_DET) return fail(GWX_ESHAPE, "D=%d", D);
  if (!is_pow2(seg_len) || seg_len < 16 || seg_len > 16384)
    return fail(GWX_ESHAPE, "seg_len=%lld must be a power of two in [16, 16384]", (long long)seg_len);
  if (stride < 1 || stride > seg_len || L < seg_len) return fail(GWX_ESHAPE, "need 1 <= stride <= seg_len <= L");
  if ((L - seg_len) / stride + 1 > 0x7fffffffLL) return fail(GWX_ESHAPE, "too many segments");
  if (!(fs > 0.0)) return fail(GWX_EINVAL, "fs must be positive");
  if (!x || !psd) return fail(GWX_EINVAL, "NULL array");
  GWX_ALIGN8(psd);
  GWX_TRY(check_ws(workspace, workspace_bytes, gwx_welch_psd_workspace(D, L, seg_len, stride)));
  GWX_TRY(ensure_init());
  return launched(launch_welch(x, D, L, fs, seg_len, stride, psd, workspace, as_stream(stream)), "welch_psd");
}

int gwx_inject(const float* noise, int D, int64_t L, const int64_t* offsets, const float* h_det, int64_t B, int64_t N,
               double fs, float* d, void* stream) {
  GWX_TRY(check_window(N));
  if (D < 1 || D > GWX_MAX_DET) return fail(GWX_ESHAPE, "D=%d", D);
  if (L < N) return fail(GWX_ESHAPE, "L < N");
  if (B < 0 || B * D > 0x7fffffffLL) return fail(GWX_ESHAPE, "B=%lld", (long long)B);
  if (!(fs > 0.0)) return fail(GWX_EINVAL, "fs must be positive");
  if (B == 0) return GWX_OK;
  if (!noise || !offsets || !h_det || !d) return fail(GWX_EINVAL, "NULL array");
  GWX_ALIGN8(offsets);
  GWX_ALIGN8(h_det);
  GWX_ALIGN8(d);
  GWX_TRY(ensure_init());
  return launched(launch_inject_rows(noise, D, L, offsets, reinterpret_cast<const float2*>(h_det), B, N, fs, d,
                                     as_stream(stream)),
                  "inject");
}

int gwx_inject_padded(const float* noise, int D, int64_t L, const int64_t* offsets, const float* h_td, int64_t B,
                      int64_t N, int64_t N_pad, double fs, float* d, void* stream) {
  GWX_TRY(check_window(N));
  GWX_TRY(check_window(N_pad));
  if (N_pad < N) return fail(GWX_ESHAPE, "N_pad=%lld < N=%lld", (long long)N_pad, (long long)N);
  if (D < 1 || D > GWX_MAX_DET) return fail(GWX_ESHAPE, "D=%d", D);
  if (L < N) return fail(GWX_ESHAPE, "L < N");
  if (B < 0 || B * D > 0x7fffffffLL) return fail(GWX_ESHAPE, "B=%lld", (long long)B);
  if (!(fs > 0.0)) return fail(GWX_EINVAL, "fs must be positive");
  if (B == 0) return GWX_OK;
  if (!noise || !offsets || !h_td || !d) return fail(GWX_EINVAL, "NULL array");
  GWX_ALIGN8(offsets);
  GWX_TRY(ensure_init());
  return launched(launch_inject_padded(noise, D, L, offsets, h_td, B, N, N_pad, fs, d, as_stream(stream)),
                  "inject_padded");
}

size_t gwx_whiten_workspace(int D, int64_t N) {
  if (D < 1 || N < 2) return 0;
  return whiten_ws_bytes(D, N);
}


static int whiten_common(bool inverse, const float* d, const double* psd, int64_t seg_len, double fs, double f_lo, int64_t B, int D,
               int64_t N, float* y, void* workspace, size_t workspace_bytes, void* stream) {
  int k_lo = 0;
  GWX_TRY(whiten_check_args(d, psd, seg_len, fs, f_lo, B, D, N, y, &k_lo));
  if (B == 0) return GWX_OK;
  GWX_TRY(check_ws(workspace, workspace_bytes, gwx_whiten_workspace(D, N)));
  GWX_TRY(ensure_init());
  float* W = reinterpret_cast<float*>(workspace);
  cudaStream_t s = as_stream(stream);
  GWX_TRY(launched(launch_whiten_filter(psd, D, seg_len, fs, k_lo, N, W, s, inverse), "whiten filter"));
  return launched(launch_whiten_rows(d, W, B * D, D, N, y, s), "whiten");
}

int gwx_whiten(const float* d, const double* psd, int64_t seg_len, double fs, double f_lo, int64_t B, int D,
               int64_t N, float* y, void* workspace, size_t workspace_bytes, void* stream) {
  return whiten_common(false, d, psd, seg_len, fs, f_lo, B, D, N, y, workspace, workspace_bytes, stream);
}

int gwx_unwhiten(const float* y, const double* psd, int64_t seg_len, double fs, double f_lo, int64_t B, int D,
                 int64_t N, float* d, void* workspace, size_t workspace_bytes, void* stream) {
  return whiten_common(true, y, psd, seg_len, fs, f_lo, B, D, N, d, workspace, workspace_bytes, stream);
}

size_t gwx_simulate_batch_workspace(int D, int64_t B, int64_t N) {
  if (D < 1 || B < 0 || N < 2) return 0;
  return whiten_ws_bytes(D, N) + coef_bytes(B);
}

int gwx_prepare_batch(const gwx_prior* prior, uint64_t seed, uint32_t step, int64_t L, int64_t N, double fs,
                      double f_lo, const int32_t* det_ids, int D, double gmst, int64_t B, double* theta,
                      int64_t* offsets, void* workspace, size_t workspace_bytes, void* stream) {
  if (!prior) return fail(GWX_EINVAL, "prior is NULL");
  DetParams dp;
  GWX_TRY(make_detparams(det_ids, D, dp));
  int k_lo = 0;
  GWX_TRY(check_sim_shapes(D, L, B, N, fs, f_lo, &k_lo));
  if (!isfinite(gmst)) return fail(GWX_EINVAL, "bad gmst");
  if (B == 0) return GWX_OK;
  if (!theta || !offsets) return fail(GWX_EINVAL, "NULL array");
  GWX_ALIGN8(theta);
  GWX_ALIGN8(offsets);
  GWX_TRY(check_ws(workspace, workspace_bytes, gwx_simulate_batch_workspace(D, B, N)));
  GWX_TRY(ensure_init());
  cudaStream_t s = as_stream(stream);
  GWX_TRY(launched(launch_sample_prior(*prior, seed, step, B, L, N, theta, offsets, s), "sample_prior"));
  return launched(launch_draw_setup(theta, B, k_lo, fs / (double)N, fs, N / 2 + 1, dp, gmst, sim_coef(workspace, D, N), s),
                  "draw set-up");
}

int gwx_prepare_theta(const double* theta, int64_t L, int64_t N, double fs, double f_lo, const int32_t* det_ids,
                      int D, double gmst, int64_t B, void* workspace, size_t workspace_bytes, void* stream) {
  DetParams dp;
  GWX_TRY(make_detparams(det_ids, D, dp));
  int k_lo = 0;
  GWX_TRY(check_sim_shapes(D, L, B, N, fs, f_lo, &k_lo));
  if (!isfinite(gmst)) return fail(GWX_EINVAL, "bad gmst");
  if (B == 0) return GWX_OK;
  if (!theta) return fail(GWX_EINVAL, "NULL array");
  GWX_ALIGN8(theta);
  GWX_TRY(check_ws(workspace, workspace_bytes, gwx_simulate_batch_workspace(D, B, N)));
  GWX_TRY(ensure_init());
  return launched(launch_draw_setup(theta, B, k_lo, fs / (double)N, fs, N / 2 + 1, dp, gmst,
                                    sim_coef(workspace, D, N), as_stream(stream)),
                  "draw set-up");
}

int gwx_simulate_prepared(const float* noise, int64_t L, const double* psd, int64_t seg_len, double fs, double f_lo,
                          int D, int64_t B, int64_t N, const int64_t* offsets, float* y, int flags, void* workspace,
                          size_t workspace_bytes, void* stream) {
  if (flags & ~GWX_SIM_FILTERS_READY) return fail(GWX_EINVAL, "flags 0x%x", flags);
  int k_lo = 0;
  GWX_TRY(check_sim_shapes(D, L, B, N, fs, f_lo, &k_lo));
  GWX_TRY(check_psd_args(seg_len, N));
  if (B == 0) return GWX_OK;
  if (!noise || !psd || !y || !offsets) return fail(GWX_EINVAL, "NULL array");
  GWX_ALIGN8(psd);
  GWX_ALIGN8(y);
  GWX_ALIGN8(offsets);
  GWX_TRY(check_ws(workspace, workspace_bytes, gwx_simulate_batch_workspace(D, B, N)));
  GWX_TRY(ensure_init());
  cudaStream_t s = as_stream(stream);
  float* W = reinterpret_cast<float*>(workspace);
  if (!(flags & GWX_SIM_FILTERS_READY))
    GWX_TRY(launched(launch_whiten_filter(psd, D, seg_len, fs, k_lo, N, W, s), "whiten filter"));
  return launched(launch_simulate_fused(sim_coef(workspace, D, N), noise, L, offsets, W, sim_filter_floats(D, N), k_lo,
                                        D, B, N, fs, y, s),
                  "simulate");
}

int gwx_simulate_shape(int64_t N, int D, int shape) {
  GWX_TRY(check_window(N));
  if (D < 1 || D > GWX_MAX_DET) return fail(GWX_ESHAPE, "D=%d outside [1, %d]", D, GWX_MAX_DET);
  if (shape < -2 || shape > 15) return fail(GWX_EINVAL, "shape %d outside [-2, 15]", shape);
  if (shape >= -1) sim_shape_set(N, D, shape);
  return sim_shape_for(N, D);
}

int gwx_simulate_autotune(const float* noise, int64_t L, const double* psd, int64_t seg_len, double fs, double f_lo,
                          int D, int64_t B, int64_t N, const int64_t* offsets, float* y, void* workspace,
                          size_t workspace_bytes, int* shape_out, void* stream) {
  int k_lo = 0;
  GWX_TRY(check_sim_shapes(D, L, B, N, fs, f_lo, &k_lo));
  GWX_TRY(check_psd_args(seg_len, N));
  if (B < 1) return fail(GWX_ESHAPE, "autotune needs at least one draw");
  if (!noise || !psd || !y || !offsets) return fail(GWX_EINVAL, "NULL array");
  GWX_ALIGN8(psd);
  GWX_ALIGN8(y);
  GWX_ALIGN8(offsets);
  GWX_TRY(check_ws(workspace, workspace_bytes, gwx_simulate_batch_workspace(D, B, N)));
  GWX_TRY(ensure_init());
  cudaStream_t s = as_stream(stream);
  float* W = reinterpret_cast<float*>(workspace);
  GWX_TRY(launched(launch_whiten_filter(psd, D, seg_len, fs, k_lo, N, W, s), "whiten filter"));
  const DrawCoef* coef = sim_coef(workspace, D, N);
  const int64_t Wcap = sim_filter_floats(D, N);
  // two-buffer passes or not x all resident blocks per SM or one, and the staged form
  const bool stage = sim_can_stage(noise, L, W, N);
  const int candidates[] = {0, 1, 2, 3, 8, 10};
  const int n_cand = stage ? 6 : 4;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return cuda_fail(cudaGetLastError(), "autotune event");
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return cuda_fail(cudaGetLastError(), "autotune event");
  }
  int best = -1;
  float best_ms = 0.f;
  cudaError_t err = cudaSuccess;
  for (int ci = 0; ci < n_cand; ++ci) {
    const int c = candidates[ci];
    err = launch_simulate_fused(coef, noise, L, offsets, W, Wcap, k_lo, D, B, N, fs, y, s, c);   // warm-up
    if (err == cudaSuccess) err = cudaEventRecord(e0, s);
    for (int rep = 0; rep < 3 && err == cudaSuccess; ++rep)
      err = launch_simulate_fused(coef, noise, L, offsets, W, Wcap, k_lo, D, B, N, fs, y, s, c);
    if (err == cudaSuccess) err = cudaEventRecord(e1, s);
    if (err == cudaSuccess) err = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    if (err != cudaSuccess) break;
    if (best < 0 || ms < best_ms) {
      best = c;
      best_ms = ms;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (err != cudaSuccess) return cuda_fail(err, "simulate autotune");
  sim_shape_set(N, D, best);
  if (shape_out) *shape_out = best;
  return GWX_OK;
}

int gwx_simulate_batch(const gwx_prior* prior, uint64_t seed, uint32_t step, const float* noise, int64_t L,
                       const double* psd, int64_t seg_len, double fs, double f_lo, const int32_t* det_ids, int D,
                       double gmst, int64_t B, int64_t N, float* y, double* theta, int64_t* offsets, void* workspace,
                       size_t workspace_bytes, void* stream) {
  GWX_TRY(check_psd_args(seg_len, N));
  if (B > 0 && (!noise || !psd || !y)) return fail(GWX_EINVAL, "NULL array");
  GWX_TRY(gwx_prepare_batch(prior, seed, step, L, N, fs, f_lo, det_ids, D, gmst, B, theta, offsets, workspace,
                            workspace_bytes, stream));
  return gwx_simulate_prepared(noise, L, psd, seg_len, fs, f_lo, D, B, N, offsets, y, 0, workspace, workspace_bytes,
                               stream);
}

size_t gwx_log_likelihood_workspace(int64_t E, int D, int64_t N, int64_t S) {
  if (E < 0 || D < 1 || N < 2 || S < 0) return 0;
  // per-event spectra, whitening filter, per-event norm partials, merger-time grid constants
  return align_up((size_t)E * D * (size_t)(N / 2 + 1) * sizeof(float2)) + whiten_ws_bytes(D, N) +
         align_up(loglike_norm_bytes(E)) + align_up(tm_rows_bytes());
}

// Shared by the two likelihood entry points: validation, data spectra, whitening filter
// and the kernels (tmarg: merger time integrated out over tc_lo + j / (u fs), j < u n_tc).
static int loglike_common(bool tmarg, int approximant, const float* y_data, int64_t E, int D, int64_t N,
                          const double* psd, int64_t seg_len, double fs, double f_lo, const int32_t* det_ids,
                          double gmst, double tc_lo, int64_t n_tc, int oversample, const double* theta,
                          const int64_t* event_offsets, int64_t S, double* lnl, void* workspace,
                          size_t workspace_bytes, void* stream) {
  if (approximant == GWX_IMRPHENOMD)
    return fail(GWX_EUNSUPPORTED, "IMRPhenomD is not available: its fitted coefficient tables are not in this build");
  if (approximant != GWX_TAYLORF2) return fail(GWX_EINVAL, "unknown approximant %d", approximant);
  GWX_TRY(check_window(N));
  GWX_TRY(check_psd_args(seg_len, N));
  DetParams dp;
  GWX_TRY(make_detparams(det_ids, D, dp));
  if (E < 0 || S < 0 || S > 0x7fffffffLL * 8 || E * D > 0x7fffffffLL) return fail(GWX_ESHAPE, "bad E or S");
  if (S > 0 && E == 0) return fail(GWX_ESHAPE, "samples without events");
  if (!(fs > 0.0) || !isfinite(gmst)) return fail(GWX_EINVAL, "bad fs or gmst");
  if (tmarg) {
    if (!isfinite(tc_lo)) return fail(GWX_EINVAL, "tc_lo must be finite");
    if (n_tc < 1 || n_tc > N) return fail(GWX_ESHAPE, "n_tc=%lld must be in [1, N=%lld]", (long long)n_tc, (long long)N);
    if (!is_pow2(oversample) || oversample > 64)
      return fail(GWX_ESHAPE, "oversample=%d must be a power of two in [1, 64]", oversample);
  }
  const double df = fs / (double)N;
  int k_lo = 0;
  GWX_TRY(band_start(f_lo, df, N / 2, &k_lo));
  if (S == 0) return GWX_OK;
  if (!y_data || !psd || !theta || !event_offsets || !lnl) return fail(GWX_EINVAL, "NULL array");
  GWX_ALIGN8(y_data);
  GWX_ALIGN8(psd);
  GWX_ALIGN8(theta);
  GWX_ALIGN8(event_offsets);
  GWX_ALIGN8(lnl);
  GWX_TRY(check_ws(workspace, workspace_bytes, gwx_log_likelihood_workspace(E, D, N, S)));
  GWX_TRY(ensure_init());
  cudaStream_t s = as_stream(stream);
  char* w = reinterpret_cast<char*>(workspace);
  float2* Y = reinterpret_cast<float2*>(w);
  w += align_up((size_t)E * D * (size_t)(N / 2 + 1) * sizeof(float2));
  float* W = reinterpret_cast<float*>(w);
  w += whiten_ws_bytes(D, N);
  double* yy_part = reinterpret_cast<double*>(w);
  w += align_up(loglike_norm_bytes(E));
  float2* tm_rows = reinterpret_cast<float2*>(w);
  GWX_TRY(launched(launch_rfft_rows(y_data, E * D, N, Y, s), "rfft of the data"));
  GWX_TRY(launched(launch_whiten_filter(psd, D, seg_len, fs, k_lo, N, W, s), "whiten filter"));
  if (tmarg)
    return launched(launch_loglike_tmarg(y_data, Y, W, theta, df, fs, dp, gmst, tc_lo, (int)n_tc, oversample,
                                         event_offsets, yy_part, tm_rows, E, D, N, k_lo, S, lnl, s),
                    "log_likelihood_tmarg");
  return launched(launch_loglike_full(y_data, Y, W, theta, df, fs, dp, gmst, event_offsets, yy_part, E, D, N, k_lo,
                                      S, lnl, s),
                  "log_likelihood");
}

int gwx_log_likelihood(int approximant, const float* y_data, int64_t E, int D, int64_t N, const double* psd,
                       int64_t seg_len, double fs, double f_lo, const int32_t* det_ids, double gmst,
                       const double* theta, const int64_t* event_offsets, int64_t S, double* lnl, void* workspace,
                       size_t workspace_bytes, void* stream) {
  return loglike_common(false, approximant, y_data, E, D, N, psd, seg_len, fs, f_lo, det_ids, gmst, 0.0, 1, 1, theta,
                        event_offsets, S, lnl, workspace, workspace_bytes, stream);
}

int gwx_log_likelihood_tmarg(int approximant, const float* y_data, int64_t E, int D, int64_t N, const double* psd,
                             int64_t seg_len, double fs, double f_lo, const int32_t* det_ids, double gmst,
                             double tc_lo, int64_t n_tc, int oversample, const double* theta,
                             const int64_t* event_offsets, int64_t S, double* lnl, void* workspace,
                             size_t workspace_bytes, void* stream) {
  return loglike_common(true, approximant, y_data, E, D, N, psd, seg_len, fs, f_lo, det_ids, gmst, tc_lo, n_tc,
                        oversample, theta, event_offsets, S, lnl, workspace, workspace_bytes, stream);
}

size_t gwx_importance_weights_workspace(int64_t E) {
  if (E < 0) return 0;
  return align_up(iw_workspace_bytes(E));
}

int gwx_importance_weights(const double* lnl, const double* log_ratio, const int64_t* event_offsets, int64_t E,
                           int64_t S, double* weights, double* ess, double* efficiency, double* ln_evidence,
                           void* workspace, size_t workspace_bytes, void* stream) {
  if (E < 0 || S < 0 || E > 0x7fffffffLL) return fail(GWX_ESHAPE, "bad E=%lld or S=%lld", (long long)E, (long long)S);
  if (S > 0 && E == 0) return fail(GWX_ESHAPE, "samples without events");
  if (E == 0) return GWX_OK;
  if (!event_offsets || (S > 0 && !lnl)) return fail(GWX_EINVAL, "NULL array");
  GWX_ALIGN8(lnl);
  GWX_ALIGN8(log_ratio);
  GWX_ALIGN8(event_offsets);
  GWX_ALIGN8(weights);
  GWX_ALIGN8(ess);
  GWX_ALIGN8(efficiency);
  GWX_ALIGN8(ln_evidence);
  GWX_TRY(check_ws(workspace, workspace_bytes, gwx_importance_weights_workspace(E)));
  GWX_TRY(ensure_init());
  return launched(launch_importance_weights(lnl, log_ratio, event_offsets, E, S, weights, ess, efficiency,
                                            ln_evidence, workspace, as_stream(stream)),
                  "importance_weights");
}

// Tuned raster bands of the product, per (M, N, K, output type); filled by
// gwx_gemm_autotune, read (without synchronising) by every product call.
namespace {
std::mutex g_tune_mu;
std::map<std::tuple<int64_t, int64_t, int64_t, int>, int> g_tune;

int tuned_group(int64_t M, int64_t N, int64_t K, int c_dtype) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tune.find(std::make_tuple(M, N, K, c_dtype));
  return it == g_tune.end() ? 0 : it->second;
}
}  // namespace

static int check_dense(const void* A, const void* B, const float* bias, const void* C, int64_t M, int64_t N, int64_t K,
                       int act, int c_dtype) {
  if (M < 1 || M > ((int64_t)1 << 23) || N < 1 || N > 0x7fffffffLL || K < 8 || K > 0x7fffffffLL || K % 8 != 0)
    return fail(GWX_ESHAPE, "gemm sizes M=%lld N=%lld K=%lld (need K %% 8 == 0)", (long long)M, (long long)N,
                (long long)K);
  if (c_dtype != GWX_F32 && c_dtype != GWX_BF16) return fail(GWX_EINVAL, "c_dtype %d", c_dtype);
  if (act != GWX_ACT_NONE && act != GWX_ACT_RELU && act != GWX_ACT_GELU) return fail(GWX_EINVAL, "act %d", act);
  if (!A || !B || !C) return fail(GWX_EINVAL, "NULL array");
  if ((((uintptr_t)A) | ((uintptr_t)B) | ((uintptr_t)C)) & 15u)
    return fail(GWX_EINVAL, "A, B and C must be 16-byte aligned");
  if (((uintptr_t)bias) & 3u) return fail(GWX_EINVAL, "bias must be 4-byte aligned");
  return GWX_OK;
}

static int dense_common(const void* A, const void* B, const float* bias, void* C, int64_t M, int64_t N, int64_t K,
                        int act, int c_dtype, void* stream) {
  GWX_TRY(check_dense(A, B, bias, C, M, N, K, act, c_dtype));
  GWX_TRY(ensure_init());
  return launched(launch_gemm_bf16(A, B, C, M, N, K, c_dtype == GWX_BF16, bias, act, tuned_group(M, N, K, c_dtype),
                                   as_stream(stream)),
                  "gemm_bf16");
}

size_t gwx_dense_bf16_backward_workspace(int64_t M, int64_t N, int64_t K) {
  if (M < 1 || N < 1 || K < 1) return 0;
  return align_up(dense_backward_ws(M, N, K));
}

int gwx_dense_bf16_backward(const void* X, const void* W, const float* bias, const float* dY, int64_t M, int64_t N,
                            int64_t K, int act, float* dX, float* dW, float* db, void* workspace,
                            size_t workspace_bytes, void* stream) {
  const int64_t lim = (int64_t)65535 * 32;
  if (M < 8 || N < 8 || K < 8 || M % 8 || N % 8 || K % 8 || M > lim || N > lim || K > lim)
    return fail(GWX_ESHAPE, "dense backward sizes M=%lld N=%lld K=%lld (multiples of 8, at most %lld)",
                (long long)M, (long long)N, (long long)K, (long long)lim);
  if (act != GWX_ACT_NONE && act != GWX_ACT_RELU && act != GWX_ACT_GELU) return fail(GWX_EINVAL, "act %d", act);
  if (!X || !W || !dY) return fail(GWX_EINVAL, "NULL array");
  if ((((uintptr_t)X) | ((uintptr_t)W) | ((uintptr_t)dX) | ((uintptr_t)dW)) & 15u)
    return fail(GWX_EINVAL, "X, W, dX and dW must be 16-byte aligned");
  if ((((uintptr_t)dY) | ((uintptr_t)bias) | ((uintptr_t)db)) & 3u)
    return fail(GWX_EINVAL, "dY, bias and db must be 4-byte aligned");
  GWX_TRY(check_ws(workspace, workspace_bytes, gwx_dense_bf16_backward_workspace(M, N, K)));
  GWX_TRY(ensure_init());
  return launched(launch_dense_backward(X, W, bias, dY, M, N, K, act, dX, dW, db, workspace,
                                        tuned_group(M, N, K, GWX_F32), as_stream(stream)),
                  "dense_bf16_backward");
}

int gwx_gemm_autotune(const void* A, const void* B, void* C, int64_t M, int64_t N, int64_t K, int c_dtype,
                      int* group_out, void* stream) {
  GWX_TRY(check_dense(A, B, nullptr, C, M, N, K, GWX_ACT_NONE, c_dtype));
  GWX_TRY(ensure_init());
  cudaStream_t s = as_stream(stream);
  const int candidates[] = {1, 2, 4, 8, 16, 32, 64};
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return cuda_fail(cudaGetLastError(), "autotune event");
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return cuda_fail(cudaGetLastError(), "autotune event");
  }
  int best = 0;
  float best_ms = 0.f;
  cudaError_t err = cudaSuccess;
  for (int g : candidates) {
    for (int rep = 0; rep < 2 && err == cudaSuccess; ++rep)   // warm-up
      err = launch_gemm_bf16(A, B, C, M, N, K, c_dtype == GWX_BF16, nullptr, GWX_ACT_NONE, g, s);
    if (err == cudaSuccess) err = cudaEventRecord(e0, s);
    for (int rep = 0; rep < 3 && err == cudaSuccess; ++rep)
      err = launch_gemm_bf16(A, B, C, M, N, K, c_dtype == GWX_BF16, nullptr, GWX_ACT_NONE, g, s);
    if (err == cudaSuccess) err = cudaEventRecord(e1, s);
    if (err == cudaSuccess) err = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    if (err != cudaSuccess) break;
    if (best == 0 || ms < best_ms) {
      best = g;
      best_ms = ms;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (err != cudaSuccess) return cuda_fail(err, "autotune");
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[std::make_tuple(M, N, K, c_dtype)] = best;
  }
  if (group_out) *group_out = best;
  return GWX_OK;
}

int gwx_gemm_bf16(const void* A, const void* B, void* C, int64_t M, int64_t N, int64_t K, int c_dtype,
                  void* stream) {
  return dense_common(A, B, nullptr, C, M, N, K, GWX_ACT_NONE, c_dtype, stream);
}

int gwx_dense_bf16(const void* X, const void* W, const float* bias, void* Y, int64_t M, int64_t N, int64_t K,
                   int act, int y_dtype, void* stream) {
  return dense_common(X, W, bias, Y, M, N, K, act, y_dtype, stream);
}

int gwx_selftest_bounded_wait(uint32_t polls, void* stream) {
  if (polls < 1 || polls > (1u << 20)) return fail(GWX_EINVAL, "polls=%u (1 .. 2^20)", polls);
  GWX_TRY(ensure_init());
  return launched(launch_selftest_wait(polls, as_stream(stream)), "selftest_bounded_wait");
}

int gwx_debug_guard(void* workspace, size_t nbytes, size_t guard_bytes, void* stream) {
  if (!workspace || guard_bytes == 0) return fail(GWX_EINVAL, "workspace is NULL or the guard empty");
  GWX_TRY(ensure_init());
  uint8_t* p = reinterpret_cast<uint8_t*>(workspace) + nbytes;
  k_guard_fill<<<(unsigned)std::min<size_t>((guard_bytes + 255) / 256, 1024), 256, 0, as_stream(stream)>>>(p, guard_bytes);
  return launched(cudaGetLastError(), "guard fill");
}

int gwx_debug_check_guard(const void* workspace, size_t nbytes, size_t guard_bytes, int* intact, void* stream) {
  if (!workspace || guard_bytes == 0 || !intact) return fail(GWX_EINVAL, "NULL argument or empty guard");
  GWX_TRY(ensure_init());
  cudaStream_t s = as_stream(stream);
  // every call queued so far, on any stream, is done before the guard is read
  GWX_TRY(launched(cudaDeviceSynchronize(), "guard check"));
  const int zero = 0;
  GWX_TRY(launched(cudaMemcpyToSymbolAsync(g_guard_bad, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, s),
                   "guard reset"));
  const uint8_t* p = reinterpret_cast<const uint8_t*>(workspace) + nbytes;
  k_guard_check<<<(unsigned)std::min<size_t>((guard_bytes + 255) / 256, 1024), 256, 0, s>>>(p, guard_bytes);
  GWX_TRY(launched(cudaGetLastError(), "guard check"));
  int bad = 0;
  GWX_TRY(launched(cudaMemcpyFromSymbolAsync(&bad, g_guard_bad, sizeof(int), 0, cudaMemcpyDeviceToHost, s),
                   "guard read"));
  GWX_TRY(launched(cudaStreamSynchronize(s), "guard read"));
  *intact = bad ? 0 : 1;
  return GWX_OK;
}

int gwx_debug_build(void) {
#ifdef GWX_DEBUG_CHECKS
  return 1;
#else
  return 0;
#endif
}

int gwx_debug_status(uint64_t* first_bad) {
  if (!first_bad) return fail(GWX_EINVAL, "first_bad is NULL");
  GWX_TRY(ensure_init());
  unsigned long long a = 0, b = 0;
  GWX_TRY(launched(cudaDeviceSynchronize(), "debug status"));
  GWX_TRY(launched(debug_take_fused(&a), "debug status"));
  GWX_TRY(launched(debug_take_waveform(&b), "debug status"));
  *first_bad = a ? a : b;
  if (*first_bad) {
    const unsigned long long v = *first_bad;
    return fail(GWX_ESHAPE, "out-of-range access skipped at site 0x%llx, index %lld", (v >> 48) & 0xFFFFull,
                (long long)(v & ((1ull << 47) - 1)));
  }
  return GWX_OK;
}

int gwx_device_status(void) {
  GWX_TRY(ensure_init());
  int st = 0, st2 = 0, st3 = 0;
  GWX_TRY(launched(gemm_status(&st), "device status"));
  GWX_TRY(launched(flow_fused_status(&st2), "device status"));
  GWX_TRY(launched(sim_status(&st3), "device status"));
  if (st != 0 || st2 != 0 || st3 != 0)
    return fail(GWX_ETIMEOUT, "a kernel gave up waiting for its own copies; its output is incomplete");
  return GWX_OK;
}

size_t gwx_spectral_features_workspace(int64_t B, int D, int64_t N) {
  if (B < 1 || D < 1 || N < 2) return 0;
  return align_up((size_t)B * D * (size_t)(N / 2 + 1) * sizeof(float2));
}

int gwx_spectral_features(const float* y, int64_t B, int D, int64_t N, double fs, double f_lo, int group, int F_pad,
                          void* features, void* workspace, size_t workspace_bytes, void* stream) {
  GWX_TRY(check_window(N));
  if (D < 1 || D > GWX_MAX_DET) return fail(GWX_ESHAPE, "D=%d", D);
  if (B < 0 || B * D > 0x7fffffffLL) return fail(GWX_ESHAPE, "B=%lld", (long long)B);
  if (!(fs > 0.0)) return fail(GWX_EINVAL, "fs must be positive");
  int k_lo = 0;
  GWX_TRY(band_start(f_lo, fs / (double)N, N / 2, &k_lo));
  if (group < 1 || group > N / 2) return fail(GWX_EINVAL, "group %d", group);
  const int64_t ng = (N / 2 - k_lo) / group;
  if (F_pad < D * ng || F_pad % 8 != 0)
    return fail(GWX_ESHAPE, "F_pad=%d must be a multiple of 8 and at least D x groups = %lld", F_pad,
                (long long)(D * ng));
  if (B == 0) return GWX_OK;
  if (!y || !features) return fail(GWX_EINVAL, "NULL array");
  GWX_ALIGN8(y);
  GWX_ALIGN8(features);
  GWX_TRY(check_ws(workspace, workspace_bytes, gwx_spectral_features_workspace(B, D, N)));
  GWX_TRY(ensure_init());
  return launched(launch_features(y, B, D, N, k_lo, group, F_pad, workspace, features, as_stream(stream)),
                  "spectral_features");
}

int gwx_cross_features(const float* y, int64_t B, int D, int64_t N, double fs, double f_lo, int group, int F_pad,
                       int col0, void* features, void* workspace, size_t workspace_bytes, void* stream) {
  GWX_TRY(check_window(N));
  if (D < 2 || D > GWX_MAX_DET) return fail(GWX_ESHAPE, "D=%d (cross spectra need two detectors or more)", D);
  if (B < 0 || B * D > 0x7fffffffLL) return fail(GWX_ESHAPE, "B=%lld", (long long)B);
  if (!(fs > 0.0)) return fail(GWX_EINVAL, "fs must be positive");
  int k_lo = 0;
  GWX_TRY(band_start(f_lo, fs / (double)N, N / 2, &k_lo));
  if (group < 1 || group > N / 2) return fail(GWX_EINVAL, "group %d", group);
  const int64_t ng = (N / 2 - k_lo) / group;
  if (col0 < 0 || F_pad % 8 != 0 || col0 + (int64_t)D * (D - 1) * ng > F_pad)
    return fail(GWX_ESHAPE, "columns col0=%d + %lld exceed F_pad=%d", col0, (long long)(D * (D - 1) * ng), F_pad);
  if (B == 0) return GWX_OK;
  if (!y || !features) return fail(GWX_EINVAL, "NULL array");
  GWX_ALIGN8(y);
  GWX_ALIGN8(features);
  GWX_TRY(check_ws(workspace, workspace_bytes, gwx_spectral_features_workspace(B, D, N)));
  GWX_TRY(ensure_init());
  return launched(launch_cross_features(y, B, D, N, k_lo, group, F_pad, col0, workspace, features, as_stream(stream)),
                  "cross_features");
}

int gwx_lag_features(const float* y, int64_t B, int D, int64_t N, double fs, double f_lo, int group, int F_pad,
                     int col0, void* features, void* workspace, size_t workspace_bytes, void* stream) {
  GWX_TRY(check_window(N));
  if (D < 1 || D > GWX_MAX_DET) return fail(GWX_ESHAPE, "D=%d", D);
  if (B < 0 || B * D > 0x7fffffffLL) return fail(GWX_ESHAPE, "B=%lld", (long long)B);
  if (!(fs > 0.0)) return fail(GWX_EINVAL, "fs must be positive");
  int k_lo = 0;
  GWX_TRY(band_start(f_lo, fs / (double)N, N / 2, &k_lo));
  if (group < 1 || group > N / 2) return fail(GWX_EINVAL, "group %d", group);
  const int64_t ng = (N / 2 - k_lo) / group;
  if (col0 < 0 || F_pad % 8 != 0 || col0 + 2 * (int64_t)D * ng > F_pad)
    return fail(GWX_ESHAPE, "columns col0=%d + %lld exceed F_pad=%d", col0, (long long)(2 * D * ng), F_pad);
  if (B == 0) return GWX_OK;
  if (!y || !features) return fail(GWX_EINVAL, "NULL array");
  GWX_ALIGN8(y);
  GWX_ALIGN8(features);
  GWX_TRY(check_ws(workspace, workspace_bytes, gwx_spectral_features_workspace(B, D, N)));
  GWX_TRY(ensure_init());
  return launched(launch_lag_features(y, B, D, N, k_lo, group, F_pad, col0, workspace, features, as_stream(stream)),
                  "lag_features");
}

int gwx_proposal_targets(const double* theta, int64_t B, const double* mean3, const double* scale3, float* targets,
                         void* stream) {
  if (B < 0) return fail(GWX_ESHAPE, "B=%lld", (long long)B);
  if (!mean3 || !scale3) return fail(GWX_EINVAL, "mean and scale (host, 3 values each) are required");
  for (int i = 0; i < 3; ++i)
    if (!(scale3[i] > 0.0) || !isfinite(mean3[i])) return fail(GWX_EINVAL, "bad mean or scale %d", i);
  if (B == 0) return GWX_OK;
  if (!theta || !targets) return fail(GWX_EINVAL, "NULL array");
  GWX_ALIGN8(theta);
  GWX_TRY(ensure_init());
  return launched(launch_targets(theta, B, mean3, scale3, targets, as_stream(stream)), "proposal_targets");
}

int gwx_gauss_nll(const float* out, int ldo, const float* targets, int P, int64_t B, float* loss_rows,
                  double* loss_mean, float* grad, void* stream) {
  if (P < 1 || ldo < 2 * P || B < 1 || B > 0x7fffffffLL) return fail(GWX_ESHAPE, "gauss_nll sizes");
  if (!out || !targets || !loss_rows || !loss_mean || !grad) return fail(GWX_EINVAL, "NULL array");
  GWX_ALIGN8(loss_mean);
  GWX_TRY(ensure_init());
  return launched(launch_gauss_nll(out, ldo, targets, P, (int)B, loss_rows, loss_mean, grad, as_stream(stream)),
                  "gauss_nll");
}

int gwx_adamw(float* param, const float* grad, float* m, float* v, int64_t n, double lr, double beta1, double beta2,
              double eps, double weight_decay, int64_t step, void* param_bf16, void* stream) {
  if (n < 0) return fail(GWX_ESHAPE, "n=%lld", (long long)n);
  if (step < 1 || !(beta1 >= 0.0 && beta1 < 1.0) || !(beta2 >= 0.0 && beta2 < 1.0) || !(eps > 0.0) || !(lr >= 0.0))
    return fail(GWX_EINVAL, "AdamW hyper-parameters (step counts from 1)");
  if (n == 0) return GWX_OK;
  if (!param || !grad || !m || !v) return fail(GWX_EINVAL, "NULL array");
  GWX_TRY(ensure_init());
  return launched(launch_adamw(param, grad, m, v, n, lr, beta1, beta2, eps, weight_decay, step, param_bf16,
                               as_stream(stream)),
                  "adamw");
}

int gwx_adamw_at(float* param, const float* grad, float* m, float* v, int64_t n, double lr, double beta1, double beta2,
                 double eps, double weight_decay, const int64_t* step, void* param_bf16, void* stream) {
  if (n < 0) return fail(GWX_ESHAPE, "n=%lld", (long long)n);
  if (!(beta1 >= 0.0 && beta1 < 1.0) || !(beta2 >= 0.0 && beta2 < 1.0) || !(eps > 0.0) || !(lr >= 0.0))
    return fail(GWX_EINVAL, "AdamW hyper-parameters");
  if (n == 0) return GWX_OK;
  if (!param || !grad || !m || !v || !step) return fail(GWX_EINVAL, "NULL array or step");
  GWX_ALIGN8(step);
  GWX_TRY(ensure_init());
  return launched(launch_adamw_at(param, grad, m, v, n, lr, beta1, beta2, eps, weight_decay, step, param_bf16,
                                  as_stream(stream)),
                  "adamw_at");
}

int gwx_vicreg(const float* x, const float* xp, int64_t B, int d, double lambda1, double lambda2, double lambda3,
               double* loss, double* terms, float* grad_x, float* grad_xp, void* stream) {
  if (B < 2 || B > 0x7fffffffLL || !vicreg_supported((int)B, d))
    return fail(GWX_ESHAPE, "B=%lld d=%d (need B >= 2, 1 <= d <= 32)", (long long)B, d);
  if (!x || !xp || !loss || !grad_x || !grad_xp) return fail(GWX_EINVAL, "NULL array");
  GWX_ALIGN8(loss);
  if (terms) GWX_ALIGN8(terms);
  GWX_TRY(ensure_init());
  return launched(launch_vicreg(x, xp, (int)B, d, lambda1, lambda2, lambda3, loss, terms, grad_x, grad_xp,
                                as_stream(stream)),
                  "vicreg");
}

int gwx_retime(const double* theta_in, double* theta_out, int64_t B, double tc_lo, double tc_hi, uint64_t seed,
               uint32_t counter, void* stream) {
  if (B < 0) return fail(GWX_ESHAPE, "B=%lld", (long long)B);
  if (!(tc_hi >= tc_lo) || !isfinite(tc_lo) || !isfinite(tc_hi)) return fail(GWX_EINVAL, "tc range");
  if (B == 0) return GWX_OK;
  if (!theta_in || !theta_out) return fail(GWX_EINVAL, "NULL array");
  GWX_ALIGN8(theta_in);
  GWX_ALIGN8(theta_out);
  GWX_TRY(ensure_init());
  return launched(launch_retime(theta_in, theta_out, B, tc_lo, tc_hi, seed, counter, as_stream(stream)), "retime");
}

// ---- ResNet-1D pieces
namespace {
// The kernels run one grid row per sample with 32-bit index arithmetic within a sample.
int check_btc(int64_t B, int T, int C) {
  if (B < 1 || T < 1 || C < 1 || B > 65535 || (int64_t)T * C >= ((int64_t)1 << 31) ||
      B * (int64_t)T >= ((int64_t)1 << 31))
    return fail(GWX_ESHAPE, "B=%lld T=%d C=%d (need 1 <= B <= 65535, T C < 2^31, B T < 2^31)", (long long)B, T, C);
  return GWX_OK;
}

int check_rows(int T, int k, int s, int p, int K) {
  const int64_t To = ((int64_t)T + 2 * p - k) / s + 1;
  if (To * K >= ((int64_t)1 << 31)) return fail(GWX_ESHAPE, "T_out K = %lld (at most 2^31 - 1)", (long long)(To * K));
  return GWX_OK;
}
}  // namespace

int gwx_im2col(const void* x, int64_t B, int T, int C, int k, int s, int p, int K, void* cols, void* stream) {
  GWX_TRY(check_btc(B, T, C));
  if (C % 8 || K % 8 || K < k * C || k < 1 || s < 1 || p < 0 || T + 2 * p < k)
    return fail(GWX_ESHAPE, "im2col C=%d K=%d k=%d s=%d p=%d (C and K multiples of 8, K >= k C)", C, K, k, s, p);
  GWX_TRY(check_rows(T, k, s, p, K));
  if (!x || !cols) return fail(GWX_EINVAL, "NULL array");
  GWX_ALIGN16(x);
  GWX_ALIGN16(cols);
  GWX_TRY(ensure_init());
  return launched(launch_im2col(x, B, T, C, k, s, p, K, cols, as_stream(stream)), "im2col");
}

int gwx_im2col_cf(const float* y, int64_t B, int D, int N, int k, int s, int p, int K, void* cols, void* stream) {
  GWX_TRY(check_btc(B, N, D));
  if (K < k * D || k < 1 || s < 1 || p < 0 || N + 2 * p < k) return fail(GWX_ESHAPE, "im2col_cf shapes");
  GWX_TRY(check_rows(N, k, s, p, K));
  if (!y || !cols) return fail(GWX_EINVAL, "NULL array");
  GWX_TRY(ensure_init());
  return launched(launch_im2col_cf(y, B, D, N, k, s, p, K, cols, as_stream(stream)), "im2col_cf");
}

int gwx_col2im(const float* dcols, int64_t B, int T, int C, int k, int s, int p, int K, const float* addend, float* dx,
               void* stream) {
  GWX_TRY(check_btc(B, T, C));
  if (K < k * C || k < 1 || s < 1 || p < 0 || T + 2 * p < k) return fail(GWX_ESHAPE, "col2im shapes");
  GWX_TRY(check_rows(T, k, s, p, K));
  if (!dcols || !dx) return fail(GWX_EINVAL, "NULL array");
  GWX_TRY(ensure_init());
  return launched(launch_col2im(dcols, B, T, C, k, s, p, K, addend, dx, as_stream(stream)), "col2im");
}

int gwx_group_norm(const float* z, int64_t B, int T, int C, int G, const float* gamma, const float* beta,
                   const float* residual32, const void* residual16, int relu, void* out16, float* out32,
                   float* mean_rstd, void* stream) {
  GWX_TRY(check_btc(B, T, C));
  if (G < 1 || C % G) return fail(GWX_ESHAPE, "C=%d not a multiple of G=%d", C, G);
  if (!z || !gamma || !beta || !mean_rstd || (!out16 && !out32)) return fail(GWX_EINVAL, "NULL array");
  GWX_TRY(ensure_init());
  return launched(launch_group_norm(z, B, T, C, G, gamma, beta, residual32, residual16, relu ? 1 : 0, out16, out32,
                                    mean_rstd, as_stream(stream)),
                  "group_norm");
}

size_t gwx_group_norm_backward_scratch(int64_t B, int C, int G) {
  if (B < 1 || C < 1 || G < 1) return 0;
  return align_up(group_norm_backward_scratch(B, C, G));
}

int gwx_group_norm_backward(const float* dy, const float* z, int64_t B, int T, int C, int G, const float* mean_rstd,
                            const float* gamma, void* scratch, float* dz, float* dgamma, float* dbeta, void* stream) {
  GWX_TRY(check_btc(B, T, C));
  if (G < 1 || C % G) return fail(GWX_ESHAPE, "C=%d not a multiple of G=%d", C, G);
  if (!dy || !z || !mean_rstd || !gamma || !scratch || !dz || !dgamma || !dbeta) return fail(GWX_EINVAL, "NULL array");
  GWX_TRY(ensure_init());
  return launched(launch_group_norm_backward(dy, z, B, T, C, G, mean_rstd, gamma, scratch, dz, dgamma, dbeta,
                                             as_stream(stream)),
                  "group_norm_backward");
}

int gwx_relu_mask(const float* dy, const void* out, int64_t n, float* d, void* stream) {
  if (n < 0) return fail(GWX_ESHAPE, "n");
  if (n == 0) return GWX_OK;
  if (!dy || !out || !d) return fail(GWX_EINVAL, "NULL array");
  GWX_TRY(ensure_init());
  return launched(launch_relu_mask(dy, out, n, d, as_stream(stream)), "relu_mask");
}

int gwx_maxpool(const void* x, int64_t B, int T, int C, void* y, uint8_t* arg, void* stream) {
  GWX_TRY(check_btc(B, T, C));
  if (!x || !y || !arg) return fail(GWX_EINVAL, "NULL array");
  GWX_TRY(ensure_init());
  return launched(launch_maxpool(x, B, T, C, y, arg, as_stream(stream)), "maxpool");
}

int gwx_maxpool_backward(const float* dy, const uint8_t* arg, int64_t B, int T, int C, float* dx, void* stream) {
  GWX_TRY(check_btc(B, T, C));
  if (!dy || !arg || !dx) return fail(GWX_EINVAL, "NULL array");
  GWX_TRY(ensure_init());
  return launched(launch_maxpool_back(dy, arg, B, T, C, dx, as_stream(stream)), "maxpool_backward");
}

int gwx_mean_time(const void* x, int64_t B, int T, int C, void* m, void* stream) {
  GWX_TRY(check_btc(B, T, C));
  if (!x || !m) return fail(GWX_EINVAL, "NULL array");
  GWX_TRY(ensure_init());
  return launched(launch_mean_time(x, B, T, C, m, as_stream(stream)), "mean_time");
}

int gwx_mean_time_backward(const float* dm, int64_t B, int T, int C, float* dx, void* stream) {
  GWX_TRY(check_btc(B, T, C));
  if (!dm || !dx) return fail(GWX_EINVAL, "NULL array");
  GWX_TRY(ensure_init());
  return launched(launch_mean_time_back(dm, B, T, C, dx, as_stream(stream)), "mean_time_backward");
}

static int check_conv(int64_t B, int64_t T, int C, int O, int k) {
  if (B < 1 || T < 128 || T % 128 || C < 64 || C % 64 || O < 64 || O % 64 || k < 1 || k > 15 || k % 2 == 0 ||
      B * T > ((int64_t)1 << 26) || (int64_t)k * C > ((int64_t)1 << 20) || (int64_t)k * O > ((int64_t)1 << 20))
    return fail(GWX_ESHAPE, "conv1d sizes B=%lld T=%lld C=%d O=%d k=%d (T %% 128 == 0, C and O multiples of 64, "
                "k odd <= 15, B T <= 2^26)", (long long)B, (long long)T, C, O, k);
  return GWX_OK;
}

int gwx_conv1d_bf16(const void* x, int64_t B, int64_t T, int C, int k, const void* W, int O, const float* addend,
                    float* z, void* stream) {
  GWX_TRY(check_conv(B, T, C, O, k));
  if (!x || !W || !z) return fail(GWX_EINVAL, "NULL array");
  if ((((uintptr_t)x) | ((uintptr_t)W) | ((uintptr_t)z) | ((uintptr_t)addend)) & 15u)
    return fail(GWX_EINVAL, "x, W, z and addend must be 16-byte aligned");
  GWX_TRY(ensure_init());
  return launched(launch_conv_forward(x, B, T, C, k, W, O, addend, z, as_stream(stream)), "conv1d_bf16");
}

size_t gwx_conv1d_bf16_backward_workspace(int64_t B, int64_t T, int C, int O, int k) {
  if (B < 1 || T < 1 || C < 1 || O < 1 || k < 1) return 0;
  return conv_backward_ws(B, T, C, O, k);
}

int gwx_conv1d_bf16_backward(const float* dz, const void* x, const void* W, int64_t B, int64_t T, int C, int O, int k,
                             const float* addend, float* dx, float* dW, void* workspace, size_t workspace_bytes,
                             void* stream) {
  GWX_TRY(check_conv(B, T, C, O, k));
  if (!dz || !x || !W) return fail(GWX_EINVAL, "NULL array");
  if ((((uintptr_t)x) | ((uintptr_t)W) | ((uintptr_t)dx) | ((uintptr_t)dW) | ((uintptr_t)addend)) & 15u)
    return fail(GWX_EINVAL, "x, W, dx, dW and addend must be 16-byte aligned");
  if (((uintptr_t)dz) & 3u) return fail(GWX_EINVAL, "dz must be 4-byte aligned");
  GWX_TRY(check_ws(workspace, workspace_bytes, conv_backward_ws(B, T, C, O, k)));
  GWX_TRY(ensure_init());
  return launched(launch_conv_backward(dz, x, W, B, T, C, O, k, addend, dx, dW, workspace, as_stream(stream)),
                  "conv1d_bf16_backward");
}

size_t gwx_skymap_workspace(void) { return kAlign; }

int gwx_skymap(const double* theta, const double* weights, int64_t S, int nside, double* map, void* workspace,
               size_t workspace_bytes, void* stream) {
  if (nside < 1 || nside > 8192 || (nside & (nside - 1))) return fail(GWX_EINVAL, "nside=%d must be a power of two", nside);
  if (S < 0 || S > ((int64_t)1 << 40)) return fail(GWX_ESHAPE, "S=%lld", (long long)S);
  if (!map || (S > 0 && !theta)) return fail(GWX_EINVAL, "NULL array");
  GWX_ALIGN8(map);
  if (theta) GWX_ALIGN8(theta);
  if (weights) GWX_ALIGN8(weights);
  GWX_TRY(check_ws(workspace, workspace_bytes, gwx_skymap_workspace()));
  GWX_TRY(ensure_init());
  return launched(launch_skymap(theta, weights, S, nside, map, workspace, as_stream(stream)), "skymap");
}

size_t gwx_adamw_clip_workspace(void) { return align_up(adamw_clip_ws()); }

int gwx_adamw_clip(float* param, const float* grad, float* m, float* v, int64_t n, double lr, double beta1,
                   double beta2, double eps, double weight_decay, int64_t step, double clip, void* param_bf16,
                   void* workspace, size_t workspace_bytes, void* stream) {
  if (n < 0) return fail(GWX_ESHAPE, "n=%lld", (long long)n);
  if (step < 1 || !(beta1 >= 0.0 && beta1 < 1.0) || !(beta2 >= 0.0 && beta2 < 1.0) || !(eps > 0.0) || !(lr >= 0.0))
    return fail(GWX_EINVAL, "AdamW hyper-parameters (step counts from 1)");
  if (!(clip > 0.0) || !isfinite(clip)) return fail(GWX_EINVAL, "clip=%g must be positive", clip);
  if (n == 0) return GWX_OK;
  if (!param || !grad || !m || !v) return fail(GWX_EINVAL, "NULL array");
  GWX_TRY(check_ws(workspace, workspace_bytes, gwx_adamw_clip_workspace()));
  GWX_TRY(ensure_init());
  return launched(launch_adamw_clip(param, grad, m, v, n, lr, beta1, beta2, eps, weight_decay, step, clip, param_bf16,
                                    workspace, as_stream(stream)),
                  "adamw_clip");
}

int gwx_sample_proposal(const float* net_out, int ldn, const double* mean3, const double* scale3,
                        const gwx_prior* prior, const double* truth, int64_t E, const int64_t* event_offsets,
                        int64_t S, uint64_t seed, uint32_t counter, int flags, double* theta, double* log_ratio,
                        void* stream) {
  if (!prior) return fail(GWX_EINVAL, "prior is NULL");
  if (flags & ~GWX_PROPOSAL_FIX_ANGLES) return fail(GWX_EINVAL, "flags 0x%x", flags);
  if (E < 0 || S < 0 || (S > 0 && E == 0) || S > 0x7fffffffLL * 64) return fail(GWX_ESHAPE, "bad E or S");
  if (net_out && (ldn < 6 || !mean3 || !scale3)) return fail(GWX_EINVAL, "net_out needs ldn >= 6, mean and scale");
  if (net_out)
    for (int i = 0; i < 3; ++i)
      if (!(scale3[i] > 0.0) || !isfinite(mean3[i])) return fail(GWX_EINVAL, "bad mean or scale %d", i);
  if (S == 0) return GWX_OK;
  if (!truth || !event_offsets || !theta || !log_ratio) return fail(GWX_EINVAL, "NULL array");
  GWX_ALIGN8(truth);
  GWX_ALIGN8(event_offsets);
  GWX_ALIGN8(theta);
  GWX_ALIGN8(log_ratio);
  GWX_TRY(ensure_init());
  return launched(launch_proposal(net_out, ldn, mean3, scale3, *prior, truth, E, event_offsets, S, seed, counter,
                                  (flags & GWX_PROPOSAL_FIX_ANGLES) ? 1 : 0, theta, log_ratio, as_stream(stream)),
                  "sample_proposal");
}

int gwx_rfft(const float* x, int64_t R, int64_t N, float* X, void* stream) {
  GWX_TRY(check_window(N));
  if (R < 0 || R > 0x7fffffffLL) return fail(GWX_ESHAPE, "R=%lld", (long long)R);
  if (R == 0) return GWX_OK;
  if (!x || !X) return fail(GWX_EINVAL, "NULL array");
  GWX_ALIGN8(x);
  GWX_ALIGN8(X);
  GWX_TRY(ensure_init());
  return launched(launch_rfft_rows(x, R, N, reinterpret_cast<float2*>(X), as_stream(stream)), "rfft");
}

int gwx_irfft(const float* X, int64_t R, int64_t N, float* x, void* stream) {
  GWX_TRY(check_window(N));
  if (R < 0 || R > 0x7fffffffLL) return fail(GWX_ESHAPE, "R=%lld", (long long)R);
  if (R == 0) return GWX_OK;
  if (!x || !X) return fail(GWX_EINVAL, "NULL array");
  GWX_ALIGN8(x);
  GWX_ALIGN8(X);
  GWX_TRY(ensure_init());
  return launched(launch_irfft_rows(reinterpret_cast<const float2*>(X), R, N, x, as_stream(stream)), "irfft");
}

}  // extern "C"

// ---------------------------------------------------------------- conditional coupling flow
namespace {


int check_flow_shape(const gwx_flow_shape* sh) {
  if (!sh) return fail(GWX_EINVAL, "flow shape is NULL");
  const int64_t lim = (int64_t)65535 * 32;
  const int w[4] = {sh->features, sh->embed_hidden, sh->context, sh->hidden};
  for (int v : w)
    if (v < 8 || v % 8 != 0 || v > lim)
      return fail(GWX_ESHAPE, "flow widths F=%d H_e=%d C=%d H=%d must be multiples of 8 in [8, %lld]", sh->features,
                  sh->embed_hidden, sh->context, sh->hidden, (long long)lim);
  if (8 + (int64_t)sh->context > lim) return fail(GWX_ESHAPE, "context width %d", sh->context);
  if (sh->layers < 1 || sh->layers > 64) return fail(GWX_ESHAPE, "layers=%d outside [1, 64]", sh->layers);
  if (sh->group < 1) return fail(GWX_EINVAL, "group=%d", sh->group);
  if (sh->extra & ~(GWX_FLOW_CROSS | GWX_FLOW_LAG)) return fail(GWX_EINVAL, "extra=%d", sh->extra);
  return GWX_OK;
}

int check_std8(const double* mean8, const double* scale8) {
  if (!mean8 || !scale8) return fail(GWX_EINVAL, "mean and scale (host, 8 values each) are required");
  for (int i = 0; i < 8; ++i)
    if (!(scale8[i] > 0.0) || !isfinite(scale8[i]) || !isfinite(mean8[i]))
      return fail(GWX_EINVAL, "bad mean or scale %d", i);
  return GWX_OK;
}

int check_prior_box(const gwx_prior* p) {
  if (!p) return fail(GWX_EINVAL, "prior is NULL");
  if (!(p->m_lo > 0.0 && p->m_hi > p->m_lo && p->d_hi > p->d_lo && p->psi_hi > p->psi_lo && p->phi_hi > p->phi_lo))
    return fail(GWX_EINVAL, "prior ranges must be non-empty with m_lo > 0");
  // spins and merger time are drawn from their ranges (a point range, lo == hi, is allowed)
  if (!(isfinite(p->chi_lo) && isfinite(p->chi_hi) && p->chi_hi >= p->chi_lo && isfinite(p->tc_lo) &&
        isfinite(p->tc_hi) && p->tc_hi >= p->tc_lo))
    return fail(GWX_EINVAL, "spin and merger-time ranges must be finite with lo <= hi");
  return GWX_OK;
}

// Features of the flow's windows: band start and the number of groups must fit F.
int check_flow_windows(const gwx_flow_shape* sh, int D, int64_t N, double fs, double f_lo, int* k_lo) {
  GWX_TRY(check_window(N));
  if (D < 1 || D > GWX_MAX_DET) return fail(GWX_ESHAPE, "D=%d", D);
  if (!(fs > 0.0)) return fail(GWX_EINVAL, "fs must be positive");
  GWX_TRY(band_start(f_lo, fs / (double)N, N / 2, k_lo));
  if (sh->group > N / 2) return fail(GWX_EINVAL, "group %d", sh->group);
  const int64_t ng = (N / 2 - *k_lo) / sh->group;
  const int64_t need = (int64_t)D * ng * (1 + ((sh->extra & GWX_FLOW_CROSS) ? D - 1 : 0) +
                                           ((sh->extra & GWX_FLOW_LAG) ? 2 : 0));
  if (sh->features < need)
    return fail(GWX_ESHAPE, "F=%d is below the %lld feature columns (D x groups x %lld)", sh->features,
                (long long)need, (long long)(need / (D * ng > 0 ? D * ng : 1)));
  if ((sh->extra & GWX_FLOW_CROSS) && D < 2) return fail(GWX_ESHAPE, "cross-spectral features need two detectors or more");
  return GWX_OK;
}

int check_flow_params(const gwx_flow_shape* sh, const float* params, const void* params_bf16) {
  if (!params || !params_bf16) return fail(GWX_EINVAL, "params and params_bf16 are required");
  GWX_ALIGN16(params);
  GWX_ALIGN16(params_bf16);
  (void)sh;
  return GWX_OK;
}

}  // namespace

extern "C" {

int gwx_flow_layout(const gwx_flow_shape* shape, int64_t* n_params, int64_t* offsets) {
  GWX_TRY(check_flow_shape(shape));
  const int64_t n = flow_layout(*shape, offsets);
  if (n_params) *n_params = n;
  return GWX_OK;
}

int gwx_flow_targets(const double* theta, int64_t B, const double* mean8, const double* scale8, float* x,
                     void* stream) {
  if (B < 0 || B > ((int64_t)1 << 31)) return fail(GWX_ESHAPE, "B=%lld", (long long)B);
  GWX_TRY(check_std8(mean8, scale8));
  if (B == 0) return GWX_OK;
  if (!theta || !x) return fail(GWX_EINVAL, "NULL array");
  GWX_ALIGN8(theta);
  GWX_ALIGN16(x);
  GWX_TRY(ensure_init());
  return launched(launch_flow_targets(theta, B, mean8, scale8, x, as_stream(stream)), "flow_targets");
}

int gwx_flow_conditioner_input(int layer, const float* v, const void* ctx, int C, const int64_t* event_offsets,
                               int64_t E, int64_t row0, int64_t B, void* X, void* stream) {
  if (layer < 0) return fail(GWX_EINVAL, "layer %d", layer);
  if (C < 8 || C % 8 != 0) return fail(GWX_ESHAPE, "C=%d must be a positive multiple of 8", C);
  if (B < 0 || B > ((int64_t)1 << 31) || row0 < 0 || (event_offsets && E < 1)) return fail(GWX_ESHAPE, "bad B, row0 or E");
  if (B == 0) return GWX_OK;
  if (!v || !ctx || !X) return fail(GWX_EINVAL, "NULL array");
  GWX_ALIGN16(v);
  GWX_ALIGN16(ctx);
  GWX_ALIGN16(X);
  if (event_offsets) GWX_ALIGN8(event_offsets);
  GWX_TRY(ensure_init());
  return launched(launch_flow_input(layer, v, ctx, C, event_offsets, E, row0, B, X, as_stream(stream)),
                  "flow_conditioner_input");
}

int gwx_flow_coupling(int layer, int direction, const float* v_in, const float* o, int64_t B, float* v_out,
                      float* sum_s, int init, void* stream) {
  if (layer < 0 || (direction != 1 && direction != -1)) return fail(GWX_EINVAL, "layer %d direction %d", layer, direction);
  if (B < 0 || B > ((int64_t)1 << 31)) return fail(GWX_ESHAPE, "B=%lld", (long long)B);
  if (B == 0) return GWX_OK;
  if (!v_in || !o || !v_out || !sum_s) return fail(GWX_EINVAL, "NULL array");
  GWX_ALIGN16(v_in);
  GWX_ALIGN16(o);
  GWX_ALIGN16(v_out);
  GWX_TRY(ensure_init());
  return launched(launch_flow_coupling(layer, direction, v_in, o, B, v_out, sum_s, init ? 1 : 0, as_stream(stream)),
                  "flow_coupling");
}

int gwx_flow_nll(const float* z, const float* sum_s, int64_t B, float* loss_rows, double* loss_mean, float* grad,
                 void* stream) {
  if (B < 1 || B > ((int64_t)1 << 31)) return fail(GWX_ESHAPE, "B=%lld", (long long)B);
  if (!z || !sum_s || !loss_rows || !loss_mean || !grad) return fail(GWX_EINVAL, "NULL array");
  GWX_ALIGN16(z);
  GWX_ALIGN16(grad);
  GWX_ALIGN8(loss_mean);
  GWX_TRY(ensure_init());
  return launched(launch_flow_nll(z, sum_s, B, loss_rows, loss_mean, grad, as_stream(stream)), "flow_nll");
}

int gwx_flow_coupling_backward(int layer, const float* w, const float* o, const float* g, int64_t B,
                               float row_weight, float* d_o, float* g_u, void* stream) {
  if (layer < 0) return fail(GWX_EINVAL, "layer %d", layer);
  if (B < 0 || B > ((int64_t)1 << 31)) return fail(GWX_ESHAPE, "B=%lld", (long long)B);
  if (B == 0) return GWX_OK;
  if (!w || !o || !g || !d_o || !g_u) return fail(GWX_EINVAL, "NULL array");
  GWX_ALIGN16(w);
  GWX_ALIGN16(o);
  GWX_ALIGN16(g);
  GWX_ALIGN16(d_o);
  GWX_ALIGN16(g_u);
  GWX_TRY(ensure_init());
  return launched(launch_flow_coupling_backward(layer, w, o, g, B, row_weight, d_o, g_u, as_stream(stream)),
                  "flow_coupling_backward");
}

int gwx_flow_input_backward(int layer, const float* dX, int C, int64_t B, float* g_u, float* d_ctx, int init,
                            void* stream) {
  if (layer < 0) return fail(GWX_EINVAL, "layer %d", layer);
  if (C < 8 || C % 8 != 0) return fail(GWX_ESHAPE, "C=%d must be a positive multiple of 8", C);
  if (B < 0 || B > ((int64_t)1 << 31)) return fail(GWX_ESHAPE, "B=%lld", (long long)B);
  if (B == 0) return GWX_OK;
  if (!dX || !g_u || !d_ctx) return fail(GWX_EINVAL, "NULL array");
  GWX_TRY(ensure_init());
  return launched(launch_flow_input_backward(layer, dX, C, B, g_u, d_ctx, init ? 1 : 0, as_stream(stream)),
                  "flow_input_backward");
}

int gwx_flow_base(uint64_t seed, uint32_t counter, int64_t row0, int64_t n, float* z, void* stream) {
  if (n < 0 || row0 < 0 || row0 + n > ((int64_t)1 << 32)) return fail(GWX_ESHAPE, "draws outside [0, 2^32)");
  if (n == 0) return GWX_OK;
  if (!z) return fail(GWX_EINVAL, "NULL array");
  GWX_ALIGN16(z);
  GWX_TRY(ensure_init());
  return launched(launch_flow_base(seed, counter, row0, n, z, as_stream(stream)), "flow_base");
}

int gwx_flow_proposal(const float* x, const float* z, const float* sum_s, int64_t S, const double* mean8,
                      const double* scale8, const gwx_prior* prior, uint64_t seed, uint32_t counter, double* theta,
                      double* log_q, double* log_ratio, void* stream) {
  GWX_TRY(check_std8(mean8, scale8));
  GWX_TRY(check_prior_box(prior));
  if (S < 0 || S > ((int64_t)1 << 32)) return fail(GWX_ESHAPE, "bad S");
  if (S == 0) return GWX_OK;
  if (!x || !z || !sum_s || !theta || !log_q || !log_ratio) return fail(GWX_EINVAL, "NULL array");
  GWX_ALIGN16(x);
  GWX_ALIGN16(z);
  GWX_ALIGN8(theta);
  GWX_ALIGN8(log_q);
  GWX_ALIGN8(log_ratio);
  GWX_TRY(ensure_init());
  return launched(launch_flow_proposal(x, z, sum_s, S, 0, S, mean8, scale8, *prior, seed, counter, theta, log_q,
                                       log_ratio, as_stream(stream)),
                  "flow_proposal");
}

size_t gwx_flow_train_workspace(const gwx_flow_shape* shape, int64_t B, int D, int64_t N) {
  if (check_flow_shape(shape) != GWX_OK || B < 1 || D < 1 || N < 2) return 0;
  return align_up(flow_train_ws(*shape, B, D, N));
}

int gwx_flow_train_step(const gwx_flow_shape* shape, float* params, void* params_bf16, float* grads, float* m,
                        float* v, int64_t step, int64_t* step_counter, double lr, double beta1, double beta2, double eps,
                        double weight_decay, double clip, const double* mean8, const double* scale8, const float* y,
                        const double* theta, int64_t B, int D, int64_t N, double fs, double f_lo,
                        const void* ctx_in, float* d_ctx_out, double* loss_mean, void* workspace,
                        size_t workspace_bytes, void* stream) {
  GWX_TRY(check_flow_shape(shape));
  GWX_TRY(check_std8(mean8, scale8));
  int k_lo = 0;
  GWX_TRY(check_flow_windows(shape, D, N, fs, f_lo, &k_lo));
  const int64_t lim = (int64_t)65535 * 32;
  if (B < 8 || B % 8 != 0 || B > lim) return fail(GWX_ESHAPE, "B=%lld must be a multiple of 8 in [8, %lld]",
                                                  (long long)B, (long long)lim);
  if (step < 0) return fail(GWX_EINVAL, "step %lld", (long long)step);
  if (step >= 1 && (!(beta1 >= 0.0 && beta1 < 1.0) || !(beta2 >= 0.0 && beta2 < 1.0) || !(eps > 0.0) || !(lr >= 0.0)))
    return fail(GWX_EINVAL, "AdamW hyper-parameters");
  GWX_TRY(check_flow_params(shape, params, params_bf16));
  if (!grads || (!y && !ctx_in) || !theta || !loss_mean || (step >= 1 && (!m || !v)) || (ctx_in && !d_ctx_out))
    return fail(GWX_EINVAL, "NULL array");
  GWX_ALIGN16(grads);
  if (y) GWX_ALIGN8(y);
  if (ctx_in) GWX_ALIGN16(ctx_in);
  GWX_ALIGN8(theta);
  GWX_ALIGN8(loss_mean);
  GWX_TRY(check_ws(workspace, workspace_bytes, gwx_flow_train_workspace(shape, B, D, N)));
  GWX_TRY(ensure_init());
  if (!(clip >= 0.0) || !isfinite(clip)) return fail(GWX_EINVAL, "clip=%g", clip);
  if (step_counter) GWX_ALIGN8(step_counter);
  return launched(flow_train_step(*shape, params, params_bf16, grads, m, v, step, step_counter, lr, beta1, beta2, eps,
                                  weight_decay, clip, mean8, scale8, y, theta, B, D, N, k_lo, ctx_in, d_ctx_out,
                                  loss_mean, workspace, as_stream(stream)),
                  "flow_train_step");
}

size_t gwx_flow_log_prob_workspace(const gwx_flow_shape* shape, int64_t B, int D, int64_t N) {
  if (check_flow_shape(shape) != GWX_OK || B < 1 || D < 1 || N < 2) return 0;
  return align_up(flow_log_prob_ws(*shape, B, D, N));
}

int gwx_flow_log_prob(const gwx_flow_shape* shape, const float* params, const void* params_bf16,
                      const double* mean8, const double* scale8, const float* y, const double* theta, int64_t B,
                      int D, int64_t N, double fs, double f_lo, const void* ctx_in, double* log_q, void* workspace,
                      size_t workspace_bytes, void* stream) {
  GWX_TRY(check_flow_shape(shape));
  GWX_TRY(check_std8(mean8, scale8));
  int k_lo = 0;
  GWX_TRY(check_flow_windows(shape, D, N, fs, f_lo, &k_lo));
  if (B < 0 || B > ((int64_t)1 << 23)) return fail(GWX_ESHAPE, "B=%lld", (long long)B);
  if (B == 0) return GWX_OK;
  GWX_TRY(check_flow_params(shape, params, params_bf16));
  if ((!y && !ctx_in) || !theta || !log_q) return fail(GWX_EINVAL, "NULL array");
  if (y) GWX_ALIGN8(y);
  if (ctx_in) GWX_ALIGN16(ctx_in);
  GWX_ALIGN8(theta);
  GWX_ALIGN8(log_q);
  GWX_TRY(check_ws(workspace, workspace_bytes, gwx_flow_log_prob_workspace(shape, B, D, N)));
  GWX_TRY(ensure_init());
  return launched(flow_log_prob(*shape, params, params_bf16, mean8, scale8, y, theta, B, D, N, k_lo, ctx_in, log_q,
                                workspace,
                                as_stream(stream)),
                  "flow_log_prob");
}

size_t gwx_sample_posterior_workspace(const gwx_flow_shape* shape, int64_t E, int D, int64_t N, int64_t S) {
  if (check_flow_shape(shape) != GWX_OK || E < 1 || D < 1 || N < 2 || S < 1) return 0;
  return align_up(flow_sample_ws(*shape, E, D, N, S));
}

size_t gwx_flow_skymap_workspace(const gwx_flow_shape* shape, int D, int64_t N, int nside) {
  if (check_flow_shape(shape) != GWX_OK || D < 1 || N < 2 || nside < 1 || nside > 8192) return 0;
  return align_up(flow_skymap_ws(*shape, D, N, nside));
}

int gwx_flow_skymap(const gwx_flow_shape* shape, const float* params, const void* params_bf16, const double* mean8,
                    const double* scale8, const float* y, int D, int64_t N, double fs, double f_lo, const void* ctx_in,
                    const double* theta, const double* log_q, int64_t S, int nside, double* map, void* workspace,
                    size_t workspace_bytes, void* stream) {
  GWX_TRY(check_flow_shape(shape));
  GWX_TRY(check_std8(mean8, scale8));
  int k_lo = 0;
  GWX_TRY(check_flow_windows(shape, D, N, fs, f_lo, &k_lo));
  if (nside < 1 || nside > 8192 || (nside & (nside - 1)) != 0)
    return fail(GWX_ESHAPE, "nside=%d must be a power of two in [1, 8192]", nside);
  if (S < 1 || S > ((int64_t)1 << 32)) return fail(GWX_ESHAPE, "S=%lld draws (need at least one)", (long long)S);
  GWX_TRY(check_flow_params(shape, params, params_bf16));
  if ((!y && !ctx_in) || !theta || !log_q || !map) return fail(GWX_EINVAL, "NULL array");
  if (y) GWX_ALIGN8(y);
  if (ctx_in) GWX_ALIGN16(ctx_in);
  GWX_ALIGN8(theta);
  GWX_ALIGN8(log_q);
  GWX_ALIGN8(map);
  GWX_TRY(check_ws(workspace, workspace_bytes, gwx_flow_skymap_workspace(shape, D, N, nside)));
  GWX_TRY(ensure_init());
  return launched(flow_skymap(*shape, params, params_bf16, mean8, scale8, y, D, N, k_lo, ctx_in, theta, log_q, S,
                              nside, map, workspace, as_stream(stream)),
                  "flow_skymap");
}

int gwx_sample_posterior(const gwx_flow_shape* shape, const float* params, const void* params_bf16,
                         const double* mean8, const double* scale8, const gwx_prior* prior, const float* y,
                         int64_t E, int D, int64_t N, double fs, double f_lo, const void* ctx_in,
                         const int64_t* event_offsets, int64_t S, uint64_t seed,
                         uint32_t counter, double* theta, double* log_q, double* log_ratio, void* workspace,
                         size_t workspace_bytes, void* stream) {
  GWX_TRY(check_flow_shape(shape));
  GWX_TRY(check_std8(mean8, scale8));
  GWX_TRY(check_prior_box(prior));
  int k_lo = 0;
  GWX_TRY(check_flow_windows(shape, D, N, fs, f_lo, &k_lo));
  if (E < 0 || E > ((int64_t)1 << 23) || S < 0 || S > ((int64_t)1 << 32) || (S > 0 && E == 0))
    return fail(GWX_ESHAPE, "bad E or S");
  if (S == 0) return GWX_OK;
  GWX_TRY(check_flow_params(shape, params, params_bf16));
  if ((!y && !ctx_in) || !event_offsets || !theta || !log_q || !log_ratio) return fail(GWX_EINVAL, "NULL array");
  if (y) GWX_ALIGN8(y);
  if (ctx_in) GWX_ALIGN16(ctx_in);
  GWX_ALIGN8(event_offsets);
  GWX_ALIGN8(theta);
  GWX_ALIGN8(log_q);
  GWX_ALIGN8(log_ratio);
  GWX_TRY(check_ws(workspace, workspace_bytes, gwx_sample_posterior_workspace(shape, E, D, N, S)));
  GWX_TRY(ensure_init());
  return launched(flow_sample(*shape, params, params_bf16, mean8, scale8, *prior, y, E, D, N, k_lo, ctx_in,
                              event_offsets, S, seed, counter, theta, log_q, log_ratio, workspace, as_stream(stream)),
                  "sample_posterior");
}

}  // extern "C"
