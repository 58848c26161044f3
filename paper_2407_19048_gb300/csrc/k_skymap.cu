// k_skymap.cu -- sky-localisation maps in the HEALPix format (the output of the paper's
// inference, Sec. 5): the importance-weighted histogram of posterior samples' (RA, dec)
// over the nested-scheme pixels of Gorski et al. 2005, normalised to unit sum.
#include "gwx_internal.h"

namespace gwx {

namespace {

constexpr double PI_S = 3.141592653589793238462643383279502884;

__device__ __forceinline__ uint32_t spread_bits(uint32_t v) {   // bit b of v -> bit 2 b
  v &= 0xFFFFu;
  v = (v | (v << 8)) & 0x00FF00FFu;
  v = (v | (v << 4)) & 0x0F0F0F0Fu;
  v = (v | (v << 2)) & 0x33333333u;
  v = (v | (v << 1)) & 0x55555555u;
  return v;
}

// Nested pixel of colatitude theta (through z = cos theta) and longitude phi.
__device__ __forceinline__ int64_t ang2pix_nest(int nside, double z, double phi) {
  const double za = fabs(z);
  double tt = fmod(phi, 2.0 * PI_S);
  if (tt < 0.0) tt += 2.0 * PI_S;
  tt /= 0.5 * PI_S;
  int face, ix, iy;
  if (za <= 2.0 / 3.0) {
    const double t1 = nside * (0.5 + tt), t2 = nside * z * 0.75;
    const int jp = (int)floor(t1 - t2), jm = (int)floor(t1 + t2);
    const int ifp = jp / nside, ifm = jm / nside;
    face = ifp == ifm ? (ifp | 4) : (ifp < ifm ? ifp : ifm + 8);
    ix = jm & (nside - 1);
    iy = nside - (jp & (nside - 1)) - 1;
  } else {
    const int ntt = min((int)tt, 3);
    const double tp = tt - ntt;
    const double s = nside * sqrt(3.0 * (1.0 - za));
    const int jp = min((int)(tp * s), nside - 1), jm = min((int)((1.0 - tp) * s), nside - 1);
    if (z > 0.0) {
      face = ntt;
      ix = nside - jm - 1;
      iy = nside - jp - 1;
    } else {
      face = ntt + 8;
      ix = jp;
      iy = jm;
    }
  }
  return (int64_t)face * nside * nside + (int64_t)(spread_bits((uint32_t)ix) | (spread_bits((uint32_t)iy) << 1));
}

__global__ void k_skymap(const double* __restrict__ theta, const double* __restrict__ w, int64_t S, int nside,
                         double* __restrict__ map, double* __restrict__ total) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double wi = 0.0;
  if (s < S) {
    wi = w ? w[s] : 1.0;
    if (wi > 0.0 && isfinite(wi)) {
      const double ra = theta[9 * S + s], dec = theta[10 * S + s];
      atomicAdd(&map[ang2pix_nest(nside, sin(dec), ra)], wi);   // z = cos(pi/2 - dec) = sin(dec)
    } else {
      wi = 0.0;
    }
  }
  for (int o = 16; o > 0; o >>= 1) wi += __shfl_down_sync(0xffffffffu, wi, o);
  if ((threadIdx.x & 31) == 0 && wi != 0.0) atomicAdd(total, wi);
}

__global__ void k_skymap_scale(double* __restrict__ map, int64_t npix, const double* __restrict__ total) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p < npix && *total > 0.0) map[p] /= *total;
}

}  // namespace

cudaError_t launch_skymap(const double* theta, const double* weights, int64_t S, int nside, double* map, void* ws,
                          cudaStream_t s) {
  const int64_t npix = 12 * (int64_t)nside * nside;
  double* total = reinterpret_cast<double*>(ws);
  cudaError_t e = cudaMemsetAsync(map, 0, (size_t)npix * sizeof(double), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(total, 0, sizeof(double), s);
  if (e != cudaSuccess) return e;
  if (S > 0) k_skymap<<<(unsigned)((S + 255) / 256), 256, 0, s>>>(theta, weights, S, nside, map, total);
  k_skymap_scale<<<(unsigned)((npix + 255) / 256), 256, 0, s>>>(map, npix, total);
  return cudaGetLastError();
}

}  // namespace gwx
