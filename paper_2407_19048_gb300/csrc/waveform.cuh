// waveform.cuh -- TaylorF2 per-draw set-up (FP64) and per-bin evaluation (FP32 +
// double-float), shared by the waveform, fused-simulation and likelihood kernels.
//
// Model (Sec. 3.1; Buonanno et al. 2009 eq. 3.18 for the non-spinning phase,
// 1.5PN aligned-spin spin-orbit term 4 beta):
//   h(f) = A(f) e^{-i Psi(f)},  A(f) = sqrt(5/24) pi^{-2/3} Mc^{5/6} f^{-7/6} / D,
//   Psi(f) = -phic - pi/4 + 3/(128 eta v^5) sum_j (a_j + l_j ln v) v^j,  v = (pi M f)^{1/3}
// with the merger at the time origin.  On the grid f = k df, v = V k^{1/3} with
// V = (pi M df)^{1/3}, so Psi/(2 pi) is a short sum of per-draw coefficients
// times fixed powers of k (see DrawCoef).  The large terms (up to ~10^3 rad at
// 20 Hz for the lightest systems) are double-float products reduced modulo one
// turn before they are added, which keeps the phase error near 1e-6 rad while
// using only FP32 arithmetic per bin.  The linear phase 2 pi f (tc + dt) of the
// projection is exact: (tc + dt) df modulo one is held as a 64-bit fixed-point
// fraction and multiplied by the integer k.
#pragma once

#include "common.cuh"

namespace gwx {

constexpr double MTSUN_S = 4.925490947641267e-6;
constexpr double MPC_M = 3.085677581491367e22;
constexpr double C_MS = 299792458.0;
constexpr double EULER_GAMMA = 0.5772156649015329;
constexpr double PI_D = 3.141592653589793238462643383279502884;

__device__ __forceinline__ float2 split_df(double x) {
  float h = (float)x;
  return make_float2(h, (float)(x - (double)h));
}

__device__ __forceinline__ double th_at(const double* th, int64_t B, int64_t b, int p) { return th[(int64_t)p * B + b]; }

constexpr double SQRT_5_24_PI_M23 = 0.21278751013966343;   // sqrt(5/24) pi^(-2/3)
constexpr double LN4 = 1.3862943611198906;
constexpr double INV_6P15_PI = 0.021658244478713226;        // 1 / (6^1.5 pi)
constexpr double INV_C = 1.0 / C_MS;

// Per-call constants of the set-up, computed once on the host.
struct SetupConsts {
  double df;         // frequency resolution
  double ln_pi_df;   // ln(pi df)
  double amp_k;      // sqrt(5/24) pi^{-2/3} (pi df)^{-5/6} df^{-7/6} c / (1 Mpc): A(df) = amp_k V^{5/2} eta^{1/2} / D[Mpc]
  double isco_bins;  // 1 / (6^1.5 pi MTSUN_S df): floor(isco_bins / (m1 + m2)) is the last bin below f_isco
};

static inline SetupConsts make_setup_consts(double df) {
  return {df, log(PI_D * df), SQRT_5_24_PI_M23 * pow(PI_D * df, -5.0 / 6.0) * pow(df, -7.0 / 6.0) * (C_MS / MPC_M),
          INV_6P15_PI / (MTSUN_S * df)};
}

// Waveform part of the set-up: PN phase coefficients in turns, amplitude and cut-off.
// Written for the GPU's scarce FP64 throughput: constant ratios are folded at compile
// time, one logarithm serves both ln V and M^(5/6), and the remaining divisions are
// the few reciprocals that depend on the draw.
__device__ inline void draw_waveform_coef(const double* th, int64_t B, int64_t b, const SetupConsts& k, int64_t F,
                                          DrawCoef& c, double* amp64 = nullptr) {
  const double m1 = th_at(th, B, b, GWX_M1), m2 = th_at(th, B, b, GWX_M2);
  const double chi1 = th_at(th, B, b, GWX_CHI1), chi2 = th_at(th, B, b, GWX_CHI2);
  const double phic = th_at(th, B, b, GWX_PHIC);
  const double iota = th_at(th, B, b, GWX_THETAJN);
  const double mt = m1 + m2;
  const double inv_mt = 1.0 / mt;
  const double M = mt * MTSUN_S;
  const double eta = m1 * m2 * inv_mt * inv_mt;
  const double eta2 = eta * eta;
  const double delta = (m1 - m2) * inv_mt;
  const double chis = 0.5 * (chi1 + chi2), chia = 0.5 * (chi1 - chi2);
  const double pi = PI_D;
  const double a2 = 3715.0 / 756.0 + (55.0 / 9.0) * eta;
  const double a3 = -16.0 * pi + (113.0 / 3.0) * delta * chia + (113.0 / 3.0 - (76.0 / 3.0) * eta) * chis;
  const double a4 = 15293365.0 / 508032.0 + (27145.0 / 504.0) * eta + (3085.0 / 72.0) * eta2;
  const double a5 = pi * (38645.0 / 756.0 - (65.0 / 9.0) * eta);
  const double l5 = 3.0 * a5;
  constexpr double a6_0 = 11583231236531.0 / 4694215680.0 - 640.0 * (PI_D * PI_D) / 3.0 -
                          6848.0 * EULER_GAMMA / 21.0 - 6848.0 * LN4 / 21.0;
  constexpr double a6_1 = -15737765635.0 / 3048192.0 + 2255.0 * (PI_D * PI_D) / 12.0;
  const double a6 = a6_0 + a6_1 * eta + (76055.0 / 1728.0) * eta2 - (127825.0 / 1296.0) * eta2 * eta;
  const double l6 = -6848.0 / 21.0;
  const double a7 = pi * (77096675.0 / 254016.0 + (378515.0 / 1512.0) * eta - (74045.0 / 756.0) * eta2);
  const double lnV = (1.0 / 3.0) * (k.ln_pi_df + log(M));   // V = (pi M df)^(1/3)
  const double V = exp(lnV);
  const double Vi = 1.0 / V;
  const double pref = (3.0 / (256.0 * PI_D)) / eta;   // 3/(128 eta) in turns
  const double Vi2 = Vi * Vi, Vi3 = Vi2 * Vi, Vi5 = Vi3 * Vi2;
  c.c0 = split_df(pref * Vi5);
  c.c2 = split_df(pref * Vi3 * a2);
  c.c3 = split_df(pref * Vi2 * a3);
  c.c4 = (float)(pref * Vi * a4);
  c.d5 = split_df(pref * a5);   // pref l5 / 3
  c.c6 = (float)(pref * V * (a6 + l6 * lnV));
  c.d6 = (float)(pref * V * (l6 / 3.0));
  c.c7 = (float)(pref * V * V * a7);
  double cph = -(phic + 0.25 * PI_D) * (1.0 / (2.0 * PI_D)) + pref * (a5 + l5 * lnV);
  cph -= rint(cph);
  c.cph = (float)cph;
  // A(df) = sqrt(5/24) pi^{-2/3} Mc^{5/6} df^{-7/6} / D with Mc^{5/6} = M^{5/6} eta^{1/2}
  // = V^2 (V eta)^{1/2} (pi df)^{-5/6}; k.amp_k folds the constants and df^{-7/6}.
  const double amp = k.amp_k * (V * V) * sqrt(V * eta) / th_at(th, B, b, GWX_DIST);
  if (amp64) *amp64 = amp;
  c.amp = (float)amp;
  const double kc = floor(k.isco_bins * inv_mt);
  c.kcut = kc > (double)(F - 1) ? (int)(F - 1) : (int)kc;
  const double ci = cos(iota);
  c.qp = (float)(0.5 * (1.0 + ci * ci));
  c.qc_im = (float)ci;
  c.pad0 = c.pad1 = c.pad2 = 0;
}

// Projection part: scale * (F+ qp - i Fx qc) per detector as a complex double-float,
// and the per-detector linear phase (tc + dt_d) df modulo one as a 2^-64 fixed point,
// for a given merger time tc (the sky position and polarisation from theta).
__device__ inline void draw_detector_coef_at(const double* th, int64_t B, int64_t b, double df, const DetParams& dp,
                                             double gmst, double qp, double qc, double scale, double tc, DrawCoef& c) {
  const double psi = th_at(th, B, b, GWX_PSI);
  const double ra = th_at(th, B, b, GWX_RA), dec = th_at(th, B, b, GWX_DEC);
  double sd, cd, sp, cp, spsi, cpsi;
  sincos(dec, &sd, &cd);
  sincos(ra - gmst, &sp, &cp);
  sincos(psi, &spsi, &cpsi);
  const double n[3] = {cd * cp, cd * sp, sd};
  const double eth[3] = {sd * cp, sd * sp, -cd};
  const double eph[3] = {-sp, cp, 0.0};
  double X[3], Y[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    X[i] = cpsi * eth[i] + spsi * eph[i];
    Y[i] = spsi * eth[i] - cpsi * eph[i];
  }
  // unrolled over the detector slots so that DetParams stays in the parameter bank
#pragma unroll
  for (int d = 0; d < GWX_MAX_DET; ++d) {
    if (d >= dp.D) {
      c.g[d] = make_float4(0.f, 0.f, 0.f, 0.f);
      c.nu[d] = 0ull;
      continue;
    }
    const double* T = dp.tensor[d];
    double DX[3], DY[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      DX[i] = T[3 * i] * X[0] + T[3 * i + 1] * X[1] + T[3 * i + 2] * X[2];
      DY[i] = T[3 * i] * Y[0] + T[3 * i + 1] * Y[1] + T[3 * i + 2] * Y[2];
    }
    const double fp = X[0] * DX[0] + X[1] * DX[1] + X[2] * DX[2] - (Y[0] * DY[0] + Y[1] * DY[1] + Y[2] * DY[2]);
    const double fc = X[0] * DY[0] + X[1] * DY[1] + X[2] * DY[2] + (Y[0] * DX[0] + Y[1] * DX[1] + Y[2] * DX[2]);
    const double dt = -(dp.pos[d][0] * n[0] + dp.pos[d][1] * n[1] + dp.pos[d][2] * n[2]) * INV_C;
    // scale (F+ qp + Fx (-i qc))
    const float2 re = split_df(scale * fp * qp), im = split_df(-scale * fc * qc);
    c.g[d] = make_float4(re.x, re.y, im.x, im.y);
    double x = (tc + dt) * df;
    x -= floor(x);
    double fx = ldexp(x, 64);
    c.nu[d] = fx >= 18446744073709551615.0 ? 0ull : (unsigned long long)fx;
  }
}

// The same with the merger time of theta.
__device__ inline void draw_detector_coef(const double* th, int64_t B, int64_t b, double df, const DetParams& dp,
                                          double gmst, double qp, double qc, double scale, DrawCoef& c) {
  draw_detector_coef_at(th, B, b, df, dp, gmst, qp, qc, scale, th_at(th, B, b, GWX_TC), c);
}

// Fractional turns of k * nu * 2^-64, in [-1/2, 1/2).
__device__ __forceinline__ float lin_turns(unsigned long long nu, int k) {
  unsigned long long p = nu * (unsigned long long)(unsigned)k;
  return (float)(int)(p >> 32) * 0x1p-32f;
}

// Phase Psi(k)/(2 pi) reduced to [-1/2, 1/2] and the factor k^{-7/6}, for 1 <= k <= KMAX.
// 1/k enters as a double-float: the hardware reciprocal estimate rh is within a few
// ulp of 1/k, and the exact residual 1 - rh k (one FMA) times rh supplies the low part.
__device__ __forceinline__ float waveform_turns(const DrawCoef& c, int k, float& k76) {
  const float4 p = __ldg(&g_kp53[k]);
  const float4 q = __ldg(&g_kq[k]);
  const float kf = (float)k;
  float rh;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rh) : "f"(kf));
  const float rl = fmaf(-rh, kf, 1.0f) * rh;
  const float t = df_frac(df_mul(c.c0.x, c.c0.y, p.x, p.y)) + df_frac(df_mul(c.c2.x, c.c2.y, rh, rl)) +
                  df_frac(df_mul(c.c3.x, c.c3.y, p.z, p.w)) + df_frac(df_mul(c.d5.x, c.d5.y, q.y, q.z));
  const float k13 = kf * p.z;   // k^{1/3}
  const float k23 = kf * q.x;   // k^{2/3}
  const float small = fmaf(c.c4, q.x, fmaf(fmaf(c.d6, q.y, c.c6), k13, fmaf(c.c7, k23, c.cph)));
  float tt = t + small;
  tt -= rintf(tt);
  k76 = q.w;   // k^{-7/6}, correctly rounded from FP64
  return tt;
}

// e^{-2 pi i turns} for |turns| < 2^21.  turns = q/4 + r with q = rint(4 turns) and
// |r| <= 1/8 (r exact); sin(2 pi r) and cos(2 pi r) from their Taylor series through
// r^9 and r^10 (the first omitted terms are below 2e-9 and 1e-10 for |2 pi r| <= pi/4),
// with the leading coefficients 2 pi and -(2 pi)^2/2 as double-float pairs: rounding
// them to one float would scale the result by ~3e-8 and bias |H|^2 systematically.  The
// quarter turns q then rotate (cos, sin) by multiples of 90 degrees.
__device__ __forceinline__ float2 expm2pi(float turns) {
  const float q = rintf(4.0f * turns);
  const float r = fmaf(q, -0.25f, turns);
  const float z = r * r;
  // coefficients (-1)^k (2 pi)^n / n! of r^n; the n = 1 and n = 2 terms as hi + lo
  const float ps = fmaf(z, fmaf(z, fmaf(z, fmaf(z, 42.058693944897655f, -76.70585975306139f), 81.60524927607506f),
                                -41.34170224039976f),
                        -1.7484555314695172e-07f);
  const float sn = fmaf(r, 6.2831854820251465f, r * ps);
  const float pc = fmaf(z, fmaf(z, fmaf(z, fmaf(z, -26.4262567833744f, 60.24464137187666f), -85.45681720669373f),
                                64.9393940226683f),
                        -5.807431762150372e-07f);
  const float cs = fmaf(z, -19.739208221435547f, fmaf(z, pc, 1.0f));
  const int qi = (int)q;
  // angle 2 pi (q/4 + r): quadrant qi & 3 rotates (cos, sin) by qi * 90 degrees
  const float c1 = (qi & 1) ? sn : cs, s1 = (qi & 1) ? cs : sn;
  const float c = ((qi + 1) & 2) ? -c1 : c1;
  const float s = (qi & 2) ? -s1 : s1;
  return make_float2(c, -s);
}

}  // namespace gwx
