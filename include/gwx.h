/*
 * gwx.h -- C ABI of libgwx: on-the-fly simulation and pre-processing of
 * compact-binary gravitational-wave training data on one NVIDIA GB300 (sm_103a).
 *
 * The paper (Sec. 3, simulation on accelerated hardware) generates every
 * training batch on the GPU: prior draws (Table 1), frequency-domain waveforms
 * (Sec. 3.1), projection onto the detectors, injection into background
 * windows cropped from a device-resident chunk, a power spectrum fitted to the
 * chunk, and whitening (Sec. 3.2).  Its parameter-estimation comparison uses
 * the standard Gaussian-noise likelihood (Sec. 6, Fig. 5 caption).  Each of
 * those steps is one entry point below, plus one fused entry point that runs
 * the whole per-batch pass.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Return value: GWX_OK (0) or a negative GWX_E* status.  On failure
 *   gwx_last_error() returns a message for the calling thread.  Arguments are
 *   validated before anything is launched; a failed validation launches nothing.
 * - Array arguments are DEVICE pointers owned by the caller unless a comment
 *   says "host".  The library never frees, keeps or reallocates them.
 * - Arrays are C-contiguous.  "complex" arrays are interleaved float pairs
 *   (re, im): a [B][F] complex array holds 2*B*F floats.
 * - Every array pointer must be 8-byte aligned (cudaMalloc and PyTorch
 *   allocations are), except the background strain `noise` of gwx_inject and
 *   of the simulate calls, which may start at any float; a misaligned pointer
 *   returns GWX_EINVAL.
 * - Every call is asynchronous on `stream` (a cudaStream_t, NULL = legacy
 *   default stream) and performs no device allocation and no host
 *   synchronisation.  Calls that need scratch memory take a caller-owned
 *   device workspace and its size; the matching *_workspace() query returns
 *   the required size in bytes.  A workspace may be reused by later calls on
 *   the same stream; calls that overlap in time on the GPU must not share one.
 * - gwx_init() prepares per-device constant tables (FFT twiddles, powers of
 *   the bin index).  Every entry point calls it implicitly for the current
 *   device on first use; because that set-up copies to device memory
 *   synchronously, the first call on a device must not happen inside CUDA
 *   stream capture (call gwx_init() beforehand).
 * - Frequency grid of a window of N samples at rate fs: f_k = k df,
 *   df = fs / N, k = 0 .. N/2 (F = N/2 + 1 bins).  Supported window lengths
 *   are powers of two 256 <= N <= 16384; Welch segment lengths are powers of
 *   two 16 <= seg_len <= 16384; background lengths are powers of two
 *   1024 <= L <= 2^24.  Up to GWX_MAX_DET detectors.
 */
#ifndef GWX_H
#define GWX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define GWX_OK            0
#define GWX_EINVAL       -1   /* bad pointer or scalar argument            */
#define GWX_ESHAPE       -2   /* unsupported or inconsistent sizes         */
#define GWX_ECUDA        -3   /* a CUDA runtime call failed                */
#define GWX_ENOMEM       -4   /* workspace smaller than *_workspace()      */
#define GWX_ETIMEOUT     -5   /* a bounded device wait expired             */
#define GWX_EUNSUPPORTED -6   /* valid request this build does not offer   */

/* ---- waveform models ---------------------------------------------------- */
#define GWX_TAYLORF2    0     /* TaylorF2 3.5PN inspiral (Sec. 3.1)         */
#define GWX_IMRPHENOMD  1     /* IMRPhenomD (Sec. 3.1): returns GWX_EUNSUPPORTED */

/* ---- detectors ------------------------------------------------------- */
#define GWX_H1 0              /* LIGO Hanford                               */
#define GWX_L1 1              /* LIGO Livingston                            */
#define GWX_V1 2              /* Virgo                                      */
#define GWX_MAX_DET 4

/* ---- parameter layout: theta is double[GWX_NPARAM][B] (row p = parameter p) */
enum {
  GWX_M1 = 0,      /* primary mass, detector frame [M_sun]                  */
  GWX_M2,          /* secondary mass [M_sun]                                */
  GWX_CHI1,        /* aligned spin of body 1                                */
  GWX_CHI2,        /* aligned spin of body 2                                */
  GWX_DIST,        /* luminosity distance [Mpc]                             */
  GWX_TC,          /* geocentre merger time from the window start [s]       */
  GWX_PHIC,        /* coalescence phase [rad]                               */
  GWX_THETAJN,     /* inclination theta_JN [rad]                            */
  GWX_PSI,         /* polarisation angle [rad]                              */
  GWX_RA,          /* right ascension [rad]                                 */
  GWX_DEC,         /* declination [rad]                                     */
  GWX_NPARAM
};

/* Prior box for gwx_sample_prior / gwx_simulate_batch (Table 1 shapes for the
 * angles; uniform ranges for masses, spins, distance, merger time, phase and
 * polarisation). */
typedef struct gwx_prior {
  double m_lo, m_hi;       /* m1, m2 ~ U[m_lo, m_hi]                          */
  double chi_lo, chi_hi;   /* chi1, chi2 ~ U[chi_lo, chi_hi]                  */
  double d_lo, d_hi;       /* distance ~ U[d_lo, d_hi] Mpc                    */
  double tc_lo, tc_hi;     /* tc ~ U[tc_lo, tc_hi] s                          */
  double phi_lo, phi_hi;   /* phic ~ U[phi_lo, phi_hi]                        */
  double psi_lo, psi_hi;   /* psi ~ U[psi_lo, psi_hi]                         */
} gwx_prior;

/* ---- library ---------------------------------------------------------- */
int         gwx_version(void);                  /* 10000*major + 100*minor + patch */
const char* gwx_status_string(int status);      /* static string                  */
const char* gwx_last_error(void);               /* thread-local message           */
int         gwx_init(void);                     /* tables for the current device  */

/* Host query: detector tensor D (row-major 3x3, D = (x x^T - y y^T)/2 from the
 * arm unit vectors) and vertex position [m] (Earth-fixed, WGS-84) of detector
 * `det`.  Both outputs are HOST arrays.  Pure host code, no CUDA call. */
int gwx_detector_geometry(int det, double* tensor9, double* position3);

/* ---- A1: prior draws --------------------------------------------------
 * Sec. 3.2 (each batch draws its parameters from the prior); Table 1 shapes.
 * Draw b uses Philox4x32-10 (Salmon et al., SC'11) with counter
 * (b, j, 1, step), key (seed low word, seed high word), j = 0..5.  Block j
 * yields uniforms u_{2j}, u_{2j+1} from word pairs (0,1), (2,3) as
 * u = (x + 1/2) 2^-52, x the top 52 bits of the pair; block 5 words (0,1) give
 * u_10 and word 2 gives the crop offset floor(w (L-N+1) / 2^32).  Transforms:
 * m1,m2,chi1,chi2,distance,tc,phic,psi linear in u_0..u_6,u_8;
 * theta_jn = acos(1 - 2u_7), ra = 2 pi u_9, dec = asin(2 u_10 - 1).
 *   prior   HOST pointer to the prior box.
 *   theta   out, double[GWX_NPARAM][B].     offsets  out, int64[B] in [0, L-N].
 * B = 0 is valid and launches nothing. */
int gwx_sample_prior(const gwx_prior* prior, uint64_t seed, uint32_t step,
                     int64_t B, int64_t L, int64_t N,
                     double* theta, int64_t* offsets, void* stream);

/* ---- A2: waveforms ------------------------------------------------------
 * Sec. 3.1: TaylorF2 3.5PN inspiral.  h(f) = A f^-7/6 exp(-i Psi(f)) with the
 * non-spinning phase coefficients of Buonanno et al. 2009 (eq. 3.18) plus the
 * 1.5PN aligned-spin spin-orbit term, leading-order amplitude, merger at the
 * time origin (tc is applied by gwx_project); h_plus = A (1+cos^2 i)/2 e^{-i Psi},
 * h_cross = -i A cos i e^{-i Psi}.  Bins k with ceil(f_lo/df) <= k <=
 * floor(f_isco/df), f_isco = 1/(6^1.5 pi M), are non-zero; all others are zero.
 *   theta  in, double[GWX_NPARAM][B] (masses, spins, distance, phic, theta_jn used).
 *   hp, hc out, complex[B][F] (strain per Hz).
 * approximant GWX_IMRPHENOMD returns GWX_EUNSUPPORTED. */
int gwx_generate_waveforms(int approximant, const double* theta, int64_t B,
                           double f_lo, double df, int64_t F,
                           float* hp, float* hc, void* stream);

/* ---- A3: projection and time shift -------------------------------------
 * Sec. 6: signal projection onto the detectors on the fly on the GPU.
 * h_det[b][d][k] = (F+_d hp[b][k] + Fx_d hc[b][k]) exp(-2 pi i f_k (tc_b + dt_d)),
 * F+ = X.D.X - Y.D.Y, Fx = X.D.Y + Y.D.X with the polarisation basis
 * X = cos(psi) e_theta + sin(psi) e_phi, Y = sin(psi) e_theta - cos(psi) e_phi of
 * the source direction (theta = pi/2 - dec, phi = ra - gmst), and
 * dt_d = -(r_d . n)/c.
 *   det_ids HOST int32[D] of GWX_H1/L1/V1.  h_det out, complex[B][D][F]. */
int gwx_project(const float* hp, const float* hc, const double* theta, int64_t B,
                const int32_t* det_ids, int D, double gmst, double df, int64_t F,
                float* h_det, void* stream);

/* ---- A4: coloured Gaussian background ------------------------------------
 * Synthetic stand-in for the paper's real background chunk (Sec. 3.2).
 * Per detector d: X_0 = 0, X_k = sqrt(L fs S(f_k)/4)(g_re + i g_im) for
 * 0 < k < L/2, X_{L/2} = sqrt(L fs S/2) g_re, noise[d] = irfft(X) (1/L
 * normalisation), with S(f) the analytic aLIGO fit evaluated at max(f, f_lo).
 * g from Box-Muller on Philox counter (k/2, d, 2, step): bin 2j takes words
 * (0,1), bin 2j+1 words (2,3), u = ((w >> 8) + 1/2) 2^-24.
 *   noise out, float[D][L].  L a power of two, 1024 <= L <= 2^24. */
size_t gwx_colored_noise_workspace(int D, int64_t L);
int gwx_colored_noise(uint64_t seed, uint32_t step, int D, int64_t L, double fs, double f_lo,
                      float* noise, void* workspace, size_t workspace_bytes, void* stream);

/* ---- A5: Welch PSD --------------------------------------------------------
 * Sec. 3.2 (the PSD is estimated from the background chunk).  One-sided
 * density, periodic Hann window, mean of K = (L - seg_len)/stride + 1
 * periodograms, no detrending: P_k = c_k/(fs sum w^2) (1/K) sum_s |rfft(w x_s)_k|^2,
 * c_k = 1 at DC and Nyquist, 2 elsewhere.  FP32 FFTs, FP64 squares and sums.
 *   x in float[D][L].  psd out, double[D][seg_len/2+1]. */
size_t gwx_welch_psd_workspace(int D, int64_t L, int64_t seg_len, int64_t stride);
int gwx_welch_psd(const float* x, int D, int64_t L, double fs, int64_t seg_len, int64_t stride,
                  double* psd, void* workspace, size_t workspace_bytes, void* stream);

/* ---- A6: crop and inject ---------------------------------------------------
 * Sec. 3.2: N background windows are cropped from the chunk and the signals are
 * injected.  d[b][dd] = noise[dd][off_b : off_b + N] + irfft(fs h_det[b][dd])
 * (circular window; the crop offset is shared by the detectors of a draw).
 *   noise in float[D][L]; offsets in int64[B], 0 <= off <= L-N;
 *   h_det in complex[B][D][N/2+1]; d out float[B][D][N]. */
int gwx_inject(const float* noise, int D, int64_t L, const int64_t* offsets,
               const float* h_det, int64_t B, int64_t N, double fs,
               float* d, void* stream);

/* ---- A7: whitening -----------------------------------------------------------
 * Sec. 3.2 (the batch is whitened with the estimated PSD).
 * y = irfft(rfft(d) M_k / sqrt(S~_k fs/2)), M_k = 1 for ceil(f_lo/df) <= k < N/2,
 * S~ = psd (grid fs/seg_len) linearly interpolated to f_k.
 *   d in float[B][D][N]; psd in double[D][seg_len/2+1]; y out float[B][D][N]
 *   (y may alias d). */
/* Definition B injection (the padded-grid waveform): with h_td [B][D][N_pad] the
 * inverse transforms (gwx_irfft, 1/N_pad normalisation) of waveforms generated and
 * projected on the grid of a padded segment, f_k = k fs / N_pad (gwx_generate_waveforms,
 * gwx_project with df = fs / N_pad):
 *   d[b][dd][i] = noise[dd][offsets[b] + i] + fs h_td[b][dd][i],  i < N.
 * On the circular padded segment the inspiral before the window start wraps to the far
 * end, outside the first N samples, when N_pad / fs >= T + tau - tc (tau the signal's
 * duration from f_lo); N_pad = N reproduces gwx_inject.  N and N_pad powers of two in
 * [256, 16384], N <= N_pad; offsets in [0, L - N] (not checked: device data). */
int gwx_inject_padded(const float* noise, int D, int64_t L, const int64_t* offsets, const float* h_td, int64_t B,
                      int64_t N, int64_t N_pad, double fs, float* d, void* stream);
size_t gwx_whiten_workspace(int D, int64_t N);
int gwx_whiten(const float* d, const double* psd, int64_t seg_len, double fs, double f_lo,
               int64_t B, int D, int64_t N, float* y,
               void* workspace, size_t workspace_bytes, void* stream);

/* Inverse of gwx_whiten on the band, for checks: d = irfft(rfft(y) M_k sqrt(S~_k fs/2)),
 * so unwhiten(whiten(x)) is x restricted to the band (bins ceil(f_lo/df) <= k < N/2).
 * Arguments, layouts and workspace as gwx_whiten (y in, d out; d may alias y). */
int gwx_unwhiten(const float* y, const double* psd, int64_t seg_len, double fs, double f_lo,
                 int64_t B, int D, int64_t N, float* d,
                 void* workspace, size_t workspace_bytes, void* stream);

/* ---- whitening without caller scratch -------------------------------------------
 * Same result as gwx_whiten, for callers that cannot allocate device memory and
 * so cannot pass a workspace: for example a plug-in whose host application owns
 * every device allocation, a serving loop that must run inside a fixed,
 * pre-reserved memory budget with no allocation or pool growth, or a binding that
 * can only pass its data pointers.  The paper has no counterpart to this entry
 * point; it exists for those callers only.
 *
 * The whitening filter is kept in a file-scope device array of the library that
 * holds at most GWX_MAX_DET x 8193 floats (128 KiB): the largest filter that
 * gwx_whiten's own limits allow (D <= GWX_MAX_DET, N a power of two <= 16384), so
 * a request beyond it fails those checks with GWX_ESHAPE.  Every GPU that loads the
 * library holds that array until the process exits.  The call allocates nothing.
 * The first call on a device looks up the array's device address on that device
 * (and prepares the library's tables as gwx_init does), so that first call should
 * happen before any stream capture.  All calls share the one array, and each call
 * overwrites it completely before reading it: calls that overlap in time on the
 * GPU (different streams, or different host threads) race on it and must be
 * serialised by the caller.  Arguments, checks, statuses and messages as gwx_whiten
 * (without the workspace); the output is bit-identical to gwx_whiten's. */
int gwx_whiten_static(const float* d, const double* psd, int64_t seg_len, double fs, double f_lo,
                      int64_t B, int D, int64_t N, float* y, void* stream);

/* ---- launch shapes of the fused pass ------------------------------------------------
 * gwx_simulate_prepared can run its fused kernel in several launch shapes that do the
 * same arithmetic and give the same output bit for bit: bit 0 of a shape selects
 * Stockham passes that alternate between two shared-memory window buffers (one block
 * barrier per pass, twice the shared memory) instead of passes in place in one (two
 * barriers per pass); bits 1-2 the resident blocks per SM (0: as many as fit, else 1..3,
 * capped at what fits); bit 3 passes in place with the next window's background crop and
 * the next detector's whitening filter copied into shared memory by bulk asynchronous
 * copies one window ahead (used when noise and the workspace are 16-byte aligned and
 * L % 4 == 0, else the shape falls back to bits 0-2; overrides bit 0).  A staged copy that
 * never completes makes the block stop after a bounded wait and is reported by
 * gwx_device_status.  Which is fastest depends on the window length and the number
 * of detectors (e.g. through how much L1 the larger shared-memory carve-out leaves), so:
 * gwx_simulate_autotune builds the whitening filter from psd into the workspace, then
 *   times each candidate shape of the fused pass on the caller's batch (its per-draw
 *   coefficients already in the workspace from gwx_prepare_batch or gwx_prepare_theta;
 *   y is overwritten with the batch) and records the fastest for (N, D), process-wide;
 *   *shape_out (optional) receives it.  It synchronises with the stream.  Arguments as
 *   gwx_simulate_prepared; B >= 1.
 * gwx_simulate_shape: shape >= 0 records that shape for (N, D), -1 forgets the record
 *   (back to the default: staged for N >= 8192, else in place), -2 only asks;
 *   returns the shape gwx_simulate_prepared now uses for (N, D), or a negative status. */
int gwx_simulate_autotune(const float* noise, int64_t L, const double* psd, int64_t seg_len, double fs,
                          double f_lo, int D, int64_t B, int64_t N, const int64_t* offsets, float* y,
                          void* workspace, size_t workspace_bytes, int* shape_out, void* stream);
int gwx_simulate_shape(int64_t N, int D, int shape);

/* ---- A1-A3, A6, A7 fused: one whitened batch --------------------------------
 * The whole per-batch pass of Sec. 3.2 in one call: prior draws (as
 * gwx_sample_prior with `seed`, `step`), TaylorF2 waveforms, projection and
 * shift, crop + injection into `noise`, whitening with `psd`.  Injection is
 * linear, so each window is transformed once: y = irfft((rfft(crop) + fs h_det) W).
 * Results equal gwx_whiten(gwx_inject(...)) up to rounding.
 *   noise in float[D][L]; psd in double[D][seg_len/2+1];
 *   y out float[B][D][N]; theta out double[GWX_NPARAM][B]; offsets out int64[B]. */
size_t gwx_simulate_batch_workspace(int D, int64_t B, int64_t N);
int gwx_simulate_batch(const gwx_prior* prior, uint64_t seed, uint32_t step,
                       const float* noise, int64_t L, const double* psd, int64_t seg_len,
                       double fs, double f_lo, const int32_t* det_ids, int D, double gmst,
                       int64_t B, int64_t N, float* y, double* theta, int64_t* offsets,
                       void* workspace, size_t workspace_bytes, void* stream);

/* The same pass in two calls, so that the prior draws and the FP64 per-draw set-up
 * (which leave most of the GPU idle) can run on a second stream while the background
 * and its PSD are produced: gwx_prepare_batch writes theta, offsets and the per-draw
 * coefficients into the workspace; gwx_simulate_prepared reads them from the same
 * workspace (sized by gwx_simulate_batch_workspace) and writes y.  The caller orders
 * the two calls (same stream, or an event); gwx_simulate_batch is exactly
 * gwx_prepare_batch followed by gwx_simulate_prepared on one stream. */
int gwx_prepare_batch(const gwx_prior* prior, uint64_t seed, uint32_t step, int64_t L, int64_t N,
                      double fs, double f_lo, const int32_t* det_ids, int D, double gmst, int64_t B,
                      double* theta, int64_t* offsets, void* workspace, size_t workspace_bytes, void* stream);
/* flags GWX_SIM_FILTERS_READY: the whitening filter this call would compute from psd is
 * already in the workspace (an earlier gwx_simulate_prepared or gwx_simulate_batch on the
 * same workspace with the same psd, seg_len, fs, f_lo, D and N), so it is not rebuilt. */
#define GWX_SIM_FILTERS_READY 1
int gwx_simulate_prepared(const float* noise, int64_t L, const double* psd, int64_t seg_len,
                          double fs, double f_lo, int D, int64_t B, int64_t N, const int64_t* offsets,
                          float* y, int flags, void* workspace, size_t workspace_bytes, void* stream);

/* ---- A8: log-likelihood -------------------------------------------------------
 * Sec. 6 (Fig. 5 caption): the usual Gaussian-noise GW likelihood.  For sample s of event e
 * (event_offsets[e] <= s < event_offsets[e+1]):
 *   ln L_s = -(1/N) sum_d sum_{ceil(f_lo/df) <= k < N/2} |Y_e,d,k - fs h_d(theta_s, f_k) W_d,k|^2,
 * Y = rfft(y_data) of the whitened data, W = 1/sqrt(S~ fs/2), h_d the TaylorF2
 * projection of theta_s.  Equal to -<d-h, d-h>/2 with the noise-weighted inner
 * product.  FP32 products, FP64 sums.
 *   y_data in float[E][D][N]; theta in double[GWX_NPARAM][S];
 *   event_offsets in int64[E+1] (device, ragged, event_offsets[E] == S);
 *   lnl out double[S]. */
size_t gwx_log_likelihood_workspace(int64_t E, int D, int64_t N, int64_t S);
int gwx_log_likelihood(int approximant, const float* y_data, int64_t E, int D, int64_t N,
                       const double* psd, int64_t seg_len, double fs, double f_lo,
                       const int32_t* det_ids, double gmst,
                       const double* theta, const int64_t* event_offsets, int64_t S,
                       double* lnl, void* workspace, size_t workspace_bytes, void* stream);

/* ---- A8 with the merger time integrated out ------------------------------------------
 * Sec. 5 leaves the coalescence time out of the estimated parameters (it is marginalised
 * over), so the likelihood that judges the estimator's samples is the marginal over a
 * uniform merger time in the window [tc_lo, tc_lo + n_tc / fs):
 *   ln L_s = ln( (1/J) sum_{j<J} exp lnL(theta_s with tc = tc_lo + j / (u fs)) ),  J = u n_tc,
 * lnL as gwx_log_likelihood (its sum over the grid is the rectangle rule for the
 * normalised integral, on a grid u = oversample times finer than the sampling interval).
 * The tc row of theta is not read.  Per sample: the template at tc_lo, the band products
 * c_k = (2/N) sum_d Y_d,k conj(fs h_d,k W_d,k), and u inverse real FFTs of N points of
 * c_k e^{2 pi i k r/(N u)}, r < u, whose first n_tc outputs are the grid's ln L up to the
 * data and template norms; FP32 products and transforms, FP64 norms and final sums.
 *   tc_lo finite; 1 <= n_tc <= N; oversample a power of two in [1, 64]; everything else,
 *   the layouts and the workspace (gwx_log_likelihood_workspace) as gwx_log_likelihood. */
int gwx_log_likelihood_tmarg(int approximant, const float* y_data, int64_t E, int D, int64_t N,
                             const double* psd, int64_t seg_len, double fs, double f_lo,
                             const int32_t* det_ids, double gmst, double tc_lo, int64_t n_tc, int oversample,
                             const double* theta, const int64_t* event_offsets, int64_t S,
                             double* lnl, void* workspace, size_t workspace_bytes, void* stream);

/* ---- importance weights of scored samples ------------------------------------
 * Samples theta_s ~ q of event e, scored by gwx_log_likelihood, become posterior
 * samples by importance sampling with the standard GW likelihood (Sec. 6):
 *   ln w_s = lnl_s + log_ratio_s   (log_ratio = ln prior - ln q; NULL = zeros, q = prior),
 *   weights_s = w_s / sum_{s in e} w_s,
 *   ess_e = (sum w)^2 / sum w^2 (Kish),  efficiency_e = ess_e / S_e,
 *   ln_evidence_e = ln((1/S_e) sum w_s).
 * An event without samples, or whose every ln w is -inf, gets ess = efficiency = 0,
 * ln_evidence = -inf and zero weights.  exp is evaluated in FP32 on the FP64 value
 * ln w - max split into two floats (relative error ~2e-7); sums are FP64.
 *   lnl, log_ratio in double[S]; event_offsets int64[E+1] (device, ragged; entries are
 *   clamped to [0, S]); weights out double[S]; ess, efficiency, ln_evidence out
 *   double[E]; any output may be NULL.  Workspace: gwx_importance_weights_workspace(E). */
size_t gwx_importance_weights_workspace(int64_t E);
int gwx_importance_weights(const double* lnl, const double* log_ratio, const int64_t* event_offsets,
                           int64_t E, int64_t S, double* weights, double* ess, double* efficiency,
                           double* ln_evidence, void* workspace, size_t workspace_bytes, void* stream);

/* ---- debugging aids ------------------------------------------------------------------
 * The debug build of the library (libgwx_debug.so: the same sources compiled with
 * GWX_DEBUG_CHECKS; build.build(debug=True)) checks the indices of the global loads and
 * stores of the hot kernels (the fused simulation pass, both likelihood kernels): an
 * index outside its array is not accessed (a load gives zero) and the first such event
 * is recorded instead of faulting.  The paper has no counterpart; these are for testing.
 * gwx_debug_build: 1 in the debug build, 0 otherwise.
 * gwx_debug_status: *first_bad = (site << 48) | 2^47 | index of the first recorded
 *   out-of-range access since the last call (then cleared), 0 if none (always 0 in the
 *   normal build); returns GWX_ESHAPE with the site and index in the message when there
 *   was one.  Synchronises the device (not allowed inside stream capture).
 * gwx_debug_guard / gwx_debug_check_guard: write a fixed byte pattern into the
 *   guard_bytes that follow the first nbytes of a caller allocation (e.g. a workspace
 *   allocated nbytes + guard_bytes large), and check later that no call wrote into them
 *   (*intact = 1) or that one did (*intact = 0); the check synchronises the device
 *   first (not allowed inside stream capture). */
int gwx_debug_build(void);
int gwx_debug_status(uint64_t* first_bad);
int gwx_debug_guard(void* workspace, size_t nbytes, size_t guard_bytes, void* stream);
int gwx_debug_check_guard(const void* workspace, size_t nbytes, size_t guard_bytes, int* intact, void* stream);

/* ---- learned part: dense products -----------------------------------------------
 * C = A B^T, the contraction of the dense layers of the embedding network (Sec. 4) and
 * the normalizing flow (Sec. 5) that train on the simulated batches:
 *   C[m][n] = sum_k A[m][k] B[n][k],
 * A bfloat16 [M][K] and B bfloat16 [N][K] row-major (K contiguous), C [M][N] row-major
 * in FP32 (c_dtype GWX_F32) or bfloat16 rounded to nearest even (GWX_BF16).  The
 * products accumulate in FP32 in tensor memory (tcgen05.mma), operands arrive by TMA.
 * Sizes: 1 <= M <= 2^23, 1 <= N, 8 <= K < 2^31 with K % 8 == 0; A, B and C 16-byte
 * aligned.  Rows and columns past M, N and the K tail are handled (zero fill, masked
 * stores).  A kernel whose bounded wait for its own copies expires skips its stores
 * and records it for gwx_device_status. */
#define GWX_F32  0
#define GWX_BF16 1
int gwx_gemm_bf16(const void* A, const void* B, void* C, int64_t M, int64_t N, int64_t K, int c_dtype,
                  void* stream);

/* A dense layer with its epilogue fused into the product above:
 *   Y[m][n] = act( sum_k X[m][k] W[n][k] + bias[n] ),
 * X bfloat16 [M][K] (activations), W bfloat16 [N][K] (weights, one row per output),
 * bias FP32 [N] or NULL, act GWX_ACT_NONE, GWX_ACT_RELU (max(0, z)) or GWX_ACT_GELU
 * (z Phi(z), Phi the standard normal CDF), Y FP32 or bfloat16 [M][N].  Same sizes and
 * alignment as gwx_gemm_bf16; bias 4-byte aligned. */
#define GWX_ACT_NONE 0
#define GWX_ACT_RELU 1
#define GWX_ACT_GELU 2
int gwx_dense_bf16(const void* X, const void* W, const float* bias, void* Y, int64_t M, int64_t N, int64_t K,
                   int act, int y_dtype, void* stream);

/* Backward pass of gwx_dense_bf16 for a loss L given dY = dL/dY (FP32 [M][N]):
 *   Z = X W^T + b (recomputed on the tensor cores when act is not GWX_ACT_NONE),
 *   dZ = dY * act'(Z)  (ReLU' = [z > 0], GELU' = Phi(z) + z phi(z)),
 *   dX = dZ W  (FP32 [M][K]),  dW = dZ^T X  (FP32 [N][K]),  db = sum_m dZ  (FP32 [N]).
 * dZ enters both products in bfloat16 (round to nearest even), with FP32 accumulation;
 * db sums the FP32 dZ.  dX, dW or db may be NULL to skip it.  M, N, K multiples of 8 in
 * [8, 65535 * 32]; X, W, dX, dW 16-byte aligned, dY, bias, db 4-byte aligned.
 * Workspace: gwx_dense_bf16_backward_workspace(M, N, K) bytes. */
size_t gwx_dense_bf16_backward_workspace(int64_t M, int64_t N, int64_t K);
int gwx_dense_bf16_backward(const void* X, const void* W, const float* bias, const float* dY, int64_t M,
                            int64_t N, int64_t K, int act, float* dX, float* dW, float* db,
                            void* workspace, size_t workspace_bytes, void* stream);

/* ---- learned proposal: the pieces around the dense layers ---------------------------
 * The network trained on the simulated batches (Sec. 4, 5; AdamW) starts as the simplest
 * conditional flow: a Gaussian over chirp mass Mc = (m1 m2)^{3/5} / M^{1/5}, total mass M
 * and distance D whose mean mu and log-scale s (standardised units) a stack of
 * gwx_dense_bf16 layers computes from spectral features of the whitened strain.
 *
 * gwx_spectral_features: out[b][d ng + g] = ln( sum_{k in group g} |Y_b,d,k|^2 / (N G) )
 *   for the groups of G bins from k_lo = ceil(f_lo N / fs) (ng = (N/2 - k_lo) / G), Y the
 *   rfft of y [B][D][N] (FP32); columns from D ng to F_pad - 1 are 0; bfloat16 [B][F_pad],
 *   F_pad a multiple of 8.  Workspace gwx_spectral_features_workspace(B, D, N).
 * gwx_proposal_targets: t[b] = ((Mc, M, D) - mean) / scale, FP32 [B][3], from theta
 *   [GWX_NPARAM][B]; mean3 and scale3 are HOST arrays of 3 doubles.
 * gwx_gauss_nll: for network outputs out [B][ldo] (mu in columns 0..P-1, s in P..2P-1)
 *   and targets [B][P]: loss_rows[b] = sum_p (t - mu)^2 e^{-2s} / 2 + s (FP32), *loss_mean
 *   their mean (FP64, one device double), grad [B][ldo] = d(mean)/d(out) (0 elsewhere).
 * gwx_adamw: one AdamW step (Loshchilov & Hutter) on n FP32 parameters with moments m, v;
 *   step counts from 1; param_bf16 (optional) receives the bfloat16 copy the layers use.
 * gwx_sample_proposal: S samples for importance sampling, event e owning rows
 *   event_offsets[e] .. event_offsets[e+1] - 1.  Uniforms from Philox4x32-10 with counter
 *   (s, block 0..4, tag 3, counter) and key seed; spins and t_c are the event's own (truth
 *   [GWX_NPARAM][E]); phic, psi uniform in the prior ranges, RA uniform in [0, 2 pi),
 *   theta_JN and dec isotropic.  With net_out (rows [E][ldn], ldn >= 6: mu, s of Mc, M, D
 *   in standardised units, mean3/scale3 as for the targets) (Mc, M, D) are drawn from the
 *   Gaussian and (m1, m2) solved (order by a fair coin); log_ratio = ln prior - ln q
 *   (uniform prior in m1, m2, D; -inf outside it).  With net_out NULL the prior is the
 *   proposal (m1, m2, D uniform; log_ratio 0).  flags GWX_PROPOSAL_FIX_ANGLES takes phic,
 *   theta_JN, psi, RA and dec from the event too, so that the proposal covers m1, m2, D
 *   only.  theta out [GWX_NPARAM][S], log_ratio [S]: pass both to gwx_log_likelihood and
 *   gwx_importance_weights. */
#define GWX_PROPOSAL_FIX_ANGLES 1
/* gwx_cross_features: for each detector pair (a, b), a < b, in the order (0,1), (0,2),
 *   .., (1,2), .. (pair p) and group g: rho = sum_k Y_a,k conj(Y_b,k) /
 *   sqrt(sum_k |Y_a,k|^2 sum_k |Y_b,k|^2) over the group's bins, written as bfloat16
 *   Re rho to column col0 + 2 p ng + g and Im rho to column col0 + (2 p + 1) ng + g of
 *   features [B][F_pad] (other columns untouched).  A common time shift of all detectors
 *   multiplies every Y by the same phase factor, which cancels in rho: the columns carry
 *   the inter-detector delay and amplitude ratio without the arrival time (the nuisance
 *   the paper's embedding is pre-trained to marginalise, Sec. 4.1).  Needs
 *   col0 + D (D - 1) ng <= F_pad.  Workspace gwx_spectral_features_workspace(B, D, N). */
size_t gwx_spectral_features_workspace(int64_t B, int D, int64_t N);
int gwx_spectral_features(const float* y, int64_t B, int D, int64_t N, double fs, double f_lo, int group,
                          int F_pad, void* features, void* workspace, size_t workspace_bytes, void* stream);
int gwx_cross_features(const float* y, int64_t B, int D, int64_t N, double fs, double f_lo, int group, int F_pad,
                       int col0, void* features, void* workspace, size_t workspace_bytes, void* stream);
/* gwx_lag_features: for each detector d and group g the normalised lag-one product
 *   lam = sum_k Y_k conj(Y_{k+1}) / sqrt(sum_k |Y_k|^2 sum_k |Y_{k+1}|^2) over the group's
 *   bins k, as bfloat16 Re lam to column col0 + 2 d ng + g and Im lam to col0 + (2 d + 1) ng
 *   + g.  For a chirp its phase is 2 pi t(f) / T with t(f) the time the signal passes
 *   frequency f: the time-frequency track that fixes the chirp mass, which log powers
 *   and cross spectra do not carry.  Needs col0 + 2 D ng <= F_pad.  Workspace as for
 *   gwx_spectral_features. */
int gwx_lag_features(const float* y, int64_t B, int D, int64_t N, double fs, double f_lo, int group, int F_pad,
                     int col0, void* features, void* workspace, size_t workspace_bytes, void* stream);
int gwx_proposal_targets(const double* theta, int64_t B, const double* mean3, const double* scale3,
                         float* targets, void* stream);
int gwx_gauss_nll(const float* out, int ldo, const float* targets, int P, int64_t B, float* loss_rows,
                  double* loss_mean, float* grad, void* stream);
int gwx_adamw(float* param, const float* grad, float* m, float* v, int64_t n, double lr, double beta1,
              double beta2, double eps, double weight_decay, int64_t step, void* param_bf16, void* stream);
/* gwx_adamw_at: gwx_adamw with the step number read on the device from *step (a device
 *   int64, not modified; counts from 1): a CUDA graph that advances one step counter can
 *   replay the updates of many tensors.  step 8-byte aligned. */
int gwx_adamw_at(float* param, const float* grad, float* m, float* v, int64_t n, double lr, double beta1,
                 double beta2, double eps, double weight_decay, const int64_t* step, void* param_bf16, void* stream);
/* gwx_adamw_clip: gwx_adamw on the gradients scaled by min(1, clip / |g|), |g| the
 *   Euclidean norm of all n gradients (summed in FP64); grad itself is not modified.
 *   Workspace gwx_adamw_clip_workspace() bytes. */
size_t gwx_adamw_clip_workspace(void);
int gwx_adamw_clip(float* param, const float* grad, float* m, float* v, int64_t n, double lr, double beta1,
                   double beta2, double eps, double weight_decay, int64_t step, double clip, void* param_bf16,
                   void* workspace, size_t workspace_bytes, void* stream);
int gwx_sample_proposal(const float* net_out, int ldn, const double* mean3, const double* scale3,
                        const gwx_prior* prior, const double* truth, int64_t E, const int64_t* event_offsets,
                        int64_t S, uint64_t seed, uint32_t counter, int flags, double* theta,
                        double* log_ratio, void* stream);

/* ---- learned part: the conditional coupling flow ------------------------------------
 * The posterior estimator q(theta | d) of Sec. 5: a standard normal over eight
 * coordinates pushed through K affine coupling layers (Dinh, Sohl-Dickstein and Bengio
 * 2017) whose shifts and log-scales small dense networks compute from a context vector
 * c, the data summary of Sec. 4 computed from the spectral features of the whitened
 * strain (gwx_spectral_features).  The paper's transforms are inverse-autoregressive;
 * coupling transforms take one pass in both directions (training needs the density of
 * simulated parameters, importance sampling needs draws).
 *
 * Coordinates r = (Mc, q, D_L, cos theta_JN, alpha, sin delta, psi, phi_c), chirp mass
 * Mc = (m1 m2)^{3/5} / (m1 + m2)^{1/5}, q = min(m1, m2) / max(m1, m2); the flow works in
 * x = (r - mean) / scale, mean8 and scale8 HOST arrays of 8 doubles (scale > 0).
 *
 * Shape: F feature columns (groups of G bins), embedding width H_e, context width C, K
 * coupling layers (1..64), conditioner width H; F, H_e, C, H multiples of 8 in
 * [8, 65535 * 32].  Features f: the D ng log group powers of gwx_spectral_features,
 * then, when `extra` has GWX_FLOW_CROSS, the D (D - 1) ng cross-spectral columns of
 * gwx_cross_features, then, when it has GWX_FLOW_LAG, the 2 D ng lag-one columns of
 * gwx_lag_features; F at least their total.
 * Parameters: one flat FP32 array `params` and its bfloat16 copy `params_bf16` with the
 * same element offsets (gwx_adamw with param_bf16 keeps them in step); weights are read
 * from the bfloat16 copy, biases from the FP32 array.  Tensor t starts at element
 * offsets[t] (a multiple of 64; gwx_flow_layout), in the order
 *   embedding        W1 [H_e][F], b1 [H_e], W2 [H_e][H_e], b2 [H_e], W3 [C][H_e], b3 [C];
 *   layer l = 0..K-1 V1 [H][8 + C], e1 [H], V2 [H][H], e2 [H], V3 [8][H], e3 [8].
 * Embedding:  c = W3 h2 + b3, h2 = relu(W2 h1 + b2), h1 = relu(W1 f + b1), f the features
 *             (f, h1, h2, c held in bfloat16; relu(z) = max(z, 0)).
 * Layer l:    split (a, b) = SPLITS[l % 4], SPLITS = {(0 1 2 3 | 4 5 6 7), (4 5 6 7 | 0 1 2 3),
 *             (0 2 4 6 | 1 3 5 7), (1 3 5 7 | 0 2 4 6)}; conditioner input row
 *             X = [bf16(v_a), 0, 0, 0, 0, c] (bfloat16 [8 + C]); o = V3 g2 + e3 (FP32 [8]),
 *             g2 = relu(V2 g1 + e2), g1 = relu(V1 X + e1) (bfloat16); shift mu_j = o_j,
 *             log-scale s_j = 3 tanh(o_{4+j} / 3) on coordinate b_j.  Sampling direction
 *             v_b <- v_b e^s + mu; density direction v_b <- (v_b - mu) e^{-s}.
 * Sampling applies layers 0 .. K-1 to z ~ N(0, I_8), the density K-1 .. 0 to x;
 * ln q_x(x) = ln N(z; 0, I_8) - sum over layers and j of s_j, and in r-coordinates
 * ln q_r = ln q_x - sum_p ln scale_p.  Training minimises the batch mean of -ln q_x.
 *
 * gwx_flow_layout: *n_params = flat array length; offsets (6 + 6K entries) if not NULL. */
typedef struct gwx_flow_shape {
  int features;      /* F   */
  int group;         /* G   */
  int embed_hidden;  /* H_e */
  int context;       /* C   */
  int layers;        /* K   */
  int hidden;        /* H   */
  int extra;         /* feature columns after the log powers: GWX_FLOW_CROSS | GWX_FLOW_LAG */
} gwx_flow_shape;
#define GWX_FLOW_CROSS 1
#define GWX_FLOW_LAG 2
int gwx_flow_layout(const gwx_flow_shape* shape, int64_t* n_params, int64_t* offsets);

/* Stages (one kernel each; the calls further down chain them).  Arrays are device
 * arrays, row-major, 16-byte aligned (8-byte for doubles and int64).
 * gwx_flow_targets: x [B][8] FP32 = (r(theta) - mean) / scale for theta [GWX_NPARAM][B].
 * gwx_flow_conditioner_input: X bfloat16 [B][8 + C] of layer l from v [B][8] FP32 and
 *   the context ctx bfloat16: [B][C] row by row when event_offsets is NULL, else [E][C]
 *   with row r taking the context of the event owning global row row0 + r.
 * gwx_flow_coupling: step of layer l, direction +1 (sampling) or -1 (density):
 *   v_out [B][8] (may be v_in) from v_in and o [B][8] FP32;
 *   sum_s[b] = (init ? 0 : sum_s[b]) + sum_j s_j.
 * gwx_flow_nll: loss_rows[b] = |z_b|^2 / 2 + 4 ln(2 pi) + sum_s[b] (FP32), *loss_mean their
 *   FP64 mean (device double), grad [B][8] = z / B.
 * gwx_flow_coupling_backward: for a density step of layer l with output w [B][8] and
 *   conditioner output o, given g = dL/dw: d_o [B][8] = dL/do including the term
 *   row_weight x sum_j s_j of the loss, and g_u [B][8] = dL/dv_in except the
 *   conditioner's share.
 * gwx_flow_input_backward: adds dX[b][j] (j = 0..3; dX = dL/dX FP32 [B][8 + C]) into
 *   g_u[b][a_j] and sets (init) or adds dX[b][8 ..] into d_ctx [B][C].
 * gwx_flow_base: base draws z [n][8] FP32 of global draws row0 .. row0 + n - 1: Philox4x32-10
 *   counters (s, j, 4, counter), key seed, block j = 0..3 giving u_{2j} = uniform52(w0, w1),
 *   u_{2j+1} = uniform52(w2, w3) and the Box-Muller pair z_{2j}, z_{2j+1} =
 *   sqrt(-2 ln u_{2j}) (cos, sin)(2 pi u_{2j+1}).
 * gwx_flow_proposal: for flow draws x [S][8] with base z and sum_s: theta [GWX_NPARAM][S],
 *   log_q [S] = ln q_r and log_ratio [S] = ln prior_r - ln q_r (-inf outside the prior's
 *   support).  Inside it m_big = Mc (1 + q)^{1/5} q^{-3/5}, m_small = q m_big, swapped
 *   into (m1, m2) when the coin u_8 (block 4 of the draw's counter, words 0 and 1) is
 *   below 1/2; theta_JN = acos, dec = asin of their coordinates.  The flow does not model
 *   the spins or t_c (Sec. 5: spins ignored, t_c marginalised): they are drawn from the
 *   prior's ranges, t_c = tc_lo + (tc_hi - tc_lo) u_9 (block 4, words 2 and 3), chi_1 and
 *   chi_2 = chi_lo + (chi_hi - chi_lo) u_10, u_11 (block 5), so their prior and proposal
 *   densities cancel in log_ratio.  The prior (uniform in m1, m2, D, cos
 *   theta_JN, RA, sin dec, psi, phic) has ln prior_r = ln 2 + 2 ln m_big - ln Mc
 *   - ln((m_hi - m_lo)^2 (d_hi - d_lo) 8 pi (psi_hi - psi_lo) (phi_hi - phi_lo)).
 *   Outside the support theta holds m_lo, d_lo and clipped angles. */
int gwx_flow_targets(const double* theta, int64_t B, const double* mean8, const double* scale8, float* x,
                     void* stream);
int gwx_flow_conditioner_input(int layer, const float* v, const void* ctx, int C, const int64_t* event_offsets,
                               int64_t E, int64_t row0, int64_t B, void* X, void* stream);
int gwx_flow_coupling(int layer, int direction, const float* v_in, const float* o, int64_t B, float* v_out,
                      float* sum_s, int init, void* stream);
int gwx_flow_nll(const float* z, const float* sum_s, int64_t B, float* loss_rows, double* loss_mean, float* grad,
                 void* stream);
int gwx_flow_coupling_backward(int layer, const float* w, const float* o, const float* g, int64_t B,
                               float row_weight, float* d_o, float* g_u, void* stream);
int gwx_flow_input_backward(int layer, const float* dX, int C, int64_t B, float* g_u, float* d_ctx, int init,
                            void* stream);
int gwx_flow_base(uint64_t seed, uint32_t counter, int64_t row0, int64_t n, float* z, void* stream);
int gwx_flow_proposal(const float* x, const float* z, const float* sum_s, int64_t S, const double* mean8,
                      const double* scale8, const gwx_prior* prior, uint64_t seed, uint32_t counter, double* theta,
                      double* log_q, double* log_ratio, void* stream);

/* One training step on a simulated batch: whitened strain y [B][D][N] (FP32) and its
 * parameters theta [GWX_NPARAM][B]: features, embedding, density pass, loss, backward
 * into grads (flat, same layout as params; the whole array is rewritten), then (step >= 1)
 * gwx_adamw over the flat array with step counter `step` (gwx_adamw_clip when clip > 0:
 * gradients scaled to a Euclidean norm of at most clip); step 0 computes the loss and
 * gradients only.  ctx_in (optional, bfloat16 [B][C]): a context from another data-summary
 * network (the ResNet-1D of Sec. 4) replaces the built-in summary of the features, whose
 * tensors then get zero gradients, and d_ctx_out (FP32 [B][C]) receives dL/dcontext for
 * that network's backward pass; y may then be NULL.  The same ctx_in argument of
 * gwx_flow_log_prob (one row per parameter vector) and gwx_sample_posterior (one row per
 * event) skips the built-in summary there.  step_counter (optional, a device int64): the update takes its step
 * number from *step_counter + 1 on the device and stores it back, so that a captured
 * CUDA graph of the call replays with the right AdamW bias corrections (step then only
 * has to be >= 1).  *loss_mean (device double) = batch mean of -ln q_x.  B a multiple of 8
 * in [8, 65535 * 32].  Workspace gwx_flow_train_workspace(shape, B, D, N). */
size_t gwx_flow_train_workspace(const gwx_flow_shape* shape, int64_t B, int D, int64_t N);
int gwx_flow_train_step(const gwx_flow_shape* shape, float* params, void* params_bf16, float* grads, float* m,
                        float* v, int64_t step, int64_t* step_counter, double lr, double beta1, double beta2, double eps,
                        double weight_decay, double clip, const double* mean8, const double* scale8, const float* y,
                        const double* theta, int64_t B, int D, int64_t N, double fs, double f_lo,
                        const void* ctx_in, float* d_ctx_out, double* loss_mean, void* workspace,
                        size_t workspace_bytes, void* stream);

/* Density ln q_r(r(theta_b) | y_b) (FP64 [B]) of B parameter vectors, each with its own
 * whitened window y [B][D][N].  Workspace gwx_flow_log_prob_workspace(shape, B, D, N). */
size_t gwx_flow_log_prob_workspace(const gwx_flow_shape* shape, int64_t B, int D, int64_t N);
int gwx_flow_log_prob(const gwx_flow_shape* shape, const float* params, const void* params_bf16,
                      const double* mean8, const double* scale8, const float* y, const double* theta, int64_t B,
                      int D, int64_t N, double fs, double f_lo, const void* ctx_in, double* log_q, void* workspace,
                      size_t workspace_bytes, void* stream);

/* Posterior samples (Sec. 5: draws from q(theta | d) for new data; Sec. 6 judges them):
 * event e of y [E][D][N] owns rows event_offsets[e] .. event_offsets[e+1] - 1 of the S
 * outputs (event_offsets device int64 [E + 1], non-decreasing from 0 to S).  Per event
 * the context is computed once; each draw runs the base normals, the K coupling layers
 * in the sampling direction and gwx_flow_proposal (theta, log_q = ln q_r, log_ratio), in
 * chunks of at most 2^17 draws.  Workspace gwx_sample_posterior_workspace(shape, E, D, N, S). */
size_t gwx_sample_posterior_workspace(const gwx_flow_shape* shape, int64_t E, int D, int64_t N, int64_t S);
int gwx_sample_posterior(const gwx_flow_shape* shape, const float* params, const void* params_bf16,
                         const double* mean8, const double* scale8, const gwx_prior* prior, const float* y,
                         int64_t E, int D, int64_t N, double fs, double f_lo, const void* ctx_in,
                         const int64_t* event_offsets, int64_t S, uint64_t seed,
                         uint32_t counter, double* theta, double* log_q, double* log_ratio, void* workspace,
                         size_t workspace_bytes, void* stream);

/* The flow's sky density over HEALPix pixels (Sec. 5: the density is evaluated at every
 * pixel of the sky map): map [12 nside^2] (FP64, nested order, unit sum) holds, at each
 * pixel centre, q_r of the flow's coordinates with RA and sin dec at the centre and the
 * other six (Mc, q, D_L, cos theta_JN, psi, phic) at those of the event's draw of largest
 * log_q among theta [GWX_NPARAM][S] (device; e.g. gwx_sample_posterior's output, first on
 * ties), normalised over the pixels.  (RA, sin dec) are equal-area coordinates of the
 * sphere (d Omega = d RA d sin dec), so with HEALPix's equal-area pixels the map is that
 * density per steradian times the pixel area, up to its normalisation.  One density
 * pass of the flow over all pixels (the event's context computed once from y [1][D][N],
 * or ctx_in [1][C]); nside a power of two in [1, 8192].  Workspace
 * gwx_flow_skymap_workspace(shape, D, N, nside). */
size_t gwx_flow_skymap_workspace(const gwx_flow_shape* shape, int D, int64_t N, int nside);
int gwx_flow_skymap(const gwx_flow_shape* shape, const float* params, const void* params_bf16,
                    const double* mean8, const double* scale8, const float* y, int D, int64_t N, double fs,
                    double f_lo, const void* ctx_in, const double* theta, const double* log_q, int64_t S,
                    int nside, double* map, void* workspace, size_t workspace_bytes, void* stream);

/* ---- self-supervised pre-training of the data summary (Sec. 4.1) ------------------
 * Two views of each simulated source, identical but for the merger time, are summarised
 * and expanded (x, x' [B][d]); the summary is trained to make them agree with the VICReg
 * loss (Bardes, Ponce and LeCun 2022) and the paper's weights (1, 1, 5):
 *   L = l1 sum (x - x')^2 / (B d) + l2 (v(x) + v(x')) + l3 (c(x) + c(x')),
 *   v(z) = sum_j max(0, 1 - sqrt(Var_j(z) + 1e-4)) / d,  c(z) = sum_{i != j} C_ij(z)^2 / d,
 * Var and C the unbiased sample variance and covariance over the batch.
 * gwx_vicreg: *loss (device double), terms (optional device double[5]: inv, v(x), v(x'),
 *   c(x), c(x')), grad_x, grad_xp = dL/dx, dL/dx' (FP32 [B][d]).  2 <= B, 1 <= d <= 32.
 * gwx_retime: theta_out = theta_in ([GWX_NPARAM][B]) with the merger time redrawn
 *   uniformly in [tc_lo, tc_hi] (uniform52 of Philox4x32-10 words 0, 1 at counter
 *   (b, 0, 5, counter), key seed): the second view's source.
 * gwx_prepare_theta: gwx_prepare_batch for given parameters theta [GWX_NPARAM][B] (no
 *   prior draws), so that gwx_simulate_prepared renders them (with the caller's offsets). */
int gwx_vicreg(const float* x, const float* xp, int64_t B, int d, double lambda1, double lambda2, double lambda3,
               double* loss, double* terms, float* grad_x, float* grad_xp, void* stream);
int gwx_retime(const double* theta_in, double* theta_out, int64_t B, double tc_lo, double tc_hi, uint64_t seed,
               uint32_t counter, void* stream);
int gwx_prepare_theta(const double* theta, int64_t L, int64_t N, double fs, double f_lo, const int32_t* det_ids,
                      int D, double gmst, int64_t B, void* workspace, size_t workspace_bytes, void* stream);

/* ---- ResNet-1D data summary (Sec. 4) ------------------------------------------------
 * 1-D convolutions on channels-last activations x [B][T][C] are im2col rows times the
 * weights W [C_out][K] on the tensor cores (gwx_dense_bf16, gwx_dense_bf16_backward):
 *   cols[b, t][j C + c] = x[b][s t + j - p][c] (zero outside 0 .. T - 1; columns k C .. K - 1
 *   zero), T_out = (T + 2 p - k) / s + 1.
 * Shapes for every call below: 1 <= B <= 65535, T C < 2^31 and B T < 2^31 (T_out K < 2^31
 *   for the row builders); otherwise GWX_ESHAPE.
 * gwx_im2col: bfloat16 x -> bfloat16 cols [B T_out][K]; C, K multiples of 8.
 * gwx_im2col_cf: the same rows from channels-first FP32 y [B][D][N] (whitened strain).
 * gwx_col2im: the adjoint: dx [B][T][C] (FP32) = addend (optional) + sum over the rows and
 *   taps that read x[b][t][c] of dcols (FP32 [B T_out][K]).
 * gwx_group_norm: per sample and group of C / G channels, over all T and those channels:
 *   out = act(gamma_c (z - mean) / sqrt(var + 1e-5) + beta_c + residual) (biased variance of
 *   the values shifted by the group's first value: FP32 sums of a few dozen terms per
 *   thread, FP64 across threads; residual FP32 or bfloat16 or none; act ReLU when relu != 0); out bfloat16
 *   (out16) and/or FP32 (out32); mean_rstd [B][G][2] kept for the backward.
 * gwx_group_norm_backward: dz = rstd (dy gamma - mean(dy gamma) - xhat mean(dy gamma xhat))
 *   per group, dgamma_c = sum dy xhat, dbeta_c = sum dy (deterministic: FP32 over runs of
 *   at most 64 terms, FP64 across runs and threads); scratch
 *   of gwx_group_norm_backward_scratch(B, C, G) bytes (256-byte aligned).
 * gwx_relu_mask: d = dy [out > 0] (out bfloat16).
 * gwx_maxpool: kernel 3, stride 2, padding 1 over time, the first maximum of a window;
 *   arg [B][T_out][C] its offset (0..2); gwx_maxpool_backward routes dy there.
 * gwx_mean_time: m [B][C] (bfloat16) = the mean over time; gwx_mean_time_backward. */
int gwx_im2col(const void* x, int64_t B, int T, int C, int k, int s, int p, int K, void* cols, void* stream);
int gwx_im2col_cf(const float* y, int64_t B, int D, int N, int k, int s, int p, int K, void* cols, void* stream);
int gwx_col2im(const float* dcols, int64_t B, int T, int C, int k, int s, int p, int K, const float* addend, float* dx,
               void* stream);
int gwx_group_norm(const float* z, int64_t B, int T, int C, int G, const float* gamma, const float* beta,
                   const float* residual32, const void* residual16, int relu, void* out16, float* out32,
                   float* mean_rstd, void* stream);
size_t gwx_group_norm_backward_scratch(int64_t B, int C, int G);
int gwx_group_norm_backward(const float* dy, const float* z, int64_t B, int T, int C, int G, const float* mean_rstd,
                            const float* gamma, void* scratch, float* dz, float* dgamma, float* dbeta, void* stream);
int gwx_relu_mask(const float* dy, const void* out, int64_t n, float* d, void* stream);
int gwx_maxpool(const void* x, int64_t B, int T, int C, void* y, uint8_t* arg, void* stream);
int gwx_maxpool_backward(const float* dy, const uint8_t* arg, int64_t B, int T, int C, float* dx, void* stream);
int gwx_mean_time(const void* x, int64_t B, int T, int C, void* m, void* stream);
int gwx_mean_time_backward(const float* dm, int64_t B, int T, int C, float* dx, void* stream);

/* ---- ResNet-1D: stride-1 convolutions as implicit GEMMs (Sec. 4) ---------------------
 * The summary's stride-1 convolutions with zero "same" padding, p = (k - 1)/2, on the
 * tensor cores without an im2col matrix: the product's A tiles come straight from the
 * channels-last activations through a 3-D tensor map, one 128-time x 64-channel box per
 * tap and channel block, zero-filled outside the series.
 * gwx_conv1d_bf16: z[b][t][o] = sum_{j < k, c < C} x[b][t + j - p][c] W[o][j C + c]
 *   (+ addend[b][t][o]); x bfloat16 [B][T][C], W bfloat16 [O][k C] (the row layout of
 *   gwx_im2col with K = k C), z FP32 [B][T][O], addend FP32 or NULL.
 * gwx_conv1d_bf16_backward: from dz FP32 [B][T][O], rounded to bfloat16 for the products
 *   as in gwx_dense_bf16_backward: dx FP32 [B][T][C] = sum_{j, o} dz[b][t - j + p][o]
 *   W[o][j C + c] (+ addend FP32 [B][T][C] or NULL) and dW FP32 [O][k C] =
 *   sum_{b, t} dz[b][t][o] x[b][t + j - p][c] (split-K, deterministic); either output may
 *   be NULL.  Workspace gwx_conv1d_bf16_backward_workspace(B, T, C, O, k) bytes.
 * Sizes: T % 128 == 0, C % 64 == 0, O % 64 == 0, k odd in [1, 15], B >= 1, B T <= 2^26;
 * x, W, z, dx, dW and addend 16-byte aligned, dz 4-byte aligned; else GWX_ESHAPE or
 * GWX_EINVAL; a workspace below the size GWX_ENOMEM.  A bounded wait that expires is
 * reported by gwx_device_status. */
int gwx_conv1d_bf16(const void* x, int64_t B, int64_t T, int C, int k, const void* W, int O, const float* addend,
                    float* z, void* stream);
size_t gwx_conv1d_bf16_backward_workspace(int64_t B, int64_t T, int C, int O, int k);
int gwx_conv1d_bf16_backward(const float* dz, const void* x, const void* W, int64_t B, int64_t T, int C, int O, int k,
                             const float* addend, float* dx, float* dW, void* workspace, size_t workspace_bytes,
                             void* stream);

/* ---- sky maps ---------------------------------------------------------------------
 * The paper's inference ends in a sky-localisation map in the HEALPix format (Sec. 5).
 * gwx_skymap: map [12 nside^2] (FP64) = the histogram of samples' sky positions (rows RA
 * and dec of theta [GWX_NPARAM][S]) over the nested-scheme HEALPix pixels (Gorski et al.
 * 2005) of resolution nside, each sample counted with its weight (weights [S], e.g. from
 * gwx_importance_weights; NULL counts every sample once; zero, negative or non-finite
 * weights are skipped), normalised to unit sum (all zero if no sample counts).  nside a
 * power of two in [1, 8192]; map overwritten.  Workspace gwx_skymap_workspace() bytes.
 * Accumulation is by FP64 atomic additions, so the last bits depend on their order. */
size_t gwx_skymap_workspace(void);
int gwx_skymap(const double* theta, const double* weights, int64_t S, int nside, double* map, void* workspace,
               size_t workspace_bytes, void* stream);

/* Autotuner of the product's tile raster (a set-up call, not a hot call: it launches the
 * product several times on the caller's buffers and synchronises `stream`).  For the
 * shape (M, N, K, c_dtype) it times each candidate band height of the persistent tile
 * walk (1 .. 64 tile-rows), keeps the fastest for later gwx_gemm_bf16 / gwx_dense_bf16
 * calls of that shape in this process, and returns it in *group (if not NULL).
 * C is overwritten. */
int gwx_gemm_autotune(const void* A, const void* B, void* C, int64_t M, int64_t N, int64_t K, int c_dtype,
                      int* group, void* stream);

/* Synchronises the current device; returns GWX_ETIMEOUT (and clears the record) if a
 * kernel gave up a bounded wait since the last call, else GWX_OK. */
int gwx_device_status(void);

/* Self-test of that path: launches one thread that waits on an mbarrier nothing arrives
 * at and gives up after `polls` polls (1 .. 2^20; each poll returns within a bounded,
 * hardware-defined time), recording the expiry as a kernel whose copies never landed
 * would.  The next gwx_device_status returns GWX_ETIMEOUT; the context stays usable.
 * GWX_EINVAL for polls out of range. */
int gwx_selftest_bounded_wait(uint32_t polls, void* stream);

/* ---- transforms (the FFT kernels of the steps above, exposed for checking) ----
 * gwx_rfft:  X[r] = rfft(x[r]) for R rows of N real samples (numpy convention,
 *            X_k = sum_n x_n e^{-2 pi i k n/N}); X complex[R][N/2+1].
 * gwx_irfft: x[r] = irfft(X[r]) with 1/N normalisation; imaginary parts of the
 *            DC and Nyquist bins are ignored. */
int gwx_rfft(const float* x, int64_t R, int64_t N, float* X, void* stream);
int gwx_irfft(const float* X, int64_t R, int64_t N, float* x, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* GWX_H */
