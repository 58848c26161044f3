// gwx_internal.h -- structures and launcher declarations shared by the
// libgwx translation units (not part of the public C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/gwx.h"

namespace gwx {

// Detector table passed by value to kernels: tensor D (row-major) and vertex
// position r [m] for each selected detector, in FP64.
struct DetParams {
  int D;
  double tensor[GWX_MAX_DET][9];
  double pos[GWX_MAX_DET][3];
};

// Per-draw waveform and projection coefficients (written by the set-up stage,
// read per frequency bin).  Phase in turns (cycles):
//   Psi(k)/2pi = c0 k^-5/3 + c2 k^-1 + c3 k^-2/3 + c4 k^-1/3 + d5 ln k
//                + (c6 + d6 ln k) k^1/3 + c7 k^2/3 + cph
// with c0, c2, c3, d5 as double-float pairs (hi, lo); amplitude of bin k is
// amp * k^-7/6.  The detector-d strain of bin k (times the sample rate) is
// g[d] * k^-7/6 * e^{-2 pi i (Psi(k)/2pi + k nu[d] 2^-64)}, with g[d] the complex
// double-float constant fs amp (F+_d qp - i Fx_d qc_im) as (re hi, re lo, im hi, im lo).
struct __align__(16) DrawCoef {
  float2 c0, c2, c3, d5;
  float c4, c6, d6, c7;
  float cph, amp, qp, qc_im;        // amp = A(df) (strain/Hz); h_plus factor qp = (1 + cos^2 i)/2,
                                    // h_cross factor -i qc_im with qc_im = cos i
  int kcut, pad0, pad1, pad2;       // last non-zero bin (inclusive), may be < k_lo
  float4 g[GWX_MAX_DET];            // fs amp (F+_d qp - i Fx_d qc_im), double-float
  unsigned long long nu[GWX_MAX_DET];
};

// ---- launchers (return cudaGetLastError() of the launch) ----
cudaError_t launch_sample_prior(const gwx_prior& p, uint64_t seed, uint32_t step, int64_t B, int64_t L,
                                int64_t N, double* theta, int64_t* offsets, cudaStream_t s);
cudaError_t launch_generate_waveforms(const double* theta, int64_t B, int k_lo, double df, int64_t F,
                                      float2* hp, float2* hc, cudaStream_t s);
cudaError_t launch_project(const float2* hp, const float2* hc, const double* theta, int64_t B,
                           const DetParams& dp, double gmst, double df, int64_t F, float2* hdet,
                           cudaStream_t s);
cudaError_t launch_draw_setup(const double* theta, int64_t B, int k_lo, double df, double fs, int64_t F,
                              const DetParams& dp, double gmst, DrawCoef* coef, cudaStream_t s);
cudaError_t launch_colored_noise(uint64_t seed, uint32_t step, int D, int64_t L, double fs, double f_lo,
                                 float* noise, void* ws, cudaStream_t s);
size_t colored_noise_ws(int D, int64_t L);
cudaError_t launch_welch(const float* x, int D, int64_t L, double fs, int64_t M, int64_t stride, double* psd,
                         void* ws, cudaStream_t s);
size_t welch_ws(int D, int64_t L, int64_t M, int64_t stride);
cudaError_t launch_whiten_filter(const double* psd, int D, int64_t M, double fs, int k_lo, int64_t N, float* W,
                                 cudaStream_t s, bool inverse = false);
// Packed-domain whitening coefficients (alpha, beta) [D][N/2] from W [D][N/2+1].
cudaError_t launch_whiten_rows(const float* d, const float* W, int64_t rows, int D, int64_t N, float* y,
                               cudaStream_t s);
cudaError_t launch_inject_rows(const float* noise, int D, int64_t L, const int64_t* offsets, const float2* hdet,
                               int64_t B, int64_t N, double fs, float* d, cudaStream_t s);
cudaError_t launch_inject_padded(const float* noise, int D, int64_t L, const int64_t* offsets, const float* htd,
                                 int64_t B, int64_t N, int64_t Np, double fs, float* d, cudaStream_t s);
cudaError_t launch_rfft_rows(const float* x, int64_t R, int64_t N, float2* X, cudaStream_t s);
cudaError_t launch_irfft_rows(const float2* X, int64_t R, int64_t N, float* x, cudaStream_t s);
// W: the whitening filter [D][N/2 + 1] at the start of an allocation of Wcap floats
// (Wcap a multiple of 4; the staged shape copies whole 16-byte words up to it).
cudaError_t launch_simulate_fused(const DrawCoef* coef, const float* noise, int64_t L, const int64_t* offsets,
                                  const float* W, int64_t Wcap, int k_lo, int D, int64_t B, int64_t N, double fs,
                                  float* y, cudaStream_t s, int shape = -1);
// Launch shape of the fused pass for windows of N samples and D detectors (bit 0: two
// shared buffers, bits 1-2: blocks per SM, 0 = the occupancy limit, bit 3: staged crop and
// filter): the tuned choice, or the default; sim_shape_set records one (a negative shape
// forgets it); sim_can_stage: whether the staged shape applies to these arrays.
int sim_shape_for(int64_t N, int D);
void sim_shape_set(int64_t N, int D, int shape);
bool sim_can_stage(const float* noise, int64_t L, const float* W, int64_t N);
// Reads and clears the record of a fused pass that gave up waiting for its staged copies.
cudaError_t sim_status(int* status);
// yy: E doubles of scratch for the per-event sum of |Y|^2 over the band.
// Per-event data norms (E x 8 FP64 partials in yy_part, loglike_norm_bytes(E)) and
// the fused per-sample set-up + likelihood.
size_t loglike_norm_bytes(int64_t E);
cudaError_t launch_loglike_full(const float* ydata, const float2* Ydata, const float* W, const double* theta,
                                double df, double fs, const DetParams& dp, double gmst, const int64_t* ev_off,
                                double* yy_part, int64_t E, int D, int64_t N, int k_lo, int64_t S, double* lnl,
                                cudaStream_t s);
// ln L with the merger time integrated out over tc_lo + j / (u fs), j < u n_tc (the tc row
// of theta unused); the same data-norm kernel and workspace as launch_loglike_full, plus
// tm_rows_bytes() of per-offset constants in rows.
size_t tm_rows_bytes();
cudaError_t launch_loglike_tmarg(const float* ydata, const float2* Ydata, const float* W, const double* theta,
                                 double df, double fs, const DetParams& dp, double gmst, double tc_lo, int n_tc,
                                 int u, const int64_t* ev_off, double* yy_part, float2* rows, int64_t E, int D,
                                 int64_t N, int k_lo, int64_t S, double* lnl, cudaStream_t s);

// Importance weights: E x iw_chunks(E) partials in ws (iw_workspace_bytes(E)).
size_t iw_workspace_bytes(int64_t E);
cudaError_t launch_importance_weights(const double* lnl, const double* ratio, const int64_t* off, int64_t E,
                                      int64_t S, double* weights, double* ess, double* eff, double* lnz, void* ws,
                                      cudaStream_t s);

// C = act(A B^T + bias), bfloat16 operands [M][K], [N][K], FP32 accumulation on the
// tensor cores; C FP32 or bfloat16 [M][N]; bias FP32 [N] or NULL; act 0/1/2.  gemm_status reads and clears the timed-out-wait record.
// group: tile-rows per raster band (0 = the default).
cudaError_t launch_gemm_bf16(const void* A, const void* B, void* C, int64_t M, int64_t N, int64_t K, bool out_bf16,
                             const float* bias, int act, int group, cudaStream_t s);
// Split-K product C [M][N] (FP32) = A B^T for few tiles and a long K: the slices' partial
// products go to `part` (gemm_splitk_ws bytes), then one kernel sums them in order.
// Implicit-GEMM 1-D convolution (stride 1, zero "same" padding): out [Bn][T][N] FP32 =
// sum_{j < k, c < C} x[b][t + dir (j - (k-1)/2)][c] W[o][j C + c] (+ addend); x bfloat16
// channels last, W bfloat16 [N][k C].  T % 128 == 0, C % 64 == 0, 16-byte aligned x, W.
cudaError_t launch_conv_gemm(const void* x, int64_t Bn, int64_t T, int64_t C, int k, int dir, const void* W, int64_t N,
                             float* out, const float* addend, cudaStream_t s);
// The ResNet's stride-1 convolutions (k_conv.cu): forward z [Bn][T][O] = conv(x, W)
// (+ addend) and its backward (dx (+ addend), dW) through implicit GEMMs; the workspace
// of the backward is conv_backward_ws bytes.
size_t conv_backward_ws(int64_t Bn, int64_t T, int C, int O, int k);
cudaError_t launch_conv_forward(const void* x, int64_t Bn, int64_t T, int C, int k, const void* W, int O,
                                const float* addend, float* z, cudaStream_t s);
cudaError_t launch_conv_backward(const float* dz, const void* x, const void* W, int64_t Bn, int64_t T, int C, int O,
                                 int k, const float* addend, float* dx, float* dW, void* ws, cudaStream_t s);
int gemm_splits(int64_t M, int64_t N, int64_t K);
size_t gemm_splitk_ws(int64_t M, int64_t N, int64_t K);
cudaError_t launch_gemm_splitk(const void* A, const void* B, float* C, int64_t M, int64_t N, int64_t K, float* part,
                               cudaStream_t s);
cudaError_t gemm_status(int* status);

// Dense-layer backward (k_dense.cu): workspace bytes and the launcher.
size_t dense_backward_ws(int64_t M, int64_t N, int64_t K);
cudaError_t launch_dense_backward(const void* X, const void* W, const float* bias, const float* dY, int64_t M,
                                  int64_t N, int64_t K, int act, float* dX, float* dW, float* db, void* ws, int group,
                                  cudaStream_t s,
                                  const void* Y = nullptr);

// Learned proposal (k_learn.cu).
cudaError_t launch_features(const float* y, int64_t B, int D, int64_t N, int k_lo, int G, int F_pad, void* ws,
                            void* out, cudaStream_t s);
// Cross-spectral columns (k_cross_features) from a spectrum Y complex [B][D][N/2+1] that
// launch_features left in its workspace, or from y (rfft into ws first).
cudaError_t launch_cross_from_spectrum(const void* Y, int64_t B, int D, int64_t N, int k_lo, int G, int F_pad,
                                       int col0, void* out, cudaStream_t s);
cudaError_t launch_cross_features(const float* y, int64_t B, int D, int64_t N, int k_lo, int G, int F_pad, int col0,
                                  void* ws, void* out, cudaStream_t s);
// Lag-one spectral products (k_lag_features), from a spectrum or from y.
cudaError_t launch_lag_from_spectrum(const void* Y, int64_t B, int D, int64_t N, int k_lo, int G, int F_pad, int col0,
                                     void* out, cudaStream_t s);
cudaError_t launch_lag_features(const float* y, int64_t B, int D, int64_t N, int k_lo, int G, int F_pad, int col0,
                                void* ws, void* out, cudaStream_t s);
cudaError_t launch_targets(const double* theta, int64_t B, const double* mean, const double* scale, float* t,
                           cudaStream_t s);
cudaError_t launch_gauss_nll(const float* out, int ldo, const float* t, int P, int B, float* loss, double* mean,
                             float* grad, cudaStream_t s);
cudaError_t launch_adamw(float* p, const float* g, float* m, float* v, int64_t n, double lr, double b1, double b2,
                         double eps, double wd, int64_t step, void* p16, cudaStream_t s);
// launch_adamw with the step number *step read on the device (a CUDA-graph step counter).
cudaError_t launch_adamw_at(float* p, const float* g, float* m, float* v, int64_t n, double lr, double b1, double b2,
                            double eps, double wd, const int64_t* step, void* p16, cudaStream_t s);
// AdamW on gradients scaled by min(1, clip / |g|) (|g| the FP64 norm of all n gradients);
// workspace adamw_clip_ws() bytes.
size_t adamw_clip_ws();
// With counter (a device int64) the step is *counter + 1, stored back, and clip <= 0
// means no clipping; without it clip must be positive and `step` is used.
cudaError_t launch_adamw_clip(float* p, const float* g, float* m, float* v, int64_t n, double lr, double b1, double b2,
                              double eps, double wd, int64_t step, double clip, void* p16, void* ws, cudaStream_t s,
                              int64_t* counter = nullptr);
cudaError_t launch_proposal(const float* net, int ldn, const double* mean, const double* scale, const gwx_prior& pr,
                            const double* truth, int64_t E, const int64_t* off, int64_t S, uint64_t seed,
                            uint32_t counter, int fix_angles, double* theta, double* lratio, cudaStream_t s);

// Conditional coupling flow (k_flow.cu).  flow_layout returns the flat parameter count
// and fills the 6 + 6K tensor offsets (when off is not NULL).
int64_t flow_layout(const gwx_flow_shape& sh, int64_t* off);
cudaError_t launch_flow_targets(const double* theta, int64_t B, const double* mean8, const double* scale8, float* x,
                                cudaStream_t s);
cudaError_t launch_flow_input(int l, const float* v, const void* ctx, int C, const int64_t* off, int64_t E,
                              int64_t row0, int64_t B, void* X, cudaStream_t s);
cudaError_t launch_flow_coupling(int l, int dir, const float* vin, const float* o, int64_t B, float* vout,
                                 float* sum_s, int init, cudaStream_t s);
cudaError_t launch_flow_nll(const float* z, const float* sum_s, int64_t B, float* loss, double* mean, float* grad,
                            cudaStream_t s);
cudaError_t launch_flow_coupling_backward(int l, const float* w, const float* o, const float* g, int64_t B,
                                          float row_weight, float* d_o, float* g_u, cudaStream_t s);
cudaError_t launch_flow_input_backward(int l, const float* dX, int C, int64_t B, float* g_u, float* d_ctx, int init,
                                       cudaStream_t s);
cudaError_t launch_flow_base(uint64_t seed, uint32_t counter, int64_t row0, int64_t n, float* z, cudaStream_t s);
cudaError_t launch_flow_proposal(const float* x, const float* z, const float* sum_s, int64_t n, int64_t row0,
                                 int64_t S, const double* mean8, const double* scale8, const gwx_prior& pr,
                                 uint64_t seed, uint32_t counter, double* theta, double* log_q, double* log_ratio,
                                 cudaStream_t s);
// The sampling pass of the coupling flow fused into one persistent tcgen05 kernel
// (k_flow_fused.cu), for conditioner widths H of 128 or 256 and 8 + C <= 128: draws
// z [n][8] of global rows row0 .. row0 + n - 1 -> x_out [n][8], ss_out [n].
bool flow_fused_supported(int C, int H, int K);
cudaError_t launch_flow_sample_fused(const void* params_bf16, const float* params, const int64_t* off_t, int C, int H,
                                     int K, const float* z, const void* ctx, const int64_t* ev_off, int64_t E,
                                     int64_t row0, int64_t n, float* x_out, float* ss_out, cudaStream_t s);
cudaError_t flow_fused_status(int* status);
size_t flow_train_ws(const gwx_flow_shape& sh, int64_t B, int D, int64_t N);
cudaError_t flow_train_step(const gwx_flow_shape& sh, float* params, void* params_bf16, float* grads, float* m,
                            float* v, int64_t step, int64_t* step_counter, double lr, double b1, double b2, double eps, double wd, double clip,
                            const double* mean8, const double* scale8, const float* y, const double* theta, int64_t B,
                            int D, int64_t N, int k_lo, const void* ctx_in, float* d_ctx_out, double* loss_mean,
                            void* ws, cudaStream_t s);
size_t flow_log_prob_ws(const gwx_flow_shape& sh, int64_t B, int D, int64_t N);
cudaError_t flow_log_prob(const gwx_flow_shape& sh, const float* params, const void* params_bf16, const double* mean8,
                          const double* scale8, const float* y, const double* theta, int64_t B, int D, int64_t N,
                          int k_lo, const void* ctx_in, double* log_q, void* ws, cudaStream_t s);
size_t flow_sample_ws(const gwx_flow_shape& sh, int64_t E, int D, int64_t N, int64_t S);
cudaError_t flow_sample(const gwx_flow_shape& sh, const float* params, const void* params_bf16, const double* mean8,
                        const double* scale8, const gwx_prior& pr, const float* y, int64_t E, int D, int64_t N,
                        int k_lo, const void* ctx_in, const int64_t* off, int64_t S,
                        uint64_t seed, uint32_t counter, double* theta, double* log_q, double* log_ratio, void* ws,
                        cudaStream_t s);
// The flow's sky density at the HEALPix (nested) pixel centres of nside, the other
// coordinates at the draw of largest log_q among theta [GWX_NPARAM][S]; map [12 nside^2].
size_t flow_skymap_ws(const gwx_flow_shape& sh, int D, int64_t N, int nside);
cudaError_t flow_skymap(const gwx_flow_shape& sh, const float* params, const void* params_bf16, const double* mean8,
                        const double* scale8, const float* y, int D, int64_t N, int k_lo, const void* ctx_in,
                        const double* theta, const double* log_q, int64_t S, int nside, double* map, void* ws,
                        cudaStream_t s);

// HEALPix sky map of weighted samples (k_skymap.cu); ws holds one double.
cudaError_t launch_skymap(const double* theta, const double* weights, int64_t S, int nside, double* map, void* ws,
                          cudaStream_t s);

// VICReg pre-training (k_vicreg.cu).
bool vicreg_supported(int B, int d);
cudaError_t launch_vicreg(const float* x, const float* xp, int B, int d, double l1, double l2, double l3,
                          double* loss, double* terms, float* gx, float* gxp, cudaStream_t s);
cudaError_t launch_retime(const double* in, double* out, int64_t B, double tc_lo, double tc_hi, uint64_t seed,
                          uint32_t counter, cudaStream_t s);

// ResNet-1D pieces (k_resnet.cu).
cudaError_t launch_im2col(const void* x, int64_t B, int T, int C, int k, int s, int p, int K, void* cols,
                          cudaStream_t st);
cudaError_t launch_im2col_cf(const float* y, int64_t B, int D, int N, int k, int s, int p, int K, void* cols,
                             cudaStream_t st);
cudaError_t launch_col2im(const float* dcols, int64_t B, int T, int C, int k, int s, int p, int K, const float* addend,
                          float* dx, cudaStream_t st);
cudaError_t launch_group_norm(const float* z, int64_t B, int T, int C, int G, const float* gamma, const float* beta,
                              const float* res32, const void* res16, int relu, void* out16, float* out32, float* ms,
                              cudaStream_t st);
size_t group_norm_backward_scratch(int64_t B, int C, int G);
cudaError_t launch_group_norm_backward(const float* dy, const float* z, int64_t B, int T, int C, int G,
                                       const float* ms, const float* gamma, void* scratch, float* dz, float* dgamma,
                                       float* dbeta, cudaStream_t st);
cudaError_t launch_relu_mask(const float* dy, const void* out, int64_t n, float* d, cudaStream_t st);
cudaError_t launch_maxpool(const void* x, int64_t B, int T, int C, void* y, uint8_t* arg, cudaStream_t st);
cudaError_t launch_maxpool_back(const float* dy, const uint8_t* arg, int64_t B, int T, int C, float* dx,
                                cudaStream_t st);
cudaError_t launch_mean_time(const void* x, int64_t B, int T, int C, void* m, cudaStream_t st);
cudaError_t launch_mean_time_back(const float* dm, int64_t B, int T, int C, float* dx, cudaStream_t st);

// Record msg as the calling thread's gwx_last_error() message; returns status.
int set_last_error(int status, const char* msg);

// The argument checks of gwx_whiten (sizes, band, NULL and alignment of d, psd, y;
// everything but the workspace), with gwx_whiten's statuses and messages; *k_lo gets
// the first band bin.
int whiten_check_args(const float* d, const double* psd, int64_t seg_len, double fs, double f_lo, int64_t B, int D,
                      int64_t N, const float* y, int* k_lo);
// gwx_init's per-device set-up; on failure the message names the failing step.
int init_device();
// GWX_OK for cudaSuccess, else GWX_ECUDA with "what: <CUDA error name> (<string>)".
int launch_status(cudaError_t e, const char* what);

// Debug build: each checked translation unit's first out-of-range access (read and
// cleared); zero when none, and always zero in the normal build.
cudaError_t debug_take_fused(unsigned long long* v);
cudaError_t debug_take_waveform(unsigned long long* v);

// per-translation-unit table set-up on the current device
cudaError_t init_tables_random();
cudaError_t init_tables_spectral();
cudaError_t init_tables_waveform();
cudaError_t init_tables_fused();

}  // namespace gwx
