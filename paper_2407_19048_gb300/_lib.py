"""ctypes declarations of the libgwx C ABI (``include/gwx.h``).

Loading fails loudly when the shared library has not been built: there is no
fallback implementation of any entry point.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
# GWX_DEBUG=1 loads the debug build (index checks in the hot kernels, workspace guards in
# the binding); it must have been built with build(debug=True)
DEBUG = os.environ.get("GWX_DEBUG", "0") not in ("", "0")
LIB_PATH = os.path.join(HERE, "libgwx_debug.so" if DEBUG else "libgwx.so")

c_i64 = ctypes.c_int64
c_u64 = ctypes.c_uint64
c_u32 = ctypes.c_uint32
c_int = ctypes.c_int
c_dbl = ctypes.c_double
c_size = ctypes.c_size_t
c_vp = ctypes.c_void_p
c_i32p = ctypes.POINTER(ctypes.c_int32)
c_dblp = ctypes.POINTER(ctypes.c_double)


class GwxPrior(ctypes.Structure):
    _fields_ = [(name, c_dbl) for name in (
        "m_lo", "m_hi", "chi_lo", "chi_hi", "d_lo", "d_hi",
        "tc_lo", "tc_hi", "phi_lo", "phi_hi", "psi_lo", "psi_hi")]


class GwxFlowShape(ctypes.Structure):
    _fields_ = [(name, c_int) for name in ("features", "group", "embed_hidden", "context", "layers", "hidden",
                                              "extra")]


c_shp = ctypes.POINTER(GwxFlowShape)
c_d8 = ctypes.POINTER(c_dbl)
c_pri = ctypes.POINTER(GwxPrior)
c_f32 = ctypes.c_float

# name -> (restype, argtypes)
SIGNATURES = {
    "gwx_version": (c_int, []),
    "gwx_status_string": (ctypes.c_char_p, [c_int]),
    "gwx_last_error": (ctypes.c_char_p, []),
    "gwx_init": (c_int, []),
    "gwx_detector_geometry": (c_int, [c_int, c_dblp, c_dblp]),
    "gwx_sample_prior": (c_int, [ctypes.POINTER(GwxPrior), c_u64, c_u32, c_i64, c_i64, c_i64, c_vp, c_vp, c_vp]),
    "gwx_generate_waveforms": (c_int, [c_int, c_vp, c_i64, c_dbl, c_dbl, c_i64, c_vp, c_vp, c_vp]),
    "gwx_project": (c_int, [c_vp, c_vp, c_vp, c_i64, c_i32p, c_int, c_dbl, c_dbl, c_i64, c_vp, c_vp]),
    "gwx_colored_noise_workspace": (c_size, [c_int, c_i64]),
    "gwx_colored_noise": (c_int, [c_u64, c_u32, c_int, c_i64, c_dbl, c_dbl, c_vp, c_vp, c_size, c_vp]),
    "gwx_welch_psd_workspace": (c_size, [c_int, c_i64, c_i64, c_i64]),
    "gwx_welch_psd": (c_int, [c_vp, c_int, c_i64, c_dbl, c_i64, c_i64, c_vp, c_vp, c_size, c_vp]),
    "gwx_inject": (c_int, [c_vp, c_int, c_i64, c_vp, c_vp, c_i64, c_i64, c_dbl, c_vp, c_vp]),
    "gwx_inject_padded": (c_int, [c_vp, c_int, c_i64, c_vp, c_vp, c_i64, c_i64, c_i64, c_dbl, c_vp, c_vp]),
    "gwx_whiten_workspace": (c_size, [c_int, c_i64]),
    "gwx_whiten": (c_int, [c_vp, c_vp, c_i64, c_dbl, c_dbl, c_i64, c_int, c_i64, c_vp, c_vp, c_size, c_vp]),
    "gwx_unwhiten": (c_int, [c_vp, c_vp, c_i64, c_dbl, c_dbl, c_i64, c_int, c_i64, c_vp, c_vp, c_size, c_vp]),
    "gwx_whiten_static": (c_int, [c_vp, c_vp, c_i64, c_dbl, c_dbl, c_i64, c_int, c_i64, c_vp, c_vp]),
    "gwx_simulate_batch_workspace": (c_size, [c_int, c_i64, c_i64]),
    "gwx_simulate_batch": (c_int, [ctypes.POINTER(GwxPrior), c_u64, c_u32, c_vp, c_i64, c_vp, c_i64, c_dbl, c_dbl,
                                   c_i32p, c_int, c_dbl, c_i64, c_i64, c_vp, c_vp, c_vp, c_vp, c_size, c_vp]),
    "gwx_prepare_batch": (c_int, [ctypes.POINTER(GwxPrior), c_u64, c_u32, c_i64, c_i64, c_dbl, c_dbl, c_i32p, c_int,
                                  c_dbl, c_i64, c_vp, c_vp, c_vp, c_size, c_vp]),
    "gwx_simulate_prepared": (c_int, [c_vp, c_i64, c_vp, c_i64, c_dbl, c_dbl, c_int, c_i64, c_i64, c_vp, c_vp,
                                      c_int, c_vp, c_size, c_vp]),
    "gwx_log_likelihood_workspace": (c_size, [c_i64, c_int, c_i64, c_i64]),
    "gwx_log_likelihood": (c_int, [c_int, c_vp, c_i64, c_int, c_i64, c_vp, c_i64, c_dbl, c_dbl, c_i32p, c_dbl,
                                   c_vp, c_vp, c_i64, c_vp, c_vp, c_size, c_vp]),
    "gwx_conv1d_bf16": (c_int, [c_vp, c_i64, c_i64, c_int, c_int, c_vp, c_int, c_vp, c_vp, c_vp]),
    "gwx_conv1d_bf16_backward_workspace": (c_size, [c_i64, c_i64, c_int, c_int, c_int]),
    "gwx_conv1d_bf16_backward": (c_int, [c_vp, c_vp, c_vp, c_i64, c_i64, c_int, c_int, c_int, c_vp, c_vp, c_vp, c_vp,
                                         c_size, c_vp]),
    "gwx_debug_build": (c_int, []),
    "gwx_debug_status": (c_int, [ctypes.POINTER(c_u64)]),
    "gwx_debug_guard": (c_int, [c_vp, c_size, c_size, c_vp]),
    "gwx_debug_check_guard": (c_int, [c_vp, c_size, c_size, ctypes.POINTER(c_int), c_vp]),
    "gwx_simulate_autotune": (c_int, [c_vp, c_i64, c_vp, c_i64, c_dbl, c_dbl, c_int, c_i64, c_i64, c_vp, c_vp, c_vp,
                                      c_size, ctypes.POINTER(c_int), c_vp]),
    "gwx_simulate_shape": (c_int, [c_i64, c_int, c_int]),
    "gwx_log_likelihood_tmarg": (c_int, [c_int, c_vp, c_i64, c_int, c_i64, c_vp, c_i64, c_dbl, c_dbl, c_i32p,
                                         c_dbl, c_dbl, c_i64, c_int, c_vp, c_vp, c_i64, c_vp, c_vp, c_size, c_vp]),
    "gwx_importance_weights_workspace": (c_size, [c_i64]),
    "gwx_importance_weights": (c_int, [c_vp, c_vp, c_vp, c_i64, c_i64, c_vp, c_vp, c_vp, c_vp, c_vp, c_size, c_vp]),
    "gwx_gemm_bf16": (c_int, [c_vp, c_vp, c_vp, c_i64, c_i64, c_i64, c_int, c_vp]),
    "gwx_dense_bf16": (c_int, [c_vp, c_vp, c_vp, c_vp, c_i64, c_i64, c_i64, c_int, c_int, c_vp]),
    "gwx_dense_bf16_backward_workspace": (c_size, [c_i64, c_i64, c_i64]),
    "gwx_dense_bf16_backward": (c_int, [c_vp, c_vp, c_vp, c_vp, c_i64, c_i64, c_i64, c_int, c_vp, c_vp, c_vp, c_vp,
                                        c_size, c_vp]),
    "gwx_spectral_features_workspace": (c_size, [c_i64, c_int, c_i64]),
    "gwx_spectral_features": (c_int, [c_vp, c_i64, c_int, c_i64, c_dbl, c_dbl, c_int, c_int, c_vp, c_vp, c_size,
                                      c_vp]),
    "gwx_cross_features": (c_int, [c_vp, c_i64, c_int, c_i64, c_dbl, c_dbl, c_int, c_int, c_int, c_vp, c_vp, c_size,
                                   c_vp]),
    "gwx_lag_features": (c_int, [c_vp, c_i64, c_int, c_i64, c_dbl, c_dbl, c_int, c_int, c_int, c_vp, c_vp, c_size,
                                 c_vp]),
    "gwx_proposal_targets": (c_int, [c_vp, c_i64, ctypes.POINTER(c_dbl), ctypes.POINTER(c_dbl), c_vp, c_vp]),
    "gwx_gauss_nll": (c_int, [c_vp, c_int, c_vp, c_int, c_i64, c_vp, c_vp, c_vp, c_vp]),
    "gwx_adamw": (c_int, [c_vp, c_vp, c_vp, c_vp, c_i64, c_dbl, c_dbl, c_dbl, c_dbl, c_dbl, c_i64, c_vp, c_vp]),
    "gwx_adamw_at": (c_int, [c_vp, c_vp, c_vp, c_vp, c_i64, c_dbl, c_dbl, c_dbl, c_dbl, c_dbl, c_vp, c_vp, c_vp]),
    "gwx_adamw_clip_workspace": (c_size, []),
    "gwx_adamw_clip": (c_int, [c_vp, c_vp, c_vp, c_vp, c_i64, c_dbl, c_dbl, c_dbl, c_dbl, c_dbl, c_i64, c_dbl, c_vp,
                               c_vp, c_size, c_vp]),
    "gwx_vicreg": (c_int, [c_vp, c_vp, c_i64, c_int, c_dbl, c_dbl, c_dbl, c_vp, c_vp, c_vp, c_vp, c_vp]),
    "gwx_retime": (c_int, [c_vp, c_vp, c_i64, c_dbl, c_dbl, c_u64, c_u32, c_vp]),
    "gwx_prepare_theta": (c_int, [c_vp, c_i64, c_i64, c_dbl, c_dbl, c_i32p, c_int, c_dbl, c_i64, c_vp, c_size,
                                  c_vp]),
    "gwx_im2col": (c_int, [c_vp, c_i64, c_int, c_int, c_int, c_int, c_int, c_int, c_vp, c_vp]),
    "gwx_im2col_cf": (c_int, [c_vp, c_i64, c_int, c_int, c_int, c_int, c_int, c_int, c_vp, c_vp]),
    "gwx_col2im": (c_int, [c_vp, c_i64, c_int, c_int, c_int, c_int, c_int, c_int, c_vp, c_vp, c_vp]),
    "gwx_group_norm": (c_int, [c_vp, c_i64, c_int, c_int, c_int, c_vp, c_vp, c_vp, c_vp, c_int, c_vp, c_vp, c_vp,
                               c_vp]),
    "gwx_group_norm_backward": (c_int, [c_vp, c_vp, c_i64, c_int, c_int, c_int, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp,
                                        c_vp]),
    "gwx_group_norm_backward_scratch": (c_size, [c_i64, c_int, c_int]),
    "gwx_relu_mask": (c_int, [c_vp, c_vp, c_i64, c_vp, c_vp]),
    "gwx_maxpool": (c_int, [c_vp, c_i64, c_int, c_int, c_vp, c_vp, c_vp]),
    "gwx_maxpool_backward": (c_int, [c_vp, c_vp, c_i64, c_int, c_int, c_vp, c_vp]),
    "gwx_mean_time": (c_int, [c_vp, c_i64, c_int, c_int, c_vp, c_vp]),
    "gwx_mean_time_backward": (c_int, [c_vp, c_i64, c_int, c_int, c_vp, c_vp]),
    "gwx_skymap_workspace": (c_size, []),
    "gwx_skymap": (c_int, [c_vp, c_vp, c_i64, c_int, c_vp, c_vp, c_size, c_vp]),
    "gwx_sample_proposal": (c_int, [c_vp, c_int, ctypes.POINTER(c_dbl), ctypes.POINTER(c_dbl),
                                    ctypes.POINTER(GwxPrior), c_vp, c_i64, c_vp, c_i64, c_u64, c_u32, c_int, c_vp, c_vp,
                                    c_vp]),
    "gwx_gemm_autotune": (c_int, [c_vp, c_vp, c_vp, c_i64, c_i64, c_i64, c_int, c_vp, c_vp]),
    "gwx_device_status": (c_int, []),
    "gwx_selftest_bounded_wait": (c_int, [c_u32, c_vp]),
    "gwx_rfft": (c_int, [c_vp, c_i64, c_i64, c_vp, c_vp]),
    "gwx_irfft": (c_int, [c_vp, c_i64, c_i64, c_vp, c_vp]),
    "gwx_flow_layout": (c_int, [c_shp, ctypes.POINTER(c_i64), ctypes.POINTER(c_i64)]),
    "gwx_flow_targets": (c_int, [c_vp, c_i64, c_d8, c_d8, c_vp, c_vp]),
    "gwx_flow_conditioner_input": (c_int, [c_int, c_vp, c_vp, c_int, c_vp, c_i64, c_i64, c_i64, c_vp, c_vp]),
    "gwx_flow_coupling": (c_int, [c_int, c_int, c_vp, c_vp, c_i64, c_vp, c_vp, c_int, c_vp]),
    "gwx_flow_nll": (c_int, [c_vp, c_vp, c_i64, c_vp, c_vp, c_vp, c_vp]),
    "gwx_flow_coupling_backward": (c_int, [c_int, c_vp, c_vp, c_vp, c_i64, c_f32, c_vp, c_vp, c_vp]),
    "gwx_flow_input_backward": (c_int, [c_int, c_vp, c_int, c_i64, c_vp, c_vp, c_int, c_vp]),
    "gwx_flow_base": (c_int, [c_u64, c_u32, c_i64, c_i64, c_vp, c_vp]),
    "gwx_flow_proposal": (c_int, [c_vp, c_vp, c_vp, c_i64, c_d8, c_d8, c_pri, c_u64, c_u32, c_vp, c_vp, c_vp,
                                  c_vp]),
    "gwx_flow_train_workspace": (c_size, [c_shp, c_i64, c_int, c_i64]),
    "gwx_flow_train_step": (c_int, [c_shp, c_vp, c_vp, c_vp, c_vp, c_vp, c_i64, c_vp, c_dbl, c_dbl, c_dbl, c_dbl, c_dbl,
                                    c_dbl, c_d8, c_d8, c_vp, c_vp, c_i64, c_int, c_i64, c_dbl, c_dbl, c_vp, c_vp, c_vp,
                                    c_vp, c_size, c_vp]),
    "gwx_flow_log_prob_workspace": (c_size, [c_shp, c_i64, c_int, c_i64]),
    "gwx_flow_log_prob": (c_int, [c_shp, c_vp, c_vp, c_d8, c_d8, c_vp, c_vp, c_i64, c_int, c_i64, c_dbl, c_dbl, c_vp,
                                  c_vp, c_vp, c_size, c_vp]),
    "gwx_sample_posterior_workspace": (c_size, [c_shp, c_i64, c_int, c_i64, c_i64]),
    "gwx_flow_skymap_workspace": (c_size, [c_shp, c_int, c_i64, c_int]),
    "gwx_flow_skymap": (c_int, [c_shp, c_vp, c_vp, c_d8, c_d8, c_vp, c_int, c_i64, c_dbl, c_dbl, c_vp, c_vp, c_vp,
                                c_i64, c_int, c_vp, c_vp, c_size, c_vp]),
    "gwx_sample_posterior": (c_int, [c_shp, c_vp, c_vp, c_d8, c_d8, c_pri, c_vp, c_i64, c_int, c_i64, c_dbl, c_dbl,
                                     c_vp, c_vp, c_i64, c_u64, c_u32, c_vp, c_vp, c_vp, c_vp, c_size, c_vp]),
}

_lib = None


def load():
    """Return the loaded libgwx (raises RuntimeError if it is missing or incomplete)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(
            "libgwx.so is not built (%s). Run `python -m paper_2407_19048_gb300.build` or "
            "`__graft_entry__.build()`; there is no CPU fallback." % LIB_PATH)
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)          # AttributeError if the library lacks a symbol
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib
