"""Workload descriptions and seeded test-input generators.

This module holds data only: the shapes, prior ranges and seeds of the
synthetic workloads, and numpy-seeded generators of arbitrary test inputs.  It
contains none of the method's arithmetic, so both the CUDA path's tests and the
CPU oracle may take their inputs from it without sharing any computation.

Workloads (synthetic stand-ins for the paper's real O3 HL background, Sec. 3.2):

* ``small``  -- TaylorF2, H1+L1, fs = 1024 Hz, 2 s windows (N = 2048),
  f_lo = 20 Hz, 64 draws; background 16 s, Welch with 1 s Hann segments and
  50 % overlap.  Masses U[10, 50], spins U[-0.5, 0.5], distance U[200, 2000] Mpc.
* ``hl3``    -- H1+L1+V1, fs = 2048 Hz, 4 s windows (N = 8192), 2048 draws;
  background 64 s, Welch with 2 s segments, 50 % overlap.  Masses U[5, 100],
  spins U[-0.99, 0.99], distance U[100, 3000] Mpc.
* ``sweep``  -- H1+L1+V1, fs = 2048 Hz, 8 s windows (N = 16384), 8192 draws;
  background 128 s, Welch with 2 s segments, 50 % overlap, ``small``'s priors.
* ``small_nonspinning`` -- ``small`` with spins fixed at zero, 512 draws: the
  learned part's training batches and the events its posteriors are judged on.

All: isotropic sky and orientation, phase and polarisation U[0, 2 pi), merger
time U[T/2, 3T/4] within the window, parameter seed 1, noise seed 2.
"""
import math

import numpy as np

TWO_PI = 2.0 * math.pi


def _prior(m, chi, d, T):
    return {"m_lo": m[0], "m_hi": m[1], "chi_lo": chi[0], "chi_hi": chi[1],
            "d_lo": d[0], "d_hi": d[1], "tc_lo": 0.5 * T, "tc_hi": 0.75 * T,
            "phi_lo": 0.0, "phi_hi": TWO_PI, "psi_lo": 0.0, "psi_hi": TWO_PI}


def _workload(name, B, dets, fs, T, L_seconds, seg_seconds, prior):
    N = int(round(fs * T))
    M = int(round(fs * seg_seconds))
    return {"name": name, "B": B, "dets": tuple(dets), "fs": float(fs), "T": float(T), "N": N,
            "L": int(round(fs * L_seconds)), "seg_len": M, "seg_stride": M // 2,
            "f_lo": 20.0, "gmst": 0.0, "param_seed": 1, "noise_seed": 2, "prior": prior}


WORKLOADS = {
    "small": _workload("small", 64, ("H1", "L1"), 1024, 2.0, 16, 1.0,
                       _prior((10.0, 50.0), (-0.5, 0.5), (200.0, 2000.0), 2.0)),
    "hl3": _workload("hl3", 2048, ("H1", "L1", "V1"), 2048, 4.0, 64, 2.0,
                     _prior((5.0, 100.0), (-0.99, 0.99), (100.0, 3000.0), 4.0)),
    "sweep": _workload("sweep", 8192, ("H1", "L1", "V1"), 2048, 8.0, 128, 2.0,
                       _prior((10.0, 50.0), (-0.5, 0.5), (200.0, 2000.0), 8.0)),
    # the learned part's generator and the events it is judged on: ``small`` with
    # non-spinning sources (the paper's estimator has no spin parameters)
    "small_nonspinning": _workload("small_nonspinning", 512, ("H1", "L1"), 1024, 2.0, 16, 1.0,
                                   _prior((10.0, 50.0), (0.0, 0.0), (200.0, 2000.0), 2.0)),
}


def tc_grid(wl, oversample=16):
    """(tc_lo, n_tc, oversample) of the merger-time marginal over the workload's prior
    window [tc_lo, tc_hi): n_tc = (tc_hi - tc_lo) fs samples."""
    p = wl["prior"]
    return p["tc_lo"], int(round((p["tc_hi"] - p["tc_lo"]) * wl["fs"])), int(oversample)


def workload(name, **overrides):
    wl = dict(WORKLOADS[name])
    wl.update(overrides)
    return wl


def resampled(name, fs, T):
    """Workload `name` at sampling rate fs and window T (N = fs T), with its detectors,
    priors (merger time in [T/2, 3T/4)), background and Welch segment lengths in seconds."""
    base = WORKLOADS[name]
    p = base["prior"]
    prior = _prior((p["m_lo"], p["m_hi"]), (p["chi_lo"], p["chi_hi"]), (p["d_lo"], p["d_hi"]), T)
    return _workload("%s_%g_%g" % (name, fs, T), base["B"], base["dets"], fs, T, base["L"] / base["fs"],
                     base["seg_len"] / base["fs"], prior)


# ---------------------------------------------------------------------------
# Seeded arbitrary inputs (numpy generator; independent of the method's Philox)
# ---------------------------------------------------------------------------

def random_theta(seed, B, prior, T=None):
    """theta [11][B] float64 uniformly inside the prior box (angles in their natural ranges)."""
    rng = np.random.default_rng(seed)
    th = np.empty((11, B))
    th[0] = rng.uniform(prior["m_lo"], prior["m_hi"], B)
    th[1] = rng.uniform(prior["m_lo"], prior["m_hi"], B)
    th[2] = rng.uniform(prior["chi_lo"], prior["chi_hi"], B)
    th[3] = rng.uniform(prior["chi_lo"], prior["chi_hi"], B)
    th[4] = rng.uniform(prior["d_lo"], prior["d_hi"], B)
    th[5] = rng.uniform(prior["tc_lo"], prior["tc_hi"], B)
    th[6] = rng.uniform(0.0, TWO_PI, B)
    th[7] = rng.uniform(0.0, math.pi, B)
    th[8] = rng.uniform(0.0, TWO_PI, B)
    th[9] = rng.uniform(0.0, TWO_PI, B)
    th[10] = rng.uniform(-0.5 * math.pi, 0.5 * math.pi, B)
    return th


def random_strain(seed, shape, scale=1e-21):
    """White Gaussian float64 array of the given shape and standard deviation."""
    return np.random.default_rng(seed).normal(0.0, scale, shape)


def random_offsets(seed, B, L, N):
    return np.random.default_rng(seed).integers(0, L - N + 1, B).astype(np.int64)


def ragged_counts(seed, E, lo, hi, zeros=0):
    """Per-event sample counts ~ U{lo..hi}; the first ``zeros`` events get none."""
    c = np.random.default_rng(seed).integers(lo, hi + 1, E).astype(np.int64)
    c[:zeros] = 0
    return c


def random_bf16_bits(seed, shape, exp_lo=-8, exp_hi=1):
    """Random bfloat16 values as their 16-bit patterns (uint16): random sign, exponent
    in [exp_lo, exp_hi] and mantissa bits.  Both sides decode the same bits."""
    rng = np.random.default_rng(seed)
    sign = rng.integers(0, 2, shape).astype(np.uint16) << 15
    exp = (rng.integers(exp_lo, exp_hi + 1, shape) + 127).astype(np.uint16) << 7
    man = rng.integers(0, 128, shape).astype(np.uint16)
    return (sign | exp | man).astype(np.uint16)


def flow_shape(features=64, group=8, embed_hidden=64, context=32, layers=4, hidden=64):
    """Sizes of the conditional flow: spectral-feature columns F, bins per feature group G,
    embedding hidden width H_e, context width C, coupling layers K, conditioner width H."""
    return {"features": features, "group": group, "embed_hidden": embed_hidden, "context": context,
            "layers": layers, "hidden": hidden}


def flow_tensor_shapes(shape):
    """The flow's parameter tensors in storage order: the embedding's three dense layers
    (weight [out][in], bias [out]), then per coupling layer its conditioner's three."""
    F, He, C = shape["features"], shape["embed_hidden"], shape["context"]
    H, K = shape["hidden"], shape["layers"]
    out = [(He, F), (He,), (He, He), (He,), (C, He), (C,)]
    for _ in range(K):
        out += [(H, 8 + C), (H,), (H, H), (H,), (8, H), (8,)]
    return out


def random_flow_params(seed, shape, gain=1.0, last_gain=0.5):
    """Random flow parameters as float32 arrays whose weights are exactly representable in
    bfloat16 (low 16 bits cleared): weights N(0, gain^2 / fan_in), the last layer of every
    conditioner scaled by last_gain, biases N(0, 0.1^2) (not rounded)."""
    rng = np.random.default_rng(seed)
    out = []
    shapes = flow_tensor_shapes(shape)
    for i, s in enumerate(shapes):
        if len(s) == 2:
            g = gain * (last_gain if (i >= 6 and i % 6 == 4) else 1.0)
            w = (rng.normal(0.0, g / math.sqrt(s[1]), s)).astype(np.float32)
            w = (w.view(np.uint32) & np.uint32(0xFFFF0000)).view(np.float32)
            out.append(w)
        else:
            out.append(rng.normal(0.0, 0.1, s).astype(np.float32))
    return out
