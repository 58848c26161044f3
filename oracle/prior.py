"""Prior draws for one batch (oracle; test infrastructure).

Sec. 3.2: each training step draws N points from the parameter prior and
generates one waveform per point.  Table 1 lists the paper's prior (chirp mass,
mass ratio, volumetric distance, isotropic orientation and sky, uniform phase
and polarisation).  The workloads here draw component masses, aligned spins and
distance uniformly between configured bounds (the configured ranges replace
Table 1's shapes; the angles keep Table 1's shapes):

* m1, m2        ~ U[m_lo, m_hi]            (independent; no ordering imposed)
* chi1, chi2    ~ U[chi_lo, chi_hi]
* distance      ~ U[d_lo, d_hi]  Mpc
* tc            ~ U[tc_lo, tc_hi] s        (geocentre merger time within the window)
* phic          ~ U[phi_lo, phi_hi]
* theta_jn      = arccos(1 - 2u)           (Table 1: "Sine(0, pi)")
* psi           ~ U[psi_lo, psi_hi]
* ra            = 2 pi u                   (Table 1: "Uniform(0, 2 pi)")
* dec           = arcsin(2u - 1)           (Table 1: "Cosine(-pi/2, pi/2)")
* crop offset   ~ U{0, ..., L - N}         (Sec. 3.2: N lazy crops of the background)

Draw b uses Philox counters (b, j, TAG_PRIOR, step) for j = 0..5; block j gives
uniforms u_{2j} (words 0,1) and u_{2j+1} (words 2,3), except block 5 whose
words 2 is the crop offset (multiply-shift) and 3 is unused.
"""
import math
import numpy as np

from . import constants as C
from .philox import TAG_PRIOR, bounded_index, key_of, philox4x32_10, uniform52


def sample_prior(prior, seed, step, B, L, N):
    """Return (theta [P][B] float64, offsets [B] int64) for draws 0..B-1 of one step.

    prior: dict with keys m_lo, m_hi, chi_lo, chi_hi, d_lo, d_hi, tc_lo, tc_hi,
    phi_lo, phi_hi, psi_lo, psi_hi.  L is the background length and N the window
    length in samples (offsets lie in [0, L - N]).
    """
    k0, k1 = key_of(seed)
    idx = np.arange(B, dtype=np.uint64).astype(np.uint32)
    u = []
    offsets = None
    for j in range(6):
        w = philox4x32_10(idx, np.uint32(j), np.uint32(TAG_PRIOR), np.uint32(step & 0xFFFFFFFF), k0, k1)
        u.append(uniform52(w[0], w[1]))
        if j < 5:
            u.append(uniform52(w[2], w[3]))
        else:
            offsets = bounded_index(w[2], L - N + 1)

    def lin(lo, hi, x):
        return lo + (hi - lo) * x

    theta = np.empty((C.P, B), dtype=np.float64)
    theta[C.M1] = lin(prior["m_lo"], prior["m_hi"], u[0])
    theta[C.M2] = lin(prior["m_lo"], prior["m_hi"], u[1])
    theta[C.CHI1] = lin(prior["chi_lo"], prior["chi_hi"], u[2])
    theta[C.CHI2] = lin(prior["chi_lo"], prior["chi_hi"], u[3])
    theta[C.DIST] = lin(prior["d_lo"], prior["d_hi"], u[4])
    theta[C.TC] = lin(prior["tc_lo"], prior["tc_hi"], u[5])
    theta[C.PHIC] = lin(prior["phi_lo"], prior["phi_hi"], u[6])
    theta[C.THETAJN] = np.arccos(1.0 - 2.0 * u[7])
    theta[C.PSI] = lin(prior["psi_lo"], prior["psi_hi"], u[8])
    theta[C.RA] = 2.0 * math.pi * u[9]
    theta[C.DEC] = np.arcsin(2.0 * u[10] - 1.0)
    return theta, offsets
