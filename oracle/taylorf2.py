"""TaylorF2 frequency-domain inspiral waveform (oracle; test infrastructure).

Sec. 3.1: the paper's IMRPhenomD builds on the inspiral phase to 3.5
post-Newtonian order, the TaylorF2 model (reviewed by Buonanno et al. 2009).  This
module evaluates that TaylorF2 model directly from its
definition, bin by bin, in float64:

    h(f)  = A(f) exp(-i Psi(f))
    A(f)  = sqrt(5/24) pi^(-2/3) Mc^(5/6) f^(-7/6) / D                 (leading order)
    Psi(f) = 2 pi f tc - phic - pi/4 + 3 / (128 eta v^5) sum_{j=0..7} alpha_j v^j,
    v     = (pi M f)^(1/3)

(Buonanno, Iyer, Ochsner, Pan, Sathyaprakash 2009, Phys. Rev. D 80, 084043,
eq. 3.18 for the non-spinning alpha_j), with masses as times (G M / c^3) and
D as a time (D / c).  alpha_5 carries (1 + 3 ln v) and alpha_6 carries ln(4v).
The aligned-spin 1.5PN spin-orbit term adds 4 beta to alpha_3, with
beta = (1/12) sum_i chi_i (113 m_i^2 / M^2 + 75 eta) (Poisson & Will 1995),
written below in the symmetric/antisymmetric spins chi_s, chi_a.

Polarisations of the (2,2) mode for aligned spins, inclination iota = theta_jn:
    h_plus  = A (1 + cos^2 iota)/2 exp(-i Psi)
    h_cross = -i A cos(iota) exp(-i Psi)

Readings (the paper states none of these):
* The waveform is generated with tc = 0 (merger at the time origin); the
  geocentre merger time tc and the detector delay are applied together by the
  projection step (``detector.project``).
* Support: bins k with ceil(f_lo/df) <= k <= floor(f_isco/df) are non-zero,
  f_isco = 1 / (6^(3/2) pi M); all other bins are exactly zero.
* Spin terms beyond 1.5PN spin-orbit are not included ("parity unpinned" for
  them is moot: neither side implements them).
"""
import math
import numpy as np

from . import constants as C


def phase_coefficients(eta, delta, chis, chia, pn_order=7):
    """Return (a, l): alpha_j(v) = a[j] + l[j] ln v for j = 0..7, zero above pn_order.

    pn_order is twice the PN order kept (0 = Newtonian, 7 = 3.5PN).
    """
    pi = math.pi
    eta = np.asarray(eta, dtype=np.float64)
    z = np.zeros_like(eta)
    a = [z + 1.0,
         z,
         3715.0 / 756.0 + 55.0 * eta / 9.0,
         -16.0 * pi + (113.0 / 3.0) * delta * chia + (113.0 / 3.0 - 76.0 * eta / 3.0) * chis,
         15293365.0 / 508032.0 + 27145.0 * eta / 504.0 + 3085.0 * eta ** 2 / 72.0,
         pi * (38645.0 / 756.0 - 65.0 * eta / 9.0),
         (11583231236531.0 / 4694215680.0 - 640.0 * pi ** 2 / 3.0
          - 6848.0 * C.EULER_GAMMA / 21.0 - 6848.0 * math.log(4.0) / 21.0
          + (-15737765635.0 / 3048192.0 + 2255.0 * pi ** 2 / 12.0) * eta
          + 76055.0 * eta ** 2 / 1728.0 - 127825.0 * eta ** 3 / 1296.0),
         pi * (77096675.0 / 254016.0 + 378515.0 * eta / 1512.0 - 74045.0 * eta ** 2 / 756.0)]
    l = [z, z, z, z, z,
         3.0 * pi * (38645.0 / 756.0 - 65.0 * eta / 9.0),
         z - 6848.0 / 21.0,
         z]
    for j in range(pn_order + 1, 8):
        a[j] = z
        l[j] = z
    return a, l


def mass_terms(m1, m2, chi1, chi2):
    """Total mass M [s], chirp mass Mc [s], eta, delta, chi_s, chi_a."""
    M = (m1 + m2) * C.MTSUN_S
    eta = m1 * m2 / (m1 + m2) ** 2
    Mc = M * eta ** 0.6
    delta = (m1 - m2) / (m1 + m2)
    chis = 0.5 * (chi1 + chi2)
    chia = 0.5 * (chi1 - chi2)
    return M, Mc, eta, delta, chis, chia


def support(theta, f_lo, df, F):
    """Boolean [B][F] mask of the non-zero bins (reading stated in the module docstring)."""
    M = (theta[C.M1] + theta[C.M2]) * C.MTSUN_S
    f_isco = 1.0 / (6.0 ** 1.5 * math.pi * M)
    k_lo = math.ceil(f_lo / df)
    k_hi = np.floor(f_isco / df)
    k = np.arange(F)
    return (k[None, :] >= k_lo) & (k[None, :] <= k_hi[:, None])


def phase(theta, f, pn_order=7):
    """Psi(f) [B][len(f)] with tc = 0, for f > 0."""
    M, Mc, eta, delta, chis, chia = mass_terms(theta[C.M1], theta[C.M2], theta[C.CHI1], theta[C.CHI2])
    a, l = phase_coefficients(eta, delta, chis, chia, pn_order)
    v = np.cbrt(math.pi * M[:, None] * f[None, :])
    lnv = np.log(v)
    s = np.zeros_like(v)
    for j in range(8):
        s += (a[j][:, None] + l[j][:, None] * lnv) * v ** j
    return -theta[C.PHIC][:, None] - math.pi / 4.0 + 3.0 / (128.0 * eta[:, None] * v ** 5) * s


def amplitude(theta, f):
    """Leading-order amplitude A(f) [B][len(f)] (strain per Hz)."""
    M, Mc, eta, delta, chis, chia = mass_terms(theta[C.M1], theta[C.M2], theta[C.CHI1], theta[C.CHI2])
    D = theta[C.DIST] * C.MPC_M / C.C_MS
    return (math.sqrt(5.0 / 24.0) * math.pi ** (-2.0 / 3.0)
            * (Mc ** (5.0 / 6.0) / D)[:, None] * f[None, :] ** (-7.0 / 6.0))


def generate_waveforms(theta, f_lo, df, F, pn_order=7):
    """h_plus, h_cross [B][F] complex128 on the grid f_k = k df, k = 0..F-1 (tc = 0)."""
    theta = np.asarray(theta, dtype=np.float64)
    B = theta.shape[1]
    hp = np.zeros((B, F), dtype=np.complex128)
    hc = np.zeros((B, F), dtype=np.complex128)
    mask = support(theta, f_lo, df, F)
    if B == 0 or not mask.any():
        return hp, hc
    f = np.arange(F, dtype=np.float64) * df
    f[0] = df  # placeholder to keep the formulas finite; bin 0 is outside the support
    A = amplitude(theta, f)
    psi = phase(theta, f, pn_order)
    base = A * np.exp(-1j * psi)
    ci = np.cos(theta[C.THETAJN])[:, None]
    hp[mask] = (base * (0.5 * (1.0 + ci ** 2)))[mask]
    hc[mask] = (base * (-1j * ci))[mask]
    return hp, hc
