"""Pins for the oracle's TaylorF2 waveform (CPU only).

Each check ties the oracle to something other than its own formulas: the
quadrupole chirp and the stationary-phase approximation, Kepler's law, the
post-Newtonian energy balance, exact symmetries, and a numerically Fourier
transformed time-domain chirp.
"""
import math

import numpy as np
import pytest

from oracle import taylorf2
from oracle import constants as C

MSUN = C.MTSUN_S


def theta_of(m1, m2, chi1=0.0, chi2=0.0, dist=1000.0, phic=0.0, iota=0.0, B=1):
    th = np.zeros((C.P, B))
    th[C.M1], th[C.M2], th[C.CHI1], th[C.CHI2] = m1, m2, chi1, chi2
    th[C.DIST], th[C.PHIC], th[C.THETAJN] = dist, phic, iota
    return th


def chirp_mass_s(m1, m2):
    return (m1 * m2) ** 0.6 / (m1 + m2) ** 0.2 * MSUN


def newtonian_td(Mc, tau):
    """Quadrupole chirp: GW frequency and phase offset (phase - phic) at time tau before merger."""
    f = (1.0 / math.pi) * (5.0 / (256.0 * tau)) ** 0.375 * Mc ** -0.625
    dphi = -2.0 * (tau / (5.0 * Mc)) ** 0.625
    return f, dphi


def tau_of_f(Mc, f):
    """Invert newtonian_td's f(tau) numerically by bisection (no closed form used)."""
    lo, hi = 1e-9, 1e6
    for _ in range(200):
        mid = math.sqrt(lo * hi)
        if newtonian_td(Mc, mid)[0] > f:
            lo = mid
        else:
            hi = mid
    return math.sqrt(lo * hi)


def test_amplitude_law_and_spa_value():
    m1, m2, dist = 23.0, 11.0, 750.0
    th = theta_of(m1, m2, dist=dist)
    df = 0.25
    hp, hc = taylorf2.generate_waveforms(th, 20.0, df, 4097)
    f = np.arange(4097) * df
    on = np.abs(hp[0]) > 0
    amp = np.abs(hp[0][on]) * f[on] ** (7.0 / 6.0)
    assert np.ptp(amp) / amp.mean() < 1e-12
    # stationary phase on the quadrupole chirp: |h~| = (A_t / 2) / sqrt(df/dt),
    # A_t = 4 Mc^(5/3) (pi f)^(2/3) / D, df/dt from differentiating f(tau)
    Mc = chirp_mass_s(m1, m2)
    D = dist * C.MPC_M / C.C_MS
    for fk in (25.0, 60.0, 110.0):
        tau = tau_of_f(Mc, fk)
        eps = tau * 1e-6
        fdot = (newtonian_td(Mc, tau - eps)[0] - newtonian_td(Mc, tau + eps)[0]) / (2 * eps)
        At = 4.0 * Mc ** (5.0 / 3.0) * (math.pi * fk) ** (2.0 / 3.0) / D
        spa = 0.5 * At / math.sqrt(fdot)
        k = int(round(fk / df))
        assert abs(abs(hp[0][k]) / spa - 1.0) < 1e-7


@pytest.mark.parametrize("m,expect_rad", [(10.0, 449.0), (5.0, 1426.0)])
def test_newtonian_phase_limit(m, expect_rad):
    th = theta_of(m, m, phic=0.3)
    Mc = chirp_mass_s(m, m)
    f = np.array([20.0, 35.0, 80.0])
    psi = taylorf2.phase(th, f, pn_order=0)[0]
    for i, fk in enumerate(f):
        tau = tau_of_f(Mc, fk)
        # Psi(f) = 2 pi f t_f - Phi(t_f) - pi/4 with tc = 0, Phi(t) = phic + dphi(tau)
        spa = 2 * math.pi * fk * (-tau) - (0.3 + newtonian_td(Mc, tau)[1]) - math.pi / 4
        assert abs(psi[i] - spa) < 1e-6 * abs(spa)
    assert abs(psi[0] + 0.3 + math.pi / 4 - expect_rad) < 1.0


def test_group_delay_newtonian():
    th = theta_of(10.0, 10.0)
    Mc = chirp_mass_s(10.0, 10.0)
    for fk in (20.0, 40.0, 100.0):
        h = fk * 1e-5
        p = taylorf2.phase(th, np.array([fk - h, fk + h]), pn_order=0)[0]
        tg = (p[1] - p[0]) / (2 * h) / (2 * math.pi)
        assert abs(tg + tau_of_f(Mc, fk)) < 1e-6 * tau_of_f(Mc, fk)
    h = 20e-5
    p = taylorf2.phase(th, np.array([20 - h, 20 + h]), pn_order=0)[0]
    assert abs(-(p[1] - p[0]) / (2 * h) / (2 * math.pi) - 5.96) < 0.01


def energy_balance_alphas(eta, delta, chis, chia):
    """alpha_j (non-log a_j and ln v coefficients l_j) derived from the PN binding
    energy E(v) and flux F(v) (Blanchet, Living Rev. Rel. 17, 2 (2014)) by the
    stationary-phase energy balance: dt/dv = -E'/F, dphi/dv = v^3 dt/dv / M,
    Psi = 2 v^3 t / M - 2 phi, expanded to relative order v^7 and integrated term by
    term.  Spin enters E and F at 1.5PN (spin-orbit) only."""
    pi, g = math.pi, C.EULER_GAMMA
    e = {2: -0.75 - eta / 12, 3: (8 / 3 - 4 * eta / 3) * chis + 8 / 3 * delta * chia,
         4: -27 / 8 + 19 * eta / 8 - eta ** 2 / 24,
         6: -675 / 64 + (34445 / 576 - 205 * pi ** 2 / 96) * eta - 155 * eta ** 2 / 96 - 35 * eta ** 3 / 5184}
    num = np.zeros((8, 2))          # -E'/(eta M v) as (value, ln v coefficient) per order
    num[0, 0] = 1.0
    for k, val in e.items():
        num[k, 0] = (k + 2) / 2 * val
    den = np.zeros((8, 2))          # F / (32/5 eta^2 v^10)
    den[0, 0] = 1.0
    den[2, 0] = -1247 / 336 - 35 * eta / 12
    den[3, 0] = 4 * pi - ((11 / 4 - 3 * eta) * chis + 11 / 4 * delta * chia)
    den[4, 0] = -44711 / 9072 + 9271 * eta / 504 + 65 * eta ** 2 / 18
    den[5, 0] = -(8191 / 672 + 583 * eta / 24) * pi
    den[6, 0] = (6643739519 / 69854400 + 16 * pi ** 2 / 3 - 1712 * g / 105 - 856 / 105 * math.log(16)
                 + (-134543 / 7776 + 41 * pi ** 2 / 48) * eta - 94403 * eta ** 2 / 3024 - 775 * eta ** 3 / 324)
    den[6, 1] = -1712 / 105         # from -(856/105) ln(16 v^2)
    den[7, 0] = (-16285 / 504 + 214745 * eta / 1728 + 193385 * eta ** 2 / 3024) * pi
    q = np.zeros((8, 2))            # series quotient tau_k
    for k in range(8):
        acc = num[k].copy()
        for j in range(1, k + 1):
            acc -= np.array([den[j, 0] * q[k - j, 0], den[j, 0] * q[k - j, 1] + den[j, 1] * q[k - j, 0]])
        q[k] = acc
    a, l = np.zeros(8), np.zeros(8)
    for k in range(8):
        t, tl = q[k]
        if k == 5:      # integral of v^-4 and v^-1 terms: (-1/3 - ln v)
            a[5], l[5] = -40 / 9 * t, -40 / 3 * t
        elif k == 6:    # t v^-3 + tl v^-3 ln v
            a[6], l[6] = -20 * t + 10 * tl, -20 * tl
        else:
            a[k] = 40 * t / ((k - 8) * (k - 5))
    return a, l


@pytest.mark.parametrize("m1,m2", [(10.0, 10.0), (30.0, 7.0), (50.0, 12.0), (5.0, 100.0)])
def test_pn_coefficients_from_energy_balance(m1, m2):
    eta = m1 * m2 / (m1 + m2) ** 2
    delta = (m1 - m2) / (m1 + m2)
    a, l = taylorf2.phase_coefficients(np.array(eta), delta, 0.0, 0.0)
    A, Lg = energy_balance_alphas(eta, delta, 0.0, 0.0)
    np.testing.assert_allclose([float(x) for x in a], A, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose([float(x) for x in l], Lg, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("chi1,chi2", [(0.4, -0.3), (-0.9, 0.8), (0.99, 0.99)])
def test_spin_orbit_term(chi1, chi2):
    m1, m2 = 30.0, 7.0
    M = m1 + m2
    eta = m1 * m2 / M ** 2
    delta = (m1 - m2) / M
    chis, chia = 0.5 * (chi1 + chi2), 0.5 * (chi1 - chi2)
    a, _ = taylorf2.phase_coefficients(np.array(eta), delta, chis, chia)
    A, _ = energy_balance_alphas(eta, delta, chis, chia)
    np.testing.assert_allclose([float(x) for x in a[:5]], A[:5], rtol=1e-12, atol=1e-12)
    beta = (chi1 * (113 * (m1 / M) ** 2 + 75 * eta) + chi2 * (113 * (m2 / M) ** 2 + 75 * eta)) / 12
    assert abs(float(a[3]) - (-16 * math.pi + 4 * beta)) < 1e-12


def test_swap_symmetry():
    th = theta_of(31.0, 12.0, 0.3, -0.7, iota=0.4, phic=1.1)
    sw = th.copy()
    sw[[C.M1, C.M2]] = th[[C.M2, C.M1]]
    sw[[C.CHI1, C.CHI2]] = th[[C.CHI2, C.CHI1]]
    a = taylorf2.generate_waveforms(th, 20.0, 0.25, 4097)
    b = taylorf2.generate_waveforms(sw, 20.0, 0.25, 4097)
    for x, y in zip(a, b):
        np.testing.assert_allclose(x, y, rtol=1e-12, atol=1e-12 * np.abs(x).max())


def test_equal_mass_ignores_antisymmetric_spin():
    a = taylorf2.generate_waveforms(theta_of(20.0, 20.0, 0.5, -0.5), 20.0, 0.25, 4097)
    b = taylorf2.generate_waveforms(theta_of(20.0, 20.0, 0.1, -0.1), 20.0, 0.25, 4097)
    np.testing.assert_allclose(a[0], b[0], rtol=1e-12, atol=1e-12 * np.abs(a[0]).max())


def test_support_is_f_lo_to_isco():
    m1, m2 = 30.0, 25.0
    df, F = 0.5, 1025
    hp, hc = taylorf2.generate_waveforms(theta_of(m1, m2), 20.0, df, F)
    # ISCO from Kepler's law at r = 6M: orbital angular frequency sqrt(M / r^3), GW frequency twice orbital
    M = (m1 + m2) * MSUN
    f_isco = 2.0 * math.sqrt(M / (6.0 * M) ** 3) / (2.0 * math.pi)
    k = np.arange(F)
    inside = (k >= 40) & (k * df <= f_isco)
    assert np.all(np.abs(hp[0][inside]) > 0) and np.all(hp[0][~inside] == 0) and np.all(hc[0][~inside] == 0)


def test_polarisation_ratio():
    iota = 0.7
    hp, hc = taylorf2.generate_waveforms(theta_of(15.0, 12.0, iota=iota), 20.0, 0.5, 1025)
    on = hp[0] != 0
    ratio = hc[0][on] / hp[0][on]
    np.testing.assert_allclose(ratio, -1j * math.cos(iota) / (0.5 * (1 + math.cos(iota) ** 2)), rtol=1e-12)


def test_matches_fourier_transform_of_time_domain_chirp():
    """The 0PN frequency-domain model equals the FFT of the quadrupole time-domain chirp
    (stationary-phase accuracy), fixing the sign of the phase, the -pi/4, phic and
    the h_cross convention h_x(t) = A_t cos(iota) sin(Phi)."""
    m1 = m2 = 10.0
    iota, phic, dist = 0.6, 1.0, 500.0
    fs, T, tc = 4096.0, 16.0, 14.0
    Mc = chirp_mass_s(m1, m2)
    D = dist * C.MPC_M / C.C_MS
    t = np.arange(int(fs * T)) / fs
    tau = tc - t
    live = tau > tau_of_f(Mc, 170.0)
    f_t = np.zeros_like(t)
    dphi = np.zeros_like(t)
    f_t[live], dphi[live] = newtonian_td(Mc, tau[live])
    At = 4.0 * Mc ** (5.0 / 3.0) * (math.pi * f_t) ** (2.0 / 3.0) / D
    # smooth turn-on between 16 and 19 Hz and turn-off between 140 and 170 Hz
    on = np.clip((f_t - 16.0) / 3.0, 0, 1)
    off = np.clip((170.0 - f_t) / 30.0, 0, 1)
    win = np.sin(0.5 * math.pi * on) ** 2 * np.sin(0.5 * math.pi * off) ** 2 * live
    Phi = phic + dphi
    hp_t = win * At * 0.5 * (1 + math.cos(iota) ** 2) * np.cos(Phi)
    hc_t = win * At * math.cos(iota) * np.sin(Phi)
    df = 1.0 / T
    F = int(fs * T) // 2 + 1
    hp_fd = np.fft.rfft(hp_t) / fs
    hc_fd = np.fft.rfft(hc_t) / fs
    th = theta_of(m1, m2, dist=dist, phic=phic, iota=iota)
    hp, hc = taylorf2.generate_waveforms(th, 10.0, df, F, pn_order=0)
    shift = np.exp(-2j * math.pi * np.arange(F) * df * tc)
    band = slice(int(22 / df), int(60 / df))     # away from both tapers
    for got_fd, model in ((hp_fd, hp[0] * shift), (hc_fd, hc[0] * shift)):
        r = got_fd[band] / model[band]
        assert np.max(np.abs(np.abs(r) - 1.0)) < 5e-3
        assert np.max(np.abs(np.angle(r))) < 5e-3
