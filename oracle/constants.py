"""Physical constants and the parameter layout (oracle's own copy; test infrastructure).

The paper states masses in solar masses in the detector frame and distances in
Mpc without cosmology (Table 1 and its note).  Conversions used here:

* G M_sun / c^3 in seconds (solar mass as a time),
* one megaparsec in metres,
* the speed of light (exact SI value),
* the Euler-Mascheroni constant (appears in the 3PN TaylorF2 phase).
"""
import math

MTSUN_S = 4.925490947641267e-6      # G M_sun / c^3 [s]
MPC_M = 3.085677581491367e22        # 1 Mpc [m]
C_MS = 299792458.0                  # speed of light [m/s]
EULER_GAMMA = 0.5772156649015329

# Parameter layout: theta is a [P][B] float64 array (structure of arrays).
M1, M2, CHI1, CHI2, DIST, TC, PHIC, THETAJN, PSI, RA, DEC = range(11)
P = 11
NAMES = ("m1", "m2", "chi1", "chi2", "distance", "tc", "phic", "theta_jn", "psi", "ra", "dec")

TWO_PI = 2.0 * math.pi
