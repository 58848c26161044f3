"""Detector geometry, antenna patterns, delays and projection (oracle; test infrastructure).

Sec. 3.2 trains on Hanford and Livingston (HL) strain; the three-detector
workload adds Virgo.  Sec. 6 notes that the projection onto the detectors is done
on the fly on the GPU, for the extrinsic parameters (ra, dec, psi).
The projection implemented here is the textbook long-wavelength response:

    h_d(f) = (F+_d h_plus(f) + Fx_d h_cross(f)) exp(-2 pi i f (tc + dt_d))
    F+ = X.D.X - Y.D.Y,   Fx = X.D.Y + Y.D.X,   D = (x x^T - y y^T)/2
    dt_d = -(r_d . n) / c

with x, y the unit arm vectors, r_d the vertex position (Earth-fixed), n the
unit vector toward the source and X, Y the polarisation basis in the plane
orthogonal to n.  For a source at polar angle th and azimuth ph (th = pi/2 - dec,
ph = ra - gmst) the basis is X = cos(psi) e_th + sin(psi) e_ph,
Y = sin(psi) e_th - cos(psi) e_ph, chosen so that a detector with arms on the
x and y axes reproduces the textbook
    F+ = (1 + cos^2 th)/2 cos 2ph cos 2psi - cos th sin 2ph sin 2psi
    Fx = (1 + cos^2 th)/2 cos 2ph sin 2psi + cos th sin 2ph cos 2psi.

Readings: arm tilts are ignored (arms tangent to the WGS-84 ellipsoid); ra is
taken Earth-fixed with gmst = 0 unless a gmst is given.

Site table (approximate published values: vertex geodetic latitude and
longitude in degrees, elevation in metres, x- and y-arm azimuths in degrees
clockwise from North).  Parity between the oracle and the GPU path does not
depend on these values; physical realism does.
"""
import math
import numpy as np

from . import constants as C

SITES = {
    # name: (lat, lon, elevation, x-arm azimuth, y-arm azimuth)
    "H1": (46.455147, -119.407657, 142.554, 324.0000, 234.0000),
    "L1": (30.562894, -90.774240, -6.574, 252.2835, 162.2835),
    "V1": (43.631415, 10.504497, 51.884, 19.4326, 289.4326),
}
DET_IDS = {"H1": 0, "L1": 1, "V1": 2}

WGS84_A = 6378137.0
WGS84_F = 1.0 / 298.257223563


def geometry(name):
    """Return (D [3][3], r [3] in metres) for a site: detector tensor and vertex position."""
    lat, lon, h, xaz, yaz = SITES[name]
    phi = math.radians(lat)
    lam = math.radians(lon)
    e_north = np.array([-math.sin(phi) * math.cos(lam), -math.sin(phi) * math.sin(lam), math.cos(phi)])
    e_east = np.array([-math.sin(lam), math.cos(lam), 0.0])

    def arm(az_deg):
        az = math.radians(az_deg)
        return math.cos(az) * e_north + math.sin(az) * e_east

    x = arm(xaz)
    y = arm(yaz)
    D = 0.5 * (np.outer(x, x) - np.outer(y, y))
    e2 = WGS84_F * (2.0 - WGS84_F)
    Nphi = WGS84_A / math.sqrt(1.0 - e2 * math.sin(phi) ** 2)
    r = np.array([(Nphi + h) * math.cos(phi) * math.cos(lam),
                  (Nphi + h) * math.cos(phi) * math.sin(lam),
                  (Nphi * (1.0 - e2) + h) * math.sin(phi)])
    return D, r


def source_frame(ra, dec, psi, gmst=0.0):
    """Unit vector n toward the source and the polarisation basis X, Y (each [3][B])."""
    ra, dec, psi = (np.asarray(a, dtype=np.float64) for a in (ra, dec, psi))
    ph = ra - gmst
    sd, cd = np.sin(dec), np.cos(dec)
    sp, cp = np.sin(ph), np.cos(ph)
    n = np.array([cd * cp, cd * sp, sd])
    e_th = np.array([sd * cp, sd * sp, -cd])        # d n / d(theta), theta = pi/2 - dec
    e_ph = np.array([-sp, cp, np.zeros_like(sp)])
    X = np.cos(psi) * e_th + np.sin(psi) * e_ph
    Y = np.sin(psi) * e_th - np.cos(psi) * e_ph
    return n, X, Y


def antenna_from_tensor(D, ra, dec, psi, gmst=0.0):
    """(F+, Fx) [B] for a detector tensor D and source angles."""
    n, X, Y = source_frame(ra, dec, psi, gmst)
    DX = np.einsum("ij,jb->ib", D, X)
    DY = np.einsum("ij,jb->ib", D, Y)
    fp = np.einsum("ib,ib->b", X, DX) - np.einsum("ib,ib->b", Y, DY)
    fc = np.einsum("ib,ib->b", X, DY) + np.einsum("ib,ib->b", Y, DX)
    return fp, fc


def antenna(name, ra, dec, psi, gmst=0.0):
    D, _ = geometry(name)
    return antenna_from_tensor(D, ra, dec, psi, gmst)


def time_delay(name, ra, dec, gmst=0.0):
    """Arrival time at the site minus arrival time at the geocentre, seconds [B]."""
    _, r = geometry(name)
    n, _, _ = source_frame(ra, dec, np.zeros_like(np.asarray(ra, dtype=np.float64)), gmst)
    return -(r @ n) / C.C_MS


def project(hp, hc, theta, dets, gmst, df):
    """h_det [B][D][F] complex128 = (F+ hp + Fx hc) exp(-2 pi i f (tc + dt_d))."""
    hp = np.asarray(hp)
    B, F = hp.shape
    f = np.arange(F, dtype=np.float64) * df
    out = np.zeros((B, len(dets), F), dtype=np.complex128)
    for i, name in enumerate(dets):
        fp, fc = antenna(name, theta[C.RA], theta[C.DEC], theta[C.PSI], gmst)
        tau = theta[C.TC] + time_delay(name, theta[C.RA], theta[C.DEC], gmst)
        shift = np.exp(-2j * math.pi * f[None, :] * tau[:, None])
        out[:, i, :] = (fp[:, None] * hp + fc[:, None] * hc) * shift
    return out
