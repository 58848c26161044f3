"""HEALPix sky maps of posterior samples (oracle; test infrastructure).

The paper turns its posterior into a sky-localisation map in the HEALPix format (Sec. 5,
the inference timings at NSIDE 32, 64 and 128).  Here a map is the importance-weighted
histogram of the samples' sky positions over the HEALPix pixels: map[p] = sum of the
normalised weights of the samples whose (RA, dec) falls in pixel p, so the map sums to
one.  Pixel indices follow the nested scheme of Gorski et al. 2005 ("HEALPix: a
framework for high-resolution discretization ...", ApJ 622, 759), restated here from its
definition:

* colatitude theta = pi/2 - dec, z = cos(theta), longitude phi = RA in [0, 2 pi),
  tt = phi / (pi/2) in [0, 4);
* equatorial zone |z| <= 2/3: with t1 = nside (1/2 + tt) and t2 = 3/4 nside z, the
  indices of the two families of pixel-boundary lines are jp = floor(t1 - t2) and
  jm = floor(t1 + t2); with ifp = jp // nside, ifm = jm // nside the base face is
  ifp + 4 when ifp == ifm, ifp when ifp < ifm, else ifm + 8; inside the face
  ix = jm mod nside and iy = nside - 1 - (jp mod nside);
* polar caps |z| > 2/3: ntt = min(floor(tt), 3), tp = tt - ntt, s = nside sqrt(3 (1 - |z|)),
  jp = min(floor(tp s), nside - 1), jm = min(floor((1 - tp) s), nside - 1); north
  (z > 0): face ntt, ix = nside - 1 - jm, iy = nside - 1 - jp; south: face ntt + 8,
  ix = jp, iy = jm;
* nested index face nside^2 + (bits of ix and iy interleaved, ix in the even bits).
"""
import math

import numpy as np


def _interleave(ix, iy):
    out = 0
    b = 0
    while (ix >> b) or (iy >> b):
        out |= ((ix >> b) & 1) << (2 * b)
        out |= ((iy >> b) & 1) << (2 * b + 1)
        b += 1
    return out


def ang2pix_nest(nside, theta, phi):
    """Nested pixel index of colatitude theta and longitude phi (scalars, radians)."""
    z = math.cos(theta)
    za = abs(z)
    tt = (phi % (2.0 * math.pi)) / (0.5 * math.pi)
    if za <= 2.0 / 3.0:
        t1 = nside * (0.5 + tt)
        t2 = nside * z * 0.75
        jp = int(math.floor(t1 - t2))
        jm = int(math.floor(t1 + t2))
        ifp, ifm = jp // nside, jm // nside
        if ifp == ifm:
            face = ifp | 4
        elif ifp < ifm:
            face = ifp
        else:
            face = ifm + 8
        ix = jm & (nside - 1)
        iy = nside - (jp & (nside - 1)) - 1
    else:
        ntt = min(int(tt), 3)
        tp = tt - ntt
        s = nside * math.sqrt(3.0 * (1.0 - za))
        jp = min(int(tp * s), nside - 1)
        jm = min(int((1.0 - tp) * s), nside - 1)
        if z > 0:
            face, ix, iy = ntt, nside - jm - 1, nside - jp - 1
        else:
            face, ix, iy = ntt + 8, jp, jm
    return face * nside * nside + _interleave(ix, iy)


def skymap(ra, dec, weights, nside):
    """Normalised importance-weighted histogram [12 nside^2] of samples at (ra, dec)."""
    ra = np.asarray(ra, dtype=np.float64)
    dec = np.asarray(dec, dtype=np.float64)
    w = np.ones(len(ra)) if weights is None else np.asarray(weights, dtype=np.float64)
    m = np.zeros(12 * nside * nside)
    for i in range(len(ra)):
        if w[i] > 0.0:
            m[ang2pix_nest(nside, 0.5 * math.pi - dec[i], ra[i])] += w[i]
    tot = m.sum()
    return m / tot if tot > 0 else m
