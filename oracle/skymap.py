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

Pixel centres (the inverse, from the same paper): for pixel p of face f with in-face
coordinates (ix, iy), the ring index counted from the north pole is
jr = jrll[f] nside - ix - iy - 1 with jrll = (2, 2, 2, 2, 3, 3, 3, 3, 4, 4, 4, 4); rings
jr < nside lie in the north cap (nr = jr pixels' worth of ring, z = 1 - nr^2 / (3 nside^2)),
jr > 3 nside in the south cap (nr = 4 nside - jr, z = -(1 - nr^2 / (3 nside^2))), the rest in
the equatorial belt (nr = nside, z = 4/3 - 2 jr / (3 nside), and rings alternate by half a
pixel: shift = (jr - nside) mod 2).  Along the ring the pixel number is
jp = (jpll[f] nr + ix - iy + 1 + shift) / 2 (jpll = (1, 3, 5, 7, 0, 2, 4, 6, 1, 3, 5, 7)),
wrapped into 1 .. 4 nr, and phi = (jp - (1 + shift) / 2) (pi / 2) / nr.

The flow's sky density (Sec. 5: the density evaluated at every pixel of the map; reading):
the normalizing flow's density over (RA, sin dec) at each pixel centre, the other six of
its coordinates held at a given point (the coordinates of the event's draw with the
largest ln q), normalised to unit sum over the pixels.  (RA, sin dec) are coordinates of
equal area on the sphere (d Omega = d RA d sin dec), so with pixels of equal area this is
the density per steradian up to its normalisation.
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


_JRLL = (2, 2, 2, 2, 3, 3, 3, 3, 4, 4, 4, 4)
_JPLL = (1, 3, 5, 7, 0, 2, 4, 6, 1, 3, 5, 7)


def _deinterleave(v):
    ix = iy = 0
    b = 0
    while v >> (2 * b):
        ix |= ((v >> (2 * b)) & 1) << b
        iy |= ((v >> (2 * b + 1)) & 1) << b
        b += 1
    return ix, iy


def pix2ang_nest(nside, p):
    """(colatitude theta, longitude phi) of the centre of nested pixel p."""
    npf = nside * nside
    f, ix, iy = p // npf, *_deinterleave(p % npf)
    jr = _JRLL[f] * nside - ix - iy - 1
    if jr < nside:
        nr, z, shift = jr, 1.0 - jr * jr / (3.0 * npf), 0
    elif jr > 3 * nside:
        nr = 4 * nside - jr
        z, shift = -(1.0 - nr * nr / (3.0 * npf)), 0
    else:
        nr, z, shift = nside, 4.0 / 3.0 - 2.0 * jr / (3.0 * nside), (jr - nside) & 1
    jp = (_JPLL[f] * nr + ix - iy + 1 + shift) // 2
    if jp > 4 * nr:
        jp -= 4 * nr
    if jp < 1:
        jp += 4 * nr
    phi = (jp - 0.5 * (1 + shift)) * 0.5 * math.pi / nr
    return math.acos(z), phi


def pixel_centres(nside):
    """(RA [12 nside^2], sin dec [12 nside^2]) of every pixel centre, nested order."""
    n = 12 * nside * nside
    ra, sd = np.empty(n), np.empty(n)
    for p in range(n):
        th, ph = pix2ang_nest(nside, p)
        ra[p], sd[p] = ph, math.cos(th)
    return ra, sd


def density_map(log_q_at, r_fixed, nside):
    """Sky density of a flow: log_q_at(r [M][8]) evaluates ln q_r for rows of flow
    coordinates (Mc, q, D, cos theta_JN, RA, sin dec, psi, phic); the map holds
    exp ln q at every pixel centre with the other coordinates at r_fixed, normalised to
    unit sum."""
    ra, sd = pixel_centres(nside)
    r = np.tile(np.asarray(r_fixed, dtype=np.float64), (len(ra), 1))
    r[:, 4], r[:, 5] = ra, sd
    lq = np.asarray(log_q_at(r), dtype=np.float64)
    w = np.exp(lq - lq.max())
    return w / w.sum()
