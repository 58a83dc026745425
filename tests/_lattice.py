"""A sky and an array for which the visibility sum is a 2-D DFT.

Sources sit on an N x N lattice of east/north direction cosines
(l, m) = ((j - N/2) d, (k - N/2) d) at one time; antennas sit on a G x G grid
of spacing lambda / (N d) in the east and north directions (coplanar).  Then
the fringe phase of baseline (p, q) grid steps at source (j, k) is
2 pi (p (j - N/2) + q (k - N/2)) / N, so with a uniform beam
V(p, q) = sum_jk I_jk exp(-2 pi i (p (j - N/2) + q (k - N/2)) / N)
        = (-1)^(p + q) FFT2(I)[p mod N, q mod N]      (N even),
which numpy's FFT evaluates independently of both the oracle and the GPU path.
The lattice is turned into RA/Dec by inverting the equatorial -> ENU rotation
(hour angle H = LST - RA): sin(dec) = n cos(lat) + u sin(lat),
cos(dec) sin(H) = -e, cos(dec) cos(H) = u cos(lat) - n sin(lat).
"""
import math

import numpy as np

C_LIGHT = 299792458.0


def lattice_case(N=16, G=5, d=0.02, nu=150e6, lst=0.7, lat=-0.5361913, seed=0):
    rng = np.random.default_rng(seed)
    j, k = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    l = ((j - N // 2) * d).ravel()
    m = ((k - N // 2) * d).ravel()
    u = np.sqrt(1.0 - l * l - m * m)
    sin_dec = m * math.cos(lat) + u * math.sin(lat)
    dec = np.arcsin(sin_dec)
    H = np.arctan2(-l, u * math.cos(lat) - m * math.sin(lat))
    ra = np.mod(lst - H, 2 * math.pi)
    I = rng.uniform(0.5, 2.0, (N, N))
    flux = I.ravel()[None, :, None].astype(np.float64)
    dx = C_LIGHT / nu / (N * d)
    a, b = np.meshgrid(np.arange(G), np.arange(G), indexing="ij")
    ant = np.stack([a.ravel() * dx, b.ravel() * dx, np.zeros(G * G)], axis=1)
    pairs = np.array([(i, jj) for i in range(G * G) for jj in range(i + 1, G * G)], dtype=np.int32)
    F = np.fft.fft2(I)
    p = a.ravel()[pairs[:, 0]] - a.ravel()[pairs[:, 1]]
    q = b.ravel()[pairs[:, 0]] - b.ravel()[pairs[:, 1]]
    expected = ((-1.0) ** (p + q)) * F[p % N, q % N]
    return dict(ant=ant, pairs=pairs, ra=ra, dec=dec, flux=flux, freqs=np.array([nu]), lsts=np.array([lst]),
                lat=lat, expected=expected, lmn=np.stack([l, m, u], 1))
