"""Seeded synthetic workloads for the visibility path.

This module only *makes inputs*: antenna layouts, source catalogues, sky maps,
frequency and time grids.  It holds none of the method's arithmetic (no
coordinate rotation to the topocentric frame, no beam, no Fourier sum), so the
CUDA path and the FP64 oracle can both consume its output without sharing any
computation.

The paper's own workloads use HERA layouts, the GSM diffuse map and GLEAM
source counts (Section 4.2, Section 5.2).  None of those are available, so the
recipes below stand in for them:

* hexagonal arrays with 14.6 m spacing (the HERA baselines quoted in the
  caption of Fig. 3 are multiples of 14.6 m);
* point sources uniform on the sphere (or on the visible hemisphere), fluxes
  log-uniform 0.1-10 Jy at 150 MHz with power-law spectral index N(-0.8, 0.2);
* a diffuse map on HEALPix RING pixel centres (Gorski et al. 2005, as used in
  Section 4.1) holding a log-normal transform of a Gaussian random field with
  power-law angular spectrum C_l ~ l^-2.5, passed as point sources at the pixel
  centres with flux = brightness x pixel solid angle (the point-source
  approximation of Section 2.1).

Every generator takes an explicit ``numpy.random.Generator`` or seed.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

HERA_LATITUDE_RAD = math.radians(-30.7215)   # site latitude (stated assumption)
SIDEREAL_DAY_S = 86164.0905


# --------------------------------------------------------------------------
# arrays
# --------------------------------------------------------------------------
def hex_array(radius: int, spacing_m: float = 14.6, n_keep: int | None = None,
              z_sigma_m: float = 0.0, rng: np.random.Generator | None = None) -> np.ndarray:
    """Antenna ENU positions [n_ant][3] of a filled hexagon of ``radius`` rings.

    A hexagon of radius r holds 3r(r+1)+1 antennas.  ``n_keep`` keeps the
    n_keep antennas closest to the centre (ties broken by azimuth), which is how
    the 350-element layout is cut from an r=11 hexagon.  ``z_sigma_m`` adds a
    Gaussian height jitter so that the array is not coplanar.
    """
    pts = []
    for j in range(-radius, radius + 1):
        for i in range(-radius, radius + 1):
            if abs(i + j) <= radius:
                pts.append((spacing_m * (i + 0.5 * j), spacing_m * (j * math.sqrt(3.0) / 2.0)))
    pts = np.array(pts, dtype=np.float64)
    if n_keep is not None:
        r = np.round(np.hypot(pts[:, 0], pts[:, 1]), 9)
        az = np.round(np.arctan2(pts[:, 0], pts[:, 1]) % (2 * np.pi), 12)
        order = np.lexsort((az, r))
        pts = pts[np.sort(order[:n_keep])]
    enu = np.zeros((len(pts), 3))
    enu[:, :2] = pts
    if z_sigma_m > 0:
        if rng is None:
            raise ValueError("z jitter needs an rng")
        enu[:, 2] = rng.normal(0.0, z_sigma_m, len(pts))
    return enu


def cross_pairs(n_ant: int) -> np.ndarray:
    """All antenna pairs (i, j) with i < j, as int32 [n_bl][2]."""
    i, j = np.triu_indices(n_ant, k=1)
    return np.stack([i, j], axis=1).astype(np.int32)


# --------------------------------------------------------------------------
# frequencies and times
# --------------------------------------------------------------------------
def channel_centres(n: int, lo_hz: float = 100e6, hi_hz: float = 200e6) -> np.ndarray:
    """Centres of n equal channels spanning [lo, hi]."""
    return lo_hz + (np.arange(n) + 0.5) * (hi_hz - lo_hz) / n


def lst_grid(n_time: int, cadence_s: float, lst0_rad: float) -> np.ndarray:
    """Local sidereal times of n_time integrations at a fixed cadence."""
    return (lst0_rad + np.arange(n_time) * cadence_s * 2 * np.pi / SIDEREAL_DAY_S) % (2 * np.pi)


# --------------------------------------------------------------------------
# point sources
# --------------------------------------------------------------------------
def uniform_sphere(n: int, rng: np.random.Generator) -> tuple[np.ndarray, np.ndarray]:
    """RA, Dec (rad) of n points uniform on the sphere."""
    ra = rng.uniform(0, 2 * np.pi, n)
    dec = np.arcsin(rng.uniform(-1, 1, n))
    return ra, dec


def visible_hemisphere(n: int, rng: np.random.Generator, lst_rad: float,
                       latitude_rad: float) -> tuple[np.ndarray, np.ndarray]:
    """RA, Dec of n points uniform on the hemisphere above the horizon at one LST.

    Points are drawn uniform in (altitude sine, azimuth) and mapped to hour
    angle and declination with the textbook alt-az to equatorial relations.
    Altitude is kept at least 1e-6 rad so that no point sits on the horizon.
    """
    sin_alt = rng.uniform(1e-6, 1.0, n)
    az = rng.uniform(0, 2 * np.pi, n)          # east of north
    alt = np.arcsin(sin_alt)
    sphi, cphi = math.sin(latitude_rad), math.cos(latitude_rad)
    sin_dec = sin_alt * sphi + np.cos(alt) * np.cos(az) * cphi
    dec = np.arcsin(np.clip(sin_dec, -1, 1))
    # hour angle from its sine and cosine
    sin_h = -np.sin(az) * np.cos(alt)
    cos_h = sin_alt * cphi - np.cos(alt) * np.cos(az) * sphi
    ha = np.arctan2(sin_h, cos_h)
    ra = (lst_rad - ha) % (2 * np.pi)
    return ra, dec


def powerlaw_fluxes(n: int, freqs_hz: np.ndarray, rng: np.random.Generator,
                    s_lo: float = 0.1, s_hi: float = 10.0, index_mean: float = -0.8,
                    index_sigma: float = 0.2, ref_hz: float = 150e6) -> np.ndarray:
    """Stokes I [n][n_freq]: log-uniform reference flux times a power law."""
    s0 = np.exp(rng.uniform(np.log(s_lo), np.log(s_hi), n))
    alpha = rng.normal(index_mean, index_sigma, n)
    return s0[:, None] * (np.asarray(freqs_hz)[None, :] / ref_hz) ** alpha[:, None]


# --------------------------------------------------------------------------
# HEALPix RING pixel centres (Gorski et al. 2005)
# --------------------------------------------------------------------------
def healpix_ring_centres(nside: int) -> tuple[np.ndarray, np.ndarray]:
    """Colatitude theta and longitude phi (rad) of all 12 nside^2 RING pixels.

    Pixels are iso-latitude rings ordered from the north pole.  The two polar
    caps hold rings 1..nside-1 with 4i pixels in ring i; the equatorial belt
    holds 2nside+1 rings of 4nside pixels each, alternate rings shifted by half
    a pixel.
    """
    npix = 12 * nside * nside
    ncap = 2 * nside * (nside - 1)
    p = np.arange(npix, dtype=np.int64)
    z = np.empty(npix)
    phi = np.empty(npix)

    north = p < ncap
    pn = p[north]
    i = (1 + np.floor(np.sqrt(1 + 2 * pn + 1e-9)).astype(np.int64)) // 2
    # guard isqrt rounding
    i = np.where(2 * i * (i - 1) > pn, i - 1, i)
    i = np.where(2 * (i + 1) * i <= pn, i + 1, i)
    j = pn + 1 - 2 * i * (i - 1)
    z[north] = 1.0 - i * i / (3.0 * nside * nside)
    phi[north] = (j - 0.5) * np.pi / (2 * i)

    belt = (p >= ncap) & (p < npix - ncap)
    pb = p[belt] - ncap
    ring = pb // (4 * nside) + nside            # ring index counted from the north pole
    j = pb % (4 * nside) + 1
    half = np.where((ring + nside) % 2 == 1, 1.0, 0.5)
    z[belt] = (2 * nside - ring) * 2.0 / (3.0 * nside)
    phi[belt] = (j - half) * np.pi / (2 * nside)

    south = p >= npix - ncap
    ps = npix - p[south]                           # 1-based index counted from the south pole
    i = (1 + np.floor(np.sqrt(2 * ps - 1 + 1e-9)).astype(np.int64)) // 2
    i = np.where(2 * i * (i - 1) >= ps, i - 1, i)
    i = np.where(2 * (i + 1) * i < ps, i + 1, i)
    j = 4 * i + 1 - (ps - 2 * i * (i - 1))
    z[south] = -1.0 + i * i / (3.0 * nside * nside)
    phi[south] = (j - 0.5) * np.pi / (2 * i)
    return np.arccos(np.clip(z, -1, 1)), phi


def healpix_radec(nside: int) -> tuple[np.ndarray, np.ndarray]:
    """RA, Dec of the RING pixel centres, taking the map in equatorial coordinates."""
    theta, phi = healpix_ring_centres(nside)
    return phi.copy(), np.pi / 2 - theta


def healpix_pixel_area(nside: int) -> float:
    return 4 * np.pi / (12 * nside * nside)


def gaussian_random_field(nside: int, rng: np.random.Generator, lmax: int | None = None,
                          slope: float = -2.5) -> np.ndarray:
    """Real Gaussian random field on the RING pixels with C_l ~ l^slope (l >= 1).

    Synthesis by spherical harmonics, ring by ring: for every ring the
    orthonormal associated Legendre functions are built by the standard
    three-term recurrence, summed against the random a_lm, and the azimuthal
    sum is evaluated with an FFT over the ring's pixels.  The result is scaled
    to unit standard deviation.
    """
    if lmax is None:
        lmax = 2 * nside
    theta, phi = healpix_ring_centres(nside)
    z = np.cos(theta)
    # ring boundaries: z is constant along a ring and rings are contiguous
    starts = np.flatnonzero(np.r_[True, np.abs(np.diff(z)) > 1e-13])
    ends = np.r_[starts[1:], len(z)]
    zr = z[starts]
    sr = np.sqrt(np.maximum(0.0, 1 - zr * zr))
    nr = len(zr)
    ells = np.arange(lmax + 1)
    cl = np.zeros(lmax + 1)
    cl[1:] = ells[1:].astype(float) ** slope
    # a_lm for m >= 0 (complex, a_l0 real)
    alm = (rng.normal(size=(lmax + 1, lmax + 1)) + 1j * rng.normal(size=(lmax + 1, lmax + 1))) / np.sqrt(2)
    alm[:, 0] = rng.normal(size=lmax + 1)
    alm *= np.sqrt(cl)[:, None]
    alm = np.tril(alm)                       # only m <= l
    F = np.zeros((nr, lmax + 1), dtype=np.complex128)   # F[ring, m]
    m = np.arange(lmax + 1)
    # lam_mm for every m: lam_00 = 1/sqrt(4 pi); lam_mm = -sqrt((2m+1)/(2m)) s lam_(m-1)(m-1)
    lam_mm = np.zeros((nr, lmax + 1))
    lam_mm[:, 0] = 1.0 / np.sqrt(4 * np.pi)
    for mm in range(1, lmax + 1):
        lam_mm[:, mm] = -np.sqrt((2 * mm + 1) / (2.0 * mm)) * sr * lam_mm[:, mm - 1]
    lam_prev2 = np.zeros((nr, lmax + 1))
    lam_prev = np.zeros((nr, lmax + 1))
    for l in range(lmax + 1):
        cur = np.zeros((nr, lmax + 1))
        cur[:, l] = lam_mm[:, l]
        if l >= 1:
            mm = m[:l]
            a = np.sqrt((4.0 * l * l - 1) / (l * l - mm * mm))
            b = np.sqrt(((l - 1.0) ** 2 - mm * mm) / (4.0 * (l - 1.0) ** 2 - 1))
            cur[:, :l] = a[None, :] * (zr[:, None] * lam_prev[:, :l] - b[None, :] * lam_prev2[:, :l])
        F += cur * alm[l][None, :]
        lam_prev2, lam_prev = lam_prev, cur
    out = np.empty(len(z))
    for r in range(nr):
        s, e = starts[r], ends[r]
        n = e - s
        phi0 = phi[s]
        coef = F[r] * np.exp(1j * m * phi0)
        # f_j = Re(F_0) + 2 Re(sum_{m>=1} coef_m e^{2 pi i m j / n})
        fold = np.zeros(n, dtype=np.complex128)
        np.add.at(fold, m[1:] % n, coef[1:])
        vals = np.fft.ifft(fold) * n
        out[s:e] = F[r, 0].real * 1.0 + 2 * vals.real
    out -= out.mean()
    sd = out.std()
    return out / sd if sd > 0 else out


# --------------------------------------------------------------------------
# composite skies
# --------------------------------------------------------------------------
@dataclass
class Sky:
    ra: np.ndarray                 # [n_src] rad
    dec: np.ndarray                # [n_src] rad
    flux: np.ndarray               # [n_stokes][n_src][n_freq] Jy
    n_point: int = 0
    n_diffuse: int = 0

    @property
    def n_src(self) -> int:
        return len(self.ra)

    @property
    def n_stokes(self) -> int:
        return self.flux.shape[0]


def diffuse_map(nside: int, freqs_hz: np.ndarray, rng: np.random.Generator,
                brightness_jy_sr: float = 1.0e3, index: float = -2.5, index_sigma: float = 0.1,
                polarized: bool = False, ref_hz: float = 150e6, lmax: int | None = None,
                dtype=np.float64) -> Sky:
    """Diffuse sky on HEALPix pixel centres as a point-source list.

    Brightness = B0 exp(0.5 g - 0.125) (log-normal of a unit GRF g), a
    per-pixel power law in frequency, times the pixel solid angle.  With
    ``polarized`` Q and U are 0.1 I times two further independent GRFs and V = 0.
    """
    ra, dec = healpix_radec(nside)
    g = gaussian_random_field(nside, rng, lmax=lmax)
    bright = brightness_jy_sr * np.exp(0.5 * g - 0.125)
    alpha = rng.normal(index, index_sigma, len(ra))
    spec = (np.asarray(freqs_hz, dtype=dtype)[None, :] / dtype(ref_hz)) ** alpha.astype(dtype)[:, None]
    stokes_i = (bright * healpix_pixel_area(nside)).astype(dtype)[:, None] * spec
    if not polarized:
        return Sky(ra, dec, stokes_i[None], 0, len(ra))
    gq = gaussian_random_field(nside, rng, lmax=lmax)
    gu = gaussian_random_field(nside, rng, lmax=lmax)
    flux = np.zeros((4,) + stokes_i.shape, dtype=dtype)
    flux[0] = stokes_i
    flux[1] = (0.1 * gq).astype(dtype)[:, None] * stokes_i
    flux[2] = (0.1 * gu).astype(dtype)[:, None] * stokes_i
    return Sky(ra, dec, flux, 0, len(ra))


def point_sky(n: int, freqs_hz: np.ndarray, rng: np.random.Generator, polarized: bool = False,
              hemisphere: tuple[float, float] | None = None, dtype=np.float64) -> Sky:
    """Power-law point sources; uniform on the sphere unless ``hemisphere=(lst, lat)``."""
    if hemisphere is None:
        ra, dec = uniform_sphere(n, rng)
    else:
        ra, dec = visible_hemisphere(n, rng, *hemisphere)
    stokes_i = powerlaw_fluxes(n, freqs_hz, rng).astype(dtype)
    if not polarized:
        return Sky(ra, dec, stokes_i[None], n, 0)
    frac = rng.uniform(0, 0.1, n)
    chi = rng.uniform(0, np.pi, n)
    flux = np.zeros((4,) + stokes_i.shape, dtype=dtype)
    flux[0] = stokes_i
    flux[1] = (frac * np.cos(2 * chi)).astype(dtype)[:, None] * stokes_i
    flux[2] = (frac * np.sin(2 * chi)).astype(dtype)[:, None] * stokes_i
    return Sky(ra, dec, flux, n, 0)


def concat_skies(*skies: Sky) -> Sky:
    ns = max(s.n_stokes for s in skies)
    parts = []
    for s in skies:
        f = s.flux
        if f.shape[0] < ns:
            f = np.concatenate([f, np.zeros((ns - f.shape[0],) + f.shape[1:], dtype=f.dtype)], axis=0)
        parts.append(f)
    return Sky(np.concatenate([s.ra for s in skies]), np.concatenate([s.dec for s in skies]),
               np.concatenate(parts, axis=1), sum(s.n_point for s in skies),
               sum(s.n_diffuse for s in skies))


# --------------------------------------------------------------------------
# full problems
# --------------------------------------------------------------------------
@dataclass
class Problem:
    """Everything one simulation needs (the inputs named in Section 2.1)."""
    name: str
    ant_enu: np.ndarray            # [n_ant][3] m
    pairs: np.ndarray              # [n_bl][2] int32
    sky: Sky
    freqs_hz: np.ndarray           # [n_freq]
    lsts_rad: np.ndarray           # [n_time]
    latitude_rad: float
    beam: str                      # "gauss" | "airy" | "uniform"
    beam_param: tuple = ()
    polarized: bool = False
    eps: float = 1e-10
    meta: dict = field(default_factory=dict)
    # per-antenna beams (Section 2.2.3): [(kind, params), ...] and the beam index of every antenna
    beams: list | None = None
    beam_of_ant: np.ndarray | None = None
    # gridded beams (Section 2.4, numerical beams): voltage samples [n_freq][n_theta][n_phi] of the
    # plan's beam (key -1, with beam == "grid") or of per-antenna beam k (beams[k] == ("grid", ()))
    beam_grids: dict | None = None
    beam_grid_order: int = 1       # 1 bilinear, 3 bicubic B-spline

    @property
    def n_vis(self) -> int:
        return len(self.pairs) * len(self.freqs_hz) * len(self.lsts_rad) * (4 if self.polarized else 1)


GAUSS_FWHM_150 = (math.radians(10.0), 150e6)   # 10 deg FWHM at 150 MHz, scaling as 1/nu


def grid_beam(freqs_hz: np.ndarray, n_theta: int, n_phi: int, fwhm_ref_rad: float = np.radians(10.0),
              ref_hz: float = 150e6, ellipticity: float = 0.0) -> np.ndarray:
    """Synthetic numerical beam standing in for a simulated (CST/HFSS-style) beam file: voltage samples
    [n_freq][n_theta][n_phi] on the grid theta_i = i (pi/2) / (n_theta - 1) (zenith angle, zenith to
    horizon) x phi_j = j 2 pi / n_phi (azimuth east of north) of an elliptical Gaussian power pattern
    exp(-4 ln2 theta^2 / FWHM^2), FWHM = fwhm_ref (ref / nu) (1 + ellipticity cos 2 phi)."""
    th = np.linspace(0.0, np.pi / 2, n_theta)
    ph = np.arange(n_phi) * (2 * np.pi / n_phi)
    nu = np.asarray(freqs_hz, dtype=np.float64)
    fwhm = fwhm_ref_rad * (ref_hz / nu)[:, None, None] * (1.0 + ellipticity * np.cos(2 * ph))[None, None, :]
    return np.sqrt(np.exp(-4.0 * np.log(2.0) * th[None, :, None] ** 2 / fwhm ** 2))


def config_small(seed: int = 0, n_src: int = 1000, eps: float = 1e-10) -> Problem:
    """37-antenna hexagon, 1 channel at 150 MHz, 1 time, n_src sources on the
    visible hemisphere, Gaussian beam (FWHM 10 deg at 150 MHz)."""
    rng = np.random.default_rng(seed)
    ant = hex_array(3)
    lst = rng.uniform(0, 2 * np.pi)
    freqs = np.array([150e6])
    sky = point_sky(n_src, freqs, rng, hemisphere=(lst, HERA_LATITUDE_RAD))
    return Problem("hex37_1ch_1t", ant, cross_pairs(len(ant)), sky, freqs, np.array([lst]),
                   HERA_LATITUDE_RAD, "gauss", GAUSS_FWHM_150, False, eps)


def config_hex127(seed: int = 1, n_chan: int = 64, n_time: int = 10, n_point: int = 20000,
                  nside: int = 64, eps: float = 1e-11, radius: int = 6) -> Problem:
    """127-antenna hexagon with 5 cm height jitter, n_chan channels over
    100-200 MHz, n_time integrations at 10.7 s, power-law point sources plus a
    HEALPix diffuse map; Gaussian beam.  Defaults are the full workload
    (8,001 baselines x 64 channels x 10 times, 69,152 sources)."""
    rng = np.random.default_rng(seed)
    ant = hex_array(radius, z_sigma_m=0.05, rng=rng)
    freqs = channel_centres(n_chan)
    lsts = lst_grid(n_time, 10.7, rng.uniform(0, 2 * np.pi))
    parts = []
    if n_point:
        parts.append(point_sky(n_point, freqs, rng))
    if nside:
        parts.append(diffuse_map(nside, freqs, rng))
    sky = concat_skies(*parts)
    return Problem(f"hex{len(ant)}_{n_chan}ch_{n_time}t", ant, cross_pairs(len(ant)), sky, freqs,
                   lsts, HERA_LATITUDE_RAD, "gauss", GAUSS_FWHM_150, False, eps)


def config_hex350_pol(seed: int = 2, n_chan: int = 256, n_time: int = 4, n_point: int = 100000,
                      nside: int = 256, eps: float = 1e-6, n_keep: int = 350,
                      radius: int = 11, dtype=np.float64) -> Problem:
    """350-antenna coplanar hexagon, polarised point + diffuse sky, 2x2 Jones
    Airy beam of a 14 m dish; defaults are the full workload."""
    rng = np.random.default_rng(seed)
    ant = hex_array(radius, n_keep=n_keep)
    freqs = channel_centres(n_chan)
    lsts = lst_grid(n_time, 10.7, rng.uniform(0, 2 * np.pi))
    parts = []
    if n_point:
        parts.append(point_sky(n_point, freqs, rng, polarized=True, dtype=dtype))
    if nside:
        parts.append(diffuse_map(nside, freqs, rng, polarized=True, dtype=dtype))
    sky = concat_skies(*parts)
    return Problem(f"hex{len(ant)}_pol_{n_chan}ch_{n_time}t", ant, cross_pairs(len(ant)), sky,
                   freqs, lsts, HERA_LATITUDE_RAD, "airy", (14.0,), True, eps)


@dataclass
class BatchSlice:
    """One independent single-slice problem of the batched workload.

    ``problem.eps`` is the slice's drawn tolerance; ``nufft_eps`` is the
    tolerance given to the transform: a tenth of it on the FP64 path, whose
    gate is a relative L2 error of 1e-9 against the direct sum (the kernel
    tolerance bounds the error relative to the summed source strengths, which
    is a few times looser in relative L2), and the tolerance itself on the
    mixed path, where FP32 rounding sets the floor."""
    problem: Problem
    precision: str          # "mixed" (eps >= 1e-6) or "fp64"
    nufft_eps: float = 0.0


def config_batch(seed: int = 4, n_slices: int = 2048, radii=(3, 4, 5, 6, 7, 8, 9, 10),
                 n_src_range=(1000, 500000), eps_choices=(1e-6, 1e-9)) -> list:
    """Ragged single-slice problems: hexagons of 37-331 antennas, skies of
    1e3-5e5 sources (log-uniform), eps from {1e-6, 1e-9}, frequency and time
    from the 127-antenna workload's ranges (100-200 MHz, 10 integrations at
    10.7 s), Gaussian beam.  Skies are prefixes of one seeded uniform-sphere
    catalogue; slices with eps < 1e-6 take the FP64 path, the others the mixed
    path."""
    rng = np.random.default_rng(seed)
    n_max = int(n_src_range[1])
    cat_ra, cat_dec = uniform_sphere(n_max, rng)
    s0 = np.exp(rng.uniform(np.log(0.1), np.log(10.0), n_max))
    alpha = rng.normal(-0.8, 0.2, n_max)
    arrays = {r: hex_array(r) for r in radii}
    pairs = {r: cross_pairs(len(a)) for r, a in arrays.items()}
    lst0 = rng.uniform(0, 2 * np.pi)
    lsts = lst_grid(10, 10.7, lst0)
    out = []
    for k in range(n_slices):
        r = int(rng.choice(radii))
        n_src = int(np.exp(rng.uniform(np.log(n_src_range[0]), np.log(n_src_range[1]))))
        eps = float(rng.choice(eps_choices))
        nu = float(rng.uniform(100e6, 200e6))
        lst = float(rng.choice(lsts))
        flux = (s0[:n_src] * (nu / 150e6) ** alpha[:n_src])[None, :, None]
        sky = Sky(cat_ra[:n_src], cat_dec[:n_src], flux, n_src, 0)
        prob = Problem(f"batch{k}_hex{len(arrays[r])}_{n_src}src", arrays[r], pairs[r], sky, np.array([nu]),
                       np.array([lst]), HERA_LATITUDE_RAD, "gauss", GAUSS_FWHM_150, False, eps)
        mixed = eps >= 1e-6
        out.append(BatchSlice(prob, "mixed" if mixed else "fp64", eps if mixed else 0.1 * eps))
    return out


SERVE_KINDS = ("hex37", "hex127", "hex350")


def serve_plans(seed: int = 5, n_chan: int = 256, n_time: int = 20, scale: float = 1.0,
                kinds=SERVE_KINDS) -> dict:
    """The resident problems the served requests draw windows from: each array
    with its sky, over n_chan channels at 100-200 MHz and n_time integrations
    at 10.7 s.  hex37: coplanar 37-antenna hexagon, 1,000 point sources;
    hex127: the 127-antenna jittered hexagon with 20,000 points + an nside-64
    map; hex350: the 350-antenna polarised sky (100,000 points + an nside-256
    map, FP32 fluxes) with Airy Jones beams.  ``scale`` < 1 shrinks the skies
    (source counts and nside) for quick tests."""
    out = {}
    if "hex37" in kinds:
        rng = np.random.default_rng(seed)
        ant = hex_array(3)
        freqs = channel_centres(n_chan)
        lsts = lst_grid(n_time, 10.7, rng.uniform(0, 2 * np.pi))
        sky = point_sky(max(10, int(1000 * scale)), freqs, rng)
        out["hex37"] = Problem(f"hex37_{n_chan}ch_{n_time}t", ant, cross_pairs(len(ant)), sky, freqs, lsts,
                               HERA_LATITUDE_RAD, "gauss", GAUSS_FWHM_150, False, 1e-6)
    if "hex127" in kinds:
        ns = 64 if scale >= 1 else max(2, int(64 * scale))
        out["hex127"] = config_hex127(seed=seed + 1, n_chan=n_chan, n_time=n_time,
                                      n_point=max(10, int(20000 * scale)), nside=ns, eps=1e-6)
    if "hex350" in kinds:
        ns = 256 if scale >= 1 else max(2, int(256 * scale))
        out["hex350"] = config_hex350_pol(seed=seed + 2, n_chan=n_chan, n_time=n_time,
                                          n_point=max(10, int(100000 * scale)), nside=ns, eps=1e-6,
                                          dtype=np.float32)
    return out


@dataclass
class ServeRequest:
    rid: int
    arrival_s: float
    kind: str
    f_range: tuple
    t_range: tuple


def serve_requests(seed: int = 5, n_requests: int = 10000, rate_hz: float = 200.0, n_chan: int = 256,
                   n_time: int = 20, kinds=SERVE_KINDS) -> list:
    """A Poisson stream of requests (exponential inter-arrival times, mean
    1/rate_hz): each names one resident problem (uniformly), a block of
    channels whose count is log-uniform in [1, n_chan] at a uniform offset,
    and a block of 1..n_time integrations (uniform) at a uniform offset."""
    rng = np.random.default_rng(seed + 100)
    t = np.cumsum(rng.exponential(1.0 / rate_hz, n_requests))
    out = []
    for i in range(n_requests):
        kind = kinds[int(rng.integers(len(kinds)))]
        nf = int(min(n_chan, max(1, round(math.exp(rng.uniform(0.0, math.log(n_chan)))))))
        f0 = int(rng.integers(0, n_chan - nf + 1))
        nt = int(rng.integers(1, n_time + 1))
        t0 = int(rng.integers(0, n_time - nt + 1))
        out.append(ServeRequest(i, float(t[i]), kind, (f0, f0 + nf), (t0, t0 + nt)))
    return out
