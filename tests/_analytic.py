"""Reference values fixed by mathematics, independent of the oracle's code.

Analytic diffuse skies (Section 4.1; profiles listed there, read with the
angle as zenith angle): for an azimuthally symmetric brightness I(theta) about
the zenith, no beam and a coplanar baseline of length |u| wavelengths, the
hemisphere integral of I e^{-2 pi i u.s} reduces to
    V(u) = 2 pi int_0^{pi/2} I(theta) J0(2 pi |u| sin theta) sin theta dtheta.
For the constant profile this has the closed form 2 pi sin(2 pi|u|)/(2 pi|u|)
(half of the full-sphere 4 pi sinc, by the up/down symmetry of the integrand).
"""
import numpy as np
from scipy import integrate, special


def monopole(u):
    u = np.asarray(u, dtype=float)
    k = 2 * np.pi * u
    return np.where(k == 0, 2 * np.pi, 2 * np.pi * np.sin(k) / np.where(k == 0, 1, k))


def profile(name, theta, sigma=0.5):
    if name == "monopole":
        return np.ones_like(theta)
    if name == "quaddome":
        return (1 - np.sin(theta) ** 2) * np.cos(theta)
    if name == "gauss":
        return np.exp(-np.sin(theta) ** 2 / (2 * sigma ** 2))
    raise KeyError(name)


def radial(name, u, sigma=0.5):
    out = []
    for uu in np.atleast_1d(u):
        f = lambda th: profile(name, np.array(th), sigma) * special.j0(2 * np.pi * uu * np.sin(th)) * np.sin(th)
        val, _ = integrate.quad(f, 0, np.pi / 2, limit=400, epsabs=1e-14, epsrel=1e-12)
        out.append(2 * np.pi * val)
    return np.array(out)
