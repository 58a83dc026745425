"""FP64 CPU oracle for the spectral-basis route (Appendix A) -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may use this module; the product never imports it.

Appendix A replaces the per-channel transforms of a wide-band simulation by
one transform per function of a compact spectral basis.  This module takes its
steps in the appendix's order, in plain numpy:

  1. the basis M (N_nu x K): here the polynomials of degree < K in the channel
     frequency, mapped to [-1, 1] over the band and orthonormalised over the
     channels (QR of the Chebyshev Vandermonde matrix).  Reading: the columns
     are orthonormal, M^T M = I; only then do the structure constants of
     Eq. A4 give the basis coefficients of the projected product, and the
     result depends on the span of M only (tested);
  2. sky coefficients per source, s_hat = (M^T M)^{-1} M^T s (Eq. A1), s the
     source's flux at the channels;
  3. at each time, the beam b at every visible source and channel, and its
     coefficients b_hat = (M^T M)^{-1} M^T b (Eq. A2).  The appendix
     interpolates coefficients stored on a beam grid to the source
     positions; here the beam is evaluated at each source's position at every
     channel (analytic, or bilinear in a gridded beam's samples, Section 2.4)
     and projected.  b is the power beam |A|^2, or A_i A_j
     for a baseline whose antennas carry different beams (Section 2.2.3);
  4. the product coefficients v_k = sum_ij s_hat_i b_hat_j d^k_ij with the
     structure constants d^k_ij = sum_q M_qi M_qj M_qk (Eqs. A3-A4);
  5. one transform per basis function, T_k(b) = sum_n v_nk e^{-i 2 pi nu b.s_n / c},
     expanded to the channels, V(b, nu_q) = sum_k M_qk T_k at nu_q.  The sum
     over k is linear, so this is the FP64 direct sum of ``oracle_vis`` with the
     per-channel strengths c~_n(nu_q) = sum_k M_qk v_nk and a unit beam, one time
     at a time.

Unpolarised skies only: Appendix A treats a scalar sky and beam.
"""
from __future__ import annotations

from dataclasses import replace

import numpy as np

from .oracle import (OracleProblem, bspline_coefficients, oracle_enu, oracle_vis, oracle_voltage,
                     oracle_voltage_grid, oracle_voltage_grid3)


def basis_matrix(freqs_hz, K: int) -> np.ndarray:
    """Orthonormal basis of the polynomials of degree < K in frequency, sampled at the channels."""
    nu = np.asarray(freqs_hz, dtype=np.float64)
    if not 1 <= K <= len(nu):
        raise ValueError("need 1 <= K <= number of channels")
    lo, hi = nu.min(), nu.max()
    x = (2.0 * nu - lo - hi) / (hi - lo) if hi > lo else np.zeros_like(nu)
    V = np.polynomial.chebyshev.chebvander(x, K - 1)
    Q, _ = np.linalg.qr(V)
    return Q


def structure_constants(M: np.ndarray) -> np.ndarray:
    """d[i, j, k] = sum_q M_qi M_qj M_qk (Eq. A4)."""
    return np.einsum("qi,qj,qk->ijk", M, M, M)


def project(M: np.ndarray, y: np.ndarray) -> np.ndarray:
    """Least-squares coefficients (M^T M)^{-1} M^T y of the rows of y [.., N_nu] (Eqs. A1-A2)."""
    return np.linalg.solve(M.T @ M, M.T @ np.asarray(y, dtype=np.float64).T).T


def product_coefficients(s_hat: np.ndarray, b_hat: np.ndarray, d: np.ndarray) -> np.ndarray:
    """v_k = sum_ij s_hat_i b_hat_j d^k_ij per source (Eq. A3)."""
    return np.einsum("ni,nj,ijk->nk", s_hat, b_hat, d)


def _beam_groups(p: OracleProblem):
    """Baselines grouped by the unordered pair of their antennas' beams: [((a, b), baseline indices)]."""
    pairs = np.asarray(p.pairs)
    if p.beam_of_ant is None or not p.beams:
        return [((0, 0), np.arange(len(pairs)))]
    boa = np.asarray(p.beam_of_ant)
    key = np.sort(np.stack([boa[pairs[:, 0]], boa[pairs[:, 1]]], axis=1), axis=1)
    out = []
    for a, b in sorted({(int(x), int(y)) for x, y in key}):
        out.append(((a, b), np.nonzero((key[:, 0] == a) & (key[:, 1] == b))[0]))
    return out


def _voltages(p: OracleProblem, beam: int, theta: np.ndarray, az: np.ndarray) -> np.ndarray:
    """[n_src][N_nu] voltage of beam `beam` (index into p.beams, or the plan's beam); gridded beams
    (Section 2.4) by the oracle's bilinear interpolation of their samples at each channel."""
    per_antenna = bool(p.beams) and p.beam_of_ant is not None
    kind, param = p.beams[beam] if per_antenna else (p.beam, p.beam_param)
    out = np.empty((len(theta), len(p.freqs_hz)))
    if kind == "grid":
        G = np.asarray(p.beam_grids[beam if per_antenna else -1], dtype=np.float64)
        cubic = p.beam_grid_order == 3
        coefs = [bspline_coefficients(G[q]) for q in range(len(p.freqs_hz))] if cubic else None
        for n, (th, a) in enumerate(zip(theta, az)):
            for q in range(len(p.freqs_hz)):
                out[n, q] = (oracle_voltage_grid3(G[q], float(th), float(a), coefs[q]) if cubic
                             else oracle_voltage_grid(G[q], float(th), float(a)))
        return out
    for n, th in enumerate(theta):
        for q, nu in enumerate(p.freqs_hz):
            out[n, q] = oracle_voltage(kind, param, float(th), float(nu))
    return out


def basis_strengths(p: OracleProblem, M: np.ndarray, t: int, beams=(0, 0)):
    """Visible sources at time t and their per-channel strengths c~ = M v (steps 2-4)."""
    if p.polarized:
        raise ValueError("the spectral-basis route is defined for unpolarised skies")
    d = structure_constants(M)
    s_hat = project(M, p.flux[0])                         # [n_src][K]
    dirs = np.array([oracle_enu(float(r), float(de), float(p.lsts_rad[t]), float(p.latitude_rad))
                     for r, de in zip(p.ra, p.dec)]).reshape(-1, 3)
    vis = np.nonzero(dirs[:, 2] > 0.0)[0]
    theta = np.arccos(np.minimum(dirs[vis, 2], 1.0))
    az = np.arctan2(dirs[vis, 0], dirs[vis, 1])
    A = _voltages(p, beams[0], theta, az)
    B = A * A if beams[0] == beams[1] else A * _voltages(p, beams[1], theta, az)
    b_hat = project(M, B)
    v = product_coefficients(s_hat[vis], b_hat, d)
    return vis, v @ M.T                                    # [n_vis][N_nu]


def basis_vis(p: OracleProblem, K: int | None = None, M: np.ndarray | None = None,
              mode: str = "literal") -> np.ndarray:
    """Complex128 visibilities [N_nu][n_time][n_bl][1] of the spectral-basis route (steps 1-5)."""
    if M is None:
        M = basis_matrix(p.freqs_hz, K)
    out = np.zeros((len(p.freqs_hz), len(p.lsts_rad), len(p.pairs), 1), dtype=np.complex128)
    for t in range(len(p.lsts_rad)):
        for beams, bls in _beam_groups(p):
            vis, c = basis_strengths(p, M, t, beams)
            if len(vis) == 0 or len(bls) == 0:
                continue
            sub = replace(p, pairs=np.asarray(p.pairs)[bls], ra=np.asarray(p.ra)[vis], dec=np.asarray(p.dec)[vis],
                          flux=c[None], lsts_rad=np.asarray(p.lsts_rad)[t:t + 1], beam="uniform",
                          beam_param=(), polarized=False, beams=None, beam_of_ant=None, beam_grids=None,
                          beam_grid_order=1)
            out[:, t, bls, :] = oracle_vis(sub, mode)[:, 0]
    return out
