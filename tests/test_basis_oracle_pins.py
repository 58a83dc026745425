"""Pins for the spectral-basis oracle (Appendix A), independent of its own code.

The facts used: with a complete basis (K = number of channels) every projection
is the identity, so the route must reproduce the plain direct sum of Eq. 3 for
any sky and beam; a sky that is a polynomial of degree < K in frequency seen
through a flat beam is represented exactly; the structure constants of Eq. A4
are fully symmetric and, for a complete basis, resolve the product of two
basis vectors; with orthonormal columns the result depends on the span of the
basis only.  Each catches a plausible slip: a transposed M, a contraction over
the wrong index of d, a beam evaluated at the wrong channel, a missing
(M^T M)^{-1}, a per-antenna voltage paired with the wrong baseline group.
"""
import itertools
import math
from dataclasses import replace

import numpy as np
import pytest

from oracle.basis import basis_matrix, basis_vis, product_coefficients, project, structure_constants
from oracle.oracle import OracleProblem, oracle_vis, rel_l2
from paper_2506_02130_gb300 import workloads as W


def _problem(n_chan=6, n_time=2, n_point=120, beam=("gauss", (math.radians(60.0), 150e6)), seed=3):
    prob = W.config_hex127(seed=seed, n_chan=n_chan, n_time=n_time, n_point=n_point, nside=0, radius=2)
    op = OracleProblem.from_workload(prob)
    return replace(op, beam=beam[0], beam_param=tuple(beam[1]))


@pytest.mark.parametrize("beam", [("gauss", (math.radians(60.0), 150e6)), ("airy", (3.0,))])
def test_complete_basis_reproduces_the_direct_sum(beam):
    p = _problem(beam=beam)
    K = len(p.freqs_hz)
    assert rel_l2(basis_vis(p, K), oracle_vis(p, "literal")) < 1e-12


def test_complete_basis_with_per_antenna_beams():
    p = _problem(n_chan=5)
    n_ant = len(p.ant_enu)
    boa = np.arange(n_ant) % 2
    p = replace(p, beams=[("gauss", (math.radians(50.0), 150e6)), ("airy", (4.0,))], beam_of_ant=boa)
    assert rel_l2(basis_vis(p, len(p.freqs_hz)), oracle_vis(p, "literal")) < 1e-12


def test_polynomial_sky_through_a_flat_beam_is_exact_at_its_degree():
    p = _problem(n_chan=7, beam=("uniform", ()))
    nu = p.freqs_hz
    x = (nu - 150e6) / 50e6
    rng = np.random.default_rng(5)
    a = rng.uniform(0.5, 2.0, size=(len(p.ra), 3))
    flux = (a[:, 0:1] + a[:, 1:2] * x[None] - 0.4 * a[:, 2:3] * x[None] ** 2)[None]
    p = replace(p, flux=flux)
    ref = oracle_vis(p, "literal")
    assert rel_l2(basis_vis(p, 3), ref) < 1e-12
    assert rel_l2(basis_vis(p, 2), ref) > 1e-4          # the quadratic term is lost


def test_structure_constants_brute_force_symmetry_and_completeness():
    rng = np.random.default_rng(1)
    M, _ = np.linalg.qr(rng.normal(size=(5, 3)))
    d = structure_constants(M)
    for i, j, k in itertools.product(range(3), repeat=3):
        assert abs(d[i, j, k] - sum(M[q, i] * M[q, j] * M[q, k] for q in range(5))) < 1e-15
        for a, b, c in itertools.permutations((i, j, k)):
            assert d[a, b, c] == pytest.approx(d[i, j, k], abs=1e-15)
    Mf, _ = np.linalg.qr(rng.normal(size=(4, 4)))
    df = structure_constants(Mf)
    # complete basis: sum_k d^k_ij M_qk = M_qi M_qj (the product of two basis vectors, re-expanded)
    np.testing.assert_allclose(np.einsum("ijk,qk->qij", df, Mf), np.einsum("qi,qj->qij", Mf, Mf), atol=1e-14)


def test_product_coefficients_of_a_complete_basis_are_the_pointwise_product():
    rng = np.random.default_rng(2)
    M = basis_matrix(np.linspace(100e6, 200e6, 6), 6)
    s, b = rng.normal(size=(3, 6)), rng.normal(size=(3, 6))
    v = product_coefficients(project(M, s), project(M, b), structure_constants(M))
    np.testing.assert_allclose(v @ M.T, s * b, atol=1e-13)


def test_basis_is_orthonormal_and_spans_the_low_degree_polynomials():
    nu = np.linspace(100e6, 200e6, 9)
    M = basis_matrix(nu, 4)
    np.testing.assert_allclose(M.T @ M, np.eye(4), atol=1e-14)
    x = (nu - 150e6) / 50e6
    P = M @ M.T
    for j in range(4):
        np.testing.assert_allclose(P @ x ** j, x ** j, atol=1e-13)
    assert np.linalg.norm(P @ x ** 4 - x ** 4) > 1e-3
    # least squares as printed in Eqs. A1-A2 returns the coefficients of a combination of the columns
    c = np.array([0.3, -1.0, 2.0, 0.5])
    np.testing.assert_allclose(project(M, (M @ c)[None])[0], c, atol=1e-13)


def test_result_depends_on_the_span_only():
    p = _problem(n_chan=7)
    M = basis_matrix(p.freqs_hz, 4)
    R, _ = np.linalg.qr(np.random.default_rng(4).normal(size=(4, 4)))
    a, b = basis_vis(p, M=M), basis_vis(p, M=M @ R)
    assert rel_l2(a, b) < 1e-12
    assert rel_l2(a, oracle_vis(p, "literal")) > 1e-9   # a truncated basis is not the direct sum


def test_truncation_error_vanishes_as_the_basis_completes():
    p = _problem(n_chan=8, beam=("gauss", (math.radians(30.0), 150e6)))
    ref = oracle_vis(p, "literal")
    errs = [rel_l2(basis_vis(p, K), ref) for K in (2, 4, 6, 8)]
    assert errs[3] < 1e-12
    assert errs[2] < errs[0]


def test_complete_basis_with_a_gridded_beam():
    p = _problem(n_chan=5)
    p = replace(p, beam="grid", beam_grids={-1: W.grid_beam(p.freqs_hz, 31, 12, math.radians(40.0), 150e6,
                                                           ellipticity=0.3)})
    assert rel_l2(basis_vis(p, len(p.freqs_hz)), oracle_vis(p, "literal")) < 1e-12
