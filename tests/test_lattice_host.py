"""Lattice test of Section 2.2.1 on the host (no GPU): filled hexagons and
grids are recognised with a reduced basis and integer antenna coordinates
that reproduce the positions; jittered heights, displaced antennas and
random layouts are not; degenerate layouts (one antenna, a line) are."""
import math

import numpy as np
import pytest

from paper_2506_02130_gb300 import fv, workloads as W


def _check(enu, basis, index, tol=1e-9):
    a1, a2 = basis[:2], basis[2:]
    rec = enu[0, :2] + index[:, :1] * a1 + index[:, 1:] * a2
    assert np.abs(rec - enu[:, :2]).max() <= tol


@pytest.mark.parametrize("radius,n_keep", [(3, None), (6, None), (10, None), (11, 350)])
def test_hexagons_are_lattices_with_hexagonal_basis(radius, n_keep):
    enu = W.hex_array(radius, n_keep=n_keep)
    res = fv.fv_lattice_detect(enu)
    assert res is not None
    basis, index, flat = res
    assert flat
    a1, a2 = basis[:2], basis[2:]
    assert np.linalg.norm(a1) == pytest.approx(14.6, rel=1e-12)
    assert np.linalg.norm(a2) == pytest.approx(14.6, rel=1e-12)
    assert abs(np.dot(a1, a2)) == pytest.approx(0.5 * 14.6 ** 2, rel=1e-9)   # 60 or 120 degrees
    _check(enu, basis, index)
    # baselines are integer combinations: the largest offset is within the hexagon's diameter
    assert np.abs(index).max() <= 2 * radius


def test_rotated_translated_rectangular_grid():
    th = math.radians(17.0)
    R = np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]])
    i, j = np.meshgrid(np.arange(5), np.arange(7), indexing="ij")
    pts = np.stack([3.0 * i.ravel(), 4.5 * j.ravel()], 1) @ R.T + [101.25, -37.5]
    enu = np.concatenate([pts, np.full((len(pts), 1), 1070.0)], 1)
    basis, index, flat = fv.fv_lattice_detect(enu)
    assert flat
    lens = sorted([np.linalg.norm(basis[:2]), np.linalg.norm(basis[2:])])
    assert lens == pytest.approx([3.0, 4.5], rel=1e-12)
    assert abs(np.dot(basis[:2], basis[2:])) < 1e-9
    _check(enu, basis, index)


def test_height_jitter_keeps_the_horizontal_lattice_but_is_not_flat():
    enu = W.hex_array(4, z_sigma_m=0.05, rng=np.random.default_rng(0))
    basis, index, flat = fv.fv_lattice_detect(enu)
    assert not flat
    _check(enu, basis, index)
    enu[:, 2] = 0.0
    assert fv.fv_lattice_detect(enu)[2]


def test_displacement_against_tolerance():
    enu = W.hex_array(3)
    enu[5, 0] += 1e-6
    assert fv.fv_lattice_detect(enu) is None                 # default tolerance 1e-10 m
    basis, index, _ = fv.fv_lattice_detect(enu, tol_m=1e-5)
    _check(enu, basis, index, tol=1e-5)           # every antenna within the tolerance of its lattice point


def test_random_layout_is_not_a_lattice():
    enu = np.zeros((40, 3))
    enu[:, :2] = np.random.default_rng(3).uniform(-100, 100, (40, 2))
    assert fv.fv_lattice_detect(enu) is None


def test_degenerate_layouts():
    one = np.array([[3.0, 4.0, 5.0]])
    basis, index, _ = fv.fv_lattice_detect(one)
    assert (index == 0).all()
    line = np.array([[2.0 * k, 0.0, 0.0] for k in (0, 1, 3, 4)])
    basis, index, _ = fv.fv_lattice_detect(line)
    assert (index[:, 1] == 0).all()
    _check(line, basis, index)
    assert np.linalg.norm(basis[:2]) == pytest.approx(2.0)
