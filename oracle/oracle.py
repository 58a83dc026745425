"""ctypes wrapper around ``oracle.c`` (test infrastructure only; see package doc)."""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass, replace

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

BEAMS = {"gauss": 0, "airy": 1, "uniform": 2, "grid": 3}


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so with gcc + OpenMP (no fast-math, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=gnu11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
               _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class _Problem(C.Structure):
    _fields_ = [("n_ant", C.c_int), ("ant_enu", C.POINTER(C.c_double)),
                ("n_bl", C.c_int), ("pairs", C.POINTER(C.c_int)),
                ("n_src", C.c_long), ("ra", C.POINTER(C.c_double)), ("dec", C.POINTER(C.c_double)),
                ("n_stokes", C.c_int), ("flux", C.POINTER(C.c_double)),
                ("n_freq", C.c_int), ("freq_hz", C.POINTER(C.c_double)),
                ("n_time", C.c_int), ("lst_rad", C.POINTER(C.c_double)),
                ("latitude_rad", C.c_double), ("beam_kind", C.c_int),
                ("beam_param", C.c_double * 3), ("polarized", C.c_int),
                ("n_beams", C.c_int), ("beam_kinds", C.POINTER(C.c_int)),
                ("beam_params", C.POINTER(C.c_double)), ("beam_of_ant", C.POINTER(C.c_int)),
                ("grid_n_theta", C.c_int), ("grid_n_phi", C.c_int), ("beam_grids", C.POINTER(C.c_double)),
                ("grid_order", C.c_int)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            lib.oracle_vis.argtypes = [C.POINTER(_Problem), C.POINTER(C.c_double), C.c_int, C.c_int]
            lib.oracle_vis.restype = C.c_int
            lib.oracle_enu.argtypes = [C.c_double] * 4 + [C.POINTER(C.c_double)]
            lib.oracle_enu.restype = None
            lib.oracle_voltage.argtypes = [C.c_int, C.POINTER(C.c_double), C.c_double, C.c_double]
            lib.oracle_voltage.restype = C.c_double
            lib.oracle_strength.argtypes = [C.c_int, C.POINTER(C.c_double), C.c_int,
                                            C.POINTER(C.c_double), C.c_double,
                                            C.POINTER(C.c_double), C.POINTER(C.c_double)]
            lib.oracle_strength.restype = None
            lib.oracle_max_threads.restype = C.c_int
            lib.oracle_voltage_grid.argtypes = [C.POINTER(C.c_double), C.c_int, C.c_int, C.c_double, C.c_double]
            lib.oracle_voltage_grid.restype = C.c_double
            lib.oracle_voltage_grid3.argtypes = [C.POINTER(C.c_double), C.c_int, C.c_int, C.c_double, C.c_double]
            lib.oracle_voltage_grid3.restype = C.c_double
            _lib = lib
    return _lib


def _p(a):
    return a.ctypes.data_as(C.POINTER(C.c_double if a.dtype == np.float64 else C.c_int))


@dataclass
class OracleProblem:
    ant_enu: np.ndarray
    pairs: np.ndarray
    ra: np.ndarray
    dec: np.ndarray
    flux: np.ndarray            # [n_stokes][n_src][n_freq]
    freqs_hz: np.ndarray
    lsts_rad: np.ndarray
    latitude_rad: float
    beam: str = "gauss"
    beam_param: tuple = ()
    polarized: bool = False
    # per-antenna beams: [(kind, params), ...] and the beam index of every antenna (None: one beam)
    beams: list | None = None
    beam_of_ant: np.ndarray | None = None
    # gridded beams: voltage samples [n_freq][n_theta][n_phi] of the plan's beam (beam == "grid") and of
    # per-antenna beam k (beams[k] == ("grid", ())), keyed by beam index (-1: the plan's beam)
    beam_grids: dict | None = None
    beam_grid_order: int = 1            # 1 bilinear, 3 bicubic B-spline

    @classmethod
    def from_workload(cls, prob, pairs=None, freq_idx=None, time_idx=None, src_idx=None):
        """Build from a workloads.Problem, optionally restricted to subsets."""
        sky = prob.sky
        flux = sky.flux
        freqs = prob.freqs_hz
        lsts = prob.lsts_rad
        ra, dec = sky.ra, sky.dec
        if src_idx is not None:
            ra, dec, flux = ra[src_idx], dec[src_idx], flux[:, src_idx]
        if freq_idx is not None:
            freqs = freqs[freq_idx]
            flux = flux[:, :, freq_idx]
        if time_idx is not None:
            lsts = lsts[time_idx]
        grids = getattr(prob, "beam_grids", None)
        if grids is not None and freq_idx is not None:
            grids = {k: np.asarray(v)[freq_idx] for k, v in grids.items()}
        return cls(prob.ant_enu, prob.pairs if pairs is None else pairs, ra, dec, flux, freqs,
                   lsts, prob.latitude_rad, prob.beam, tuple(prob.beam_param), prob.polarized,
                   getattr(prob, "beams", None), getattr(prob, "beam_of_ant", None), grids,
                   getattr(prob, "beam_grid_order", 1))


def oracle_vis(p: OracleProblem, mode: str = "factored", n_threads: int = 0) -> np.ndarray:
    """Complex128 visibilities [n_freq][n_time][n_bl][n_pol] by FP64 direct sum."""
    lib = _load()
    ant = np.ascontiguousarray(p.ant_enu, dtype=np.float64)
    pairs = np.ascontiguousarray(p.pairs, dtype=np.int32)
    ra = np.ascontiguousarray(p.ra, dtype=np.float64)
    dec = np.ascontiguousarray(p.dec, dtype=np.float64)
    flux = np.ascontiguousarray(p.flux, dtype=np.float64)
    freqs = np.ascontiguousarray(p.freqs_hz, dtype=np.float64)
    lsts = np.ascontiguousarray(p.lsts_rad, dtype=np.float64)
    n_pol = 4 if p.polarized else 1
    bp = (C.c_double * 3)(*(list(p.beam_param) + [0.0] * (3 - len(p.beam_param))))
    nb, kinds_p, params_p, boa_p = 0, None, None, None
    grids = p.beam_grids or {}
    if p.beam == "grid" and not (p.beam_of_ant is not None and p.beams):
        # one gridded beam for every antenna: the per-antenna form with a single beam
        p = replace(p, beams=[("grid", ())], beam_of_ant=np.zeros(len(ant), dtype=np.int32),
                    beam_grids={0: grids[-1]})
        grids = p.beam_grids
    gth, gph, grid_p = 0, 0, None
    if p.beam_of_ant is not None and p.beams:
        kinds = np.ascontiguousarray([BEAMS[k] for k, _ in p.beams], dtype=np.int32)
        params = np.ascontiguousarray([list(v) + [0.0] * (3 - len(v)) for _, v in p.beams], dtype=np.float64)
        boa = np.ascontiguousarray(p.beam_of_ant, dtype=np.int32)
        if len(boa) != len(ant):
            raise ValueError("beam_of_ant needs one entry per antenna")
        nb, kinds_p, params_p = len(kinds), kinds.ctypes.data_as(C.POINTER(C.c_int)), _p(params)
        boa_p = boa.ctypes.data_as(C.POINTER(C.c_int))
        gridded = [k for k, (kind, _) in enumerate(p.beams) if kind == "grid"]
        if gridded:
            shape = np.asarray(grids[gridded[0]]).shape
            if len(shape) != 3 or shape[0] != len(freqs):
                raise ValueError("gridded beams need [n_freq][n_theta][n_phi] samples")
            allg = np.zeros((len(kinds),) + shape)
            for k in gridded:
                g = np.asarray(grids[k], dtype=np.float64)
                allg[k] = g if p.beam_grid_order == 1 else np.stack([bspline_coefficients(pl) for pl in g])
            allg = np.ascontiguousarray(allg)
            gth, gph, grid_p = shape[1], shape[2], _p(allg)
        keep = (kinds, params, boa, grid_p and allg)     # alive for the call
    prob = _Problem(len(ant), _p(ant), len(pairs), pairs.ctypes.data_as(C.POINTER(C.c_int)),
                    len(ra), _p(ra), _p(dec), flux.shape[0], _p(flux), len(freqs), _p(freqs),
                    len(lsts), _p(lsts), float(p.latitude_rad), BEAMS[p.beam], bp,
                    1 if p.polarized else 0, nb, kinds_p, params_p, boa_p, gth, gph, grid_p,
                    int(p.beam_grid_order))
    out = np.zeros((len(freqs), len(lsts), len(pairs), n_pol, 2), dtype=np.float64)
    rc = lib.oracle_vis(C.byref(prob), _p(out), 0 if mode == "literal" else 1, int(n_threads))
    if rc != 0:
        raise RuntimeError(f"oracle_vis failed with code {rc}")
    return out[..., 0] + 1j * out[..., 1]


def oracle_enu(ra: float, dec: float, lst: float, lat: float) -> np.ndarray:
    out = np.zeros(3)
    _load().oracle_enu(ra, dec, lst, lat, _p(out))
    return out


def oracle_voltage(beam: str, param, theta: float, nu: float) -> float:
    bp = np.array(list(param) + [0.0] * (3 - len(param)), dtype=np.float64)
    return _load().oracle_voltage(BEAMS[beam], _p(bp), theta, nu)


def oracle_strength(beam: str, param, polarized: bool, s, nu: float, stokes) -> np.ndarray:
    bp = np.array(list(param) + [0.0] * (3 - len(param)), dtype=np.float64)
    s = np.ascontiguousarray(s, dtype=np.float64)
    st = np.ascontiguousarray(list(stokes) + [0.0] * (4 - len(stokes)), dtype=np.float64)
    n_pol = 4 if polarized else 1
    out = np.zeros(2 * n_pol)
    _load().oracle_strength(BEAMS[beam], _p(bp), 1 if polarized else 0, _p(s), nu, _p(st), _p(out))
    return out[0::2] + 1j * out[1::2]


def oracle_voltage_grid(plane, theta: float, az: float) -> float:
    """Bilinear voltage of a gridded beam's samples plane[n_theta][n_phi] (see oracle.c)."""
    a = np.ascontiguousarray(plane, dtype=np.float64)
    return _load().oracle_voltage_grid(_p(a), a.shape[0], a.shape[1], float(theta), float(az))


def _collocation(n: int, periodic: bool) -> np.ndarray:
    """Cubic B-spline collocation matrix of n knots at the knots: sample i = (c[i-1] + 4 c[i] + c[i+1]) / 6,
    the out-of-range knots mirrored about the end samples (c[-1] = c[1], c[n] = c[n-2]) or wrapped."""
    B = np.zeros((n, n))
    for i in range(n):
        for off, wgt in ((-1, 1.0 / 6.0), (0, 4.0 / 6.0), (1, 1.0 / 6.0)):
            k = i + off
            if periodic:
                k %= n
            else:
                if k < 0:
                    k = -k
                if k > n - 1:
                    k = 2 * (n - 1) - k
            B[i, k] += wgt
    return B


def bspline_coefficients(plane) -> np.ndarray:
    """B-spline coefficients [n_theta][n_phi] that interpolate the samples plane[n_theta][n_phi] at the
    grid nodes (mirror ends along zenith angle, periodic along azimuth): dense solves of the two
    collocation systems, one axis after the other."""
    F = np.asarray(plane, dtype=np.float64)
    nth, nph = F.shape
    Cth = np.linalg.solve(_collocation(nth, False), F) if nth > 1 else F.copy()
    return np.linalg.solve(_collocation(nph, True), Cth.T).T


def oracle_voltage_grid3(plane, theta: float, az: float, coef=None) -> float:
    """Bicubic B-spline voltage of a gridded beam's samples plane[n_theta][n_phi] (see oracle.c); coef:
    the plane's coefficients if already computed."""
    c = np.ascontiguousarray(bspline_coefficients(plane) if coef is None else coef, dtype=np.float64)
    return _load().oracle_voltage_grid3(_p(c), c.shape[0], c.shape[1], float(theta), float(az))


def max_threads() -> int:
    return _load().oracle_max_threads()


def rel_l2(a, b) -> float:
    """Relative L2 error ||a - b|| / ||b||."""
    a = np.asarray(a); b = np.asarray(b)
    nb = np.linalg.norm(b.ravel())
    return float(np.linalg.norm((a - b).ravel()) / nb) if nb > 0 else float(np.linalg.norm(a.ravel()))
