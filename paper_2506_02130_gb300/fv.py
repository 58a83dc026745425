"""Python binding of libfftvis_gb300.so (argument marshalling only).

The names follow the C ABI of ``include/fv.h``: ``fv_plan``, ``fv_set_array``,
``fv_set_sky``, ``fv_execute``, ``fv_destroy`` (plus ``fv_opts_default``,
``fv_get_info``, ``fv_last_error``).  Every step of the visibility path runs
in the library's CUDA kernels; this module never computes visibilities and
has no CPU fallback: if the library is missing or no GPU is usable, calls
raise.

Host inputs are numpy arrays.  Device buffers may be passed as torch CUDA
tensors (their data pointer is handed to the library, which borrows it).
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libfftvis_gb300.so")

ABI_VERSION = 5          # FV_ABI_VERSION of include/fv.h that the structs below mirror
FV_OK, FV_ERR_ARG, FV_ERR_OOM, FV_ERR_CUDA, FV_ERR_STATE, FV_ERR_TIMEOUT, FV_ERR_UNSUPPORTED = range(7)
FV_FP64, FV_MIXED = 0, 1
SPREAD = {"auto": 0, "gather": 1, "scatter": 2, "atomic": 3, "tensor": 4}
BEAMS = {"gauss": 0, "airy": 1, "uniform": 2, "grid": 3}
TRANSFORMS = {"auto": 0, "type3": 1, "lattice": 2, "basis": 3}
TRANSFORM_NAMES = {0: "auto", 1: "type3", 2: "lattice", 3: "basis"}
HEIGHTS = {"auto": 0, "grid": 1, "terms": 2}
STATUS_NAMES = {0: "FV_OK", 1: "FV_ERR_ARG", 2: "FV_ERR_OOM", 3: "FV_ERR_CUDA", 4: "FV_ERR_STATE",
                5: "FV_ERR_TIMEOUT", 6: "FV_ERR_UNSUPPORTED"}


class FvError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class fv_opts(C.Structure):
    _fields_ = [("precision", C.c_int), ("eps", C.c_double),
                ("n_freq", C.c_int), ("freq_hz", C.POINTER(C.c_double)),
                ("n_time", C.c_int), ("lst_rad", C.POINTER(C.c_double)),
                ("latitude_rad", C.c_double), ("beam", C.c_int), ("beam_param", C.c_double * 3),
                ("polarized", C.c_int), ("dims", C.c_int), ("upsampfac", C.c_double),
                ("kernel_width", C.c_int), ("cuda_stream", C.c_void_p), ("device", C.c_int),
                ("n_streams", C.c_int), ("spread_method", C.c_int), ("fft_max_radix", C.c_int),
                ("transform", C.c_int), ("lattice_tol_m", C.c_double), ("n_basis", C.c_int),
                ("bin_size", C.c_int * 2),
                ("heights", C.c_int)]


class fv_info(C.Structure):
    _fields_ = [("dims", C.c_int), ("kernel_width", C.c_int), ("beta", C.c_double),
                ("upsampfac", C.c_double), ("n_unique", C.c_int), ("n_bl", C.c_int), ("n_src", C.c_long),
                ("nf1_max", C.c_int * 3), ("nf2_max", C.c_int * 3), ("src_centre", C.c_double * 3),
                ("src_halfwidth", C.c_double * 3), ("workspace_bytes", C.c_longlong),
                ("transform", C.c_int), ("lattice", C.c_int), ("lattice_modes", C.c_int * 2),
                ("lattice_grid", C.c_int * 2), ("lattice_terms", C.c_int), ("lattice_basis", C.c_double * 4),
                ("beam_groups", C.c_int), ("basis_terms", C.c_int), ("basis_grid", C.c_int * 3),
                ("basis_fit_error", C.c_double),
                ("height_terms", C.c_int), ("spread_method", C.c_int)]


PROFILE_CLASSES = 12


class fv_profile_data(C.Structure):
    _fields_ = [("name", C.c_char_p * PROFILE_CLASSES), ("total_ms", C.c_double * PROFILE_CLASSES),
                ("launches", C.c_longlong * PROFILE_CLASSES), ("bytes", C.c_double * PROFILE_CLASSES)]


# Every function the header declares, with its C signature.
SIGNATURES = {
    "fv_opts_default": (None, [C.POINTER(fv_opts)]),
    "fv_lattice_detect": (C.c_int, [C.c_int, C.c_void_p, C.c_double, C.c_void_p, C.c_void_p]),
    "fv_plan": (C.c_int, [C.POINTER(fv_opts), C.POINTER(C.c_void_p)]),
    "fv_set_array": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_void_p]),
    "fv_set_beams": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]),
    "fv_set_beam_grid": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p]),
    "fv_set_sky": (C.c_int, [C.c_void_p, C.c_long, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_int]),
    "fv_execute": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int]),
    "fv_destroy": (C.c_int, [C.c_void_p]),
    "fv_last_error": (C.c_char_p, [C.c_void_p]),
    "fv_get_info": (C.c_int, [C.c_void_p, C.POINTER(fv_info)]),
    "fv_abi_version": (C.c_int, []),
    "fv_selftest_wait": (C.c_int, [C.c_void_p]),
    "fv_profile_enable": (C.c_int, [C.c_void_p, C.c_int]),
    "fv_profile_read": (C.c_int, [C.c_void_p, C.POINTER(fv_profile_data)]),
    "fv_execute_static": (C.c_int, [C.c_void_p, C.c_void_p]),
    "fv_batch_create": (C.c_int, [C.c_int, C.c_void_p, C.c_int, C.POINTER(C.c_void_p)]),
    "fv_batch_add": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int]),
    "fv_batch_add_range": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int,
                                     C.c_int, C.c_int, C.c_int]),
    "fv_batch_execute": (C.c_int, [C.c_void_p, C.c_int]),
    "fv_batch_clear": (C.c_int, [C.c_void_p]),
    "fv_batch_destroy": (C.c_int, [C.c_void_p]),
    "fv_batch_last_error": (C.c_char_p, [C.c_void_p]),
    "fv_batch_workspace_bytes": (C.c_longlong, [C.c_void_p]),
}

_lib = None


def load_library(path: str = LIB_PATH):
    """Load the CUDA library; raise if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise FvError(FV_ERR_CUDA, f"{path} not built: run __graft_entry__.build() (no CPU fallback)")
        lib = C.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        # the structs above mirror include/fv.h of this version; a library built from another one would
        # read them with another layout
        if lib.fv_abi_version() != ABI_VERSION:
            raise FvError(FV_ERR_STATE, f"{path} has ABI version {lib.fv_abi_version()}, this binding "
                                        f"expects {ABI_VERSION}: rebuild with __graft_entry__.build()")
        _lib = lib
    return _lib


def _ptr(a):
    """Data pointer of a numpy array or torch tensor."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return C.c_void_p(a.data_ptr())
    return C.c_void_p(a.ctypes.data)


def _check(status, plan=None):
    if status != FV_OK:
        msg = load_library().fv_last_error(plan)
        raise FvError(status, msg.decode() if msg else "")


# ---------------------------------------------------------------- C-named calls
def fv_opts_default() -> fv_opts:
    o = fv_opts()
    load_library().fv_opts_default(C.byref(o))
    return o


def fv_plan(opts: fv_opts) -> C.c_void_p:
    h = C.c_void_p()
    _check(load_library().fv_plan(C.byref(opts), C.byref(h)))
    return h


def fv_set_array(plan, enu_m: np.ndarray, pairs: np.ndarray | None = None) -> None:
    enu = np.ascontiguousarray(enu_m, dtype=np.float64)
    pr = None if pairs is None else np.ascontiguousarray(pairs, dtype=np.int32)
    _check(load_library().fv_set_array(plan, len(enu), _ptr(enu), 0 if pr is None else len(pr), _ptr(pr)), plan)


def fv_set_sky(plan, ra: np.ndarray, dec: np.ndarray, flux) -> None:
    """flux: numpy [n_stokes][n_src][n_freq] (float32/float64) or a CUDA tensor of that shape."""
    ra = np.ascontiguousarray(ra, dtype=np.float64)
    dec = np.ascontiguousarray(dec, dtype=np.float64)
    on_dev = hasattr(flux, "is_cuda") and flux.is_cuda
    if on_dev:
        if not flux.is_contiguous():
            raise ValueError("device flux must be contiguous")
        fp64 = str(flux.dtype) == "torch.float64"
        n_stokes = flux.shape[0]
    else:
        flux = np.ascontiguousarray(flux)
        if flux.dtype not in (np.float32, np.float64):
            flux = flux.astype(np.float64)
        fp64 = flux.dtype == np.float64
        n_stokes = flux.shape[0]
    _check(load_library().fv_set_sky(plan, len(ra), _ptr(ra), _ptr(dec), n_stokes, _ptr(flux), int(fp64),
                                     int(on_dev)), plan)


def fv_lattice_detect(enu_m, tol_m: float = 0.0):
    """(basis [a1_e, a1_n, a2_e, a2_n], index [n_ant][2], flat) if the antennas'
    horizontal positions form a lattice within tol_m (0 = 1e-10 m), flat telling
    whether the heights agree too; None otherwise (host only)."""
    enu = np.ascontiguousarray(enu_m, dtype=np.float64)
    n = len(enu)
    basis = np.zeros(4)
    index = np.zeros((max(n, 1), 2), dtype=np.int32)
    ok = load_library().fv_lattice_detect(n, _ptr(enu), float(tol_m), _ptr(basis), _ptr(index))
    return (basis, index[:n], ok == 1) if ok else None


def fv_execute(plan, vis) -> None:
    """vis: numpy complex array (host) or CUDA tensor (device) of the full output shape."""
    on_dev = hasattr(vis, "is_cuda") and vis.is_cuda
    _check(load_library().fv_execute(plan, _ptr(vis), int(on_dev)), plan)


STATIC_SCRATCH_BYTES = 64 << 20


def fv_execute_static(plan, vis) -> None:
    """fv_execute into a device buffer with the library's static scratch (allocates nothing)."""
    _check(load_library().fv_execute_static(plan, _ptr(vis)), plan)


def fv_selftest_wait(plan) -> None:
    """Enqueue the bounded-wait check on the plan's stream: its next execution raises FV_ERR_TIMEOUT."""
    _check(load_library().fv_selftest_wait(plan), plan)


def fv_destroy(plan) -> None:
    _check(load_library().fv_destroy(plan))


def fv_get_info(plan) -> dict:
    i = fv_info()
    _check(load_library().fv_get_info(plan, C.byref(i)), plan)
    return {"dims": i.dims, "kernel_width": i.kernel_width, "beta": i.beta, "upsampfac": i.upsampfac,
            "n_unique": i.n_unique, "n_bl": i.n_bl, "n_src": i.n_src, "nf1_max": list(i.nf1_max),
            "nf2_max": list(i.nf2_max), "src_centre": list(i.src_centre),
            "src_halfwidth": list(i.src_halfwidth), "workspace_bytes": i.workspace_bytes,
            "transform": TRANSFORM_NAMES[i.transform], "lattice": bool(i.lattice),
            "lattice_modes": list(i.lattice_modes), "lattice_grid": list(i.lattice_grid),
            "lattice_terms": i.lattice_terms, "beam_groups": i.beam_groups,
            "lattice_basis": list(i.lattice_basis), "basis_terms": i.basis_terms,
            "basis_grid": list(i.basis_grid), "basis_fit_error": i.basis_fit_error,
            "height_terms": i.height_terms,
            "spread": {v: k for k, v in SPREAD.items()}.get(i.spread_method, str(i.spread_method))}


def fv_profile_enable(plan, enable: bool = True) -> None:
    _check(load_library().fv_profile_enable(plan, int(enable)), plan)


def fv_profile_read(plan) -> dict:
    """Per kernel class: {name: {"ms", "launches", "bytes"}} since the last read."""
    d = fv_profile_data()
    _check(load_library().fv_profile_read(plan, C.byref(d)), plan)
    out = {}
    for c in range(PROFILE_CLASSES):
        name = d.name[c].decode() if d.name[c] else ""
        if name:
            out[name] = {"ms": d.total_ms[c], "launches": d.launches[c], "bytes": d.bytes[c]}
    return out


def _check_batch(status, b):
    if status != FV_OK:
        msg = load_library().fv_batch_last_error(b)
        raise FvError(status, msg.decode() if msg else "")


class Batch:
    """Slices of many plans executed together on shared lanes (fv_batch_*)."""

    def __init__(self, device: int = -1, stream=None, n_lanes: int = 0):
        if stream == 0:
            raise ValueError("pass a non-default stream, or None for a batch-owned stream")
        h = C.c_void_p()
        _check_batch(load_library().fv_batch_create(device, None if stream is None else C.c_void_p(stream),
                                                    n_lanes, C.byref(h)), None)
        self.handle = h
        self._keep = []

    def add(self, plan: "Plan", vis, t_range=None, f_range=None, window=None):
        """Slices t_range x f_range of plan into vis.  vis has the plan's full
        output shape, or with window = (f0, t0, nt) holds the channels from f0
        and nt times from t0: slice (t, f) at index (f - f0) * nt + (t - t0)."""
        t_lo, t_hi = t_range or (0, plan.n_time)
        f_lo, f_hi = f_range or (0, plan.n_freq)
        self._keep.append((plan, vis))
        lib = load_library()
        if window is None:
            st = lib.fv_batch_add(self.handle, plan.handle, _ptr(vis), t_lo, t_hi, f_lo, f_hi)
        else:
            f0, t0, nt = window
            st = lib.fv_batch_add_range(self.handle, plan.handle, _ptr(vis), t_lo, t_hi, f_lo, f_hi, f0, t0, nt)
        _check_batch(st, self.handle)

    def execute(self, use_graph: bool = False):
        _check_batch(load_library().fv_batch_execute(self.handle, int(use_graph)), self.handle)

    def clear(self):
        _check_batch(load_library().fv_batch_clear(self.handle), self.handle)
        self._keep = []

    @property
    def workspace_bytes(self) -> int:
        return int(load_library().fv_batch_workspace_bytes(self.handle))

    def close(self):
        if self.handle:
            load_library().fv_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- convenience
@dataclass
class Plan:
    """Owns one fv_plan_t; ``run`` fills a host or device output."""
    handle: C.c_void_p
    n_freq: int
    n_time: int
    n_bl: int
    n_pol: int
    precision: int
    _keep: tuple = ()

    @classmethod
    def create(cls, freqs_hz, lsts_rad, latitude_rad, beam="gauss", beam_param=(), precision=FV_FP64,
               eps=1e-10, polarized=False, dims=0, upsampfac=0.0, kernel_width=0, stream=None, device=-1,
               n_streams=0, spread="auto", fft_max_radix=0, transform="auto", lattice_tol_m=0.0, n_basis=0,
               bin_size=(0, 0), heights="auto"):
        o = fv_opts_default()
        freqs = np.ascontiguousarray(freqs_hz, dtype=np.float64)
        lsts = np.ascontiguousarray(lsts_rad, dtype=np.float64)
        o.precision = precision
        o.eps = eps
        o.n_freq = len(freqs)
        o.freq_hz = freqs.ctypes.data_as(C.POINTER(C.c_double))
        o.n_time = len(lsts)
        o.lst_rad = lsts.ctypes.data_as(C.POINTER(C.c_double))
        o.latitude_rad = latitude_rad
        o.beam = BEAMS[beam]
        for k, v in enumerate(beam_param):
            o.beam_param[k] = v
        o.polarized = int(polarized)
        o.dims = dims
        o.upsampfac = upsampfac
        o.kernel_width = kernel_width
        if stream == 0:
            raise ValueError("stream 0 (the legacy default stream) cannot be passed as a handle: "
                             "pass a non-default stream, or None for a plan-owned stream")
        o.cuda_stream = None if stream is None else C.c_void_p(stream)
        o.device = device
        o.n_streams = n_streams
        o.spread_method = SPREAD[spread]
        o.fft_max_radix = fft_max_radix
        o.transform = TRANSFORMS[transform]
        o.lattice_tol_m = lattice_tol_m
        o.n_basis = n_basis
        o.bin_size[0], o.bin_size[1] = int(bin_size[0]), int(bin_size[1])
        o.heights = HEIGHTS[heights]
        h = fv_plan(o)
        return cls(h, len(freqs), len(lsts), 0, 4 if polarized else 1, precision)

    @classmethod
    def from_problem(cls, prob, precision=FV_FP64, eps=None, **kw):
        grid = prob.beam == "grid"
        p = cls.create(prob.freqs_hz, prob.lsts_rad, prob.latitude_rad, "uniform" if grid else prob.beam,
                       () if grid else prob.beam_param, precision, prob.eps if eps is None else eps,
                       prob.polarized, **kw)
        p.set_array(prob.ant_enu, prob.pairs)
        if grid:
            p.set_beam_grid(-1, prob.beam_grids[-1], getattr(prob, "beam_grid_order", 1))
        return p

    def set_array(self, enu_m, pairs=None):
        fv_set_array(self.handle, enu_m, pairs)
        self.n_bl = fv_get_info(self.handle)["n_bl"]

    def set_beams(self, beams, beam_of_ant, grids=None, grid_order=1):
        """Per-antenna beams: beams = [(kind, params), ...], beam_of_ant = beam index per antenna
        (None or an empty list: the plan's single beam).  A beam of kind "grid" takes its samples
        [n_freq][n_theta][n_phi] from grids[k] (fv_set_beam_grid, interpolation order grid_order)."""
        if not beams or beam_of_ant is None:
            _check(load_library().fv_set_beams(self.handle, 0, None, None, None), self.handle)
            return
        kinds = np.ascontiguousarray([BEAMS["uniform" if k == "grid" else k] for k, _ in beams], dtype=np.int32)
        params = np.ascontiguousarray([list(v) + [0.0] * (3 - len(v)) for _, v in beams], dtype=np.float64)
        boa = np.ascontiguousarray(beam_of_ant, dtype=np.int32)
        _check(load_library().fv_set_beams(self.handle, len(kinds), _ptr(kinds), _ptr(params), _ptr(boa)),
               self.handle)
        for k, (kind, _) in enumerate(beams):
            if kind == "grid":
                self.set_beam_grid(k, grids[k], grid_order)

    def set_beam_grid(self, beam, samples, order=1):
        """Gridded beam (fv_set_beam_grid): voltage samples [n_freq][n_theta][n_phi] for beam index
        `beam` (-1: the plan's beam), interpolated bilinearly (order 1) or by bicubic B-splines (3)."""
        a = np.ascontiguousarray(samples, dtype=np.float64)
        if a.ndim != 3 or a.shape[0] != self.n_freq:
            raise ValueError("beam samples must be [n_freq][n_theta][n_phi]")
        _check(load_library().fv_set_beam_grid(self.handle, int(beam), a.shape[1], a.shape[2], int(order),
                                               _ptr(a)), self.handle)

    def set_sky(self, ra, dec, flux):
        self._keep = (flux,)          # a device flux is borrowed by the plan
        fv_set_sky(self.handle, ra, dec, flux)

    @property
    def out_shape(self):
        return (self.n_freq, self.n_time, self.n_bl, self.n_pol)

    @property
    def out_dtype(self):
        return np.complex128 if self.precision == FV_FP64 else np.complex64

    def run(self, out=None):
        if out is None:
            out = np.empty(self.out_shape, dtype=self.out_dtype)
        fv_execute(self.handle, out)
        return out

    def info(self):
        return fv_get_info(self.handle)

    def close(self):
        if self.handle:
            fv_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
