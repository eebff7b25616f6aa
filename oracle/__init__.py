"""ORACLE -- TEST INFRASTRUCTURE ONLY.

Plain CPU L.A.Cosmic (``lacosmic.cpp``) and the POISSON work function
(``poisson.cpp``) used to check the CUDA library. Only
the test suite, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package; the product path never does.

``clean``/``iterate`` take ``precision="f64"`` (the reference) or ``"f32"``
(the same steps in single precision, in the same order, for decision-exact
comparisons with an FP32 kernel).
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_POISSON_PATH = os.path.join(_HERE, "_build", "libpoisson.so")
_lock = threading.Lock()
_lib = None
_plib = None

MAP_NAMES = ("m5", "lplus", "noise", "s", "sprime", "m3", "f", "r", "cand", "g1", "g2")


class _Params(ctypes.Structure):
    _fields_ = [("gain", ctypes.c_double), ("readnoise", ctypes.c_double),
                ("sigclip", ctypes.c_double), ("sigfrac", ctypes.c_double),
                ("objlim", ctypes.c_double), ("objlim_form", ctypes.c_int)]


@dataclass
class Params:
    """Cleaning parameters. Values are rounded to float32 first, as the C API takes floats."""
    gain: float = 7.0
    readnoise: float = 5.0
    sigclip: float = 4.5
    sigfrac: float = 0.5
    objlim: float = 1.0
    objlim_form: int = 0  # 0: script form (default); 1: article form

    def _c(self):
        f = lambda v: float(np.float32(v))  # noqa: E731
        return _Params(f(self.gain), f(self.readnoise), f(self.sigclip), f(self.sigfrac),
                       f(self.objlim), int(self.objlim_form))


def build(force: bool = False, src: str | None = None, out: str | None = None,
          defines: tuple = ()) -> str:
    """Compile the oracle into a shared library (OpenMP if available).

    ``src``/``out`` default to ``lacosmic.cpp`` and ``_build/liboracle.so``.
    """
    src = src or os.path.join(_HERE, "lacosmic.cpp")
    out = out or _LIB_PATH
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(src):
        return out
    os.makedirs(os.path.dirname(out), exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    base = ["g++", "-std=c++17", "-O2", "-fPIC", "-shared", "-ffp-contract=off",
            *[f"-D{d}" for d in defines], src, "-o", tmp]
    try:
        subprocess.run(base[:5] + ["-fopenmp"] + base[5:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True)
    os.replace(tmp, out)
    return out


def _bind(path: str):
    lib = ctypes.CDLL(path)
    P = ctypes.POINTER(_Params)
    vp, ci = ctypes.c_void_p, ctypes.c_int
    for name in ("oracle_iter_f64", "oracle_iter_f32"):
        fn = getattr(lib, name)
        fn.restype = ci
        fn.argtypes = [vp, vp, ci, ci, P, vp, vp, vp, vp, vp]
    for name in ("oracle_clean_f64", "oracle_clean_f32"):
        fn = getattr(lib, name)
        fn.restype = ci
        fn.argtypes = [vp, ci, ci, P, ci, vp, vp, vp, vp]
    for name in ("oracle_replace_f64", "oracle_replace_f32"):
        fn = getattr(lib, name)
        fn.restype = ci
        fn.argtypes = [vp, vp, ci, ci, vp, vp]
    lib.oracle_median_filter_f64.restype = ci
    lib.oracle_median_filter_f64.argtypes = [vp, ci, ci, ci, vp]
    lib.oracle_lplus_f64.restype = ci
    lib.oracle_lplus_f64.argtypes = [vp, ci, ci, vp]
    lib.oracle_set_threads.argtypes = [ci]
    lib.oracle_set_threads.restype = None
    lib.oracle_max_threads.restype = ci
    lib.oracle_num_maps.restype = ci
    assert lib.oracle_num_maps() == len(MAP_NAMES)
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _bind(build())
    return _lib


class Oracle:
    """The oracle API bound to one compiled library (the default one, or a test's variant)."""

    def __init__(self, path: str | None = None):
        self._path = path

    @property
    def lib(self):
        return _load() if self._path is None else _bind_cached(self._path)

    def median_filter(self, img, r):
        return median_filter(img, r, lib=self.lib)

    def lplus(self, img):
        return lplus(img, lib=self.lib)

    def replace(self, J, Mk, precision="f64"):
        return replace(J, Mk, precision, lib=self.lib)

    def iterate(self, J, Mprev, params, **kw):
        return iterate(J, Mprev, params, lib=self.lib, **kw)

    def clean(self, I0, params, niter=4, **kw):
        return clean(I0, params, niter, lib=self.lib, **kw)


_bound = {}


def _bind_cached(path):
    with _lock:
        if path not in _bound:
            _bound[path] = _bind(path)
        return _bound[path]


def set_threads(n: int) -> None:
    _load().oracle_set_threads(int(n))


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _u8(a):
    return np.ascontiguousarray(a, dtype=np.uint8)


def median_filter(img, r: int, *, lib=None):
    """Clamped (2r+1)^2 median filter in float64."""
    a = np.ascontiguousarray(img, dtype=np.float64)
    h, w = a.shape
    out = np.empty_like(a)
    if (lib or _load()).oracle_median_filter_f64(a.ctypes.data, w, h, int(r), out.ctypes.data) != 0:
        raise ValueError("oracle_median_filter_f64 rejected its arguments")
    return out


def lplus(img, *, lib=None):
    """Stage (a) L+ in float64."""
    a = np.ascontiguousarray(img, dtype=np.float64)
    h, w = a.shape
    out = np.empty_like(a)
    if (lib or _load()).oracle_lplus_f64(a.ctypes.data, w, h, out.ctypes.data) != 0:
        raise ValueError("oracle_lplus_f64 rejected its arguments")
    return out


def replace(J, Mk, precision: str = "f64", *, lib=None):
    """Stage (e) alone. Returns (I_k, count of flagged pixels with no unflagged neighbour)."""
    J = _f32(J)
    Mk = _u8(Mk)
    h, w = J.shape
    out = np.empty_like(J)
    c = ctypes.c_longlong(0)
    fn = getattr(lib or _load(), f"oracle_replace_{precision}")
    if fn(J.ctypes.data, Mk.ctypes.data, w, h, out.ctypes.data, ctypes.byref(c)) != 0:
        raise ValueError("oracle_replace rejected its arguments")
    return out, int(c.value)


@dataclass
class IterResult:
    Ik: np.ndarray
    Mk: np.ndarray
    maps: dict | None
    fragile: np.ndarray | None
    n_new: int
    n_none_left: int


def iterate(J, Mprev, params: Params, *, precision: str = "f64", maps: bool = False,
            fragile: bool = False, lib=None) -> IterResult:
    """One iteration from (J = I_{k-1}, M_{k-1}); Mprev may be None (no flags)."""
    J = _f32(J)
    h, w = J.shape
    Mp = None if Mprev is None else _u8(Mprev)
    Ik = np.empty_like(J)
    Mk = np.empty((h, w), dtype=np.uint8)
    dt = np.float64 if precision == "f64" else np.float32
    mp = np.empty((len(MAP_NAMES), h, w), dtype=dt) if maps else None
    fr = np.empty((h, w), dtype=np.uint8) if fragile else None
    counts = (ctypes.c_longlong * 2)()
    fn = getattr(lib or _load(), f"oracle_iter_{precision}")
    rc = fn(J.ctypes.data, None if Mp is None else Mp.ctypes.data, w, h, ctypes.byref(params._c()),
            Ik.ctypes.data, Mk.ctypes.data, None if mp is None else mp.ctypes.data,
            None if fr is None else fr.ctypes.data, counts)
    if rc != 0:
        raise ValueError("oracle_iter rejected its arguments")
    md = {n: mp[i] for i, n in enumerate(MAP_NAMES)} if maps else None
    return IterResult(Ik, Mk, md, fr, int(counts[0]), int(counts[1]))


@dataclass
class CleanResult:
    clean: np.ndarray
    mask: np.ndarray
    n_new: list
    n_none_left: list
    fragile: np.ndarray | None


def clean(I0, params: Params, niter: int = 4, *, precision: str = "f64",
          fragile: bool = False, lib=None) -> CleanResult:
    """niter iterations from I0; returns the cleaned frame and the cumulative mask."""
    I0 = _f32(I0)
    h, w = I0.shape
    out = np.empty_like(I0)
    mask = np.empty((h, w), dtype=np.uint8)
    counts = (ctypes.c_longlong * max(2 * niter, 1))()
    fr = np.empty((h, w), dtype=np.uint8) if fragile else None
    fn = getattr(lib or _load(), f"oracle_clean_{precision}")
    rc = fn(I0.ctypes.data, w, h, ctypes.byref(params._c()), int(niter), out.ctypes.data,
            mask.ctypes.data, counts, None if fr is None else fr.ctypes.data)
    if rc != 0:
        raise ValueError("oracle_clean rejected its arguments")
    return CleanResult(out, mask, [int(counts[2 * k]) for k in range(niter)],
                       [int(counts[2 * k + 1]) for k in range(niter)], fr)


# --- POISSON work function (Sec. 6.3.2) -------------------------------------------------------


def build_poisson(force: bool = False) -> str:
    """Compile ``poisson.cpp`` into ``_build/libpoisson.so``."""
    return build(force, src=os.path.join(_HERE, "poisson.cpp"), out=_POISSON_PATH)


def _load_poisson():
    global _plib
    with _lock:
        if _plib is None:
            lib = ctypes.CDLL(build_poisson())
            lib.oracle_exp_neg.restype = ctypes.c_double
            lib.oracle_exp_neg.argtypes = [ctypes.c_double]
            lib.oracle_stream_value.restype = ctypes.c_uint64
            lib.oracle_stream_value.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
            lib.oracle_algorithm_q.restype = ctypes.c_int
            lib.oracle_algorithm_q.argtypes = [ctypes.c_double, ctypes.c_void_p, ctypes.c_int]
            lib.oracle_poisson.restype = ctypes.c_int
            lib.oracle_poisson.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_uint64,
                                           ctypes.c_void_p]
            _plib = lib
    return _plib


def exp_neg(mu: float) -> float:
    """e^-mu by the fixed double-precision steps the work function uses (0 <= mu <= 700)."""
    return float(_load_poisson().oracle_exp_neg(float(mu)))


def stream_value(s: int, j: int) -> int:
    """The j-th value of the counter-based SplitMix64 stream with key s."""
    return int(_load_poisson().oracle_stream_value(s & (2**64 - 1), j & (2**64 - 1)))


def algorithm_q(mu: float, u) -> int:
    """Algorithm Q on the given uniforms; -1 if it needs more of them."""
    u = np.ascontiguousarray(u, dtype=np.float64)
    return int(_load_poisson().oracle_algorithm_q(float(mu), u.ctypes.data, int(u.size)))


def poisson(img, seed: int) -> np.ndarray:
    """The POISSON work function on one frame: a deviate of mean img[p] per pixel (float32)."""
    a = _f32(img)
    h, w = a.shape
    out = np.empty_like(a)
    if _load_poisson().oracle_poisson(a.ctypes.data, w, h, seed & (2**64 - 1), out.ctypes.data) != 0:
        raise ValueError("oracle_poisson rejected its arguments")
    return out
