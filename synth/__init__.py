"""Seeded synthetic CCD frames (inputs only; none of the cleaning arithmetic).

The generator is C++ (``synth.cpp``) loaded through ctypes. It is shared by the
CUDA path's tests and benchmark and by the oracle's tests, so both sides read
the same bytes. ``workloads`` lists the five benchmark workloads.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_build", "libsynth.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``synth.cpp`` into ``_build/libsynth.so`` (OpenMP if available)."""
    src = os.path.join(_HERE, "synth.cpp")
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(src):
        return _LIB_PATH
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    base = ["g++", "-std=c++17", "-O2", "-fPIC", "-shared", "-ffp-contract=off", src, "-o", tmp]
    try:
        subprocess.run(base[:5] + ["-fopenmp"] + base[5:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.synth_frame.restype = ctypes.c_int
            lib.synth_frame.argtypes = [
                ctypes.c_int, ctypes.c_int, ctypes.c_uint64, ctypes.c_int, ctypes.c_double,
                ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                ctypes.c_void_p, ctypes.c_void_p,
            ]
            _lib = lib
    return _lib


# Densities of the 800x800 workload (200 stars, 1500 cosmic rays on 0.64 Mpix),
# used to scale star and cosmic-ray counts with frame area.
STAR_DENSITY = 200 / 640000.0
CR_DENSITY = 1500 / 640000.0


def frame(w: int, h: int, *, seed: int = 0, index: int = 0, sky: float = 100.0, gain: float = 7.0,
          readnoise: float = 5.0, nstars: int | None = None, ncr: int | None = None,
          truth: bool = False):
    """One frame in DN as a float32 array of shape (h, w).

    ``nstars``/``ncr`` default to the 800x800 workload densities scaled by area.
    With ``truth=True`` also returns the uint8 cosmic-ray truth mask.
    """
    if nstars is None:
        nstars = int(round(STAR_DENSITY * w * h))
    if ncr is None:
        ncr = int(round(CR_DENSITY * w * h))
    out = np.empty((h, w), dtype=np.float32)
    tr = np.empty((h, w), dtype=np.uint8) if truth else None
    rc = _load().synth_frame(w, h, seed, index, sky, gain, readnoise, nstars, ncr,
                             out.ctypes.data, tr.ctypes.data if truth else None)
    if rc != 0:
        raise ValueError(f"synth_frame rejected w={w} h={h} gain={gain}")
    return (out, tr) if truth else out


def flat(w: int, h: int, *, seed: int = 0, index: int = 0, sky: float = 100.0, gain: float = 7.0,
         readnoise: float = 5.0):
    """Noise-only flat field: Poisson sky plus read noise, no stars, no cosmic rays."""
    return frame(w, h, seed=seed, index=index, sky=sky, gain=gain, readnoise=readnoise,
                 nstars=0, ncr=0)
