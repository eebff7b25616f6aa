"""ctypes binding of the C ABI in include/crb.h (argument marshalling only).

Every function keeps its C name. The library is the in-tree
``_build/libcrb.so``; if it cannot be built or loaded, importing fails loudly:
there is no CPU fallback.
"""

from __future__ import annotations

import ctypes
import threading

from . import build as _build

_lock = threading.Lock()
_lib = None

CRB_OK, CRB_EINVAL, CRB_ENOMEM, CRB_ECUDA, CRB_ETIMEOUT, CRB_EBUSY, CRB_EALIAS, CRB_EDEVICE = range(8)
NUM_MAPS = 11
MAP_NAMES = ("m5", "lplus", "noise", "s", "sprime", "m3", "f", "r", "cand", "g1", "g2")


class crb_options(ctypes.Structure):
    _fields_ = [("objlim_form", ctypes.c_int), ("early_exit", ctypes.c_int),
                ("tile_shape", ctypes.c_int), ("use_graphs", ctypes.c_int), ("profile", ctypes.c_int),
                ("no_fusion", ctypes.c_int), ("pipeline", ctypes.c_int), ("autotune", ctypes.c_int),
                ("fuse2", ctypes.c_int)]


class crb_rect(ctypes.Structure):
    _fields_ = [("x0", ctypes.c_int), ("y0", ctypes.c_int), ("w", ctypes.c_int), ("h", ctypes.c_int),
                ("cx0", ctypes.c_int), ("cy0", ctypes.c_int), ("cw", ctypes.c_int), ("ch", ctypes.c_int)]


# (name, restype, argtypes)
_vp, _ci, _cf = ctypes.c_void_p, ctypes.c_int, ctypes.c_float
_PP = ctypes.POINTER(ctypes.c_void_p)
_PI = ctypes.POINTER(ctypes.c_int)
_PF = ctypes.POINTER(ctypes.c_float)
SIGNATURES = {
    "crb_create": (_vp, [_cf, _cf, _cf, _cf, _cf, _ci]),
    "crb_create_ex": (_vp, [_cf, _cf, _cf, _cf, _cf, _ci, ctypes.POINTER(crb_options)]),
    "crb_destroy": (None, [_vp]),
    "crb_clean": (_ci, [_vp, _vp, _ci, _ci, _vp, _vp, _vp]),
    "crb_clean_batch": (_ci, [_vp, _ci, _PP, _PI, _PI, _PF, _PF, _PP, _PP, _vp]),
    "crb_clean_batch_host": (_ci, [_vp, _ci, _PP, _PI, _PI, _PF, _PF, _PP, _PP, _vp]),
    "crb_clean_noalloc": (_ci, [_cf, _cf, _cf, _cf, _cf, _ci, _vp, _ci, _ci, _vp, _vp, _vp]),
    "crb_sync_status": (_ci, [_vp, _vp]),
    "crb_last_counts": (_ci, [_vp, ctypes.POINTER(ctypes.c_longlong), _ci]),
    "crb_last_work": (_ci, [_vp, ctypes.POINTER(ctypes.c_longlong), _ci]),
    "crb_last_launches": (_ci, [_vp]),
    "crb_iterate": (_ci, [_vp, _vp, _vp, _ci, _ci, _vp, _vp, _vp, _vp]),
    "crb_profile_read": (_ci, [_vp, ctypes.POINTER(ctypes.c_double), _PI, ctypes.POINTER(ctypes.c_double), _PI,
                               _ci]),
    "crb_alu_peak": (_ci, [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double), _vp]),
    "crb_fadd_peak": (_ci, [ctypes.POINTER(ctypes.c_double), _vp]),
    "crb_profile_kernels": (_ci, [_vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_ci), _ci, _ci]),
    "crb_server_create": (_vp, [_cf, _cf, _cf, _cf, _cf, _ci, ctypes.POINTER(crb_options), ctypes.c_size_t, _ci,
                                _ci]),
    "crb_server_submit": (_ci, [_vp, _vp, _ci, _ci, _cf, _cf, _vp, _vp, ctypes.c_uint64]),
    "crb_server_poll": (_ci, [_vp, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_double), _PI, _ci,
                              _ci]),
    "crb_server_stats": (_ci, [_vp, ctypes.POINTER(ctypes.c_longlong), _ci]),
    "crb_server_frame_bytes": (ctypes.c_size_t, [_ci, _ci]),
    "crb_server_destroy": (None, [_vp]),
    "crb_tuned_config": (_ci, [_vp, _PI, _ci, _PI, _PI]),
    "crb_selftest_wait_timeout": (_ci, [_vp, ctypes.c_uint, _vp]),
    "crb_num_tile_shapes": (_ci, []),
    "crb_tile_shape": (_ci, [_ci, _PI, _PI]),
    "crb_partition": (_ci, [_ci, _ci, _ci, _ci, _ci, ctypes.POINTER(crb_rect), _ci, _PI, _PI]),
    "crb_clean_rects": (_ci, [_vp, _vp, _ci, _ci, _ci, ctypes.POINTER(crb_rect), _vp, _vp, _vp]),
    "crb_poisson": (_ci, [_vp, _ci, _ci, ctypes.c_uint64, _vp, _vp]),
    "crb_poisson_batch": (_ci, [_ci, _PP, _PI, _PI, ctypes.POINTER(ctypes.c_uint64), _PP, _vp]),
    "crb_last_error": (ctypes.c_char_p, []),
    "crb_strerror": (ctypes.c_char_p, [_ci]),
}


def load():
    """Builds (if stale) and loads the CUDA library; raises if that is impossible."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            lib = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def lib_path() -> str:
    return _build.LIB


class CrbError(RuntimeError):
    def __init__(self, status: int, where: str):
        lib = load()
        msg = lib.crb_last_error().decode() or lib.crb_strerror(status).decode()
        super().__init__(f"{where}: status {status} ({lib.crb_strerror(status).decode()}): {msg}")
        self.status = status


def check(status: int, where: str) -> None:
    if status != CRB_OK:
        raise CrbError(status, where)


def __getattr__(name):  # crb_* functions by their C names
    if name.startswith("crb_"):
        return getattr(load(), name)
    raise AttributeError(name)
