"""ctypes binding of libptrig_cpu (include/ptrig_cpu.h): numpy float32 arrays
in, numpy float32 arrays out."""
from __future__ import annotations

import ctypes
import threading

import numpy as np

from . import build as _build

FUNCS = {"sin": 0, "cos": 1, "tan": 2, "sincos": 3}
_lib = None
_lock = threading.Lock()


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(_build.build())
            L.ptrig_cpu_f32.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_size_t, ctypes.c_int]
            L.ptrig_cpu_f32.restype = ctypes.c_int
            L.ptrig_cpu_default_threads.argtypes = []
            L.ptrig_cpu_default_threads.restype = ctypes.c_int
            L.ptrig_cpu_libm_f64.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                             ctypes.c_size_t, ctypes.c_int]
            L.ptrig_cpu_libm_f64.restype = ctypes.c_int
            _lib = L
    return _lib


def default_threads() -> int:
    return lib().ptrig_cpu_default_threads()


def evaluate(func: str, x: np.ndarray, threads: int = 0, out=None):
    """func of float32 array x; returns y (or (sin, cos) for "sincos")."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    n = x.size
    y0 = np.empty_like(x) if out is None else out[0]
    y1 = (np.empty_like(x) if out is None else out[1]) if func == "sincos" else None
    st = lib().ptrig_cpu_f32(FUNCS[func], x.ctypes.data, y0.ctypes.data,
                             None if y1 is None else y1.ctypes.data, n, threads)
    if st != 0:
        raise RuntimeError(f"ptrig_cpu_f32({func}) returned {st}")
    return (y0, y1) if func == "sincos" else y0


def libm(func: str, x: np.ndarray, threads: int = 0):
    """The C library's double sin/cos/tan of x (context, not the method)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    y0 = np.empty_like(x)
    y1 = np.empty_like(x) if func == "sincos" else None
    st = lib().ptrig_cpu_libm_f64(FUNCS[func], x.ctypes.data, y0.ctypes.data,
                                  None if y1 is None else y1.ctypes.data, x.size, threads)
    if st != 0:
        raise RuntimeError(f"ptrig_cpu_libm_f64({func}) returned {st}")
    return (y0, y1) if func == "sincos" else y0
