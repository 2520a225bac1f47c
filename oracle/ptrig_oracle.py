"""Plain FP64 CPU oracle of the pi/12 piecewise trigonometric method
(arXiv 2502.10831): Python loader for ``ptrig_oracle.c``.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline / reference legs may import this module.  It is
independent of the CUDA library: it imports nothing from the package, shares
no header, table or constant generator with it, and its constants (pi and the
bits of 2/pi used by the exact reduction of Sec. 3) come from Machin's formula
evaluated here in exact integer arithmetic.

Function selectors: 0 = sin, 1 = cos, 2 = tan.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from fractions import Fraction

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ptrig_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libptrig_oracle.so")

SIN, COS, TAN = 0, 1, 2
FUNCS = {"sin": SIN, "cos": COS, "tan": TAN}

# ----------------------------------------------------------------- constants

_PI_BITS = 1600  # fixed-point bits carried for pi and 2/pi (doubles need ~1200)


def _arctan_inv(x: int, one: int) -> int:
    """arctan(1/x) * one, by its alternating Taylor series in integers."""
    total = term = one // x
    x2 = x * x
    n = 1
    sign = -1
    while term:
        term //= x2
        total += sign * (term // (2 * n + 1))
        sign = -sign
        n += 1
    return total


def pi_fixed(bits: int = _PI_BITS) -> int:
    """floor-ish pi * 2**bits from Machin's formula pi = 16 atan(1/5) - 4 atan(1/239),
    carried with 64 guard bits."""
    guard = 64
    one = 1 << (bits + guard)
    pi = 16 * _arctan_inv(5, one) - 4 * _arctan_inv(239, one)
    return pi >> guard


def two_over_pi_words(nwords: int = 48) -> np.ndarray:
    """Big-endian 32-bit words of the fraction of 2/pi (2/pi < 1)."""
    bits = 32 * nwords
    pi = pi_fixed(bits + 64)                      # pi * 2^(bits+64)
    top = (1 << (2 * (bits + 64) + 1)) // pi       # 2/pi * 2^(bits+64)
    top >>= 64                                     # 2/pi * 2^bits
    return np.array([(top >> (bits - 32 * (i + 1))) & 0xFFFFFFFF for i in range(nwords)],
                    dtype=np.uint32)


def pi_double_double() -> tuple[float, float]:
    """pi as hi + lo with hi the correctly rounded double."""
    p = Fraction(pi_fixed(), 1 << _PI_BITS)
    hi = float(p)
    lo = float(p - Fraction(hi))
    return hi, lo


# ------------------------------------------------------------------ building


def build(force: bool = False) -> str:
    """Compile ptrig_oracle.c into a shared library with the system C compiler.
    No fast-math and no FMA contraction, so x86-64 and aarch64 round alike."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        os.makedirs(os.path.dirname(_LIB), exist_ok=True)
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-ffp-contract=off",
               "-fno-fast-math", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = ctypes.CDLL(path)
        d = ctypes.c_double
        i = ctypes.c_int
        sz = ctypes.c_size_t
        P = ctypes.c_void_p
        L.ptro_init.argtypes = [P, i, d, d]
        L.ptro_init.restype = i
        for name, args in [("ptro_proposed", [i, d]), ("ptro_taylor", [i, i, d]),
                           ("ptro_derivative", [i, d]), ("ptro_faithful", [i, d]),
                           ("ptro_proposed_seg", [i, i, d]), ("ptro_fisr", [d])]:
            f = getattr(L, name)
            f.argtypes = args
            f.restype = d
        L.ptro_proposed_array.argtypes = [i, P, P, sz]
        L.ptro_proposed_seg_array.argtypes = [i, i, P, P, sz]
        L.ptro_taylor_array.argtypes = [i, i, P, P, sz]
        L.ptro_derivative_array.argtypes = [i, P, P, sz]
        L.ptro_faithful_array.argtypes = [i, P, P, sz]
        L.ptro_reduce_array.argtypes = [P, P, P, P, P, P, sz]
        L.ptro_coeffs.argtypes = [i, P]
        L.ptro_coeffs.restype = i
        L.ptro_quadruple.argtypes = [i, P]
        L.ptro_quadruple.restype = i
        w = np.ascontiguousarray(two_over_pi_words(48))
        hi, lo = pi_double_double()
        rc = L.ptro_init(w.ctypes.data, len(w), hi, lo)
        if rc != 0:
            raise RuntimeError("ptro_init failed")
        _lib = L
    return _lib


# ------------------------------------------------------------------ array API


def _fid(func) -> int:
    return FUNCS[func] if isinstance(func, str) else int(func)


def _as_f64(x) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x, dtype=np.float64))


def proposed(func, x) -> np.ndarray:
    """The paper's piecewise sin/cos/tan (Sec. 2) of every element of x, FP64."""
    x = _as_f64(x)
    y = np.empty_like(x)
    lib().ptro_proposed_array(_fid(func), x.ctypes.data, y.ctypes.data, x.size)
    return y


def proposed_neighbour(func, dk: int, x) -> np.ndarray:
    """Like proposed() but evaluated with the segment index shifted by dk."""
    x = _as_f64(x)
    y = np.empty_like(x)
    lib().ptro_proposed_seg_array(_fid(func), int(dk), x.ctypes.data, y.ctypes.data, x.size)
    return y


def taylor(func, nterms: int, x) -> np.ndarray:
    """Taylor-n baseline: n non-zero Maclaurin terms on the reduced angle."""
    x = _as_f64(x)
    y = np.empty_like(x)
    lib().ptro_taylor_array(_fid(func), int(nterms), x.ctypes.data, y.ctypes.data, x.size)
    return y


def derivative(func, x) -> np.ndarray:
    """d/dx of the paper's piecewise function."""
    x = _as_f64(x)
    y = np.empty_like(x)
    lib().ptro_derivative_array(_fid(func), x.ctypes.data, y.ctypes.data, x.size)
    return y


def faithful(func, x) -> np.ndarray:
    """Algorithms 1-6 as printed: FISR, 0.261 selector, tan pole guard."""
    x = _as_f64(x)
    y = np.empty_like(x)
    lib().ptro_faithful_array(_fid(func), x.ctypes.data, y.ctypes.data, x.size)
    return y


def reduce(x):
    """Per-element reduction: (u, q, neg, seg, node_dist)."""
    x = _as_f64(x)
    n = x.size
    u = np.empty(n)
    q = np.empty(n, dtype=np.int32)
    neg = np.empty(n, dtype=np.int32)
    seg = np.empty(n, dtype=np.int32)
    nd = np.empty(n)
    lib().ptro_reduce_array(x.ctypes.data, u.ctypes.data, q.ctypes.data, neg.ctypes.data,
                            seg.ctypes.data, nd.ctypes.data, n)
    return u, q, neg, seg, nd


def fisr(v: float) -> float:
    return lib().ptro_fisr(float(v))


def coeffs(k: int) -> np.ndarray:
    """Radian coefficients (a, b, c, d) the oracle uses on segment k."""
    out = np.zeros(4)
    if lib().ptro_coeffs(int(k), out.ctypes.data) != 0:
        raise ValueError(k)
    return out


def quadruple(k: int) -> tuple:
    """Integer degree-domain quadruple (A, B, C, D) the oracle holds for segment k."""
    out = np.zeros(4, dtype=np.int32)
    if lib().ptro_quadruple(int(k), out.ctypes.data) != 0:
        raise ValueError(k)
    return tuple(int(v) for v in out)

