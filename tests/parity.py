"""Comparison rules between the CUDA library and the FP64 oracle.

  * segment index: bit-exact, except within 2 FP32 ulps of a node k pi/12,
    where the GPU may take the adjacent segment; its value is then compared
    with the oracle's value of that adjacent segment's formula.
  * quadrant: bit-exact.
  * FP32 sin / cos: |delta| <= 1e-6.
  * FP32 tan: relative error <= 1e-5 where |cos interpolant| >= 1e-3 (plus one
    subnormal ulp, 2^-149, for results below FLT_MIN).
"""
from __future__ import annotations

import functools
import math

import numpy as np

SIN_COS_ATOL = 1e-6
TAN_RTOL = 1e-5
TAN_COS_FLOOR = 1e-3
STEP = math.pi / 12


def near_node(u: np.ndarray) -> np.ndarray:
    """|u - m pi/12| within 2 FP32 ulps of the node (m = 1..5)."""
    m = np.round(u / STEP)
    node = m * STEP
    ulp = np.spacing(np.abs(node).astype(np.float32)).astype(np.float64)
    return (np.abs(u - node) <= 2 * ulp) & (m >= 1) & (m <= 5)


def reference_with_gpu_segments(oracle, func: str, xd: np.ndarray, seg_gpu: np.ndarray):
    """Oracle values evaluated with the segment the GPU chose (checked to be
    the oracle's own segment or, near a node, an adjacent one)."""
    u, q, neg, seg_o, _ = oracle.reduce(xd)
    finite = np.isfinite(xd)
    gseg = (seg_gpu & 0x0F).astype(np.int32)
    gq = (seg_gpu >> 4).astype(np.int32)
    assert np.all(seg_gpu[~finite] == 0xFF)
    assert np.array_equal(gq[finite], q[finite]), "quadrant mismatch"
    diff = finite & (gseg != seg_o)
    nn = near_node(u)
    bad = diff & ~(nn & (np.abs(gseg - seg_o) == 1))
    assert not bad.any(), f"segment mismatch away from nodes at x={xd[bad][:5]}"
    ref = oracle.proposed(func, xd)
    for dk in (-1, 1):
        m = diff & (gseg - seg_o == dk)
        if m.any():
            ref[m] = oracle.proposed_neighbour(func, dk, xd[m])
    return ref, diff


def check_values(oracle, func: str, xd: np.ndarray, y: np.ndarray, ref: np.ndarray,
                 atol: float = SIN_COS_ATOL, rtol: float = TAN_RTOL):
    finite = np.isfinite(xd)
    assert np.all(np.isnan(y[~finite])), "NaN/inf input must give NaN"
    yf = y[finite].astype(np.float64)
    rf = ref[finite]
    if func in ("sin", "cos"):
        err = np.abs(yf - rf)
        worst = int(np.argmax(err)) if err.size else 0
        assert err.size == 0 or err.max() <= atol, (
            f"{func}: max |delta| {err.max():.3e} at x={xd[finite][worst]!r}")
        return float(err.max()) if err.size else 0.0
    c = np.abs(oracle.proposed("cos", xd[finite]))
    keep = c >= TAN_COS_FLOOR
    err = np.abs(yf[keep] - rf[keep])
    # relative bound, plus one subnormal ulp (2^-149) for results below FLT_MIN
    excess = err - (rtol * np.abs(rf[keep]) + 2.0 ** -149)
    worst = int(np.argmax(excess)) if excess.size else 0
    assert excess.size == 0 or excess.max() <= 0, (
        f"tan: |delta| {err[worst]:.3e} vs ref {rf[keep][worst]:.3e} at x={xd[finite][keep][worst]!r}")
    nz = rf[keep] != 0
    return float((err[nz] / np.abs(rf[keep][nz])).max()) if nz.any() else 0.0


@functools.lru_cache(maxsize=4)
def closest_to_half_pi_multiples(oracle, e_lo: int = -1, e_hi: int = 20, k: int = 6) -> np.ndarray:
    """The k positive floats of each binade [2^e, 2^(e+1)), e_lo <= e <= e_hi,
    that lie closest to a nonzero multiple of pi/2, and their negatives: the
    inputs whose reduced angle cancels most.  Exhaustive over each binade; the
    distance is computed in double with pi/2 split into four 26-bit pieces
    (j times a piece is exact for |j| < 2^27).  Cached per arguments: treat
    the returned array as read-only."""
    half_pi = oracle.pi_fixed(200) // 2  # pi/2 * 2^200, truncated
    pieces = []
    rem = half_pi
    for _ in range(4):
        e = rem.bit_length() - 26
        p = (rem >> e) << e
        pieces.append(math.ldexp(p >> e, e - 200))
        rem -= p
    c = 2.0 / math.pi
    out = []
    for e in range(e_lo, e_hi + 1):
        lo = int(np.float32(2.0 ** e).view(np.uint32))
        bits = np.arange(lo, lo + (1 << 23), dtype=np.uint32)
        x = bits.view(np.float32).astype(np.float64)
        j = np.rint(x * c)
        r = x - j * pieces[0]
        for p in pieces[1:]:
            r = r - j * p
        a = np.where(j == 0, np.inf, np.abs(r))
        idx = np.argpartition(a, k)[:k]
        out.append(x[idx])
    v = np.concatenate(out).astype(np.float32)
    return np.concatenate([v, -v])
