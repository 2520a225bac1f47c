"""Generate ptrig_constants.h: the numeric constants of the CUDA kernels.

Run from the repository root:  python paper_2502_10831_gb300/csrc/gen_constants.py

Everything is derived here in exact integer / rational arithmetic and rounded
once to the target format (round-to-nearest-even, or truncation where a
Cody-Waite split needs trailing zero bits).  pi comes from the Gauss-Legendre
(Brent-Salamin) AGM iteration in fixed point.

Constants
  * Cody-Waite splits of pi/2 (Cody & Waite 1980): FP32 24+24+24 bits
    (three positive floats, used with FMA) for |x| <= 2^20, FP64 21+53+53
    bits for |x| < 2^31.
  * 2/pi as 32-bit words for the Payne-Hanek reduction of larger |x|
    (Payne & Hanek 1983).
  * The pi/12 coefficient table of the paper's Sec. 2 formulas in the
    kernels' reduced variable t = |r| (see the table comment below).
  * Taylor-n coefficients (Maclaurin series of sin, cos, tan).
"""
from __future__ import annotations

import math
import os
from fractions import Fraction

PREC = 2200  # fixed-point bits carried for pi


def pi_agm(bits: int = PREC) -> Fraction:
    """pi by the Gauss-Legendre AGM iteration with `bits` fractional bits."""
    g = 64
    one = 1 << (bits + g)
    a = one
    b = math.isqrt(one * one // 2)
    t = one // 4
    p = 1
    for _ in range(40):
        an = (a + b) // 2
        b = math.isqrt(a * b)
        t -= p * (a - an) * (a - an) // one
        a = an
        p <<= 1
        if abs(a - b) <= 1:
            break
    pi = (a + b) * (a + b) // (4 * t)
    return Fraction(pi >> g, 1 << bits)


PI = pi_agm()
HALF_PI = PI / 2


def _round_bits(v: Fraction, bits: int, mode: str = "nearest") -> Fraction:
    """Round v to `bits` significant bits (nearest-even or toward zero)."""
    if v == 0:
        return Fraction(0)
    s = -1 if v < 0 else 1
    a = abs(v)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    if Fraction(2) ** e > a:
        e -= 1
    scale = Fraction(2) ** (bits - 1 - e)
    m = a * scale
    if mode == "trunc":
        mi = m.numerator // m.denominator
    else:
        fl = m.numerator // m.denominator
        rem = m - fl
        if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and fl % 2 == 1):
            mi = fl + 1
        else:
            mi = fl
    return s * Fraction(mi) / scale


def f32(v: Fraction, mode: str = "nearest") -> float:
    r = _round_bits(v, 24, mode)
    return float(r)  # exact: 24 bits fit in a double


def f64(v: Fraction, mode: str = "nearest") -> float:
    return float(_round_bits(v, 53, mode))


def lit32(x: float) -> str:
    if x == 0:
        return "-0.0f" if math.copysign(1.0, x) < 0 else "0.0f"
    return f"{x.hex()}f"


def lit64(x: float) -> str:
    return "0.0" if x == 0 else x.hex()


def main() -> str:
    lines = []
    w = lines.append
    w("/* Generated by gen_constants.py -- do not edit.  Numeric constants of the")
    w(" * pi/12 trigonometry kernels, each rounded once from an exact value. */")
    w("#pragma once")
    w("#include <stdint.h>")
    w("")

    # ---- FP32 Cody-Waite with FMA (|x| <= 2^20, |j| < 2^20)
    # P1 = pi/2 truncated to 24 bits has ulp 2^-23, so x - j P1 (one FMA) has
    # no bit below 2^-24 and magnitude < 1 for |x| <= 2^20: it is exact.  P2
    # (truncated) and P3 (nearest) carry the next 48 bits; the rounding of the
    # two later FMAs and the dropped tail give |error| <= 2^-23 |r| + 2^-49.65,
    # and no float in (0.5, 2^20] lies closer than 2^-27.8 to a multiple of
    # pi/2.  All three pieces are positive, so x = -0 keeps its sign.
    p1 = _round_bits(HALF_PI, 24, "trunc")
    p2 = _round_bits(HALF_PI - p1, 24, "trunc")
    p3 = _round_bits(HALF_PI - p1 - p2, 24)
    assert p1 > 0 and p2 > 0 and p3 > 0
    w("/* pi/2 = PIO2_F1 + PIO2_F2 + PIO2_F3 (+ < 2^-70): three positive 24-bit floats, used with FMA */")
    w(f"#define PTRIG_PIO2_F1 {lit32(float(p1))}")
    w(f"#define PTRIG_PIO2_F2 {lit32(float(p2))}")
    w(f"#define PTRIG_PIO2_F3 {lit32(float(p3))}")
    # two pieces for |x| < 2^16 (fp16 storage): P1 and the rest rounded to
    # nearest; the dropped tail is below 2^-48, so |j| < 2^16 gives at most
    # 2^-32 on top of the one rounding of the second FMA
    p2r = _round_bits(HALF_PI - p1, 24)
    assert abs(HALF_PI - p1 - p2r) <= Fraction(1, 2 ** 48)
    w("/* pi/2 = PIO2_F1 + PIO2_F2R (+ < 2^-48): the two-piece split for |x| < 2^16 */")
    w(f"#define PTRIG_PIO2_F2R {lit32(float(p2r))}")
    w(f"#define PTRIG_2_OVER_PI_F {lit32(f32(2 / PI))}")
    w(f"#define PTRIG_12_OVER_PI_F {lit32(f32(12 / PI))}")
    w(f"#define PTRIG_PIO2_F {lit32(f32(HALF_PI))}")
    w("/* 1.5 * 2^23: adding it rounds a float to an integer held in the low mantissa bits */")
    w(f"#define PTRIG_RINT_MAGIC_F {lit32(1.5 * 2.0 ** 23)}")
    w("/* FP32 reduction bound 2^20 of the Taylor kernels (Payne-Hanek above) */")
    w(f"#define PTRIG_FAST_LIMIT_F {lit32(2.0 ** 20)}")
    w("/* Bound of the two-piece FP32 reduction (16-bit storage): every fp16 and")
    w(" * bf16 value below 2^16 keeps its row code and r within 2^-21 of the")
    w(" * three-piece reduction; larger angles take the full path */")
    w(f"#define PTRIG_TWO_PIECE_LIMIT_F {lit32(65535.0)}")
    w("/* FP32 reduction bound of the signed-row kernels: M + 8 j stays exact")
    w(" * in [2^23, 2^24) for |j| <= 2^19 * 2/pi + 1 < 2^19 */")
    w(f"#define PTRIG_SEG_LIMIT_F {lit32(2.0 ** 19)}")
    w("/* bits of 1.5 * 2^23, and -7 * 1.5 * 2^23: fma(8, M + j, -7 M) = M + 8 j exactly */")
    w("#define PTRIG_RINT_MAGIC_BITS 0x4b400000u")
    w(f"#define PTRIG_SEG_BASE_C {lit32(-7 * 1.5 * 2.0 ** 23)}")
    w("")

    # ---- FP64 Cody-Waite (|j| < 2^31)
    d1 = _round_bits(HALF_PI, 21, "trunc")
    d2 = _round_bits(HALF_PI - d1, 53, "trunc")
    d3 = _round_bits(HALF_PI - d1 - d2, 53)
    w("/* pi/2 = PIO2_D1 + PIO2_D2 + PIO2_D3 (+ ~2^-127): 21 + 53 + 53 bits */")
    w(f"#define PTRIG_PIO2_D1 {lit64(float(d1))}")
    w(f"#define PTRIG_PIO2_D2 {lit64(float(d2))}")
    w(f"#define PTRIG_PIO2_D3 {lit64(float(d3))}")
    w(f"#define PTRIG_2_OVER_PI_D {lit64(f64(2 / PI))}")
    w(f"#define PTRIG_12_OVER_PI_D {lit64(f64(12 / PI))}")
    w(f"#define PTRIG_PIO2_D {lit64(f64(HALF_PI))}")
    w(f"#define PTRIG_PIO2_D_LO {lit64(f64(HALF_PI - Fraction(f64(HALF_PI))))}")
    w(f"#define PTRIG_RINT_MAGIC_D {lit64(1.5 * 2.0 ** 52)}")
    w("/* FP64 Cody-Waite bound 2^31 (|j| < 2^31 keeps j * PIO2_D1 exact) */")
    w(f"#define PTRIG_CW64_LIMIT {lit64(2.0 ** 31)}")
    w("")

    # ---- 2/pi words for Payne-Hanek
    nwords = 40
    two_over_pi = 2 / PI
    fixed = (two_over_pi.numerator << (32 * nwords)) // two_over_pi.denominator
    words = [(fixed >> (32 * (nwords - 1 - i))) & 0xFFFFFFFF for i in range(nwords)]
    w("/* fraction bits of 2/pi, big-endian: 2/pi = sum_i W[i] 2^(-32(i+1)) */")
    w(f"#define PTRIG_TWO_OVER_PI_NWORDS {nwords}")
    w("#define PTRIG_TWO_OVER_PI_WORDS \\")
    for i in range(0, nwords, 6):
        chunk = ", ".join(f"0x{v:08x}u" for v in words[i:i + 6])
        w(f"  {chunk}{',' if i + 6 < nwords else ''} \\")
    w("")

    # ---- coefficient table in t = |r|
    # Appendix integer rationals tan(x deg) ~ (A x + B)/(C x + D) (Eqs. 9, 5-8, 10)
    Q = [(11, 0, -1, 632), (10, 10, -4, 657), (6, 46, -5, 541),
         (10, 217, -13, 1252), (4, 297, -10, 910), (1, 542, -11, 990)]
    R = Fraction(180) / PI
    rows = []
    for p in (0, 1):
        for kq in range(4):
            if p == 0:
                A, B, C, D = Q[kq]          # u = t, segment kq
                rows.append((A * R, Fraction(B), C * R, Fraction(D), kq))
            else:
                k = 5 - kq                  # u = pi/2 - t, segment 5 - kq
                A, B, C, D = Q[k]
                rows.append((-A * R, Fraction(90 * A + B), -C * R, Fraction(90 * C + D), k))
    w("/* Sec. 2 formulas in the kernels' variable t = |r|, r = x - j pi/2:")
    w(" *   index (p << 2) | kq, p = j & 1, kq = floor(t 12/pi) in 0..3")
    w(" *   p = 0: u = t,        segment kq:     N = A R t + B,          D = C R t + D")
    w(" *   p = 1: u = pi/2 - t, segment 5 - kq: N = (90A+B) - A R t,    D = (90C+D) - C R t")
    w(" * with R = 180/pi; entries {aN, bN, aD, bD}, N = aN t + bN, D = aD t + bD. */")
    w("#define PTRIG_TABLE_F32 \\")
    for i, (aN, bN, aD, bD, k) in enumerate(rows):
        sep = "," if i < 7 else ""
        w(f"  {{{lit32(f32(aN))}, {lit32(f32(bN))}, {lit32(f32(aD))}, {lit32(f32(bD))}}}{sep} /* seg {k} */ \\")
    w("")
    w("#define PTRIG_TABLE_F64 \\")
    for i, (aN, bN, aD, bD, k) in enumerate(rows):
        sep = "," if i < 7 else ""
        w(f"  {lit64(f64(aN))}, {lit64(f64(bN))}, {lit64(f64(aD))}, {lit64(f64(bD))}{sep} /* seg {k} */ \\")
    w("")

    # ---- signed rows: the same formulas in the signed r, indexed by
    # i = (8 j + f) mod 16 with f = floor(r 12/pi) in [-4, 3].  j' = j - [r < 0]
    # (the quadrant below x) has j' & 1 = bit 3 of i; f' = i & 7 is f for r >= 0
    # (kq = f') and f + 8 for r < 0 (kq = 7 - f', and j = j' + 1).  In every row
    # N >= 0 and D carries the sign (-1)^(j' & 1); sin and cos take the further
    # sign (-1)^((j' >> 1) & 1) from bit 4 of (8 j + f), tan none.
    srows = []
    for i in range(16):
        jp, fp = i >> 3, i & 7
        if fp <= 3:
            kq, p, sr = fp, jp, 0
        else:
            kq, p, sr = 7 - fp, 1 - jp, 1
        aN, bN, aD, bD, k = rows[(p << 2) | kq]
        if sr:  # t = -r
            aN, aD = -aN, -aD
        if jp:
            aD, bD = -aD, -bD
        srows.append((aN, bN, aD, bD, k, jp, sr))
    w("/* Signed rows: index i = (8 j + f) mod 16, f = floor(r 12/pi) in [-4, 3];")
    w(" * N = aN r + bN >= 0, D = aD r + bD with the sign of (j - [r < 0]) & 1")
    w(" * folded in; A holds {aN, aD}, B {bN, bD}.  Row 0's bN is -0 so that")
    w(" * x = -0 gives N = -0. */")
    w("#define PTRIG_SROW_A_F32 \\")
    for i, (aN, bN, aD, bD, k, jp, sr) in enumerate(srows):
        sep = "," if i < 15 else ""
        w(f"  {{{lit32(f32(aN))}, {lit32(f32(aD))}}}{sep} /* {i}: seg {k}, j' odd {jp}, r<0 {sr} */ \\")
    w("")
    w("#define PTRIG_SROW_B_F32 \\")
    for i, (aN, bN, aD, bD, k, jp, sr) in enumerate(srows):
        sep = "," if i < 15 else ""
        bn = -0.0 if i == 0 else f32(bN)
        w(f"  {{{lit32(bn)}, {lit32(f32(bD))}}}{sep} \\")
    w("")

    # ---- u-form FP64 coefficients for the paper-faithful kernels
    w("/* Sec. 2 formulas in the paper's variable u for segments 0..5:")
    w(" * {a, b, c, d} = {A R, B, C R, D}, then the sin/cos radicand coefficients")
    w(" * {x, y, z} = {a^2 + c^2, 2(ab + cd), b^2 + d^2} (appendix A.4). */")
    w("#define PTRIG_UFORM_F64 \\")
    for k, (A, B, C, D) in enumerate(Q):
        a, b, c, d = A * R, Fraction(B), C * R, Fraction(D)
        vals = [a, b, c, d, a * a + c * c, 2 * (a * b + c * d), b * b + d * d]
        sep = "," if k < 5 else ""
        w("  " + ", ".join(lit64(f64(v)) for v in vals) + sep + " \\")
    w("")

    # ---- Taylor coefficients (Horner in u^2)
    sin_c = [Fraction((-1) ** i, math.factorial(2 * i + 1)) for i in range(9)]
    cos_c = [Fraction((-1) ** i, math.factorial(2 * i)) for i in range(9)]
    # tan: coefficients from t' = 1 + t^2
    c = [Fraction(0)] * 20
    c[1] = Fraction(1)
    for k in range(1, 18):
        sq = sum(c[i] * c[k - i] for i in range(k + 1))
        c[k + 1] = sq / (k + 1)
    tan_c = [c[2 * i + 1] for i in range(9)]
    for name, cs in (("SIN", sin_c), ("COS", cos_c), ("TAN", tan_c)):
        w(f"#define PTRIG_TAYLOR_{name}_F32 {', '.join(lit32(f32(v)) for v in cs)}")
        w(f"#define PTRIG_TAYLOR_{name}_F64 {', '.join(lit64(f64(v)) for v in cs)}")
    w("")
    return "\n".join(lines) + "\n"


if __name__ == "__main__":
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "ptrig_constants.h")
    with open(out, "w") as f:
        f.write(main())
    print(out)
