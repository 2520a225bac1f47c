"""The FP32 reduction's error bound, checked on the CPU from its constants.

The kernels reduce |x| <= PTRIG_FAST_LIMIT_F with three FMAs against
pi/2 = P1 + P2 + P3 + tail.  The bound |r - (x - j pi/2)| <= 2^-23 |r| + 2^-49.65
rests on: P1 having ulp 2^-23 (first FMA exact), positive pieces (x = -0 keeps
its sign), |j| < 2^20, a tail below 2^-70, and no float up to the limit lying
within 2^-27.8 of a nonzero multiple of pi/2 (relative error of r below 2^-21.2).
"""
import math
import os
import re
from fractions import Fraction

import numpy as np

import parity as P

HDR = os.path.join(os.path.dirname(__file__), "..", "paper_2502_10831_gb300", "csrc", "ptrig_constants.h")


def _const(name):
    m = re.search(rf"#define {name} (\S+)f\n", open(HDR).read())
    return float.fromhex(m.group(1))


def _half_pi(oracle):
    return Fraction(oracle.pi_fixed(400), 1 << 401)


def test_pieces_positive_and_sum_to_half_pi(oracle):
    p = [_const(f"PTRIG_PIO2_F{k}") for k in (1, 2, 3)]
    assert all(v > 0 for v in p)
    for v in p:
        assert np.float32(v) == v
    assert math.frexp(p[0])[1] == 1  # P1 in [1, 2): ulp 2^-23
    tail = _half_pi(oracle) - sum(Fraction(v) for v in p)
    assert abs(tail) < Fraction(1, 2 ** 70)


def test_limit_and_quotient_range():
    lim = _const("PTRIG_FAST_LIMIT_F")
    assert lim == 2.0 ** 20
    jmax = lim * _const("PTRIG_2_OVER_PI_F") + 1
    assert jmax < 2 ** 20 and jmax < 2 ** 22  # |j| fits the 1.5*2^23 rounding trick


def test_no_float_closer_than_bound_to_half_pi_multiple(oracle):
    worst = P.closest_to_half_pi_multiples(oracle, -1, 20, 6)
    u, _, _, _, _ = oracle.reduce(worst.astype(np.float64))
    d = np.minimum(u, np.pi / 2 - u)
    assert np.log2(d.min()) > -27.9
    # relative error of r at the closest float stays below 2^-21.2
    assert 2.0 ** -23 + 2.0 ** -49.65 / d.min() < 2.0 ** -21.2


def _rn32(v):
    """v rounded to the nearest FP32 (ties to even), exactly (normal range)."""
    if v == 0:
        return Fraction(0)
    s = -1 if v < 0 else 1
    a = abs(v)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    if Fraction(2) ** e > a:
        e -= 1
    sc = Fraction(2) ** (23 - e)
    m = a * sc
    fl = m.numerator // m.denominator
    rem = m - fl
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and fl % 2):
        fl += 1
    return s * Fraction(fl) / sc


def _two_piece_worst(values):
    """Over the given nonzero values, emulated exactly: asserts that the
    two-piece reduction selects the same signed row as the three-piece one and
    returns the largest relative difference of the two reduced angles."""
    c = {n: Fraction(_const(n)) for n in ("PTRIG_PIO2_F1", "PTRIG_PIO2_F2", "PTRIG_PIO2_F3", "PTRIG_PIO2_F2R",
                                          "PTRIG_2_OVER_PI_F", "PTRIG_12_OVER_PI_F", "PTRIG_RINT_MAGIC_F")}
    M = c["PTRIG_RINT_MAGIC_F"]
    worst = Fraction(0)
    for xv in values:
        x = Fraction(float(xv))
        y = _rn32(x * c["PTRIG_2_OVER_PI_F"] + M)
        jf = y - M
        r1 = _rn32(x - jf * c["PTRIG_PIO2_F1"])  # exact
        r3 = _rn32(_rn32(r1 - jf * c["PTRIG_PIO2_F2"]) - jf * c["PTRIG_PIO2_F3"])
        r2 = _rn32(r1 - jf * c["PTRIG_PIO2_F2R"])
        base = M + 8 * jf
        assert math.floor(base + r3 * c["PTRIG_12_OVER_PI_F"]) == math.floor(base + r2 * c["PTRIG_12_OVER_PI_F"]), xv
        if r3 != 0 and jf != 0:
            worst = max(worst, abs(r2 - r3) / abs(r3))
    return worst


def test_two_piece_limit_covers_fp16():
    lim = _const("PTRIG_TWO_PIECE_LIMIT_F")
    assert 65504.0 <= lim < 65536.0  # every finite fp16, no bf16 from 2^16 up


def test_two_piece_reduction_for_bf16_storage():
    """bf16 storage reduces with two pieces below 2^16 (larger angles take the
    full path): over every finite nonzero bf16 value below the limit the
    two-piece r selects the same signed row and stays within 2^-21 of the
    three-piece r."""
    lim = _const("PTRIG_TWO_PIECE_LIMIT_F")
    bits = np.arange(1 << 16, dtype=np.uint32) << 16
    with np.errstate(invalid="ignore"):
        xs = bits.view(np.float32).astype(np.float64)
    xs = xs[np.isfinite(xs) & (xs != 0) & (np.abs(xs) <= lim)]
    assert xs.size > 36000
    assert _two_piece_worst(xs) < Fraction(1, 2 ** 21)


def test_two_piece_reduction_for_fp16_storage():
    """fp16 storage reduces with two pieces of pi/2 (|x| < 2^16): over every
    finite nonzero fp16 value, emulated exactly, the two-piece r stays within
    2^-21 (relative) of the three-piece r and selects the same signed row,
    so the FP32 segment dump describes the fp16 kernels too."""
    bits = np.arange(1 << 16, dtype=np.uint32).astype(np.uint16)
    with np.errstate(invalid="ignore"):
        xs = bits.view(np.float16).astype(np.float64)
    assert _two_piece_worst(xs[np.isfinite(xs) & (xs != 0)]) < Fraction(1, 2 ** 21)


def _table_words():
    h = open(HDR).read()
    body = h[h.index("#define PTRIG_TWO_OVER_PI_WORDS"):]
    body = body[:body.index("\n\n")] if "\n\n" in body else body
    return [int(w, 16) for w in re.findall(r"0x([0-9a-fA-F]{8})u", body)]


def _ph_f32_model(xv, words):
    """The FP32 side path's Payne-Hanek steps on one float, integer steps
    exactly and each FP32 operation rounded once: returns (r, j mod 4)."""
    c1, c2r = Fraction(_const("PTRIG_PIO2_F1")), Fraction(_const("PTRIG_PIO2_F2R"))
    b = int(np.float32(xv).view(np.uint32))
    e = ((b >> 23) & 0xff) - 150
    m = (b & 0x7fffff) | 0x800000
    tw = [0] + list(words)  # b_k of 2/pi is bit k + 31 of this table, MSB first
    t0 = e + 30
    iw, sh = t0 >> 5, t0 & 31
    window = ((tw[iw] << 96 | tw[iw + 1] << 64 | tw[iw + 2] << 32 | tw[iw + 3]) << sh >> 32) & ((1 << 96) - 1)
    p = m * window  # 120 bits; bits 94-95 are j mod 4, bits 0-93 the fraction
    q = (p >> 94) & 3
    f = p & ((1 << 94) - 1)
    up = f >> 93
    if up:
        f = (1 << 94) - f
    fhi = f >> 30
    lz = min(64 - fhi.bit_length(), 63)
    g = (f << lz >> 30) & ((1 << 64) - 1)
    a, bb = Fraction(g >> 40), Fraction((g >> 16) & 0xffffff)
    hi = _rn32(a * c1)
    tail = _rn32(a * c2r + _rn32(_rn32(bb / (1 << 24)) * c1 + (a * c1 - hi)))
    r = _rn32(hi + tail) / Fraction(2) ** (24 + lz)
    jj = (q + up) & 3
    if up:
        r = -r
    if b >> 31:
        r, jj = -r, (-jj) & 3
    return r, jj


def test_fp32_payne_hanek_model(oracle):
    """FP32 angles beyond the fast range reduce by an integer product of the
    24-bit significand with a 96-bit window of 2/pi: over the floats of
    2^19 .. 2^26 closest to a multiple of pi/2, binade edges up to the largest
    float and random angles, the model takes the nearest multiple (ties
    aside) and the reduced angle's relative error stays below 2^-23.9 (one
    FP32 rounding of the sum and the dropped bits of the product and of pi/2:
    leaving out the second piece of pi/2 already gives 2^-23.2)."""
    words = _table_words()
    assert words[:8] == [int(w) for w in oracle.two_over_pi_words(8)]
    half_pi = _half_pi(oracle)
    r = np.random.default_rng(3)
    xs = list(P.closest_to_half_pi_multiples(oracle, 19, 26, 2))
    xs += [np.float32(2.0 ** k) for k in range(8, 128)]
    xs += [np.nextafter(np.float32(2.0 ** k), np.float32(0)) for k in range(9, 128)]
    xs += list((2.0 ** r.uniform(8, 127.99, 600) * r.choice([-1.0, 1.0], 600)).astype(np.float32))
    xs.append(np.finfo(np.float32).max)
    worst = Fraction(0)
    for xv in xs:
        x = Fraction(float(xv))
        j = round(x / half_pi)
        exact = x - j * half_pi
        got, jj = _ph_f32_model(xv, words)
        if jj != j % 4:  # only within rounding of an odd multiple of pi/4
            assert abs(abs(exact) - half_pi / 2) < Fraction(1, 2 ** 20), xv
            continue
        worst = max(worst, abs(got - exact) / abs(exact))
    assert math.log2(worst) < -23.9
