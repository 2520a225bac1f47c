"""The forward kernels' signed-row table and row code, checked on the CPU.

The kernels index 16 rows by (8 j + f) mod 16 with f = floor(r 12/pi) and take
the quadrant sign of sin and cos from bit 4 of 8 j + f (see ptrig_device.cuh).
Here the generated table is evaluated with that index in float64 over many
angles and compared with the FP64 oracle, the exactness conditions of the index
FMA are checked, and x = -0 is followed through row 0.
"""
import math
import os
import re

import numpy as np

import parity as P
from paper_2502_10831_gb300 import workloads

HDR = os.path.join(os.path.dirname(__file__), "..", "paper_2502_10831_gb300", "csrc", "ptrig_constants.h")


def _num(t):
    t = t.strip().rstrip("f")
    return float.fromhex(t) if "x" in t else float(t)


def _rows(name):
    text = open(HDR).read()
    body = re.search(rf"#define {name} \\\n(.*?)\n\n", text, re.S).group(1)
    return np.array([[_num(v) for v in g.split(",")] for g in re.findall(r"\{([^}]*)\}", body)])


def _const(name):
    return _num(re.search(rf"#define {name} (\S+)\n", open(HDR).read()).group(1))


def _signed_eval(x):
    a, b = _rows("PTRIG_SROW_A_F32"), _rows("PTRIG_SROW_B_F32")
    j = np.rint(x * 2 / np.pi)
    r = x - j * (np.pi / 2)
    code = (8 * j + np.floor(r * 12 / np.pi)).astype(np.int64)
    i = code & 15
    sg = np.where((code >> 4) & 1, -1.0, 1.0)
    N = a[i, 0] * r + b[i, 0]
    D = a[i, 1] * r + b[i, 1]
    h = np.sqrt(N * N + D * D)
    return N, D, {"sin": sg * N / h, "cos": sg * D / h, "tan": N / D}


def test_signed_rows_reproduce_the_oracle(oracle):
    x = np.concatenate([workloads.bandwidth(1 << 19).astype(np.float64),
                        workloads.parity(1 << 17).astype(np.float64),
                        np.random.default_rng(2).uniform(-2e5, 2e5, 1 << 17)])
    N, _, got = _signed_eval(x)
    assert np.all(N >= 0)
    u, *_ = oracle.reduce(x)
    far = np.abs(u - np.round(u / P.STEP) * P.STEP) > 1e-9
    for f, g in got.items():
        ref = oracle.proposed(f, x)
        if f == "tan":
            k = far & (np.abs(oracle.proposed("cos", x)) > 1e-3)
            err = np.abs(g[k] - ref[k]) / np.abs(ref[k])
            assert err.max() < 1e-6, (f, err.max())
        else:
            err = np.abs(g[far] - ref[far])
            assert err.max() < 1e-6, (f, err.max())


def test_row_code_fma_is_exact_within_the_limit():
    """c = fma(8, M + j, -7 M) = M + 8 j and M + 8 j + f stay integers of
    [2^23, 2^24) -- where the float ulp is 1 and rounding toward -inf is the
    floor -- for every j the FP32 reduction produces below the limit."""
    M = _const("PTRIG_RINT_MAGIC_F")
    lim = _const("PTRIG_SEG_LIMIT_F")
    assert M == 1.5 * 2 ** 23 and _const("PTRIG_SEG_BASE_C") == -7 * M
    bits = re.search(r"#define PTRIG_RINT_MAGIC_BITS (0x[0-9a-f]+)u", open(HDR).read()).group(1)
    assert int(bits, 16) == int(np.float32(M).view(np.uint32))
    jmax = math.ceil(lim * 2 / math.pi) + 1
    for j in (-jmax, jmax):
        for f in (-4, 3):
            v = M + 8 * j + f
            assert 2 ** 23 <= v < 2 ** 24
    assert np.float32(-7 * M) == -7 * M  # the constant is exact in FP32
    assert _const("PTRIG_FAST_LIMIT_F") >= lim


def test_negative_zero_keeps_its_sign():
    """Row 0's bN is -0: N = aN (-0) + (-0) = -0, so sin(-0) = tan(-0) = -0."""
    b = _rows("PTRIG_SROW_B_F32")
    assert b[0, 0] == 0 and math.copysign(1.0, b[0, 0]) < 0
    a = _rows("PTRIG_SROW_A_F32")
    n_neg = np.float32(a[0, 0]) * np.float32(-0.0) + np.float32(b[0, 0])
    n_pos = np.float32(a[0, 0]) * np.float32(0.0) + np.float32(b[0, 0])
    assert math.copysign(1.0, n_neg) < 0 and math.copysign(1.0, n_pos) > 0


def test_rows_are_the_t_form_rows_with_signs():
    """Each signed row is an 8-row t-form row (t = |r|) with the sign of r
    folded into the slopes and (-1)^(j' & 1) into D."""
    t8 = _rows("PTRIG_TABLE_F32")
    a, b = _rows("PTRIG_SROW_A_F32"), _rows("PTRIG_SROW_B_F32")
    for i in range(16):
        jp, fp = i >> 3, i & 7
        if fp <= 3:
            kq, p, sr = fp, jp, 0
        else:
            kq, p, sr = 7 - fp, 1 - jp, 1
        aN, bN, aD, bD = t8[(p << 2) | kq]
        s_r = -1.0 if sr else 1.0
        s_d = -1.0 if jp else 1.0
        assert a[i, 0] == s_r * aN and b[i, 0] == bN
        assert a[i, 1] == s_d * s_r * aD and b[i, 1] == s_d * bD
