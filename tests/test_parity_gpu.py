"""GPU parity of libptrig against the FP64 oracle (element by element), through
the C ABI.  Needs a CUDA GPU; run with -m gpu."""
import math

import numpy as np
import pytest

import parity as P
from paper_2502_10831_gb300 import workloads

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

FUNCS = ("sin", "cos", "tan")


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_10831_gb300 import binding, build
    build.build()
    return binding


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _run(B, func, x_np, dtype="f32"):
    x = _dev(x_np)
    y = torch.empty_like(x)
    getattr(B, f"ptrig_{func}_{dtype}")(x, y)
    torch.cuda.synchronize()
    return y.cpu().numpy()


def _segments(B, x_np):
    x = _dev(x_np.astype(np.float32))
    s = torch.empty(x.shape, dtype=torch.uint8, device="cuda")
    B.ptrig_segment_f32(x, s)
    torch.cuda.synchronize()
    return s.cpu().numpy()


# ----------------------------------------------------------------- FP32 core


@pytest.fixture(scope="module")
def c1():
    return workloads.parity(1 << 20)


@pytest.mark.parametrize("func", FUNCS)
def test_f32_parity_parity_workload(B, oracle, c1, func):
    xd = c1.astype(np.float64)
    y = _run(B, func, c1)
    ref, _ = P.reference_with_gpu_segments(oracle, func, xd, _segments(B, c1))
    P.check_values(oracle, func, xd, y, ref)


def test_sincos_equals_sin_and_cos(B, c1):
    x = _dev(c1)
    s = torch.empty_like(x)
    c = torch.empty_like(x)
    B.ptrig_sincos_f32(x, s, c)
    s1 = _run(B, "sin", c1)
    c1v = _run(B, "cos", c1)
    torch.cuda.synchronize()
    assert np.array_equal(s.cpu().numpy(), s1) and np.array_equal(c.cpu().numpy(), c1v)


def test_segment_indices_bit_exact_away_from_nodes(B, oracle, c1):
    extra = workloads.bandwidth(1 << 18)
    x = np.concatenate([c1, extra])
    seg = _segments(B, x)
    u, q, neg, seg_o, _ = oracle.reduce(x.astype(np.float64))
    same = (seg & 0x0F) == seg_o
    assert np.all(same | P.near_node(u))
    assert np.array_equal(seg >> 4, q)
    # the near-node share of the node-heavy workload is small but not empty
    assert (~same).sum() < 0.01 * x.size


def test_edge_values(B, oracle):
    x = workloads.edge_values()
    xd = x.astype(np.float64)
    seg = _segments(B, x)
    for func in FUNCS:
        y = _run(B, func, x)
        ref, _ = P.reference_with_gpu_segments(oracle, func, xd, seg)
        P.check_values(oracle, func, xd, y, ref)
        z = np.array([0.0, -0.0], dtype=np.float32)
        yz = _run(B, func, z)
        if func == "cos":
            assert np.all(yz == 1.0)
        else:
            assert np.all(yz == 0.0) and list(np.signbit(yz)) == [False, True]


@pytest.mark.parametrize("func", ("sin", "cos", "tan", "sincos"))
def test_large_arguments(B, oracle, func):
    """|x| log-uniform in [1, 1e5] (FP32 reduction), in (2^19, 2^31) and up
    to the largest float (the Payne-Hanek side path), for every function
    (sincos: both outputs)."""
    big = workloads.large(1 << 20)
    r = np.random.default_rng(4)
    mid = (2.0 ** r.uniform(19.0, 31.0, 1 << 16) * r.choice([-1, 1], 1 << 16)).astype(np.float32)
    huge = (10.0 ** r.uniform(9.5, 38.5, 4096) * r.choice([-1, 1], 4096)).astype(np.float32)
    x = np.concatenate([big, mid, huge[np.isfinite(huge)]])
    xd = x.astype(np.float64)
    seg = _segments(B, x)
    if func == "sincos":
        xt = _dev(x)
        s, c = torch.empty_like(xt), torch.empty_like(xt)
        B.ptrig_sincos_f32(xt, s, c)
        torch.cuda.synchronize()
        outs = {"sin": s.cpu().numpy(), "cos": c.cpu().numpy()}
    else:
        outs = {func: _run(B, func, x)}
    for f, y in outs.items():
        ref, _ = P.reference_with_gpu_segments(oracle, f, xd, seg)
        P.check_values(oracle, f, xd, y, ref)


def _scattered(n, frac, seed, lo=19.0):
    """The bandwidth mixture with a fraction of its angles, at random
    positions, replaced by |x| log-uniform in [2^lo, 2^60) (both side paths)."""
    x = workloads.bandwidth(n)
    r = np.random.default_rng(seed)
    idx = r.choice(n, max(1, int(n * frac)), replace=False)
    x[idx] = (2.0 ** r.uniform(lo, 60.0, idx.size) * r.choice([-1, 1], idx.size)).astype(np.float32)
    return x


@pytest.mark.parametrize("func", ("sin", "cos", "tan", "sincos"))
@pytest.mark.parametrize("frac", (1e-3, 3e-2))
def test_scattered_large_arguments(B, oracle, func, frac):
    """Angles beyond the FP32 reduction range scattered through an ordinary
    array (2^20 + 37 angles: whole chunks, a partial chunk and a ragged tail),
    so that many threads meet one in the middle of their work: every output
    against the oracle."""
    x = _scattered((1 << 20) + 37, frac, 12)
    xd = x.astype(np.float64)
    seg = _segments(B, x)
    if func == "sincos":
        xt = _dev(x)
        s, c = torch.empty_like(xt), torch.empty_like(xt)
        B.ptrig_sincos_f32(xt, s, c)
        torch.cuda.synchronize()
        outs = {"sin": s.cpu().numpy(), "cos": c.cpu().numpy()}
    else:
        outs = {func: _run(B, func, x)}
    for f, y in outs.items():
        ref, _ = P.reference_with_gpu_segments(oracle, f, xd, seg)
        P.check_values(oracle, f, xd, y, ref)


@pytest.mark.parametrize("func", ("sin", "cos", "sincos"))
def test_scattered_large_arguments_bf16(B, oracle, func):
    """The same with bf16 storage (which holds angles up to 3.4e38): 1% of
    2^20 + 45 angles with |x| from 2^15 up, across the 2^16 bound of the
    two-piece reduction and the FP32 range."""
    bits = workloads.f32_to_bf16_bits(_scattered((1 << 20) + 45, 1e-2, 13, lo=15.0))
    xd = workloads.bf16_bits_to_f32(bits).astype(np.float64)
    xt = _dev(bits.view(np.int16))
    y0 = torch.empty_like(xt)
    if func == "sincos":
        y1 = torch.empty_like(xt)
        B.ptrig_sincos_bf16(xt, y0, y1)
        outs = {"sin": y0, "cos": y1}
    else:
        getattr(B, f"ptrig_{func}_bf16")(xt, y0)
        outs = {func: y0}
    torch.cuda.synchronize()
    seg = _segments(B, xd.astype(np.float32))
    for f, t in outs.items():
        got = workloads.bf16_bits_to_f32(t.cpu().numpy().view(np.uint16)).astype(np.float64)
        ref, _ = P.reference_with_gpu_segments(oracle, f, xd, seg)
        assert np.abs(got - ref).max() <= _half_ref_tol(f, "bf16"), (f, np.abs(got - ref).max())


@pytest.fixture(scope="module")
def worst_reduction():
    return P.closest_to_half_pi_multiples(oracle_module(), -1, 20, 6)


def oracle_module():
    from oracle import ptrig_oracle as O
    return O


@pytest.mark.parametrize("func", FUNCS)
def test_reduction_worst_cases(B, oracle, worst_reduction, func):
    """The floats of every binade up to 2^21 that lie closest to a multiple of
    pi/2 (the largest cancellation in the FP32 reduction): the usual bounds,
    and a relative bound of 2^-18 wherever the result is small (sin at even,
    cos at odd multiples) or for tan everywhere (zero or pole)."""
    x = worst_reduction
    xd = x.astype(np.float64)
    y = _run(B, func, x)
    ref, _ = P.reference_with_gpu_segments(oracle, func, xd, _segments(B, x))
    P.check_values(oracle, func, xd, y, ref)
    small = np.ones(x.shape, bool) if func == "tan" else np.abs(ref) < 1e-2
    assert small.sum() >= 40
    err = np.abs(y[small].astype(np.float64) - ref[small])
    bound = 2.0 ** -18 * np.abs(ref[small]) + 2.0 ** -149
    assert np.all(err <= bound), (func, xd[small][np.argmax(err / bound)], float((err / bound).max()))


@pytest.mark.parametrize("func", FUNCS + ("sincos",))
def test_side_path_worst_cases(B, oracle, func):
    """The 6 floats of every binade [2^19, 2^27) closest to a multiple of pi/2,
    and their negatives: they take the side path (Payne-Hanek in integer
    arithmetic), and the result keeps the relative bound of 2^-18 wherever it
    is small (for tan everywhere).  sincos: both outputs."""
    x = P.closest_to_half_pi_multiples(oracle, 19, 26, 6)
    xd = x.astype(np.float64)
    seg = _segments(B, x)
    if func == "sincos":
        xt = _dev(x)
        s, c = torch.empty_like(xt), torch.empty_like(xt)
        B.ptrig_sincos_f32(xt, s, c)
        torch.cuda.synchronize()
        outs = {"sin": s.cpu().numpy(), "cos": c.cpu().numpy()}
    else:
        outs = {func: _run(B, func, x)}
    for f, y in outs.items():
        ref, _ = P.reference_with_gpu_segments(oracle, f, xd, seg)
        P.check_values(oracle, f, xd, y, ref)
        small = np.ones(x.shape, bool) if f == "tan" else np.abs(ref) < 1e-2
        err = np.abs(y[small].astype(np.float64) - ref[small])
        bound = 2.0 ** -18 * np.abs(ref[small]) + 2.0 ** -149
        assert np.all(err <= bound), (f, xd[small][np.argmax(err / bound)], float((err / bound).max()))


# ------------------------------------------------- sizes, alignment, in place


@pytest.mark.parametrize("offset", [0, 1, 2, 3])
def test_sizes_alignment_and_guard_bands(B, oracle, offset):
    sizes = [0, 1, 2, 3, 4, 5, 7, 8, 9, 15, 16, 17, 31, 33, 1000, 4099, 70001]
    base = workloads.parity(80000)
    canary = np.float32(-7777.5)
    for n in sizes:
        for func in ("sin", "tan", "sincos"):
            pad = 64
            xbuf = np.full(n + 2 * pad, np.float32(0.25), dtype=np.float32)
            xbuf[pad + offset: pad + offset + n] = base[:n]
            xb = _dev(xbuf)
            yb = _dev(np.full(n + 2 * pad, canary, dtype=np.float32))
            zb = _dev(np.full(n + 2 * pad, canary, dtype=np.float32))
            xs = xb[pad + offset: pad + offset + n]
            ys = yb[pad + offset: pad + offset + n]
            zs = zb[pad + offset: pad + offset + n]
            if func == "sincos":
                B.ptrig_sincos_f32(xs, ys, zs, n)
            else:
                getattr(B, f"ptrig_{func}_f32")(xs, ys, n)
            torch.cuda.synchronize()
            yh = yb.cpu().numpy()
            zh = zb.cpu().numpy()
            lo, hi = pad + offset, pad + offset + n
            assert np.all(yh[:lo] == canary) and np.all(yh[hi:] == canary)
            if func != "sincos":
                assert np.all(zh == canary)
            else:
                assert np.all(zh[:lo] == canary) and np.all(zh[hi:] == canary)
            if n:
                f0 = "sin" if func == "sincos" else func
                ref = _run(B, f0, base[:n].copy())  # aligned, vector path
                assert np.array_equal(yh[lo:hi], ref), (n, offset, func)
                if func == "sincos":
                    assert np.array_equal(zh[lo:hi], _run(B, "cos", base[:n].copy()))


def test_in_place(B):
    x = workloads.parity(10007)
    for func in FUNCS:
        t = _dev(x)
        getattr(B, f"ptrig_{func}_f32")(t, t)
        torch.cuda.synchronize()
        assert np.array_equal(t.cpu().numpy(), _run(B, func, x))


# ------------------------------------------------------------------ Taylor


@pytest.mark.parametrize("nterms", [5, 7, 9])
@pytest.mark.parametrize("func", FUNCS)
def test_taylor_parity(B, oracle, func, nterms):
    x = workloads.parity(1 << 18)
    xd = x.astype(np.float64)
    xt = _dev(x)
    y = torch.empty_like(xt)
    if nterms == 5:
        getattr(B, f"ptrig_taylor_{func}_f32")(xt, y)
    else:
        B.ptrig_taylor_n_f32(FUNCS.index(func), nterms, xt, y)
    torch.cuda.synchronize()
    yh = y.cpu().numpy().astype(np.float64)
    ref = oracle.taylor(func, nterms, xd)
    if func == "tan":
        rel = np.abs(yh - ref) / np.maximum(np.abs(ref), 1e-30)
        assert rel.max() <= 1e-5
    else:
        assert np.abs(yh - ref).max() <= 1e-6


# --------------------------------------------------------------- derivatives


@pytest.mark.parametrize("func", FUNCS)
def test_bwd_f32_parity(B, oracle, func):
    x = workloads.parity(1 << 18)
    xd = x.astype(np.float64)
    g = np.random.default_rng(9).standard_normal(x.size).astype(np.float32)
    xt, gt = _dev(x), _dev(g)
    gx = torch.empty_like(xt)
    getattr(B, f"ptrig_{func}_bwd_f32")(xt, gt, gx)
    torch.cuda.synchronize()
    got = gx.cpu().numpy().astype(np.float64)
    u, *_ = oracle.reduce(xd)
    keep = ~P.near_node(u)
    if func == "tan":
        keep &= np.abs(oracle.proposed("cos", xd)) >= 1e-3
    ref = g.astype(np.float64) * oracle.derivative(func, xd)
    err = np.abs(got - ref)[keep] / np.maximum(1.0, np.abs(ref[keep]))
    assert err.max() <= 2e-5, err.max()


@pytest.mark.parametrize("func", FUNCS)
def test_bwd_f32_scattered_large_arguments(B, oracle, func):
    """The derivative kernels on 2^20 + 37 angles with 1% of them beyond the
    FP32 reduction range at random positions (whole chunks, a partial chunk
    and a ragged tail), against the oracle's derivative."""
    x = _scattered((1 << 20) + 37, 1e-2, 14)
    xd = x.astype(np.float64)
    g = np.random.default_rng(10).standard_normal(x.size).astype(np.float32)
    xt, gt = _dev(x), _dev(g)
    gx = torch.empty_like(xt)
    getattr(B, f"ptrig_{func}_bwd_f32")(xt, gt, gx)
    torch.cuda.synchronize()
    got = gx.cpu().numpy().astype(np.float64)
    u, *_ = oracle.reduce(xd)
    keep = ~P.near_node(u)
    if func == "tan":
        keep &= np.abs(oracle.proposed("cos", xd)) >= 1e-3
    ref = g.astype(np.float64) * oracle.derivative(func, xd)
    err = np.abs(got - ref)[keep] / np.maximum(1.0, np.abs(ref[keep]))
    assert err.max() <= 2e-5, err.max()


@pytest.mark.parametrize("func", FUNCS)
def test_f64_forward_and_derivative(B, oracle, func):
    r = np.random.default_rng(21)
    x = np.concatenate([workloads.parity(1 << 16).astype(np.float64), r.uniform(-1e6, 1e6, 1 << 14),
                        10.0 ** r.uniform(9, 300, 2048), [0.0, -0.0, math.pi / 2, 1e-300]])
    xt = _dev(x)
    y = torch.empty_like(xt)
    getattr(B, f"ptrig_{func}_f64")(xt, y)
    g = torch.ones_like(xt)
    dy = torch.empty_like(xt)
    getattr(B, f"ptrig_{func}_bwd_f64")(xt, g, dy)
    torch.cuda.synchronize()
    yh, dyh = y.cpu().numpy(), dy.cpu().numpy()
    u, *_ = oracle.reduce(x)
    nn = np.abs(u - np.round(u / P.STEP) * P.STEP) < 1e-13
    ref = oracle.proposed(func, x)
    dref = oracle.derivative(func, x)
    keep = ~nn
    if func == "tan":
        keep &= np.abs(oracle.proposed("cos", x)) >= 1e-3
        assert np.max(np.abs(yh - ref)[keep] / np.abs(ref[keep])) <= 1e-11
    else:
        assert np.max(np.abs(yh - ref)[keep]) <= 1e-12
    assert np.max(np.abs(dyh - dref)[keep] / np.maximum(1.0, np.abs(dref[keep]))) <= 1e-10


# ---------------------------------------------------------------- f16 / bf16


def _half_ref_tol(func, dt):
    if func in ("sin", "cos"):
        return 2e-3
    return 2.0 ** -11 + 1e-6 if dt == "f16" else 2.0 ** -8 + 1e-6


@pytest.mark.parametrize("dt", ["f16", "bf16"])
@pytest.mark.parametrize("func", ("sin", "cos", "tan", "sincos"))
def test_half_parity(B, oracle, func, dt):
    n = 1 << 20
    if dt == "f16":
        xh = workloads.half16(n)
        bits = xh.view(np.uint16)
        xd = xh.astype(np.float64)
    else:
        bits = workloads.half_bf16(n)
        xd = workloads.bf16_bits_to_f32(bits).astype(np.float64)
    xt = _dev(bits.view(np.int16))
    y0 = torch.empty_like(xt)
    if func == "sincos":
        y1 = torch.empty_like(xt)
        getattr(B, f"ptrig_sincos_{dt}")(xt, y0, y1)
        outs = {"sin": y0, "cos": y1}
    else:
        getattr(B, f"ptrig_{func}_{dt}")(xt, y0)
        outs = {func: y0}
    torch.cuda.synchronize()
    seg = _segments(B, xd.astype(np.float32))
    for f, t in outs.items():
        raw = t.cpu().numpy().view(np.uint16)
        got = raw.view(np.float16).astype(np.float64) if dt == "f16" else \
            workloads.bf16_bits_to_f32(raw).astype(np.float64)
        ref, _ = P.reference_with_gpu_segments(oracle, f, xd, seg)
        tol = _half_ref_tol(f, dt)
        if f in ("sin", "cos"):
            assert np.abs(got - ref).max() <= tol, (f, dt, np.abs(got - ref).max())
        else:
            big = 65504.0 if dt == "f16" else 3.0e38
            keep = (np.abs(oracle.proposed("cos", xd)) >= 1e-3) & (np.abs(ref) < 0.99 * big) & \
                   (np.abs(ref) > 1e-4)
            rel = np.abs(got[keep] - ref[keep]) / np.abs(ref[keep])
            assert rel.max() <= tol, (dt, rel.max())


# 16-bit storage: significand bits, smallest normal exponent, largest finite
_HALF_FMT = {"f16": (11, -14, 65504.0), "bf16": (8, -126, float(np.float32(3.3895313892515355e38)))}
# Relative bound on the FP32 value before the final rounding: the reduction's
# 2^-21.2 times a conditioning of at most 2 (no formula row cancels: N or D is
# exactly proportional to t where it vanishes), plus a few FP32 roundings and
# the hardware rsqrt / rcp approximations.
_HALF_EPS = 2.0 ** -18


def _round_neighbours(ref, fmt):
    """For |ref|: the two storage-grid values around it (lo <= |ref| <= hi),
    the round-to-nearest-even choice, and whether |ref| lies within
    _HALF_EPS relative of the midpoint between lo and hi."""
    p, emin, maxf = _HALF_FMT[fmt]
    a = np.abs(ref)
    _, ex = np.frexp(np.where(a > 0, a, 1.0))
    e = np.maximum(ex - 1, emin)
    ulp = np.ldexp(1.0, e - (p - 1))
    lo = np.floor(a / ulp) * ulp
    hi = lo + ulp
    mid = lo + ulp / 2
    even_lo = (np.floor(a / ulp) % 2) == 0
    rn = np.where(a < mid, lo, np.where(a > mid, hi, np.where(even_lo, lo, hi)))
    rn = np.where(rn > maxf, np.inf, rn)
    hi = np.where(hi > maxf, np.inf, hi)
    near = np.abs(a - mid) <= _HALF_EPS * a
    return lo, hi, rn, near


@pytest.mark.parametrize("dt", ["f16", "bf16"])
@pytest.mark.parametrize("func", ("sin", "cos", "tan"))
def test_half_exhaustive_correctly_rounded(B, oracle, func, dt):
    """Every one of the 65536 bit patterns: NaN for NaN / inf inputs, and
    otherwise the oracle value rounded to nearest in the storage type -- or,
    only where the oracle value lies within 2^-18 relative of a rounding
    midpoint, the other neighbour.  Signs must agree."""
    bits = np.arange(1 << 16, dtype=np.uint32).astype(np.uint16)
    with np.errstate(invalid="ignore"):  # signalling-NaN patterns
        xd = (bits.view(np.float16).astype(np.float64) if dt == "f16"
              else workloads.bf16_bits_to_f32(bits).astype(np.float64))
    xt = _dev(bits.view(np.int16))
    y = torch.empty_like(xt)
    getattr(B, f"ptrig_{func}_{dt}")(xt, y)
    torch.cuda.synchronize()
    raw = y.cpu().numpy().view(np.uint16)
    with np.errstate(invalid="ignore"):
        got = (raw.view(np.float16).astype(np.float64) if dt == "f16"
               else workloads.bf16_bits_to_f32(raw).astype(np.float64))
    fin = np.isfinite(xd)
    assert np.all(np.isnan(got[~fin]))
    xf, gf = xd[fin], got[fin]
    ref, _ = P.reference_with_gpu_segments(oracle, func, xf, _segments(B, xf.astype(np.float32)))
    lo, hi, rn, near = _round_neighbours(ref, dt)
    ga = np.abs(gf)
    ok = (ga == rn) | (near & ((ga == lo) | (ga == hi)))
    nz = (ref != 0) & (gf != 0)
    ok &= ~nz | (np.signbit(gf) == np.signbit(ref))
    bad = np.flatnonzero(~ok)
    assert bad.size == 0, (dt, func, bad.size, xf[bad[:4]], gf[bad[:4]], ref[bad[:4]])


@pytest.mark.parametrize("dt", ["f16", "bf16"])
def test_half_vector_and_scalar_paths_agree(B, dt):
    """Aligned arrays take the 16-byte vector path (packed FP32 pairs);
    misaligned ones and n % 8 tails the element path.  Both round alike."""
    n = 40003
    bits = workloads.half16(n).view(np.uint16) if dt == "f16" else workloads.half_bf16(n)
    ref = {}
    for off in range(0, 8):
        buf = np.zeros(n + 16, dtype=np.uint16)
        buf[off: off + n] = bits
        xb = _dev(buf.view(np.int16))
        ys = torch.zeros_like(xb)
        yc = torch.zeros_like(xb)
        getattr(B, f"ptrig_sincos_{dt}")(xb[off: off + n], ys[off: off + n], yc[off: off + n], n)
        yt = torch.zeros_like(xb)
        getattr(B, f"ptrig_tan_{dt}")(xb[off: off + n], yt[off: off + n], n)
        torch.cuda.synchronize()
        got = [t.cpu().numpy()[off: off + n] for t in (ys, yc, yt)]
        if off == 0:
            ref = got
        else:
            for g, r in zip(got, ref):
                assert np.array_equal(g, r), (dt, off)


@pytest.mark.parametrize("dt", ["f16", "bf16"])
def test_half_sizes_alignment_and_guard_bands(B, dt):
    """16-bit sin, cos, tan and sincos on sizes around the whole-chunk
    boundaries (2048 angles per fp16 chunk, 4096 per bf16 sin / cos / tan
    chunk), aligned and misaligned: canaries around each output stay
    untouched, and every value equals the one computed in a large aligned
    array."""
    canary = 0x7BCD
    pad = 64
    full_n = 3 * 4096 + 40
    bits = workloads.half16(full_n).view(np.uint16) if dt == "f16" else workloads.half_bf16(full_n)
    ref = {}
    xt = _dev(bits.view(np.int16))
    for f in ("sin", "cos", "tan"):
        y = torch.empty_like(xt)
        getattr(B, f"ptrig_{f}_{dt}")(xt, y)
        ref[f] = y.cpu().numpy().view(np.uint16)
    torch.cuda.synchronize()
    for n in (0, 1, 7, 8, 9, 2047, 2048, 2049, 4095, 4096, 4097, 8200, 3 * 4096 + 5):
        for off in (0, 3):
            buf = np.zeros(n + 2 * pad, dtype=np.uint16)
            buf[pad + off: pad + off + n] = bits[:n]
            xb = _dev(buf.view(np.int16))
            outs = {}
            for f in ("sin", "cos", "tan", "sincos"):
                ya = _dev(np.full(n + 2 * pad, canary, dtype=np.uint16).view(np.int16))
                yb = _dev(np.full(n + 2 * pad, canary, dtype=np.uint16).view(np.int16))
                xs = xb[pad + off: pad + off + n]
                if f == "sincos":
                    getattr(B, f"ptrig_sincos_{dt}")(xs, ya[pad + off: pad + off + n], yb[pad + off: pad + off + n], n)
                else:
                    getattr(B, f"ptrig_{f}_{dt}")(xs, ya[pad + off: pad + off + n], n)
                torch.cuda.synchronize()
                outs[f] = (ya.cpu().numpy().view(np.uint16), yb.cpu().numpy().view(np.uint16))
            lo, hi = pad + off, pad + off + n
            for f, (a, b) in outs.items():
                assert np.all(a[:lo] == canary) and np.all(a[hi:] == canary), (dt, f, n, off)
                if f == "sincos":
                    assert np.all(b[:lo] == canary) and np.all(b[hi:] == canary), (dt, f, n, off)
                    assert np.array_equal(a[lo:hi], ref["sin"][:n]) and np.array_equal(b[lo:hi], ref["cos"][:n])
                else:
                    assert np.all(b == canary)
                    assert np.array_equal(a[lo:hi], ref[f][:n]), (dt, f, n, off)


def test_mapped_host_buffers(B):
    """Inputs and outputs in pinned host memory, which the ABI accepts (the
    device reads and writes it over the host link): the same values as with
    device buffers, for FP32 and both 16-bit types (whose kernels then stage
    their inputs in registers rather than through cp.async)."""
    n = 3 * 4096 + 40
    cases = {"f32": workloads.bandwidth(n), "f16": workloads.half16(n).view(np.int16),
             "bf16": workloads.half_bf16(n).view(np.int16)}
    for dt, x in cases.items():
        xd = _dev(x)
        xh = torch.from_numpy(np.ascontiguousarray(x)).pin_memory()
        for f in ("sin", "cos", "tan"):
            yd = torch.empty_like(xd)
            getattr(B, f"ptrig_{f}_{dt}")(xd, yd)
            for src, dst in ((xh, torch.empty_like(xh).pin_memory()), (xh, torch.empty_like(xd)),
                             (xd, torch.empty_like(xh).pin_memory())):
                getattr(B, f"ptrig_{f}_{dt}")(src, dst, n)
                torch.cuda.synchronize()
                assert np.array_equal(dst.cpu().numpy(), yd.cpu().numpy()), (dt, f, src.is_cuda, dst.is_cuda)


# -------------------------------------------------------------------- batch


def _make_batch(n_arrays=60, seed=3):
    r = np.random.default_rng(seed)
    lengths = list(r.integers(0, 20000, n_arrays)) + [0, 1, 3, 5, 4096, 65537, 2047, 2049]
    funcs = list(r.integers(0, 4, len(lengths)))
    offs = list(r.integers(0, 4, len(lengths)))
    # output offsets: equal to the input's (congruent misalignment) for most
    # arrays, different for every fifth (element path throughout)
    yoffs = [o if i % 5 else (o + 1 + i) % 4 for i, o in enumerate(offs)]
    return lengths, funcs, offs, yoffs


GUARD = 8


def test_batch_matches_single_kernels_and_oracle(B, oracle):
    lengths, funcs, offs, yoffs = _make_batch()
    xs, ys, zs, descs, bufs = [], [], [], [], []
    for i, (n, f, o, oy) in enumerate(zip(lengths, funcs, offs, yoffs)):
        xh = workloads.batch_array(i, n)
        xb = _dev(np.concatenate([np.zeros(o, np.float32), xh, np.zeros(GUARD, np.float32)]))
        yb = torch.full((oy + n + GUARD,), -5.0, dtype=torch.float32, device="cuda")
        zb = torch.full_like(yb, -5.0)
        x, y, z = xb[o:o + n], yb[oy:oy + n], zb[oy:oy + n]
        bufs.append((yb, zb, oy))
        xs.append(xh)
        ys.append(y)
        zs.append(z)
        descs.append((x, y, z if f == 3 else None, n, f))
    for flags in (0, B.BATCH_GRAPH):
        for yb, zb, _ in bufs:
            yb.fill_(-5.0)
            zb.fill_(-5.0)
        plan = B.BatchPlan(descs, flags)
        plan.set_config(128, 8)
        plan.run()
        torch.cuda.synchronize()
        for i, (n, f) in enumerate(zip(lengths, funcs)):
            yb, zb, oy = bufs[i]
            for buf in (yb, zb):  # nothing written outside each array
                hb = buf.cpu().numpy()
                assert np.all(hb[:oy] == -5.0) and np.all(hb[oy + n:] == -5.0), (i, n, f)
            if f != 3:
                assert np.all(zb.cpu().numpy() == -5.0)
            if n == 0:
                continue
            got = ys[i].cpu().numpy()[:n]
            name = ("sin", "cos", "tan", "sin")[f]
            assert np.array_equal(got, _run(B, name, xs[i])), (i, n, f)
            if f == 3:
                assert np.array_equal(zs[i].cpu().numpy()[:n], _run(B, "cos", xs[i]))
            xd = xs[i].astype(np.float64)
            ref, _ = P.reference_with_gpu_segments(oracle, name, xd, _segments(B, xs[i]))
            P.check_values(oracle, name, xd, got, ref)
        res = plan.autotune(reps=2, candidates=[(128, 8), (256, 16), (512, 4)])
        assert res["block"] in (128, 256, 512)
        plan.run()
        plan.run_per_array()
        torch.cuda.synchronize()
        plan.close()


# --------------------------------------------------------- full-size sample


def test_full_size_bandwidth_workload_sampled(B, oracle):
    """2^28 angles of the bandwidth workload in the benchmark's launch
    configuration: a random sample of outputs against the oracle, and
    sin^2 + cos^2 = 1 (up to FP32 rounding) at every element."""
    n = 1 << 28
    x = workloads.bandwidth(n)
    xt = _dev(x)
    s = torch.empty_like(xt)
    c = torch.empty_like(xt)
    t = torch.empty_like(xt)
    B.ptrig_sincos_f32(xt, s, c)
    B.ptrig_tan_f32(xt, t)
    torch.cuda.synchronize()
    dev = (s * s + c * c - 1).abs().max().item()
    assert dev <= 2e-6
    r = np.random.default_rng(17)
    idx = np.unique(np.concatenate([r.integers(0, n, 1 << 16), np.arange(1000), np.arange(n - 1000, n)]))
    xi = x[idx]
    xd = xi.astype(np.float64)
    seg = _segments(B, xi)
    it = torch.from_numpy(idx).cuda()
    for f, out in (("sin", s), ("cos", c), ("tan", t)):
        got = out[it].cpu().numpy()
        ref, _ = P.reference_with_gpu_segments(oracle, f, xd, seg)
        P.check_values(oracle, f, xd, got, ref)
    del xt, s, c, t
    torch.cuda.empty_cache()


# ------------------------------------------------------------ misc behaviour


def test_cuda_math_comparison_kernels(B):
    x = workloads.parity(1 << 16)
    xt = _dev(x)
    for fast in (0, 1):
        for fi, f in enumerate(FUNCS):
            y = torch.empty_like(xt)
            B.ptrig_cudamath_f32(fi, fast, xt, y)
            torch.cuda.synchronize()
            xd = x.astype(np.float64)
            ref = getattr(np, f)(xd)
            err = np.abs(y.cpu().numpy() - ref)
            if f == "tan":
                # the __tanf intrinsic loses accuracy next to the poles
                keep = np.abs(np.cos(xd)) > 1e-2
                err = err[keep] / np.maximum(1.0, np.abs(ref[keep]))
            assert err.max() < (1e-5 if not fast else 2e-2)


def test_errors_on_gpu(B):
    from paper_2502_10831_gb300.binding import PtrigError
    x = torch.zeros(16, device="cuda")
    with pytest.raises(PtrigError):
        B.ptrig_sincos_f32(x, x, None)
    with pytest.raises(PtrigError):
        B.ptrig_taylor_n_f32(1, 4, x, x)
    B.ptrig_sin_f32(x, x, 0)  # n == 0 is a no-op
    assert B.ptrig_version() >= 10000
