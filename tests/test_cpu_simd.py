"""The CPU SIMD baseline (cpu_simd/, include/ptrig_cpu.h) against the FP64
oracle, with the GPU path's comparison rules (FP32 sin / cos within 1e-6,
tan within 1e-5 relative where |cos| >= 1e-3; near a pi/12 node either
adjacent segment's formula is accepted)."""
import ctypes

import numpy as np
import pytest

import parity as P
from paper_2502_10831_gb300 import workloads

FUNCS = ("sin", "cos", "tan")


@pytest.fixture(scope="module")
def C():
    from cpu_simd import ptrig_cpu
    ptrig_cpu.lib()
    return ptrig_cpu


def _check(oracle, func, x, y):
    xd = x.astype(np.float64)
    ref = oracle.proposed(func, xd)
    u = oracle.reduce(xd)[0]
    nn = P.near_node(u) & np.isfinite(xd)
    if nn.any():  # near a node: compare with whichever adjacent formula is closer
        for dk in (-1, 1):
            alt = oracle.proposed_neighbour(func, dk, xd[nn])
            closer = np.abs(alt - y[nn]) < np.abs(ref[nn] - y[nn])
            sub = ref[nn]
            sub[closer] = alt[closer]
            ref[nn] = sub
    return P.check_values(oracle, func, xd, y, ref)


@pytest.mark.parametrize("func", FUNCS)
def test_parity_workload(C, oracle, func):
    x = workloads.parity(1 << 18)
    _check(oracle, func, x, C.evaluate(func, x))


def test_sincos_matches_sin_and_cos(C):
    x = workloads.bandwidth(1 << 16)
    s, c = C.evaluate("sincos", x)
    assert np.array_equal(s.view(np.uint32), C.evaluate("sin", x).view(np.uint32))
    assert np.array_equal(c.view(np.uint32), C.evaluate("cos", x).view(np.uint32))


@pytest.mark.parametrize("func", FUNCS)
def test_bandwidth_and_large_arguments(C, oracle, func):
    r = np.random.default_rng(11)
    huge = (10.0 ** r.uniform(6.0, 38.5, 8192) * r.choice([-1, 1], 8192)).astype(np.float32)
    x = np.concatenate([workloads.bandwidth(1 << 16), workloads.large(1 << 16), huge[np.isfinite(huge)]])
    _check(oracle, func, x, C.evaluate(func, x))


@pytest.mark.parametrize("func", FUNCS)
def test_edge_values(C, oracle, func):
    x = workloads.edge_values()
    _check(oracle, func, x, C.evaluate(func, x))
    z = C.evaluate(func, np.array([0.0, -0.0], np.float32))
    if func == "cos":
        assert np.all(z == 1.0)
    else:
        assert np.all(z == 0.0) and list(np.signbit(z)) == [False, True]


@pytest.mark.parametrize("func", FUNCS)
def test_reduction_worst_cases(C, oracle, func):
    """Floats closest to multiples of pi/2 up to 2^21: relative error 2^-18
    where the result is small (and for tan everywhere)."""
    x = P.closest_to_half_pi_multiples(oracle, -1, 20, 6)
    y = C.evaluate(func, x)
    ref = oracle.proposed(func, x.astype(np.float64))
    small = np.ones(x.shape, bool) if func == "tan" else np.abs(ref) < 1e-2
    err = np.abs(y[small].astype(np.float64) - ref[small])
    assert np.all(err <= 2.0 ** -18 * np.abs(ref[small]) + 2.0 ** -149)


def test_sizes_threads_and_in_place(C):
    base = workloads.bandwidth(5000)
    base[::97] = np.float32(3.0e9)  # some angles on the Payne-Hanek path
    full = {f: C.evaluate(f, base, threads=1) for f in FUNCS}
    for n in (0, 1, 3, 255, 256, 257, 1000, 4099, 5000):
        for threads in (1, 3, 16, 0):
            for f in FUNCS:
                y = C.evaluate(f, base[:n], threads=threads)
                assert np.array_equal(y.view(np.uint32), full[f][:n].view(np.uint32)), (n, threads, f)
    for f in FUNCS:  # in place
        buf = base.copy()
        C.evaluate(f, buf, out=(buf, None))
        assert np.array_equal(buf.view(np.uint32), full[f].view(np.uint32))


def test_invalid_arguments(C):
    L = C.lib()
    x = np.zeros(4, np.float32)
    y = np.zeros(4, np.float32)
    assert L.ptrig_cpu_f32(0, None, y.ctypes.data, None, 4, 1) == 1
    assert L.ptrig_cpu_f32(3, x.ctypes.data, y.ctypes.data, None, 4, 1) == 1
    assert L.ptrig_cpu_f32(4, x.ctypes.data, y.ctypes.data, None, 4, 1) == 1
    assert L.ptrig_cpu_f32(-1, x.ctypes.data, y.ctypes.data, None, 4, 1) == 1
    assert L.ptrig_cpu_f32(0, None, None, None, 0, 1) == 0
    assert C.default_threads() >= 1


def test_header_symbols_exported(C):
    import os
    import re
    hdr = open(os.path.join(os.path.dirname(__file__), "..", "include", "ptrig_cpu.h")).read()
    names = set(re.findall(r"\b(ptrig_cpu_\w+)\s*\(", hdr))
    assert names == {"ptrig_cpu_f32", "ptrig_cpu_default_threads", "ptrig_cpu_libm_f64"}
    L = ctypes.CDLL(C.lib()._name)
    for nm in names:
        assert hasattr(L, nm)


def test_libm_loop_matches_numpy_and_validates():
    """The C library loop the bench times for context: double sin/cos/tan of
    every element (sincos into two arrays), threaded, same argument checks."""
    from cpu_simd import ptrig_cpu as C
    x = np.random.default_rng(6).uniform(-1e3, 1e3, 100003)
    for f in ("sin", "cos", "tan"):
        assert np.allclose(C.libm(f, x, threads=5), getattr(np, f)(x), rtol=1e-12, atol=1e-12)
    s, c = C.libm("sincos", x, threads=3)
    assert np.allclose(s, np.sin(x), atol=1e-12) and np.allclose(c, np.cos(x), atol=1e-12)
    L = C.lib()
    assert L.ptrig_cpu_libm_f64(7, x.ctypes.data, x.ctypes.data, None, 4, 1) == 1
    assert L.ptrig_cpu_libm_f64(0, None, x.ctypes.data, None, 4, 1) == 1
    assert L.ptrig_cpu_libm_f64(3, x.ctypes.data, x.ctypes.data, None, 4, 1) == 1
    assert L.ptrig_cpu_libm_f64(0, None, None, None, 0, 1) == 0
