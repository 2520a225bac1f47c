"""Arrays past 2^31 and 2^32 elements: every index computation must stay in
64 bits.  Inputs are drawn on the device from a seeded generator (U[-100pi,
100pi]); outputs are compared with the oracle at both ends, around the 2^31
and 2^32 element boundaries and at random positions."""
import math

import numpy as np
import pytest

import parity as P

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_10831_gb300 import binding, build
    build.build()
    return binding


def _positions(n, seed):
    r = np.random.default_rng(seed)
    edges = [np.arange(0, 64), np.arange(n - 64, n)]
    for b in (1 << 31, 1 << 32, (1 << 32) // 4 * 4):
        if b < n:
            edges.append(np.arange(max(0, b - 40), min(n, b + 40)))
    return np.unique(np.concatenate(edges + [r.integers(0, n, 1 << 16)]))


def _device_uniform(n, seed):
    g = torch.Generator(device="cuda").manual_seed(seed)
    x = torch.empty(n, dtype=torch.float32, device="cuda")
    x.uniform_(-100 * math.pi, 100 * math.pi, generator=g)
    return x


def test_f32_past_2_pow_32(B, oracle):
    n = (1 << 32) + 5
    x = _device_uniform(n, 71)
    ys = torch.empty_like(x)
    yc = torch.empty_like(x)
    B.ptrig_sincos_f32(x, ys, yc)
    torch.cuda.synchronize()
    idx = torch.from_numpy(_positions(n, 5)).cuda()
    xs = x[idx].cpu().numpy()
    xd = xs.astype(np.float64)
    for name, t in (("sin", ys), ("cos", yc)):
        got = t[idx].cpu().numpy()
        ref, _ = P.reference_with_gpu_segments(oracle, name, xd, _segments(B, xs))
        P.check_values(oracle, name, xd, got, ref)
    del ys, yc
    y = torch.empty_like(x)
    B.ptrig_tan_f32(x, y)
    torch.cuda.synchronize()
    got = y[idx].cpu().numpy()
    ref, _ = P.reference_with_gpu_segments(oracle, "tan", xd, _segments(B, xs))
    P.check_values(oracle, "tan", xd, got, ref)
    del x, y
    torch.cuda.empty_cache()


def test_f16_past_2_pow_32(B, oracle):
    n = (1 << 32) + 9
    g = torch.Generator(device="cuda").manual_seed(72)
    x = torch.empty(n, dtype=torch.float16, device="cuda")
    x.uniform_(-60.0, 60.0, generator=g)
    y = torch.empty_like(x)
    B.ptrig_sin_f16(x.view(torch.int16), y.view(torch.int16))
    torch.cuda.synchronize()
    idx = torch.from_numpy(_positions(n, 6)).cuda()
    xd = x[idx].float().cpu().numpy().astype(np.float64)
    got = y[idx].float().cpu().numpy().astype(np.float64)
    ref = oracle.proposed("sin", xd)
    assert np.abs(got - ref).max() <= 2e-3
    del x, y
    torch.cuda.empty_cache()


def _segments(B, xs):
    xt = torch.from_numpy(xs.astype(np.float32)).cuda()
    s = torch.empty(xt.shape, dtype=torch.uint8, device="cuda")
    B.ptrig_segment_f32(xt, s)
    torch.cuda.synchronize()
    return s.cpu().numpy()


def test_batch_array_past_2_pow_31(B, oracle):
    """A ragged batch whose first array has 2^31 + 77 elements (tile offsets
    past 2^31) next to two small arrays, as one graph launch."""
    n_big = (1 << 31) + 77
    x = _device_uniform(n_big, 73)
    ys = torch.empty_like(x)
    yc = torch.empty_like(x)
    xs_small = _device_uniform(1000, 74)
    ya = torch.empty_like(xs_small)
    yb = torch.empty_like(xs_small)
    descs = [(x, ys, yc, n_big, B.SINCOS), (xs_small, ya, None, 1000, B.SIN), (xs_small[3:], yb[3:], None, 997, B.TAN)]
    plan = B.BatchPlan(descs, B.BATCH_GRAPH)
    plan.run()
    torch.cuda.synchronize()
    idx = torch.from_numpy(_positions(n_big, 8)).cuda()
    xv = x[idx].cpu().numpy()
    xd = xv.astype(np.float64)
    for name, t in (("sin", ys), ("cos", yc)):
        ref, _ = P.reference_with_gpu_segments(oracle, name, xd, _segments(B, xv))
        P.check_values(oracle, name, xd, t[idx].cpu().numpy(), ref)
    xsd = xs_small.cpu().numpy()
    ref, _ = P.reference_with_gpu_segments(oracle, "sin", xsd.astype(np.float64), _segments(B, xsd))
    P.check_values(oracle, "sin", xsd.astype(np.float64), ya.cpu().numpy(), ref)
    ref, _ = P.reference_with_gpu_segments(oracle, "tan", xsd[3:].astype(np.float64), _segments(B, xsd[3:]))
    P.check_values(oracle, "tan", xsd[3:].astype(np.float64), yb[3:].cpu().numpy(), ref)
    plan.close()
    del x, ys, yc
    torch.cuda.empty_cache()
