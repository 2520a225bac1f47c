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
