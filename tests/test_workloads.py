"""The seeded input generators produce the workloads the docs describe:
component fractions, ranges, dtypes, the ragged batch's lengths and total,
bf16 rounding, and chunk-wise determinism.  CPU only."""
import math

import numpy as np
import pytest

from paper_2502_10831_gb300 import workloads as W

PI = math.pi


def _dist_to_grid(x, step, offset=0.0):
    """Distance of each x to the nearest offset + k step."""
    k = np.rint((x - offset) / step)
    return np.abs(x - offset - k * step), k


def test_parity_mixture():
    x = W.parity(1 << 20).astype(np.float64)
    assert x.dtype == np.float64 and np.all(np.abs(x) <= 2 * PI + 1e-3)
    d, k = _dist_to_grid(x, PI, PI / 2)  # odd multiples of pi/2
    near = (d <= 1.001e-3) & (np.abs(PI / 2 + k * PI) <= 1.5 * PI + 1e-9)
    # 10% drawn near the four poles, plus the uniform part's own share of those windows
    expect = 0.10 + 0.90 * 4 * 2e-3 / (4 * PI)
    assert abs(near.mean() - expect) < 0.003


def test_bandwidth_mixture():
    # the array is the FP32 rounding of a float64 mixture drawn per chunk
    m = 1 << 22
    v = W._mixture(W._rng("bandwidth", 0), m, 100 * PI, 0.8, 0.1, 1200, 1e-4, 1e-3)
    assert np.array_equal(W.bandwidth(m), v.astype(np.float32))
    assert np.all(np.abs(v) <= 100 * PI + 1e-3)
    dn, kn = _dist_to_grid(v, PI / 12)
    dp, _ = _dist_to_grid(v, PI, PI / 2)
    # near a node: the 10% node component, the uniform part's share of the
    # windows, and the pole component within 1e-4 of its pole (a node too)
    expect_node = 0.10 + 0.80 * 2e-4 / (PI / 12) + 0.10 * 0.1
    # near a pole: the 10% pole component, the uniform part's share, and the
    # nodes that are poles (k an odd multiple of 6: 1 in 12)
    expect_pole = 0.10 + 0.80 * 2e-3 / PI + 0.10 / 12
    assert np.all(np.abs(kn[dn <= 1e-4]) <= 1200)
    assert abs((dn <= 1e-4).mean() - expect_node) < 0.002
    assert abs((dp <= 1e-3).mean() - expect_pole) < 0.002


def test_half_workloads():
    h = W.half16(1 << 20)
    assert h.dtype == np.float16
    assert np.all(np.isfinite(h)) and np.all(np.abs(h.astype(np.float64)) <= 60.1)
    b = W.half_bf16(1 << 20)
    assert b.dtype == np.uint16
    x = W.bf16_bits_to_f32(b).astype(np.float64)
    assert np.all(np.abs(x) <= 100 * PI * 1.01)


def test_bf16_rounding_is_nearest_even():
    torch = pytest.importorskip("torch")
    r = np.random.default_rng(5)
    x = np.concatenate([r.standard_normal(1 << 16).astype(np.float32) * 1e3,
                        (r.integers(0, 1 << 32, 1 << 16, dtype=np.uint64).astype(np.uint32)).view(np.float32),
                        np.array([np.inf, -np.inf, 0.0, -0.0, 3.0e38, 1e-40], dtype=np.float32)])
    x = x[~np.isnan(x)]
    want = torch.from_numpy(x).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    assert np.array_equal(W.f32_to_bf16_bits(x), want)
    assert W.f32_to_bf16_bits(np.array([np.nan], dtype=np.float32))[0] == 0x7FC0


def test_large_is_log_uniform_with_random_sign():
    x = W.large(1 << 20).astype(np.float64)
    a = np.log10(np.abs(x))
    assert a.min() >= -1e-6 and a.max() <= 5 + 1e-6
    # log-uniform: each decade holds a fifth of the angles
    counts = np.histogram(a, bins=5, range=(0, 5))[0] / x.size
    assert np.all(np.abs(counts - 0.2) < 0.005)
    assert abs((x < 0).mean() - 0.5) < 0.005


def test_batch_spec_total_and_ranges():
    lengths, sel = W.batch_spec()
    assert lengths.size == 4096 and int(lengths.sum()) == 458_624_309
    assert lengths.min() >= 100 and lengths.max() < 1_000_000
    assert set(np.unique(sel)) == {0, 1, 2, 3}
    assert np.all(np.abs(np.bincount(sel) / 4096 - 0.25) < 0.03)
    v = W.batch_array(7, 5000)
    assert v.dtype == np.float32 and np.all(np.abs(v) <= 8 * PI)


def test_autograd_inputs():
    x, w, v, u = W.autograd((64, 1024))
    assert x.shape == (64, 1024) and all(a.shape == x.shape and a.dtype == np.float32 for a in (w, v, u))
    assert np.all(np.abs(x) <= 4 * PI)
    assert abs(float(w.mean())) < 0.05 and abs(float(w.std()) - 1) < 0.05


def test_deterministic_and_chunk_stable():
    a = W.bandwidth(W.CHUNK + 1000)
    b = W.bandwidth(W.CHUNK + 1000)
    assert np.array_equal(a, b)
    # a whole chunk's values do not depend on the array's length
    assert np.array_equal(W.bandwidth(W.CHUNK)[:W.CHUNK], a[:W.CHUNK])
    assert np.array_equal(W.bandwidth(2 * W.CHUNK + 7)[:W.CHUNK], a[:W.CHUNK])
    assert not np.array_equal(W.bandwidth(1000, seed=1), a[:1000])
