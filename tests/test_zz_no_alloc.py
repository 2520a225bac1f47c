"""The batch entry point that allocates nothing (ptrig_batch_run_noalloc).

It serves callers that may not call cudaMalloc (during stream capture, inside
an allocator, on latency-critical paths).  Its outputs must match the
plan-based ptrig_batch_run within the tolerances of the parity tests, on two
calls in a row with different batches, since the second call reuses the
library's one scratch table.  Kept in a file that pytest collects last.
"""
import ctypes

import numpy as np
import pytest

from paper_2502_10831_gb300 import workloads

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

SIN_COS_ATOL = 1e-6
TAN_RTOL = 1e-5


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_10831_gb300 import binding, build
    build.build()
    binding.lib()
    return binding


def _make(seed, count):
    """Ragged batch on the device: arrays of random length (some empty, some
    odd, some starting off the 16-byte grid) and random selectors."""
    r = np.random.default_rng(seed)
    lengths = [int(v) for v in r.integers(0, 30000, count)] + [0, 1, 3, 70001]
    funcs = [int(v) for v in r.integers(0, 4, len(lengths))]
    offs = [int(v) for v in r.integers(0, 4, len(lengths))]
    arrays = []
    for i, (n, f, o) in enumerate(zip(lengths, funcs, offs)):
        xh = workloads.batch_array(1000 * seed + i, n)
        xb = torch.from_numpy(np.concatenate([np.zeros(o, np.float32), xh])).cuda()
        yb = torch.full_like(xb, -9.0)
        zb = torch.full_like(xb, -9.0)
        arrays.append((xb[o:], yb[o:], zb[o:], n, f))
    return arrays


def _descs(B, arrays):
    arr = (B.ptrig_desc * len(arrays))()
    for i, (x, y, z, n, f) in enumerate(arrays):
        arr[i] = B.ptrig_desc(x.data_ptr(), y.data_ptr(), z.data_ptr() if f == B.SINCOS else 0, n, f, 0)
    raw = np.frombuffer(bytes(arr), dtype=np.uint8).copy()
    return torch.from_numpy(raw).cuda(), len(arrays)


def _outputs(arrays):
    torch.cuda.synchronize()
    return [(y.cpu().numpy()[:n].copy(), z.cpu().numpy()[:n].copy()) for (x, y, z, n, f) in arrays]


def _reset(arrays):
    for (x, y, z, n, f) in arrays:
        y.fill_(-9.0)
        z.fill_(-9.0)


def _close(func, got, ref):
    if got.size == 0:
        return True
    if func == "tan":
        scale = np.maximum(np.abs(ref.astype(np.float64)), 1e-30)
        return bool(np.all(np.abs(got.astype(np.float64) - ref) <= TAN_RTOL * scale))
    return bool(np.all(np.abs(got.astype(np.float64) - ref) <= SIN_COS_ATOL))


def test_noalloc_batch_matches_plan_batch_on_two_calls_in_a_row(B):
    batches = [_make(1, 70), _make(2, 45)]
    expected = []
    for arrays in batches:
        plan = B.BatchPlan([(x, y, z if f == B.SINCOS else None, n, f) for (x, y, z, n, f) in arrays])
        plan.run()
        expected.append(_outputs(arrays))
        plan.close()
        _reset(arrays)
    descs = [_descs(B, arrays) for arrays in batches]
    # two calls in a row; the second reuses (and must rewrite) the scratch table
    for (d, count) in descs:
        B.ptrig_batch_run_noalloc(d, count)
    got = [_outputs(arrays) for arrays in batches]
    for arrays, exp, out in zip(batches, expected, got):
        for (x, y, z, n, f), (ey, ez), (gy, gz) in zip(arrays, exp, out):
            name = ("sin", "cos", "tan", "sin")[f]
            assert _close(name, gy, ey), (n, f)
            if f == B.SINCOS:
                assert _close("cos", gz, ez), (n, f)
            else:
                assert np.all(gz == -9.0)  # untouched


def test_noalloc_batch_limits(B):
    from paper_2502_10831_gb300.binding import PtrigError
    d = torch.zeros(40 * 16385, dtype=torch.uint8, device="cuda")
    with pytest.raises(PtrigError):
        B.ptrig_batch_run_noalloc(d, 16385)  # more arrays than the scratch table holds
    with pytest.raises(PtrigError):
        B.ptrig_batch_run_noalloc(None, 3)
    B.ptrig_batch_run_noalloc(None, 0)  # empty batch: no-op
    assert ctypes.sizeof(B.ptrig_desc) == 40
