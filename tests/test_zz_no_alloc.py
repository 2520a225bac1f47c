"""The batch entry point that allocates nothing (ptrig_batch_run_noalloc).

It serves callers that may not call cudaMalloc (inside an allocator or memory
pool, on latency-critical paths where an allocation could synchronize the
device).  Its outputs must match the
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


def _segments(B, x):
    s = torch.empty(x.shape, dtype=torch.uint8, device="cuda")
    B.ptrig_segment_f32(x, s)
    torch.cuda.synchronize()
    return s.cpu().numpy()


def test_noalloc_batch_matches_the_oracle(B, oracle):
    """Each array of a no-allocation batch against the FP64 oracle directly
    (near a node with the segment the GPU chose)."""
    import parity as P
    arrays = _make(3, 40)
    d, count = _descs(B, arrays)
    B.ptrig_batch_run_noalloc(d, count)
    out = _outputs(arrays)
    for (x, y, z, n, f), (gy, gz) in zip(arrays, out):
        if n == 0:
            continue
        xs = x[:n]
        xd = xs.cpu().numpy().astype(np.float64)
        seg = _segments(B, xs)
        names = [("sin", gy), ("cos", gz)] if f == B.SINCOS else [(("sin", "cos", "tan")[f], gy)]
        for name, got in names:
            ref, _ = P.reference_with_gpu_segments(oracle, name, xd, seg)
            P.check_values(oracle, name, xd, got, ref)


def test_noalloc_batch_at_the_array_limit(B, oracle):
    """16384 arrays (the scratch table's limit) of 1 to 64 elements each,
    packed into one allocation: every output against the oracle."""
    import parity as P
    count = 16384
    r = np.random.default_rng(8)
    lengths = r.integers(1, 65, count)
    funcs = r.integers(0, 4, count)
    offs = np.concatenate([[0], np.cumsum(lengths)[:-1]])
    total = int(lengths.sum())
    xh = workloads.batch_array(77, total)
    x = torch.from_numpy(xh).cuda()
    y = torch.full_like(x, -9.0)
    z = torch.full_like(x, -9.0)
    arr = (B.ptrig_desc * count)()
    for i in range(count):
        o, n, f = int(offs[i]), int(lengths[i]), int(funcs[i])
        arr[i] = B.ptrig_desc(x.data_ptr() + 4 * o, y.data_ptr() + 4 * o,
                              z.data_ptr() + 4 * o if f == B.SINCOS else 0, n, f, 0)
    d = torch.from_numpy(np.frombuffer(bytes(arr), dtype=np.uint8).copy()).cuda()
    B.ptrig_batch_run_noalloc(d, count)
    torch.cuda.synchronize()
    yh, zh = y.cpu().numpy(), z.cpu().numpy()
    xd = xh.astype(np.float64)
    seg = _segments(B, x)
    fe = np.repeat(funcs, lengths)  # selector of every element
    for f, name in ((0, "sin"), (1, "cos"), (2, "tan"), (3, "sin")):
        m = fe == f
        ref, _ = P.reference_with_gpu_segments(oracle, name, xd[m], seg[m])
        P.check_values(oracle, name, xd[m], yh[m], ref)
    m = fe == 3
    ref, _ = P.reference_with_gpu_segments(oracle, "cos", xd[m], seg[m])
    P.check_values(oracle, "cos", xd[m], zh[m], ref)
    assert np.all(zh[fe != 3] == -9.0)


def test_noalloc_batch_skips_invalid_descriptors(B):
    """Descriptors with an unknown selector, a nonzero reserved field or a
    NULL input (or output) pointer with n > 0 are skipped: their outputs keep
    the fill, and the valid arrays around them are computed."""
    n = 5000
    xs = [torch.from_numpy(workloads.batch_array(900 + i, n)).cuda() for i in range(7)]
    ys = [torch.full_like(x, -9.0) for x in xs]
    zs = [torch.full_like(x, -9.0) for x in xs]
    D = B.ptrig_desc
    arr = (D * 7)(
        D(xs[0].data_ptr(), ys[0].data_ptr(), 0, n, B.SIN, 0),        # valid
        D(xs[1].data_ptr(), ys[1].data_ptr(), 0, n, 7, 0),            # unknown func
        D(xs[2].data_ptr(), ys[2].data_ptr(), 0, n, B.COS, 1),        # reserved != 0
        D(0, ys[3].data_ptr(), 0, n, B.TAN, 0),                       # NULL x
        D(xs[4].data_ptr(), ys[4].data_ptr(), 0, n, B.SINCOS, 0),     # sincos without y1
        D(xs[5].data_ptr(), 0, 0, n, B.SIN, 0),                       # NULL y0
        D(xs[6].data_ptr(), ys[6].data_ptr(), zs[6].data_ptr(), n, B.SINCOS, 0),  # valid
    )
    d = torch.from_numpy(np.frombuffer(bytes(arr), dtype=np.uint8).copy()).cuda()
    B.ptrig_batch_run_noalloc(d, 7)
    torch.cuda.synchronize()
    for i in (1, 2, 3, 4, 5):
        assert torch.all(ys[i] == -9.0).item() and torch.all(zs[i] == -9.0).item(), i
    s0 = torch.empty_like(xs[0])
    B.ptrig_sin_f32(xs[0], s0)
    s6, c6 = torch.empty_like(xs[6]), torch.empty_like(xs[6])
    B.ptrig_sincos_f32(xs[6], s6, c6)
    torch.cuda.synchronize()
    assert torch.equal(ys[0], s0) and torch.equal(ys[6], s6) and torch.equal(zs[6], c6)
    assert torch.all(zs[0] == -9.0).item()
