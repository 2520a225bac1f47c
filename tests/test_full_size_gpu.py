"""The other configurations at their full sizes, in the launch configurations
bench.py times, checked on sampled outputs against the oracle (and through
properties that hold at any size)."""
import numpy as np
import pytest

import parity as P
from paper_2502_10831_gb300 import workloads

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_10831_gb300 import binding, build
    build.build()
    return binding


def _sample(n, k=1 << 15, seed=23):
    r = np.random.default_rng(seed)
    return np.unique(np.concatenate([r.integers(0, n, k), np.arange(min(n, 512)), np.arange(max(0, n - 512), n)]))


@pytest.mark.parametrize("dt", ["f16", "bf16"])
def test_half_full_size_sampled(B, oracle, dt):
    n = 1 << 28
    if dt == "f16":
        bits = workloads.half16(n).view(np.uint16)
        vals = bits.view(np.float16)
    else:
        bits = workloads.half_bf16(n)
        vals = None
    xt = torch.from_numpy(bits.view(np.int16)).cuda()
    ys = torch.empty_like(xt)
    yc = torch.empty_like(xt)
    getattr(B, f"ptrig_sincos_{dt}")(xt, ys, yc)
    torch.cuda.synchronize()
    idx = _sample(n)
    it = torch.from_numpy(idx).cuda()
    xs = bits[idx]
    xd = (vals[idx].astype(np.float64) if dt == "f16" else workloads.bf16_bits_to_f32(xs).astype(np.float64))
    for name, t in (("sin", ys), ("cos", yc)):
        raw = t[it].cpu().numpy().view(np.uint16)
        got = raw.view(np.float16).astype(np.float64) if dt == "f16" else \
            workloads.bf16_bits_to_f32(raw).astype(np.float64)
        ref = oracle.proposed(name, xd)
        assert np.abs(got - ref).max() <= 2e-3, (dt, name)
    del xt, ys, yc
    torch.cuda.empty_cache()


def test_batch_full_size_sampled(B, oracle):
    """4096 ragged arrays (about 4.5e8 angles) in one graph launch, with the
    plan's autotuned configuration; sampled arrays against the oracle."""
    lengths, sel = workloads.batch_spec(4096)
    total = int(sum((int(n) + 63) // 64 * 64 for n in lengths))
    xs = torch.empty(total, dtype=torch.float32, device="cuda")
    y0 = torch.empty_like(xs)
    y1 = torch.empty_like(xs)
    descs, offs, off = [], [], 0
    for i, (n, f) in enumerate(zip(lengths, sel)):
        n = int(n)
        xs[off:off + n] = torch.from_numpy(workloads.batch_array(i, n)).cuda()
        descs.append((xs[off:off + n], y0[off:off + n], y1[off:off + n] if f == 3 else None, n, int(f)))
        offs.append(off)
        off += (n + 63) // 64 * 64
    plan = B.BatchPlan(descs, B.BATCH_GRAPH)
    plan.autotune(reps=2)
    plan.run()
    torch.cuda.synchronize()
    r = np.random.default_rng(3)
    for i in r.choice(len(lengths), 48, replace=False):
        n, f, o = int(lengths[i]), int(sel[i]), offs[i]
        xh = workloads.batch_array(int(i), n).astype(np.float64)
        pick = np.unique(np.concatenate([r.integers(0, n, 256), [0, n - 1]]))
        for name, buf in ((("sin", "cos", "tan", "sin")[f], y0),) + ((("cos", y1),) if f == 3 else ()):
            got = buf[o:o + n].cpu().numpy()[pick].astype(np.float64)
            ref = oracle.proposed(name, xh[pick])
            if name == "tan":
                keep = np.abs(oracle.proposed("cos", xh[pick])) >= 1e-3
                u, *_ = oracle.reduce(xh[pick])
                keep &= ~P.near_node(u)
                assert np.all(np.abs(got[keep] - ref[keep]) <= 1e-5 * np.abs(ref[keep]))
            else:
                u, *_ = oracle.reduce(xh[pick])
                keep = ~P.near_node(u)
                assert np.abs(got - ref)[keep].max() <= 1e-6
    plan.close()


def test_fused_loss_full_size(B, oracle):
    """[8192, 4096] loss and gradient: gradient sampled against the oracle's
    analytic derivative; loss within FP32 summation error of the oracle's."""
    x, w, v, u = workloads.autograd((8192, 4096))
    n = x.size
    xt, wt, vt, ut = (torch.from_numpy(a.reshape(-1)).cuda() for a in (x, w, v, u))
    loss = torch.empty((), dtype=torch.float64, device="cuda")
    gx = torch.empty_like(xt)
    B.ptrig_sincostan_loss_f32(xt, wt, vt, ut, -50.0, 50.0, loss, gx)
    torch.cuda.synchronize()
    idx = _sample(n)
    xd = x.reshape(-1)[idx].astype(np.float64)
    wd, vd, ud = (a.reshape(-1)[idx].astype(np.float64) for a in (w, v, u))
    t = oracle.proposed("tan", xd)
    g_ref = (wd * oracle.derivative("sin", xd) + vd * oracle.derivative("cos", xd)
             + ud * oracle.derivative("tan", xd) * ((t >= -50) & (t <= 50)))
    uu, *_ = oracle.reduce(xd)
    keep = ~P.near_node(uu) & (np.abs(oracle.proposed("cos", xd)) >= 1e-3) & (np.abs(np.abs(t) - 50) > 1e-2)
    got = gx.cpu().numpy()[idx].astype(np.float64)
    assert np.max(np.abs(got - g_ref)[keep] / np.maximum(1.0, np.abs(g_ref[keep]))) <= 5e-5
    # loss: the full oracle sum (33.5M terms, about 10 s of CPU)
    xf = x.reshape(-1).astype(np.float64)
    tf = oracle.proposed("tan", xf)
    l_ref = float(np.sum(w.reshape(-1) * oracle.proposed("sin", xf) + v.reshape(-1) * oracle.proposed("cos", xf)
                         + u.reshape(-1) * np.clip(tf, -50, 50)))
    assert abs(loss.item() - l_ref) <= 1e-5 * abs(l_ref) + 5e-2
