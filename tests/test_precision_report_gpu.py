"""Per-function error of the GPU results against the FP64 oracle (the kernels'
own rounding error), and of the oracle against libm FP64 (the method's own
approximation error), for FP32, fp16 and bf16 storage.

The asserts are the parity tolerances; the figures are written to
$PTRIG_REPORT_DIR/precision_report.json when that variable is set.
"""
import json
import os

import numpy as np
import pytest

import parity as P
from paper_2502_10831_gb300 import workloads

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

TOL = {  # abs for sin/cos, relative (|cos| >= 1e-3) for tan
    ("f32", "sin"): 1e-6, ("f32", "cos"): 1e-6, ("f32", "tan"): 1e-5,
    ("f16", "sin"): 2e-3, ("f16", "cos"): 2e-3, ("f16", "tan"): 2.0 ** -11 + 1e-6,
    ("bf16", "sin"): 2e-3, ("bf16", "cos"): 2e-3, ("bf16", "tan"): 2.0 ** -8 + 1e-6,
}


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_10831_gb300 import binding, build
    build.build()
    return binding


def _inputs(dt):
    n = 1 << 20
    if dt == "f32":
        x = workloads.parity(n)
        return x, x.astype(np.float64)
    if dt == "f16":
        h = workloads.half16(n)
        return h.view(np.int16), h.astype(np.float64)
    b = workloads.half_bf16(n)
    return b.view(np.int16), workloads.bf16_bits_to_f32(b).astype(np.float64)


def _decode(raw, dt):
    if dt == "f32":
        return raw.astype(np.float64)
    if dt == "f16":
        return raw.view(np.float16).astype(np.float64)
    return workloads.bf16_bits_to_f32(raw.view(np.uint16)).astype(np.float64)


def test_precision_report(B, oracle):
    report = {}
    for dt in ("f32", "f16", "bf16"):
        x_store, xd = _inputs(dt)
        xt = torch.from_numpy(np.ascontiguousarray(x_store)).cuda()
        seg_x = torch.from_numpy(xd.astype(np.float32)).cuda()
        seg = torch.empty(seg_x.shape, dtype=torch.uint8, device="cuda")
        B.ptrig_segment_f32(seg_x, seg)
        cosr = np.abs(oracle.proposed("cos", xd))
        for f in ("sin", "cos", "tan"):
            y = torch.empty_like(xt)
            getattr(B, f"ptrig_{f}_{dt}")(xt, y)
            torch.cuda.synchronize()
            got = _decode(y.cpu().numpy(), dt)
            ref, _ = P.reference_with_gpu_segments(oracle, f, xd, seg.cpu().numpy())
            exact = getattr(np, f)(xd)
            if f == "tan":
                keep = (cosr >= 1e-3) & np.isfinite(got) & (np.abs(ref) > 1e-4)
                if dt == "f16":
                    keep &= np.abs(ref) < 6.5e4
                e_gpu = np.abs(got[keep] - ref[keep]) / np.abs(ref[keep])
                e_method = np.abs(ref[keep] - exact[keep]) / np.abs(exact[keep])
                kind = "relative, |cos| >= 1e-3"
            else:
                e_gpu = np.abs(got - ref)
                e_method = np.abs(ref - exact)
                kind = "absolute"
            report[f"{f}_{dt}"] = {
                "vs_oracle": {"max": float(e_gpu.max()), "mean": float(e_gpu.mean()), "kind": kind,
                              "tolerance": TOL[(dt, f)]},
                "method_vs_libm_fp64": {"max": float(e_method.max()), "mean": float(e_method.mean()),
                                        "kind": kind},
                "n": int(e_gpu.size)}
            assert e_gpu.max() <= TOL[(dt, f)], (dt, f, e_gpu.max())
    out = os.environ.get("PTRIG_REPORT_DIR")
    if out:
        os.makedirs(out, exist_ok=True)
        with open(os.path.join(out, "precision_report.json"), "w") as fh:
            json.dump(report, fh, indent=1)


def _threaded(fn, x, parts=16):
    """fn over slices of x on host threads (the oracle's C calls release the GIL)."""
    from concurrent.futures import ThreadPoolExecutor
    chunks = np.array_split(x, parts)
    with ThreadPoolExecutor(max_workers=parts) as ex:
        return np.concatenate(list(ex.map(fn, chunks)))


def test_precision_report_large_arguments(B, oracle):
    """The precision configuration's large-argument set: 2^24 FP32 angles with
    |x| log-uniform in [1, 1e5] (FP32 reduction), and 2^20 samples of each
    FP32 Payne-Hanek side path in two ranges -- |x| log-uniform in
    [2^19, 2^31) and in [2^31, 2^127).  Per function (sincos: both outputs
    of the fused kernel) the error against the FP64 oracle and the oracle's
    against numpy's float64 functions (the method's own error)."""
    r = np.random.default_rng(11)
    sets = {"log_uniform_1_1e5_2p24": workloads.large(1 << 24)}
    for name, lo, hi in (("side_2p19_2p31", 19.0, 31.0), ("side_2p31_2p127", 31.0, 127.0)):
        sets[name] = (2.0 ** r.uniform(lo, hi, 1 << 20) * r.choice([-1.0, 1.0], 1 << 20)).astype(np.float32)
    report = {}
    for sname, x in sets.items():
        xd = x.astype(np.float64)
        xt = torch.from_numpy(x).cuda()
        seg = torch.empty(xt.shape, dtype=torch.uint8, device="cuda")
        B.ptrig_segment_f32(xt, seg)
        ys = {}
        for f in ("sin", "cos", "tan"):
            y = torch.empty_like(xt)
            getattr(B, f"ptrig_{f}_f32")(xt, y)
            ys[f] = y
        s, c = torch.empty_like(xt), torch.empty_like(xt)
        B.ptrig_sincos_f32(xt, s, c)
        torch.cuda.synchronize()
        segh = seg.cpu().numpy()
        cosr = np.abs(_threaded(lambda a: oracle.proposed("cos", a), xd))
        # the oracle with the segment the GPU chose (near a node either is valid)
        idx = np.arange(xd.size)
        refs = {f: _threaded(lambda i: P.reference_with_gpu_segments(oracle, f, xd[i], segh[i])[0], idx)
                for f in ("sin", "cos", "tan")}
        outs = [(f, f, ys[f]) for f in ("sin", "cos", "tan")] + [("sincos.sin", "sin", s), ("sincos.cos", "cos", c)]
        sec = {}
        for label, f, t in outs:
            got = t.cpu().numpy().astype(np.float64)
            ref = refs[f]
            exact = getattr(np, f)(xd)
            if f == "tan":
                keep = cosr >= 1e-3
                e_gpu = np.abs(got[keep] - ref[keep]) / np.abs(ref[keep])
                e_method = np.abs(ref[keep] - exact[keep]) / np.abs(exact[keep])
                kind = "relative, |cos| >= 1e-3"
                tol = 1e-5
            else:
                e_gpu = np.abs(got - ref)
                e_method = np.abs(ref - exact)
                kind = "absolute"
                tol = 1e-6
            sec[label] = {"vs_oracle": {"max": float(e_gpu.max()), "mean": float(e_gpu.mean()), "kind": kind,
                                        "tolerance": tol},
                          "method_vs_numpy_fp64": {"max": float(e_method.max()), "mean": float(e_method.mean()),
                                                   "kind": kind},
                          "n": int(e_gpu.size)}
            assert e_gpu.max() <= tol, (sname, label, e_gpu.max())
        report[sname] = sec
        del xt, seg, ys, s, c
        torch.cuda.empty_cache()
    out = os.environ.get("PTRIG_REPORT_DIR")
    if out:
        os.makedirs(out, exist_ok=True)
        with open(os.path.join(out, "precision_report_large.json"), "w") as fh:
            json.dump(report, fh, indent=1)


def test_precision_report_derivatives_and_fp64(B, oracle):
    """The differentiation configuration's inputs (2^22 angles of x ~
    U[-4pi, 4pi], w, v, u ~ N(0, 1)): each FP32 derivative kernel and the
    fused loss kernel against the oracle's derivative and loss, away from the
    pi/12 nodes (where the two adjacent formulas have different slopes); and
    the FP64 forward and derivative kernels on the 2^20-angle parity set.
    Derivative errors are |got - ref| / max(1, |ref|)."""
    n = 1 << 22
    x, w, v, u = (a.reshape(-1)[:n].copy() for a in workloads.autograd((8192, 512)))
    xd = x.astype(np.float64)
    ured, *_ = oracle.reduce(xd)
    keep = ~P.near_node(ured)
    idx = np.arange(n)
    dref = {f: _threaded(lambda i: oracle.derivative(f, xd[i]), idx) for f in ("sin", "cos", "tan")}
    cosr = np.abs(_threaded(lambda i: oracle.proposed("cos", xd[i]), idx))
    report = {}
    xt = torch.from_numpy(x).cuda()
    gy = torch.ones_like(xt)
    for f in ("sin", "cos", "tan"):
        gx = torch.empty_like(xt)
        getattr(B, f"ptrig_{f}_bwd_f32")(xt, gy, gx)
        torch.cuda.synchronize()
        got = gx.cpu().numpy().astype(np.float64)
        k = keep & (cosr >= 1e-3) if f == "tan" else keep
        e = np.abs(got[k] - dref[f][k]) / np.maximum(1.0, np.abs(dref[f][k]))
        report[f"{f}_bwd_f32"] = {"max": float(e.max()), "mean": float(e.mean()), "n": int(e.size),
                                  "kind": "|got - ref| / max(1, |ref|), away from nodes", "tolerance": 2e-5}
        assert e.max() <= 2e-5, (f, e.max())
    # fused loss: loss and dL/dx with clamp(tan, -50, 50)
    lo, hi = -50.0, 50.0
    tref = _threaded(lambda i: oracle.proposed("tan", xd[i]), idx)
    sref = _threaded(lambda i: oracle.proposed("sin", xd[i]), idx)
    cref = _threaded(lambda i: oracle.proposed("cos", xd[i]), idx)
    inside = (tref >= lo) & (tref <= hi)
    g_ref = w * dref["sin"] + v * dref["cos"] + u * dref["tan"] * inside
    loss_ref = float(np.sum(w * sref + v * cref + u * np.clip(tref, lo, hi)))
    wt, vt, ut = (torch.from_numpy(a).cuda() for a in (w, v, u))
    loss = torch.zeros((), dtype=torch.float64, device="cuda")
    gx = torch.empty_like(xt)
    B.ptrig_sincostan_loss_f32(xt, wt, vt, ut, lo, hi, loss, gx)
    torch.cuda.synchronize()
    got = gx.cpu().numpy().astype(np.float64)
    k = keep & (cosr >= 1e-3) & (np.abs(np.abs(tref) - 50.0) > 1e-2)
    e = np.abs(got[k] - g_ref[k]) / np.maximum(1.0, np.abs(g_ref[k]))
    rel_loss = abs(loss.item() - loss_ref) / max(1.0, abs(loss_ref))
    report["fused_loss_f32"] = {"gradient": {"max": float(e.max()), "mean": float(e.mean()), "n": int(e.size),
                                             "kind": "|got - ref| / max(1, |ref|), away from nodes, poles and "
                                                     "the clamp edges"},
                                "loss": {"relative": rel_loss, "value": loss.item(), "oracle": loss_ref}}
    assert e.max() <= 5e-5 and abs(loss.item() - loss_ref) <= 1e-5 * max(1.0, abs(loss_ref)) + 1e-3
    # FP64 data path on the parity set
    xp = workloads.parity(1 << 20).astype(np.float64)
    up, *_ = oracle.reduce(xp)
    kp = np.abs(up - np.round(up / P.STEP) * P.STEP) >= 1e-13
    cp = np.abs(oracle.proposed("cos", xp))
    xpt = torch.from_numpy(xp).cuda()
    for f in ("sin", "cos", "tan"):
        y = torch.empty_like(xpt)
        dy = torch.empty_like(xpt)
        getattr(B, f"ptrig_{f}_f64")(xpt, y)
        getattr(B, f"ptrig_{f}_bwd_f64")(xpt, torch.ones_like(xpt), dy)
        torch.cuda.synchronize()
        ref = oracle.proposed(f, xp)
        dr = oracle.derivative(f, xp)
        k = kp & (cp >= 1e-3) if f == "tan" else kp
        yh, dyh = y.cpu().numpy(), dy.cpu().numpy()
        ev = np.abs(yh[k] - ref[k]) / (np.abs(ref[k]) if f == "tan" else 1.0)
        ed = np.abs(dyh[k] - dr[k]) / np.maximum(1.0, np.abs(dr[k]))
        report[f"{f}_f64"] = {"value": {"max": float(ev.max()), "mean": float(ev.mean()),
                                        "kind": "relative, |cos| >= 1e-3" if f == "tan" else "absolute"},
                              "derivative": {"max": float(ed.max()), "mean": float(ed.mean()),
                                             "kind": "|got - ref| / max(1, |ref|)"},
                              "n": int(k.sum())}
        assert ev.max() <= (1e-11 if f == "tan" else 1e-12) and ed.max() <= 1e-10
    out = os.environ.get("PTRIG_REPORT_DIR")
    if out:
        os.makedirs(out, exist_ok=True)
        with open(os.path.join(out, "precision_report_derivatives.json"), "w") as fh:
            json.dump(report, fh, indent=1)
