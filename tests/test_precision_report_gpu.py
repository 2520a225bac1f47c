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
