#!/usr/bin/env python
"""Throughput of the pi/12 piecewise trigonometric hot path (arXiv 2502.10831)
on GB300.

One step = one pass of the whole FP32 hot path over the bandwidth workload
(2^28 angles: 80% U[-100pi, 100pi], 10% within 1e-4 of k pi/12, 10% within
1e-3 of odd multiples of pi/2): proposed sin, cos, tan, sincos and the
Taylor-5 sin, cos, tan baseline, one kernel launch each.  value = angles
evaluated per second (Gelem/s, summed over the step's seven kernels), inputs
resident in HBM; the 1 GiB input and outputs exceed the 129 MB L2, so no
flush is needed between kernels.

Extra objects on the JSON line: per-kernel times and HBM fractions, the
roofline of the dominant kernel, fp16 / bf16 packed storage against the plain
FP32 kernels, CUDA's own sinf / __sinf on the same array, the end-to-end rate
through the C ABI from pinned host buffers, the FP64 oracle timed on the host
cores (cpu_baseline) and SM clocks sampled during the timed region.

  python bench.py [--steps K] [--warmup W] [--gpus N] [--impl {ptrig,reference}]
Under torchrun (N > 1) every rank evaluates its own 2^28-angle shard
(replicas, weak scaling); rank 0 prints the line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2502_10831_gb300 import replicas as R  # noqa: E402

METRIC = "Gelem/s & % HBM peak, π/12 sin/cos/tan on 2^28 fp32; packed-half vs plain"
NOMINAL_HBM_GBS = 8000.0  # GB300 HBM3e nominal rate, for context beside the measured copy peak
WORKLOAD = ("bandwidth: 2^28 fp32 angles, 80% U[-100pi,100pi], 10% within 1e-4 of k*pi/12, "
            "10% within 1e-3 of odd multiples of pi/2; step = proposed sin, cos, tan, sincos + "
            "Taylor-5 sin, cos, tan (one launch each)")


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ------------------------------------------------------------------ clocks


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line.strip()))

    def stop(self):
        if self.proc is None:
            return
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)

    def window(self, t0=None, t1=None):
        """Summary of the samples taken between t0 and t1 (perf_counter)."""
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.12)  # let the sampler read past t1
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ts, line in list(self.lines):
            if t0 is not None and not (t0 - 0.05 <= ts <= t1 + 0.05):
                continue
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm), "interval_ms": 50}


# -------------------------------------------------------------- CPU oracle


def _oracle_pass(O, xd, threads):
    """The step's seven functions with the oracle over xd on `threads` host
    threads (the C calls release the GIL); returns seconds."""
    import numpy as np
    from concurrent.futures import ThreadPoolExecutor

    parts = np.array_split(xd, threads)

    def work(part):
        for f in ("sin", "cos", "tan"):
            O.proposed(f, part)
        O.proposed("sin", part)  # sincos = sin and cos of the same angle
        O.proposed("cos", part)
        for f in ("sin", "cos", "tan"):
            O.taylor(f, 5, part)
        return part.size

    t0 = time.perf_counter()
    if threads == 1:
        work(xd)
    else:
        with ThreadPoolExecutor(max_workers=threads) as ex:
            list(ex.map(work, parts))
    return time.perf_counter() - t0


def cpu_model() -> str:
    """The host CPU's model string (lscpu's "Model name", else /proc/cpuinfo)."""
    import subprocess
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def oracle_rate(x_host, threads: int | None = None, full: bool = True):
    """The FP64 oracle, as it stands, over bounded samples of the workloads:
    the step's seven functions on the first 2^24 angles of the bandwidth
    workload on every host core (`value`), and with `full` also on 2^20 of
    them on one core, on the 2^20-angle parity workload on every core, and the
    host C library's double sin / cos / tan on the same 2^24 angles (context:
    the inbuilt functions the paper compares against)."""
    import numpy as np

    from oracle import ptrig_oracle as O

    O.lib()
    threads = threads or os.cpu_count() or 1
    m = min(x_host.size, 1 << 24)
    xd = x_host[:m].astype(np.float64)
    dt = _oracle_pass(O, xd, threads)
    out = {"value": 7 * m / dt / 1e9, "unit": "Gelem/s", "cores": threads, "kind": "oracle",
           "sample": f"first {m} angles of the bandwidth workload x 7 functions (sincos counted once), "
                     f"{threads} threads, {dt:.2f} s wall", "cpu_model": cpu_model()}
    if not full:
        return out
    m1 = min(m, 1 << 20)
    t1 = _oracle_pass(O, xd[:m1], 1)
    out["one_core"] = {"value": round(7 * m1 / t1 / 1e9, 5), "sample": f"first {m1} angles x 7 functions, 1 thread"}
    from paper_2502_10831_gb300 import workloads as W
    xc1 = W.parity(1 << 20).astype(np.float64)
    tc = _oracle_pass(O, xc1, threads)
    out["parity_workload"] = {"value": round(7 * xc1.size / tc / 1e9, 5),
                              "sample": f"the 2^20-angle parity workload x 7 functions, {threads} threads"}
    try:
        from cpu_simd import ptrig_cpu as C
        lib = {}
        for label, th, xs in (("all_cores", threads, xd), ("one_core", 1, xd[:m1])):
            t0 = time.perf_counter()
            for f in ("sin", "cos", "tan"):
                C.libm(f, xs, th)
            lib[label] = {"value": round(3 * xs.size / (time.perf_counter() - t0) / 1e9, 4),
                          "sample": f"{xs.size} angles x sin, cos, tan (C library, double), {th} threads"}
        out["libm_f64"] = lib
    except (ImportError, OSError, RuntimeError) as e:
        out["libm_f64"] = {"unavailable": str(e)}
    return out


def cpu_simd_rate(x_host):
    """The CPU SIMD baseline (cpu_simd/, vectorised across angles, one thread
    per online core) over the whole workload: each proposed function of the
    step once, outputs pre-touched, wall-clock timed."""
    import numpy as np

    from cpu_simd import ptrig_cpu as C

    threads = C.default_threads()
    y0 = np.zeros_like(x_host)
    y1 = np.zeros_like(x_host)
    C.evaluate("sincos", x_host[: 1 << 20], threads, out=(y0[: 1 << 20], y1[: 1 << 20]))
    per = {}
    total_t = 0.0
    for f in ("sin", "cos", "tan", "sincos"):
        t0 = time.perf_counter()
        C.evaluate(f, x_host, threads, out=(y0, y1))
        dt = time.perf_counter() - t0
        total_t += dt
        per[f] = {"s": round(dt, 4), "gelem_s": round(x_host.size / dt / 1e9, 3)}
    return {"value": round(4 * x_host.size / total_t / 1e9, 3), "unit": "Gelem/s", "cores": threads,
            "kind": "cpu_simd", "per_function": per,
            "sample": f"all {x_host.size} angles of the workload x the 4 proposed functions (sin, cos, tan, "
                      f"sincos; sincos counted once), FP32, {threads} threads"}


# ---------------------------------------------------------------- reference


def run_reference(args, rank, world):
    """--impl reference: the FP64 CPU oracle on the host cores, same workload,
    metric and unit; each step a bounded sample."""
    if rank != 0:
        return 0
    import numpy as np

    from paper_2502_10831_gb300 import workloads as W

    x = W.bandwidth(1 << 22)
    for _ in range(args.warmup):
        oracle_rate(x[: 1 << 18], full=False)
    vals = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        vals.append(oracle_rate(x, full=False))
    dt = time.perf_counter() - t0
    v = statistics.median(r["value"] for r in vals)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "Gelem/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "n": 1 << 22},
            "cpu_baseline": {"kind": "oracle", "cores": vals[0]["cores"], "sample": vals[0]["sample"], "value": v,
                             "unit": "Gelem/s"},
            "e2e": {"value": v, "unit": "Gelem/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "gpu_launches": 0}
    print(json.dumps(line))
    return 0


# --------------------------------------------------------------------- GPU


class Kernel:
    """One kernel launch of a step: name, algorithmic bytes per launch,
    angles evaluated per launch, and the call that launches it."""

    def __init__(self, name, nbytes, elems, call, launches=1):
        self.name, self.nbytes, self.elems, self.call, self.launches = name, nbytes, elems, call, launches


def workload_bandwidth(B, W, torch, dev, rank, log2n):
    n = 1 << log2n
    x_host = W.bandwidth(n, seed=R.shard_seed(W.SEED, rank))
    x = torch.from_numpy(x_host).to(dev)
    o = [torch.empty_like(x) for _ in range(2)]
    s = torch.cuda.current_stream().cuda_stream
    ks = [Kernel("sin_f32", 8 * n, n, lambda: B.ptrig_sin_f32(x, o[0], n, s)),
          Kernel("cos_f32", 8 * n, n, lambda: B.ptrig_cos_f32(x, o[0], n, s)),
          Kernel("tan_f32", 8 * n, n, lambda: B.ptrig_tan_f32(x, o[0], n, s)),
          Kernel("sincos_f32", 12 * n, n, lambda: B.ptrig_sincos_f32(x, o[0], o[1], n, s)),
          Kernel("taylor_sin_f32", 8 * n, n, lambda: B.ptrig_taylor_sin_f32(x, o[0], n, s)),
          Kernel("taylor_cos_f32", 8 * n, n, lambda: B.ptrig_taylor_cos_f32(x, o[0], n, s)),
          Kernel("taylor_tan_f32", 8 * n, n, lambda: B.ptrig_taylor_tan_f32(x, o[0], n, s))]
    meta = {"metric": METRIC, "dtype": "f32", "workload": WORKLOAD.replace("2^28", f"2^{log2n}"), "n_per_gpu": n,
            "l2": f"inputs larger than L2 ({4 * n / 2**30:g} GiB vs 129 MB), no flush"}
    return ks, meta, {"x": x, "x_host": x_host, "n": n}


def workload_half(B, W, torch, dev, rank, log2n):
    import numpy as np
    n = 1 << log2n
    xs = {"f16": torch.from_numpy(W.half16(n, seed=R.shard_seed(W.SEED, rank)).view(np.int16)).to(dev),
          "bf16": torch.from_numpy(W.half_bf16(n, seed=R.shard_seed(W.SEED, rank)).view(np.int16)).to(dev)}
    o = [torch.empty_like(xs["f16"]) for _ in range(2)]
    s = torch.cuda.current_stream().cuda_stream
    ks = []
    for dt, x in xs.items():
        for f in ("sin", "cos", "tan"):
            ks.append(Kernel(f"{f}_{dt}", 4 * n, n, (lambda f=f, dt=dt, x=x: getattr(B, f"ptrig_{f}_{dt}")(x, o[0], n, s))))
        ks.append(Kernel(f"sincos_{dt}", 6 * n, n, (lambda dt=dt, x=x: getattr(B, f"ptrig_sincos_{dt}")(x, o[0], o[1], n, s))))
    meta = {"metric": f"Gelem/s, pi/12 sin/cos/tan/sincos on 2^{log2n} angles stored as fp16 and bf16 (FP32 math)",
            "dtype": "f16/bf16 storage, f32 math",
            "workload": f"precision: bandwidth mixture as fp16 (uniform part |x| <= 60) and as bf16, 2^{log2n} each; "
                        "step = sin, cos, tan, sincos for both types", "n_per_gpu": n,
            "l2": "inputs larger than L2 (512 MiB vs 129 MB), no flush"}
    return ks, meta, {}


def workload_large(B, W, torch, dev, rank, log2n):
    n = 1 << min(log2n, 26)
    x = torch.from_numpy(W.large(n, seed=R.shard_seed(W.SEED, rank))).to(dev)
    o = [torch.empty_like(x) for _ in range(2)]
    s = torch.cuda.current_stream().cuda_stream
    ks = [Kernel("sin_f32", 8 * n, n, lambda: B.ptrig_sin_f32(x, o[0], n, s)),
          Kernel("cos_f32", 8 * n, n, lambda: B.ptrig_cos_f32(x, o[0], n, s)),
          Kernel("tan_f32", 8 * n, n, lambda: B.ptrig_tan_f32(x, o[0], n, s)),
          Kernel("sincos_f32", 12 * n, n, lambda: B.ptrig_sincos_f32(x, o[0], o[1], n, s))]
    meta = {"metric": f"Gelem/s, pi/12 sin/cos/tan/sincos on 2^{n.bit_length() - 1} fp32 angles with |x| "
                      "log-uniform in [1, 1e5]",
            "dtype": "f32 (integer Payne-Hanek reduction above 2^19)",
            "workload": f"precision: 2^{n.bit_length() - 1} fp32 (the 2^24-angle precision mixture drawn at 4x the "
                        "size so the arrays exceed L2), |x| log-uniform in [1, 1e5], random sign; all within the "
                        "FP32 reduction range", "n_per_gpu": n,
            "l2": "inputs larger than L2 (256 MiB vs 129 MB), no flush"}
    return ks, meta, {"n": n}


def workload_batch(B, W, torch, dev, rank, log2n, arrays=4096, config=None):
    lengths, sel = W.batch_spec(arrays, seed=R.shard_seed(W.SEED, rank))
    total = int(lengths.sum())
    padded = int(sum((int(n) + 63) // 64 * 64 for n in lengths))
    xs = torch.empty(padded, dtype=torch.float32, device=dev)
    y0 = torch.empty_like(xs)
    y1 = torch.empty_like(xs)
    descs, off, nbytes = [], 0, 0
    for i, (n, f) in enumerate(zip(lengths, sel)):
        n = int(n)
        xs[off:off + n] = torch.from_numpy(W.batch_array(i, n, seed=R.shard_seed(W.SEED, rank))).to(dev)
        descs.append((xs[off:off + n], y0[off:off + n], y1[off:off + n] if f == 3 else None, n, int(f)))
        nbytes += (12 if f == 3 else 8) * n
        off += (n + 63) // 64 * 64  # each array starts on a 256-byte boundary, as separate allocations would
    plan = B.BatchPlan(descs, B.BATCH_GRAPH)
    if config:
        plan.set_config(*config)
        tuned = {"block": config[0], "items_per_thread": config[1], "fixed": True}
    else:
        tuned = plan.autotune(reps=3)
    s = torch.cuda.current_stream().cuda_stream
    ks = [Kernel("batch_graph", nbytes, total, lambda: plan.run(s))]
    meta = {"metric": f"Gelem/s, ragged batch of {arrays} fp32 arrays (per-array sin/cos/tan/sincos), one kernel "
                      "launch over a tile table, captured in a CUDA graph",
            "dtype": "f32", "workload": f"batching: {arrays} arrays, lengths floor(exp U[ln 100, ln 1e6]) "
                                        f"(total {total}), values U[-8pi, 8pi], selectors uniform",
            "n_per_gpu": total, "l2": "inputs larger than L2, no flush", "autotuned": tuned}
    return ks, meta, {"plan": plan, "descs": descs}


def workload_autograd(B, W, torch, dev, rank, log2n):
    from paper_2502_10831_gb300 import functional as Fn
    x_h, w_h, v_h, u_h = W.autograd((8192, 4096), seed=R.shard_seed(W.SEED, rank))
    x = torch.from_numpy(x_h).to(dev).requires_grad_(True)
    w, v, u = (torch.from_numpy(a).to(dev) for a in (w_h, v_h, u_h))
    n = x.numel()

    def fwd_bwd():
        x.grad = None
        loss = (w * Fn.sin(x) + v * Fn.cos(x) + u * torch.clamp(Fn.tan(x), -50, 50)).sum()
        loss.backward()

    def fused():
        x.grad = None
        Fn.sincostan_loss(x, w, v, u, -50.0, 50.0).backward()

    # algorithmic bytes of the unfused step: forward reads x three times and
    # writes three outputs; backward reads x and the incoming gradient and
    # writes a gradient for each function (the torch elementwise ops between
    # them are not counted)
    ks = [Kernel("loss_fwd_bwd", 4 * n * 15, n, fwd_bwd, launches=6)]
    meta = {"metric": "Gelem/s, forward + backward of sum(w sin + v cos + u clamp(tan, -50, 50)) over [8192, 4096] "
                      "fp32 (autograd.Function, hand-written derivative kernels)",
            "dtype": "f32", "workload": "differentiation: x U[-4pi, 4pi], w, v, u ~ N(0,1), [8192, 4096]",
            "n_per_gpu": n, "l2": "inputs larger than L2, no flush"}
    loss_buf = torch.empty((), dtype=torch.float64, device=dev)
    gx_buf = torch.empty_like(x)

    def fused_kernel():
        B.ptrig_sincostan_loss_f32(x.detach(), w, v, u, -50.0, 50.0, loss_buf, gx_buf, n,
                                   torch.cuda.current_stream().cuda_stream)

    gy = torch.randn(x.shape, device=dev)

    def bwd_kernel(f):
        return lambda: getattr(B, f"ptrig_{f}_bwd_f32")(x.detach(), gy, gx_buf, n,
                                                        torch.cuda.current_stream().cuda_stream)

    return ks, meta, {"fused": fused, "fused_kernel": fused_kernel, "n": n,
                      "bwd": {f: bwd_kernel(f) for f in ("sin", "cos", "tan")}}


def workload_fp64(B, W, torch, dev, rank, log2n):
    """The FP64 data path (Sec. 4 evaluates in double) and the paper-faithful
    FP64 kernels on 2^26 doubles of the bandwidth workload; FP64-issue-bound."""
    import numpy as np
    n = 1 << min(log2n, 26)
    x = torch.from_numpy(W.bandwidth(n, seed=R.shard_seed(W.SEED, rank)).astype(np.float64)).to(dev)
    y = torch.empty_like(x)
    s = torch.cuda.current_stream().cuda_stream
    ks = [Kernel(f"{f}_f64", 16 * n, n, (lambda f=f: getattr(B, f"ptrig_{f}_f64")(x, y, n, s)))
          for f in ("sin", "cos", "tan")]
    ks += [Kernel(f"faithful_{f}_f64", 16 * n, n, (lambda fi=fi: B.ptrig_faithful_f64(fi, x, y, n, s)))
           for fi, f in enumerate(("sin", "cos", "tan"))]
    meta = {"metric": f"Gelem/s, pi/12 sin/cos/tan in FP64 (proposed and paper-faithful) on 2^{n.bit_length() - 1} "
                      "doubles", "dtype": "f64",
            "workload": f"fp64: 2^{n.bit_length() - 1} doubles of the bandwidth mixture; step = FP64 sin, cos, tan and "
                        "the paper-faithful FP64 sin, cos, tan (one launch each)", "n_per_gpu": n,
            "l2": "inputs larger than L2 (512 MiB vs 129 MB), no flush"}
    return ks, meta, {"n": n}


def fp64_peak(B, torch, dev, stream):
    """FP64 FMA throughput of the probe kernel (GFLOP/s, CUDA events)."""
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    sink = torch.empty(sms * 8 * 256, dtype=torch.float64, device=dev)
    iters = 2048
    ms = _time_call(lambda: B.ptrig_fp64_fma_probe(sink, iters, sink.numel(), stream.cuda_stream), 5, stream)
    return sink.numel() * iters * 16 / ms / 1e6, f"ptrig_fp64_fma_probe: {sink.numel()} threads x {iters} x 8 FMA " \
                                                 "chains, CUDA events"


def fp64_flops():
    """FP64 FLOPs per angle of each FP64 kernel (profiles/fp64_ops.json)."""
    p = os.path.join(ROOT, "profiles", "fp64_ops.json")
    return json.load(open(p)).get("kernels", {}) if os.path.exists(p) else {}


WORKLOADS = {"bandwidth": workload_bandwidth, "half": workload_half, "large": workload_large,
             "batch": workload_batch, "autograd": workload_autograd, "fp64": workload_fp64}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ptrig", choices=["ptrig", "reference"])
    ap.add_argument("--workload", default="bandwidth", choices=sorted(WORKLOADS))
    ap.add_argument("--log2n", type=int, default=28)
    ap.add_argument("--batch-arrays", type=int, default=4096,
                    help="arrays in the batch workload (4096 is the configured batch; fewer for profiling)")
    ap.add_argument("--batch-config", default=None,
                    help="BLOCK,ITEMS: fixed batch tile shape instead of the autotuner (for profiling)")
    ap.add_argument("--no-extras", action="store_true", help="skip half/cuda-math/e2e/cpu legs")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3

    rank, world, local = R.rank_env()
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch

    from paper_2502_10831_gb300 import binding as B
    from paper_2502_10831_gb300 import build as Bld
    from paper_2502_10831_gb300 import workloads as W

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if local == 0:  # one build per node; the other ranks load what it wrote
        Bld.build()
    if dist:
        dist.barrier()
    B.lib()
    dev = torch.device("cuda", local)
    wl_kw = {}
    if args.workload == "batch":
        wl_kw["arrays"] = args.batch_arrays
        if args.batch_config:
            wl_kw["config"] = tuple(int(v) for v in args.batch_config.split(","))
    kernels_list, meta, state = WORKLOADS[args.workload](B, W, torch, dev, rank, args.log2n, **wl_kw)
    stream = torch.cuda.current_stream()

    def step():
        for k in kernels_list:
            k.call()

    # the clock sampler starts first; the warm-up steps then run right before
    # the timed region, so that its first kernel does not start on a GPU that
    # sat idle while the sampler came up
    nk = len(kernels_list)
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(nk + 1)] for _ in range(args.steps)]
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    # timed region: K steps, events around every kernel on the launching stream
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    if hasattr(torch.cuda, "_sleep"):
        # a short device-side spin ahead of the start event, so that the host
        # has queued the first launches by the time the GPU reaches it (the
        # first kernel's launch latency then stays out of the device time)
        torch.cuda._sleep(200_000)
    wall0 = time.perf_counter()
    t0.record(stream)
    for s in range(args.steps):
        ev[s][0].record(stream)
        for k, kern in enumerate(kernels_list):
            kern.call()
            ev[s][k + 1].record(stream)
    t1.record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    if dist:
        dist.barrier()
    clk = clocks.window(wall0, wall0 + wall)
    total_ms = R.max_over_ranks(t0.elapsed_time(t1), dist, dev)
    per_kernel_ms = [statistics.mean(ev[s][k].elapsed_time(ev[s][k + 1]) for s in range(args.steps))
                     for k in range(nk)]
    per_kernel_med = [statistics.median(ev[s][k].elapsed_time(ev[s][k + 1]) for s in range(args.steps))
                      for k in range(nk)]
    ms_per_step = total_ms / args.steps
    value = R.job_throughput(sum(k.elems for k in kernels_list), world, ms_per_step * 1e-3) / 1e9
    peak, peak_kind = _peaks()
    kernels = {}
    for kern, ms, med in zip(kernels_list, per_kernel_ms, per_kernel_med):
        gbs = kern.nbytes / (ms * 1e-3) / 1e9
        kernels[kern.name] = {"ms": round(ms, 4), "gelem_s": round(kern.elems / (ms * 1e-3) / 1e9, 2),
                              "gb_s": round(gbs, 1), "hbm_frac": round(gbs / peak, 4),
                              "hbm_frac_nominal": round(gbs / NOMINAL_HBM_GBS, 4),
                              "ms_median": round(med, 4),
                              "gelem_s_median": round(kern.elems / (med * 1e-3) / 1e9, 2)}
    dom_i = max(range(nk), key=lambda k: per_kernel_ms[k])
    dom = kernels_list[dom_i]
    achieved = dom.nbytes / (per_kernel_ms[dom_i] * 1e-3) / 1e9
    traffic, traffic_src = lookup_traffic(dom.name, meta["n_per_gpu"], args.workload)
    roofline = {"bound": "hbm", "kernel": dom.name, "achieved": round(achieved, 1), "peak": peak,
                "peak_kind": "measured (MEASURED_PEAKS.json hbm_gbs, copy)" if peak_kind == "measured" else peak_kind,
                "unit": "GB/s", "frac": round(achieved / peak, 4),
                "frac_of_nominal": round(achieved / NOMINAL_HBM_GBS, 4), "nominal_gbs": NOMINAL_HBM_GBS,
                "algorithmic_bytes_per_launch": dom.nbytes, "traffic": traffic, "traffic_source": traffic_src}
    if args.workload == "fp64":  # FP64-issue-bound: the roofline is the FP64 FMA rate
        pk, how = fp64_peak(B, torch, dev, stream)
        fl = fp64_flops().get(dom.name, {}).get("flops_per_element")
        ach = fl * dom.elems / (per_kernel_ms[dom_i] * 1e-3) / 1e9 if fl else None
        roofline = {"bound": "fp64", "kernel": dom.name, "achieved": round(ach, 1) if ach else None,
                    "peak": round(pk, 1), "peak_kind": "measured (" + how + ")", "unit": "GFLOP/s",
                    "frac": round(ach / pk, 4) if ach else None, "flops_per_element": fl,
                    "flops_source": "profiles/fp64_ops.json", "traffic": None}
    config = {"workload": meta["workload"], "n_per_gpu": meta["n_per_gpu"], "l2": meta["l2"],
              "launch_configs": {name: B.ptrig_get_launch_config(fam) for name, fam in (
                  ("f32", B.FAMILY_F32), ("f32_sincos", B.FAMILY_F32_SINCOS), ("taylor", B.FAMILY_TAYLOR),
                  ("half", B.FAMILY_HALF), ("half_sincos", B.FAMILY_HALF_SINCOS), ("bf16", B.FAMILY_BF16),
                  ("bf16_sincos", B.FAMILY_BF16_SINCOS), ("half_tan", B.FAMILY_HALF_TAN),
                  ("bf16_tan", B.FAMILY_BF16_TAN), ("bwd", B.FAMILY_BWD))},
              "launch_config_fields": "threads per block, 16-byte loads in flight per thread (0: four below 2^27 "
                                      "elements, two from there), persistent blocks per SM (0: one-shot)"}
    if "autotuned" in meta:
        config["batch_autotuned"] = meta["autotuned"]
    line = {"metric": meta["metric"], "value": round(value, 2), "unit": "Gelem/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": meta["dtype"],
            "data": "synthetic", "config": config, "roofline": roofline, "kernels": kernels,
            "gpu_launches": sum(k.launches for k in kernels_list) * args.steps, "clocks": clk,
            "wall_s_timed": round(wall, 3)}
    if args.workload != "bandwidth":
        line["workload"] = args.workload
    if args.workload == "batch" and rank == 0:
        plan = state["plan"]
        ms = _time_call(lambda: plan.run_per_array(stream.cuda_stream), 3, stream)
        line["per_array_launches"] = {"ms": round(ms, 3), "gelem_s": round(meta["n_per_gpu"] / ms / 1e6, 2),
                                      "launches": len(state["descs"])}
    if args.workload == "autograd" and rank == 0:
        nn = state["n"]
        ms = _time_call(state["fused"], 5, stream)
        kms = _time_call(state["fused_kernel"], 20, stream)
        line["fused_loss"] = {"ms": round(ms, 3), "gelem_s": round(nn / ms / 1e6, 2),
                              "speedup_vs_unfused": round(ms_per_step / ms, 2),
                              "kernel_ms": round(kms, 4), "kernel_gelem_s": round(nn / kms / 1e6, 2),
                              "kernel_gb_s": round(20 * nn / kms / 1e6, 1),
                              "kernel_hbm_frac": round(20 * nn / kms / 1e6 / peak, 4),
                              "how": "autograd step: one kernel computes the loss and dL/dx (sin, cos, tan and "
                                     "their derivatives from one reduction; reads x, w, v, u, writes dL/dx, "
                                     "20 B/angle), then backward scales dL/dx by the incoming gradient (a torch "
                                     "multiply, 8 B/angle); kernel_* times the library call alone"}
        bk = {}
        for f, call in state["bwd"].items():
            bms = _time_call(call, 20, stream)
            bk[f"{f}_bwd_f32"] = {"ms": round(bms, 4), "gelem_s": round(nn / bms / 1e6, 2),
                                  "hbm_frac": round(12 * nn / bms / 1e6 / peak, 4)}
        line["backward_kernels"] = bk
    if args.workload == "large" and rank == 0:
        line["side_paths"] = side_paths(B, torch, dev, stream, peak)
    if args.workload == "bandwidth" and not args.no_extras and rank == 0:
        line.update(extras(args, B, W, state, stream, peak, kernels, clocks, rank))
    clocks.stop()
    if rank == 0:
        print(json.dumps(line))
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def lookup_traffic(kernel, n, workload):
    """ncu DRAM bytes (read + write) of one launch of `kernel` on `n` angles of
    `workload`, from profiles/traffic.json; (None, None) when no capture of
    exactly that launch exists."""
    tpath = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(tpath):
        return None, None
    for e in json.load(open(tpath)).get("captures", []):
        if e.get("kernel") == kernel and e.get("n") == n and e.get("workload") == workload:
            return e.get("bytes_per_launch"), e.get("source")
    return None, None


def side_paths(B, torch, dev, stream, peak):
    """sin_f32 throughput of the Payne-Hanek side path on 2^26 angles in each
    of two ranges: |x| log-uniform in [2^19, 2^31) and in [2^31, 2^127]."""
    import numpy as np
    n = 1 << 26
    out = {}
    for name, lo, hi in (("ph_2p19_2p31", 19.0, 31.0), ("ph_2p31_2p127", 31.0, 127.0)):
        r = np.random.default_rng(7)
        xh = (2.0 ** r.uniform(lo, hi, n) * r.choice([-1.0, 1.0], n)).astype(np.float32)
        xh = np.clip(xh, -np.float32(2.0 ** hi), np.float32(2.0 ** hi))
        x = torch.from_numpy(xh).to(dev)
        y = torch.empty_like(x)
        ms = _time_call(lambda: B.ptrig_sin_f32(x, y, n, stream.cuda_stream), 5, stream)
        out[name] = {"range": f"|x| log-uniform in [2^{lo:g}, 2^{hi:g})", "ms": round(ms, 3),
                     "gelem_s": round(n / ms / 1e6, 2), "hbm_frac": round(8 * n / ms / 1e6 / peak, 4)}
        del x, y
    return out


def _time_call(fn, reps, stream):
    import torch
    for _ in range(2):
        fn()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def _timed(fn, stream, clocks, min_s=0.3, max_reps=4000, flush=None):
    """Average CUDA-event time of fn on `stream` after 3 warm-up calls, over
    enough calls to fill about min_s seconds (so that the clock sampler sees
    the window), and the clock summary of that window.  With `flush`, an L2
    flush runs before every call, outside the timed events."""
    import torch
    for _ in range(3):
        fn()
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    fn()
    b.record(stream)
    torch.cuda.synchronize()
    est = max(a.elapsed_time(b), 1e-3)
    reps = int(min(max_reps, max(3, min_s * 1e3 / est)))
    w0 = time.perf_counter()
    if flush is None:
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / reps
    else:
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        for e0, e1 in evs:
            flush()
            e0.record(stream)
            fn()
            e1.record(stream)
        torch.cuda.synchronize()
        ms = sum(e0.elapsed_time(e1) for e0, e1 in evs) / reps
    w1 = time.perf_counter()
    return ms, reps, clocks.window(w0, w1)


def leg_large(B, W, torch, dev, stream, peak, clocks):
    """The precision configuration's large-argument set: 2^24 FP32 angles,
    |x| log-uniform in [1, 1e5] (64 MiB, under L2: the L2 is flushed before
    every timed call), the four functions; plus sin on 2^24 angles of each
    reduction side path."""
    import numpy as np
    n = 1 << 24
    sp = stream.cuda_stream
    x = torch.from_numpy(W.large(n)).to(dev)
    y0, y1 = torch.empty_like(x), torch.empty_like(x)
    scratch = torch.empty(64 << 20, dtype=torch.float32, device=dev)  # 256 MiB > L2
    clean = torch.ones(64 << 20, dtype=torch.float32, device=dev)
    acc = torch.empty((), dtype=torch.float32, device=dev)

    def flush():
        # write 256 MiB, then read another 256 MiB: the inputs leave L2, and the
        # lines it holds afterwards are clean, so the timed call does not pay
        # for writing back the flush's own dirty lines
        scratch.fill_(1.0)
        torch.sum(clean, dim=0, out=acc)

    out = {"n": n, "workload": "2^24 fp32 angles, |x| log-uniform in [1, 1e5], random sign (FP32 reduction)",
           "l2": "64 MiB arrays; before every timed call the L2 is flushed by a 256 MiB write followed by a "
                 "256 MiB read (no dirty flush lines left for the timed call to write back)"}
    for f, nb in (("sin", 8), ("cos", 8), ("tan", 8), ("sincos", 12)):
        if f == "sincos":
            fn = (lambda: B.ptrig_sincos_f32(x, y0, y1, n, sp))
        else:
            fn = (lambda f=f: getattr(B, f"ptrig_{f}_f32")(x, y0, n, sp))
        ms, reps, clk = _timed(fn, stream, clocks, flush=flush)
        out[f"{f}_f32"] = {"ms": round(ms, 4), "gelem_s": round(n / ms / 1e6, 2),
                           "hbm_frac": round(nb * n / ms / 1e6 / peak, 4), "reps": reps, "clocks": clk}
    # the same distribution at 4x the size (256 MiB arrays, above L2, no flush):
    # the 2^24 launches are short enough for their start-up to show
    n4 = 1 << 26
    x4 = torch.from_numpy(W.large(n4)).to(dev)
    z0, z1 = torch.empty_like(x4), torch.empty_like(x4)
    big = {"n": n4}
    for f, nb in (("sin", 8), ("cos", 8), ("tan", 8), ("sincos", 12)):
        if f == "sincos":
            fn = (lambda: B.ptrig_sincos_f32(x4, z0, z1, n4, sp))
        else:
            fn = (lambda f=f: getattr(B, f"ptrig_{f}_f32")(x4, z0, n4, sp))
        ms, reps, clk = _timed(fn, stream, clocks)
        big[f"{f}_f32"] = {"ms": round(ms, 4), "gelem_s": round(n4 / ms / 1e6, 2),
                           "hbm_frac": round(nb * n4 / ms / 1e6 / peak, 4), "clocks": clk}
    out["at_2p26"] = big
    del x4, z0, z1
    side = {}
    for name, lo, hi in (("ph_2p19_2p31", 19.0, 31.0), ("ph_2p31_2p127", 31.0, 127.0)):
        r = np.random.default_rng(7)
        xh = (2.0 ** r.uniform(lo, hi, n) * r.choice([-1.0, 1.0], n)).astype(np.float32)
        x.copy_(torch.from_numpy(xh))
        ms, reps, clk = _timed(lambda: B.ptrig_sin_f32(x, y0, n, sp), stream, clocks, flush=flush)
        side[name] = {"range": f"|x| log-uniform in [2^{lo:g}, 2^{hi:g})", "ms": round(ms, 3),
                      "gelem_s": round(n / ms / 1e6, 2), "clocks": clk}
    out["side_paths_sin_f32"] = side
    del x, y0, y1, scratch, clean
    torch.cuda.empty_cache()
    return out


def leg_batch(B, W, torch, dev, stream, peak, clocks, rank):
    """The batching configuration: 4096 ragged FP32 arrays with per-array
    selectors, one graph-captured launch (autotuned tile shape) against one
    launch per array."""
    ks, meta, st = workload_batch(B, W, torch, dev, rank, 0)
    k = ks[0]
    ms, reps, clk = _timed(k.call, stream, clocks)
    plan = st["plan"]
    pms, preps, pclk = _timed(lambda: plan.run_per_array(stream.cuda_stream), stream, clocks, min_s=0.3)
    total = meta["n_per_gpu"]
    out = {"arrays": len(st["descs"]), "elements": total, "workload": meta["workload"],
           "autotuned": meta["autotuned"],
           "graph": {"ms": round(ms, 4), "gelem_s": round(total / ms / 1e6, 2),
                     "hbm_frac": round(k.nbytes / ms / 1e6 / peak, 4), "bytes": k.nbytes, "reps": reps,
                     "clocks": clk},
           "per_array_launches": {"ms": round(pms, 3), "gelem_s": round(total / pms / 1e6, 2),
                                  "launches": len(st["descs"]), "reps": preps, "clocks": pclk},
           "speedup_vs_per_array": round(pms / ms, 2)}
    plan.close()
    del ks, st
    torch.cuda.empty_cache()
    return out


def leg_autograd(B, W, torch, dev, stream, peak, clocks, rank):
    """The differentiation configuration at [8192, 4096]: the unfused autograd
    step (sin, cos, tan forward and backward kernels with torch's elementwise
    ops between them), the fused loss+gradient kernel through autograd and
    alone, and each derivative kernel."""
    ks, meta, st = workload_autograd(B, W, torch, dev, rank, 0)
    nn = st["n"]
    ums, ureps, uclk = _timed(ks[0].call, stream, clocks)
    fms, freps, fclk = _timed(st["fused"], stream, clocks)
    kms, kreps, kclk = _timed(st["fused_kernel"], stream, clocks)
    out = {"shape": [8192, 4096], "workload": meta["workload"],
           "unfused_step": {"ms": round(ums, 3), "gelem_s": round(nn / ums / 1e6, 2), "clocks": uclk,
                            "how": "forward sin, cos, tan + backward through autograd.Function (6 ptrig kernels "
                                   "and torch's elementwise ops)"},
           "fused_step": {"ms": round(fms, 3), "gelem_s": round(nn / fms / 1e6, 2),
                          "speedup_vs_unfused": round(ums / fms, 2), "clocks": fclk},
           "fused_kernel": {"ms": round(kms, 4), "gelem_s": round(nn / kms / 1e6, 2),
                            "gb_s": round(20 * nn / kms / 1e6, 1), "hbm_frac": round(20 * nn / kms / 1e6 / peak, 4),
                            "bytes_per_angle": 20, "clocks": kclk}}
    bk = {}
    for f, call in st["bwd"].items():
        bms, _, bclk = _timed(call, stream, clocks)
        bk[f"{f}_bwd_f32"] = {"ms": round(bms, 4), "gelem_s": round(nn / bms / 1e6, 2),
                              "hbm_frac": round(12 * nn / bms / 1e6 / peak, 4), "clocks": bclk}
    out["backward_kernels"] = bk
    del ks, st
    torch.cuda.empty_cache()
    return out


def extras(args, B, W, state, stream, peak, kernels, clocks, rank):
    import numpy as np
    import torch

    x, x_host, n = state["x"], state["x_host"], state["n"]
    out = {}
    s_ptr = stream.cuda_stream
    y0 = torch.empty_like(x)
    y1 = torch.empty_like(x)
    # CUDA's own math library on the same array
    cm = {}
    for fast in (0, 1):
        for fi, f in enumerate(("sin", "cos", "tan")):
            ms = _time_call(lambda: B.ptrig_cudamath_f32(fi, fast, x, y0, None, n, s_ptr), 5, stream)
            cm[("__" if fast else "") + f + "f"] = {"ms": round(ms, 4), "gelem_s": round(n / ms / 1e6, 2)}
    out["cuda_math"] = cm
    tm = {}
    for f in ("sin", "cos", "tan"):  # PyTorch's own elementwise kernels, for context
        fn = getattr(torch, f)
        ms = _time_call(lambda: fn(x, out=y0), 5, stream)
        tm[f"torch.{f}"] = {"ms": round(ms, 4), "gelem_s": round(n / ms / 1e6, 2)}
    out["torch_math"] = tm
    del y0, y1
    # packed half storage against the plain FP32 kernels
    half = {}
    xh16 = torch.from_numpy(W.half16(n).view(np.int16)).to(x.device)
    xbf = torch.from_numpy(W.half_bf16(n).view(np.int16)).to(x.device)
    h0 = torch.empty_like(xh16)
    h1 = torch.empty_like(xh16)
    for dt, xt in (("f16", xh16), ("bf16", xbf)):
        for f in ("sin", "cos", "tan"):
            ms, reps, clk = _timed(lambda: getattr(B, f"ptrig_{f}_{dt}")(xt, h0, n, s_ptr), stream, clocks, min_s=0.1)
            plain = kernels[f"{f}_f32"]["gelem_s"]
            g = n / ms / 1e6
            half[f"{f}_{dt}"] = {"ms": round(ms, 4), "gelem_s": round(g, 2), "hbm_frac": round(4 * n / ms / 1e6 / peak, 4),
                                 "vs_plain_f32": round(g / plain, 3), "clocks": clk}
        ms, reps, clk = _timed(lambda: getattr(B, f"ptrig_sincos_{dt}")(xt, h0, h1, n, s_ptr), stream, clocks, min_s=0.1)
        g = n / ms / 1e6
        half[f"sincos_{dt}"] = {"ms": round(ms, 4), "gelem_s": round(g, 2), "hbm_frac": round(6 * n / ms / 1e6 / peak, 4),
                                "vs_plain_f32": round(g / kernels["sincos_f32"]["gelem_s"], 3), "clocks": clk}
    out["packed_half"] = half
    del xh16, xbf, h0, h1
    torch.cuda.empty_cache()
    # FP64 data path (Sec. 4 evaluates in double) and the paper-faithful FP64
    # kernels, on 2^26 doubles of the same workload: FP64-issue-bound on GB300
    m = min(n, 1 << 26)
    xd = x[:m].double()
    yd = torch.empty_like(xd)
    f64 = {}
    for f in ("sin", "cos", "tan"):
        ms = _time_call(lambda: getattr(B, f"ptrig_{f}_f64")(xd, yd, m, s_ptr), 5, stream)
        f64[f"{f}_f64"] = {"ms": round(ms, 4), "gelem_s": round(m / ms / 1e6, 2)}
    for fi, f in enumerate(("sin", "cos", "tan")):
        ms = _time_call(lambda: B.ptrig_faithful_f64(fi, xd, yd, m, s_ptr), 5, stream)
        f64[f"faithful_{f}_f64"] = {"ms": round(ms, 4), "gelem_s": round(m / ms / 1e6, 2)}
    # the FP64 roofline: FMA throughput of the probe kernel (events), and each
    # kernel's FP64 FLOPs per angle (2 DFMA + DMUL + DADD, counted by ncu)
    peak64, how = fp64_peak(B, torch, x.device, stream)
    ops = fp64_flops()
    for k, v in f64.items():
        fl = ops.get(k, {}).get("flops_per_element")
        if fl:
            v["fp64_gflops"] = round(fl * v["gelem_s"], 1)
            v["fp64_frac"] = round(fl * v["gelem_s"] / peak64, 4)
            v["flops_per_element"] = fl
            # DMUL and DADD take an issue slot as a DFMA does but count one
            # FLOP: the share of the FP64 pipe's instruction rate in use
            ins = sum(ops[k].get(o, 0.0) for o in ("dfma", "dmul", "dadd"))
            v["fp64_inst_per_element"] = ins
            v["fp64_pipe_frac"] = round(ins * v["gelem_s"] / (peak64 / 2), 4)
    out["fp64"] = {"n": m, "kernels": f64, "bound": "FP64 issue (GB300 runs FP64 at a small fraction of FP32)",
                   "peak_gflops": round(peak64, 1), "peak_how": how,
                   "flops_source": "profiles/fp64_ops.json (ncu DFMA, DMUL, DADD thread instructions per angle)"}
    del xd, yd
    torch.cuda.empty_cache()
    # the other configurations, each with its own event timing and clock window
    out["large_arguments"] = leg_large(B, W, torch, x.device, stream, peak, clocks)
    out["batch"] = leg_batch(B, W, torch, x.device, stream, peak, clocks, rank)
    out["autograd"] = leg_autograd(B, W, torch, x.device, stream, peak, clocks, rank)
    out["e2e"] = e2e(B, x_host, n, x.device, stream, clocks)
    out["cpu_baseline"] = oracle_rate(x_host)
    out["cpu_simd"] = cpu_simd_rate(x_host)
    return out


def _gpu_numa_cpus(device):
    """(NUMA node, CPU list) of the GPU from sysfs, or (None, None)."""
    import torch
    try:
        p = torch.cuda.get_device_properties(device)
        bus = f"{p.pci_domain_id:04x}:{p.pci_bus_id:02x}:{p.pci_device_id:02x}.0"
        node = int(open(f"/sys/bus/pci/devices/{bus}/numa_node").read())
        if node < 0:
            return None, None
        cpus = open(f"/sys/devices/system/node/node{node}/cpulist").read().strip()
        return node, cpus
    except (AttributeError, OSError, ValueError):
        return None, None


def _parse_cpulist(text):
    cpus = set()
    for part in text.split(","):
        if "-" in part:
            a, b = part.split("-")
            cpus.update(range(int(a), int(b) + 1))
        elif part:
            cpus.add(int(part))
    return cpus


def e2e(B, x_host, n, device, stream, clocks):
    """The step through the C ABI with the data in pinned HOST memory, timed
    end to end (host clock around synchronized runs of steps).  Every output
    array of a step -- eight per step -- lands in its own pinned host buffer,
    so every result is delivered.  The pinned buffers are allocated (and
    first touched) from the CPUs of the GPU's NUMA node when sysfs names one.
    Two ways are measured, three runs of 5 steps each, and the faster
    median is reported:
      copy:      each step uploads its angles, runs the seven kernels into
                 device buffers and downloads the eight output arrays; the
                 downloads run on their own stream behind each kernel, and the
                 next step's upload goes into a second input buffer on a third
                 stream while this step's results travel back;
      zero-copy: upload of the angles, then the seven kernels writing their
                 outputs straight into pinned host memory over NVLink-C2C (the
                 ABI takes any pointer the device can dereference)."""
    import torch

    node, cpulist = _gpu_numa_cpus(device)
    old_aff = None
    if cpulist:
        try:
            old_aff = os.sched_getaffinity(0)
            os.sched_setaffinity(0, _parse_cpulist(cpulist))
        except OSError:
            old_aff = None
    hx = torch.from_numpy(x_host).pin_memory()
    hy = [torch.empty(n, dtype=torch.float32).pin_memory() for _ in range(8)]
    for h in hy:
        h.fill_(0)  # first touch on this node
    if old_aff is not None:
        os.sched_setaffinity(0, old_aff)
    dxs = [torch.empty(n, dtype=torch.float32, device=device) for _ in range(2)]
    dx = dxs[0]
    s_ptr = stream.cuda_stream
    seq = [("sin_f32", 1), ("cos_f32", 1), ("tan_f32", 1), ("sincos_f32", 2), ("taylor_sin_f32", 1),
           ("taylor_cos_f32", 1), ("taylor_tan_f32", 1)]

    def launch(name, src, o):
        fn = getattr(B, f"ptrig_{name}")
        if name == "sincos_f32":
            fn(src, o[0], o[1], n, s_ptr)
        else:
            fn(src, o[0], n, s_ptr)

    douts = [torch.empty(n, dtype=torch.float32, device=device) for _ in range(3)]
    copy_stream = torch.cuda.Stream(device=device)
    h2d_stream = torch.cuda.Stream(device=device)
    slot = [0]
    copy_done = [None, None, None]

    def upload(buf, after):
        if after is not None:  # the kernels that read this buffer last have finished
            h2d_stream.wait_event(after)
        with torch.cuda.stream(h2d_stream):
            dxs[buf].copy_(hx, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(h2d_stream)
        return ev

    def run_copy(steps):
        kern_done = [None, None]
        ready = upload(0, None)
        for st in range(steps):
            b = st % 2
            stream.wait_event(ready)
            k = 0  # output array index within the step: 0..7
            for name, nout in seq:
                bufs = [(slot[0] + i) % 3 for i in range(nout)]
                for ob in bufs:  # an output buffer is reused only after its download finished
                    if copy_done[ob] is not None:
                        stream.wait_event(copy_done[ob])
                launch(name, dxs[b], [douts[ob] for ob in bufs])
                done = torch.cuda.Event()
                done.record(stream)
                copy_stream.wait_event(done)
                with torch.cuda.stream(copy_stream):
                    for ob in bufs:
                        hy[k].copy_(douts[ob], non_blocking=True)
                        k += 1
                        ce = torch.cuda.Event()
                        ce.record(copy_stream)
                        copy_done[ob] = ce
                slot[0] = (slot[0] + nout) % 3
            kern_done[b] = torch.cuda.Event()
            kern_done[b].record(stream)
            if st + 1 < steps:  # next step's input, into the buffer this step does not read
                ready = upload(1 - b, kern_done[1 - b])
        stream.wait_stream(copy_stream)

    def run_zero_copy(steps):
        for _ in range(steps):
            dx.copy_(hx, non_blocking=True)
            k = 0
            for name, nout in seq:
                launch(name, dx, hy[k:k + nout])
                k += nout

    res, runs = {}, {}
    w0 = time.perf_counter()
    for mode, run in (("copy", run_copy), ("zero-copy", run_zero_copy)):
        run(2)
        torch.cuda.synchronize()
        ts = []
        for _ in range(3):
            t0 = time.perf_counter()
            run(5)
            torch.cuda.synchronize()
            ts.append((time.perf_counter() - t0) / 5)
        runs[mode] = [round(t * 1e3, 3) for t in ts]
        res[mode] = statistics.median(ts)
    w1 = time.perf_counter()

    # the host link alone: pinned copies of the angle array each way, the
    # best of five single copies (a copy that another user of the host link
    # slows down would otherwise make the bound look longer than the step)
    def link(fn):
        fn()
        torch.cuda.synchronize()
        best = 0.0
        for _ in range(5):
            t0 = time.perf_counter()
            fn()
            torch.cuda.synchronize()
            best = max(best, 4 * n / (time.perf_counter() - t0) / 1e9)
        return best

    h2d = link(lambda: dx.copy_(hx, non_blocking=True))
    d2h = link(lambda: hy[0].copy_(douts[0], non_blocking=True))
    del douts
    best = min(res, key=res.get)
    dt = res[best]
    bound_s = 8 * 4 * n / (d2h * 1e9)  # the step's device-to-host bytes at the link's copy rate
    return {"value": round(7 * n / dt / 1e9, 2), "unit": "Gelem/s", "h2d_bytes_per_step": 4 * n,
            "d2h_bytes_per_step": 8 * 4 * n, "ms_per_step": round(dt * 1e3, 3), "mode": best,
            "ms_per_step_by_mode": {k: round(v * 1e3, 3) for k, v in res.items()}, "runs_ms": runs,
            "link_gbs": {"h2d": round(h2d, 1), "d2h": round(d2h, 1)},
            "link_bound_ms": round(bound_s * 1e3, 3), "link_frac": round(bound_s / dt, 4),
            "host_numa_node": node, "host_cpus": cpulist, "clocks": clocks.window(w0, w1),
            "how": "pinned host angles -> device, the 7 kernels of the step, each of the 8 output arrays into its "
                   "own pinned host buffer; per mode the median of 3 runs of 5 steps, timed with the host clock "
                   "around each synchronized run, every step's upload and downloads inside it.  link_frac = the "
                   "step's device-to-host bytes at the pinned-copy rate (best of five single 1 GiB copies) / the "
                   "step time"}


if __name__ == "__main__":
    sys.exit(main())
