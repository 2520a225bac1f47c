"""ctypes binding of libptrig's C ABI (include/ptrig.h), same names as the C
entry points.  Argument marshalling only: every computation runs in the CUDA
library.  Arguments may be torch tensors (their data pointer and element count
are used) or raw integer addresses; `stream` defaults to torch's current CUDA
stream.  A nonzero status raises PtrigError.

The library must have been built (python -m paper_2502_10831_gb300.build);
loading fails loudly otherwise -- there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os
import threading

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_build", "libptrig.so")

SIN, COS, TAN, SINCOS = 0, 1, 2, 3
FAMILY_F32, FAMILY_HALF, FAMILY_TAYLOR, FAMILY_BWD, FAMILY_BF16, FAMILY_CUDAMATH = 0, 1, 2, 3, 4, 5
FAMILY_F32_SINCOS, FAMILY_HALF_SINCOS, FAMILY_BF16_SINCOS = 6, 7, 8
FAMILY_HALF_TAN, FAMILY_BF16_TAN = 9, 10
FAMILY_COUNT = 11
BATCH_GRAPH = 1

_P = ctypes.c_void_p
_SZ = ctypes.c_size_t
_I = ctypes.c_int

# name -> argument types (all return ptrig_status as int unless listed in _RESTYPE)
SIGNATURES = {
    "ptrig_status_string": [_I],
    "ptrig_last_cuda_error": [],
    "ptrig_version": [],
    "ptrig_sin_f32": [_P, _P, _SZ, _P],
    "ptrig_cos_f32": [_P, _P, _SZ, _P],
    "ptrig_tan_f32": [_P, _P, _SZ, _P],
    "ptrig_sincos_f32": [_P, _P, _P, _SZ, _P],
    "ptrig_sin_f16": [_P, _P, _SZ, _P],
    "ptrig_cos_f16": [_P, _P, _SZ, _P],
    "ptrig_tan_f16": [_P, _P, _SZ, _P],
    "ptrig_sincos_f16": [_P, _P, _P, _SZ, _P],
    "ptrig_sin_bf16": [_P, _P, _SZ, _P],
    "ptrig_cos_bf16": [_P, _P, _SZ, _P],
    "ptrig_tan_bf16": [_P, _P, _SZ, _P],
    "ptrig_sincos_bf16": [_P, _P, _P, _SZ, _P],
    "ptrig_sin_f64": [_P, _P, _SZ, _P],
    "ptrig_cos_f64": [_P, _P, _SZ, _P],
    "ptrig_tan_f64": [_P, _P, _SZ, _P],
    "ptrig_taylor_sin_f32": [_P, _P, _SZ, _P],
    "ptrig_taylor_cos_f32": [_P, _P, _SZ, _P],
    "ptrig_taylor_tan_f32": [_P, _P, _SZ, _P],
    "ptrig_taylor_n_f32": [_I, _I, _P, _P, _SZ, _P],
    "ptrig_sin_bwd_f32": [_P, _P, _P, _SZ, _P],
    "ptrig_cos_bwd_f32": [_P, _P, _P, _SZ, _P],
    "ptrig_tan_bwd_f32": [_P, _P, _P, _SZ, _P],
    "ptrig_sin_bwd_f64": [_P, _P, _P, _SZ, _P],
    "ptrig_cos_bwd_f64": [_P, _P, _P, _SZ, _P],
    "ptrig_tan_bwd_f64": [_P, _P, _P, _SZ, _P],
    "ptrig_sincostan_loss_f32": [_P, _P, _P, _P, _SZ, ctypes.c_float, ctypes.c_float, _P, _P, _P],
    "ptrig_faithful_f64": [_I, _P, _P, _SZ, _P],
    "ptrig_segment_f32": [_P, _P, _SZ, _P],
    "ptrig_cudamath_f32": [_I, _I, _P, _P, _P, _SZ, _P],
    "ptrig_fp64_fma_probe": [_P, _SZ, _I, _P],
    "ptrig_set_launch_config": [_I, _I, _I, _I],
    "ptrig_get_launch_config": [_I, _P, _P, _P],
    "ptrig_batch_plan_create": [_P, _P, _SZ, _I],
    "ptrig_batch_run": [_P, _P],
    "ptrig_batch_run_per_array": [_P, _P],
    "ptrig_batch_plan_set_config": [_P, _I, _I],
    "ptrig_batch_plan_get_config": [_P, _P, _P, _P, _P],
    "ptrig_batch_plan_autotune": [_P, _P, _I, _P, _P, _I, _P, _P, _P],
    "ptrig_batch_plan_destroy": [_P],
    "ptrig_batch_run_noalloc": [_P, _SZ, _P],
}
_RESTYPE = {"ptrig_status_string": ctypes.c_char_p, "ptrig_batch_plan_destroy": None}


class PtrigError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        lib = _load()
        msg = lib.ptrig_status_string(status).decode()
        if status == 2:
            msg += f" (cudaError {lib.ptrig_last_cuda_error()})"
        super().__init__(f"{where}: {msg}")


class ptrig_desc(ctypes.Structure):
    """Mirror of the C struct ptrig_desc (40 bytes)."""
    _fields_ = [("x", ctypes.c_void_p), ("y0", ctypes.c_void_p), ("y1", ctypes.c_void_p),
                ("n", ctypes.c_uint64), ("func", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]


_lib = None
_lock = threading.Lock()


def _load():
    global _lib
    if _lib is None:
        with _lock:
            if _lib is None:
                if not os.path.exists(LIB_PATH):
                    raise ImportError(
                        f"libptrig.so is not built ({LIB_PATH}); run "
                        "`python -m paper_2502_10831_gb300.build` (needs nvcc). "
                        "There is no CPU fallback.")
                L = ctypes.CDLL(LIB_PATH)
                for name, args in SIGNATURES.items():
                    f = getattr(L, name)
                    f.argtypes = args
                    f.restype = _RESTYPE.get(name, ctypes.c_int)
                _lib = L
    return _lib


def lib():
    """The loaded ctypes library (raises ImportError if it was not built)."""
    return _load()


def exported_symbols() -> list[str]:
    return list(SIGNATURES)


# --------------------------------------------------------------- marshalling

# bytes per element of each entry point's arrays, by name suffix
_ESIZE = {"f32": 4, "f16": 2, "bf16": 2, "f64": 8}


def _esize(name: str) -> int:
    return _ESIZE[name.rsplit("_", 1)[1]]


def _ptr(a) -> int | None:
    if a is None:
        return None
    if isinstance(a, int):
        return a
    return a.data_ptr()


def _count(a) -> int:
    return a.numel()


def _buffers(name: str, n: int, *bufs):
    """Checks the tensors among `bufs` -- (tensor or int or None, bytes per
    element) pairs -- before any launch: each must be a contiguous CUDA tensor
    (or pinned host tensor, which the device reaches directly) holding at
    least n elements of that width, the CUDA ones all on one device.  Raw
    integer addresses are the caller's responsibility.  Returns that device
    (None if no CUDA tensor was passed)."""
    dev = None
    for b, esize in bufs:
        if b is None or isinstance(b, int):
            continue
        if not b.is_cuda and not b.is_pinned():
            raise ValueError(f"{name}: arrays must be CUDA tensors or pinned host tensors")
        if not b.is_contiguous():
            raise ValueError(f"{name}: arrays must be contiguous")
        if b.element_size() != esize:
            raise ValueError(f"{name}: arrays hold {esize}-byte elements, got {b.dtype}")
        if b.numel() < n:
            raise ValueError(f"{name}: an array holds {b.numel()} elements, fewer than n = {n}")
        if not b.is_cuda:
            continue
        if dev is None:
            dev = b.device
        elif b.device != dev:
            raise ValueError(f"{name}: arrays on different devices ({dev}, {b.device})")
    return dev


class _on:
    """Makes `dev` torch's current device for the launch (no-op for None)."""

    def __init__(self, dev):
        self.dev = dev

    def __enter__(self):
        if self.dev is not None:
            import torch
            self.ctx = torch.cuda.device(self.dev)
            self.ctx.__enter__()

    def __exit__(self, *exc):
        if self.dev is not None:
            self.ctx.__exit__(*exc)


def _stream(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _check(status: int, where: str):
    if status != 0:
        raise PtrigError(status, where)


def _unary(name, out_esize=None):
    es = _esize(name)
    oes = es if out_esize is None else out_esize

    def f(x, y, n=None, stream=None):
        n = _count(x) if n is None else n
        with _on(_buffers(name, n, (x, es), (y, oes))):
            _check(getattr(_load(), name)(_ptr(x), _ptr(y), n, _stream(stream)), name)
    f.__name__ = name
    f.__doc__ = f"{name}(x, y, n=None, stream=None): see include/ptrig.h"
    return f


def _binary_out(name):
    es = _esize(name)

    def f(x, y0, y1, n=None, stream=None):
        n = _count(x) if n is None else n
        with _on(_buffers(name, n, (x, es), (y0, es), (y1, es))):
            _check(getattr(_load(), name)(_ptr(x), _ptr(y0), _ptr(y1), n, _stream(stream)), name)
    f.__name__ = name
    f.__doc__ = f"{name}(x, a, b, n=None, stream=None): see include/ptrig.h"
    return f


for _name, _args in SIGNATURES.items():
    if _args == [_P, _P, _SZ, _P]:
        globals()[_name] = _unary(_name, 1 if _name == "ptrig_segment_f32" else None)
    elif _args == [_P, _P, _P, _SZ, _P]:
        globals()[_name] = _binary_out(_name)


def ptrig_taylor_n_f32(func, nterms, x, y, n=None, stream=None):
    n = _count(x) if n is None else n
    with _on(_buffers("ptrig_taylor_n_f32", n, (x, 4), (y, 4))):
        _check(_load().ptrig_taylor_n_f32(func, nterms, _ptr(x), _ptr(y), n, _stream(stream)),
               "ptrig_taylor_n_f32")


def ptrig_faithful_f64(func, x, y, n=None, stream=None):
    """The paper's Algorithms 1-6 (FISR, 0.261 selector, pole guard) in FP64."""
    n = _count(x) if n is None else n
    with _on(_buffers("ptrig_faithful_f64", n, (x, 8), (y, 8))):
        _check(_load().ptrig_faithful_f64(func, _ptr(x), _ptr(y), n, _stream(stream)), "ptrig_faithful_f64")


def ptrig_cudamath_f32(func, fast, x, y0, y1=None, n=None, stream=None):
    n = _count(x) if n is None else n
    with _on(_buffers("ptrig_cudamath_f32", n, (x, 4), (y0, 4), (y1, 4))):
        _check(_load().ptrig_cudamath_f32(func, fast, _ptr(x), _ptr(y0), _ptr(y1), n, _stream(stream)),
               "ptrig_cudamath_f32")


def ptrig_sincostan_loss_f32(x, w, v, u, clamp_lo, clamp_hi, loss, gx, n=None, stream=None):
    """Fused loss sum(w sin + v cos + u clamp(tan)) into the device double
    `loss`, and its gradient into gx.  See include/ptrig.h."""
    n = _count(x) if n is None else n
    with _on(_buffers("ptrig_sincostan_loss_f32", n, (x, 4), (w, 4), (v, 4), (u, 4), (gx, 4))):
        _buffers("ptrig_sincostan_loss_f32", 1, (loss, 8))
        _check(_load().ptrig_sincostan_loss_f32(_ptr(x), _ptr(w), _ptr(v), _ptr(u), n, clamp_lo, clamp_hi,
                                                _ptr(loss), _ptr(gx), _stream(stream)),
               "ptrig_sincostan_loss_f32")


def ptrig_fp64_fma_probe(sink, iters, nsink=None, stream=None):
    """Measurement kernel: nsink / 256 blocks of 256 threads, each thread
    16 * iters FP64 FLOPs (8 FMA chains); sink receives one double per thread."""
    nsink = _count(sink) if nsink is None else nsink
    with _on(_buffers("ptrig_fp64_fma_probe", nsink, (sink, 8))):
        _check(_load().ptrig_fp64_fma_probe(_ptr(sink), nsink, iters, _stream(stream)), "ptrig_fp64_fma_probe")


def ptrig_status_string(status: int) -> str:
    return _load().ptrig_status_string(status).decode()


def ptrig_last_cuda_error() -> int:
    return _load().ptrig_last_cuda_error()


def ptrig_version() -> int:
    return _load().ptrig_version()


def ptrig_set_launch_config(family, block, vec_per_thread, blocks_per_sm):
    _check(_load().ptrig_set_launch_config(family, block, vec_per_thread, blocks_per_sm),
           "ptrig_set_launch_config")


def ptrig_get_launch_config(family):
    b, v, s = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(_load().ptrig_get_launch_config(family, ctypes.byref(b), ctypes.byref(v), ctypes.byref(s)),
           "ptrig_get_launch_config")
    return b.value, v.value, s.value


# ----------------------------------------------------------------- batch


def ptrig_batch_run_noalloc(device_descs, count, stream=None):
    """Ragged batch without any device allocation: device_descs is the device
    address (or a CUDA tensor of at least count * 40 bytes) of `count`
    ptrig_desc structs.  See include/ptrig.h."""
    dev = None
    if device_descs is not None and not isinstance(device_descs, int):
        need = count * ctypes.sizeof(ptrig_desc)
        have = device_descs.numel() * device_descs.element_size()
        if not device_descs.is_cuda or not device_descs.is_contiguous() or have < need:
            raise ValueError(f"ptrig_batch_run_noalloc: descriptors need a contiguous CUDA tensor of at least "
                             f"{need} bytes, got {have} bytes")
        dev = device_descs.device
    with _on(dev):
        _check(_load().ptrig_batch_run_noalloc(_ptr(device_descs), count, _stream(stream)),
               "ptrig_batch_run_noalloc")


class BatchPlan:
    """Owner of a ptrig_batch_plan: descriptors of (x, y0, y1, n, func)."""

    def __init__(self, descs, flags: int = 0):
        arr = (ptrig_desc * len(descs))()
        for i, (x, y0, y1, n, func) in enumerate(descs):
            arr[i] = ptrig_desc(_ptr(x), _ptr(y0), _ptr(y1), int(n), int(func), 0)
        self._keep = arr
        self.handle = ctypes.c_void_p()
        _check(_load().ptrig_batch_plan_create(ctypes.byref(self.handle), arr, len(descs), flags),
               "ptrig_batch_plan_create")

    def run(self, stream=None):
        _check(_load().ptrig_batch_run(self.handle, _stream(stream)), "ptrig_batch_run")

    def run_per_array(self, stream=None):
        _check(_load().ptrig_batch_run_per_array(self.handle, _stream(stream)), "ptrig_batch_run_per_array")

    def set_config(self, block: int, items_per_thread: int):
        _check(_load().ptrig_batch_plan_set_config(self.handle, block, items_per_thread),
               "ptrig_batch_plan_set_config")

    def config(self):
        b, it, g = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        t = ctypes.c_uint64()
        _check(_load().ptrig_batch_plan_get_config(self.handle, ctypes.byref(b), ctypes.byref(it),
                                                   ctypes.byref(t), ctypes.byref(g)),
               "ptrig_batch_plan_get_config")
        return {"block": b.value, "items_per_thread": it.value, "tiles": t.value, "grid": g.value}

    def autotune(self, reps: int = 5, candidates=None, stream=None):
        bb, bi, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_float()
        if candidates:
            cb = (ctypes.c_int * len(candidates))(*[c[0] for c in candidates])
            ci = (ctypes.c_int * len(candidates))(*[c[1] for c in candidates])
            nc = len(candidates)
        else:
            cb = ci = None
            nc = 0
        _check(_load().ptrig_batch_plan_autotune(self.handle, _stream(stream), reps, cb, ci, nc,
                                                 ctypes.byref(bb), ctypes.byref(bi), ctypes.byref(ms)),
               "ptrig_batch_plan_autotune")
        return {"block": bb.value, "items_per_thread": bi.value, "ms": ms.value}

    def close(self):
        if self.handle:
            _load().ptrig_batch_plan_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
