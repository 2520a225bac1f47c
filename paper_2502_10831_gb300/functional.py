"""Tensor-level API over libptrig: the paper's sin/cos/tan of CUDA tensors.

torch provides device memory and the current stream; the arithmetic runs in
the CUDA library.  float32, float16, bfloat16 and float64 tensors are
accepted (f16 / bf16 compute in FP32 and round once).  Autograd support
(forward + the hand-written derivative kernels) is available through
``sin``, ``cos``, ``tan`` for float32 and float64 inputs.
"""
from __future__ import annotations

import torch

from . import binding as B

_FUNCS = ("sin", "cos", "tan")
_SUFFIX = {torch.float32: "f32", torch.float16: "f16", torch.bfloat16: "bf16", torch.float64: "f64"}


def _prep(x: torch.Tensor) -> torch.Tensor:
    if not isinstance(x, torch.Tensor) or not x.is_cuda:
        raise ValueError("ptrig functions take CUDA tensors")
    if x.dtype not in _SUFFIX:
        raise TypeError(f"unsupported dtype {x.dtype}")
    return x.contiguous()


def _check_out(out: torch.Tensor, x: torch.Tensor, what: str = "out") -> None:
    """out must match x: a contiguous tensor of the same shape, dtype and
    device (checked before any launch)."""
    if not isinstance(out, torch.Tensor):
        raise TypeError(f"{what} must be a tensor")
    if out.shape != x.shape or out.dtype != x.dtype or out.device != x.device or not out.is_contiguous():
        raise ValueError(f"{what} must be a contiguous tensor of x's shape {tuple(x.shape)}, dtype {x.dtype} "
                         f"and device {x.device}; got {tuple(out.shape)}, {out.dtype}, {out.device}"
                         f"{'' if out.is_contiguous() else ', non-contiguous'}")


def forward(func: str, x: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
    """Paper's sin/cos/tan of x (no autograd)."""
    x = _prep(x)
    if out is None:
        y = torch.empty_like(x)
    else:
        _check_out(out, x)
        y = out
    getattr(B, f"ptrig_{func}_{_SUFFIX[x.dtype]}")(x, y)
    return y


def sincos(x: torch.Tensor):
    """(sin, cos) of x from one reduction and one square root per element."""
    x = _prep(x)
    if x.dtype == torch.float64:
        return forward("sin", x), forward("cos", x)
    s = torch.empty_like(x)
    c = torch.empty_like(x)
    getattr(B, f"ptrig_sincos_{_SUFFIX[x.dtype]}")(x, s, c)
    return s, c


def taylor(func: str, x: torch.Tensor, nterms: int = 5) -> torch.Tensor:
    """Taylor-n baseline (n in 5, 7, 9) on the same reduced angle, FP32."""
    x = _prep(x)
    if x.dtype != torch.float32:
        raise TypeError("the Taylor baseline is FP32")
    y = torch.empty_like(x)
    B.ptrig_taylor_n_f32(_FUNCS.index(func), nterms, x, y)
    return y


def derivative(func: str, x: torch.Tensor, gy: torch.Tensor) -> torch.Tensor:
    """gy * d f(x)/dx with f the paper's piecewise function (f32 / f64)."""
    x = _prep(x)
    gy = gy.contiguous()
    if x.dtype not in (torch.float32, torch.float64) or gy.dtype != x.dtype or gy.shape != x.shape:
        raise TypeError("derivative needs matching float32 or float64 x and gy")
    if gy.device != x.device:
        raise ValueError(f"gy is on {gy.device}, x on {x.device}")
    gx = torch.empty_like(x)
    getattr(B, f"ptrig_{func}_bwd_{_SUFFIX[x.dtype]}")(x, gy, gx)
    return gx


class _Ptrig(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, func):
        ctx.func = func
        ctx.save_for_backward(x)
        return forward(func, x)

    @staticmethod
    def backward(ctx, gy):
        (x,) = ctx.saved_tensors
        return derivative(ctx.func, x, gy), None


def sin(x: torch.Tensor) -> torch.Tensor:
    return _Ptrig.apply(x, "sin") if x.requires_grad else forward("sin", x)


def cos(x: torch.Tensor) -> torch.Tensor:
    return _Ptrig.apply(x, "cos") if x.requires_grad else forward("cos", x)


def tan(x: torch.Tensor) -> torch.Tensor:
    return _Ptrig.apply(x, "tan") if x.requires_grad else forward("tan", x)


def segment(x: torch.Tensor) -> torch.Tensor:
    """Per element: segment index | quadrant << 4 (uint8), FP32 inputs."""
    x = _prep(x)
    out = torch.empty(x.shape, dtype=torch.uint8, device=x.device)
    B.ptrig_segment_f32(x, out)
    return out


def cudamath(func: str, x: torch.Tensor, fast: bool = False):
    """CUDA's own sinf/cosf/tanf/sincosf (or intrinsics) for comparison."""
    x = _prep(x)
    y0 = torch.empty_like(x)
    if func == "sincos":
        y1 = torch.empty_like(x)
        B.ptrig_cudamath_f32(B.SINCOS, int(fast), x, y0, y1)
        return y0, y1
    B.ptrig_cudamath_f32(_FUNCS.index(func), int(fast), x, y0)
    return y0


class _FusedLoss(torch.autograd.Function):
    """L = sum(w sin(x) + v cos(x) + u clamp(tan(x), lo, hi)) and dL/dx from one
    kernel pass; the gradient is kept for backward.  w, v, u are constants."""

    @staticmethod
    def forward(ctx, x, w, v, u, lo, hi):
        x, w, v, u = (t.contiguous() for t in (x, w, v, u))
        loss = torch.empty((), dtype=torch.float64, device=x.device)
        gx = torch.empty_like(x)
        B.ptrig_sincostan_loss_f32(x, w, v, u, float(lo), float(hi), loss, gx)
        ctx.save_for_backward(gx)
        return loss.to(x.dtype)

    @staticmethod
    def backward(ctx, g):
        (gx,) = ctx.saved_tensors
        return g.to(gx.dtype) * gx, None, None, None, None, None


def sincostan_loss(x: torch.Tensor, w: torch.Tensor, v: torch.Tensor, u: torch.Tensor,
                   lo: float = -50.0, hi: float = 50.0) -> torch.Tensor:
    """Fused sum(w sin(x) + v cos(x) + u clamp(tan(x), lo, hi)) for float32 CUDA
    tensors of one shape, differentiable in x."""
    for t in (x, w, v, u):
        if not t.is_cuda or t.dtype != torch.float32 or t.shape != x.shape or t.device != x.device:
            raise TypeError("sincostan_loss takes float32 CUDA tensors of one shape on one device")
    return _FusedLoss.apply(x, w, v, u, lo, hi)
