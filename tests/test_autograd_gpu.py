"""Differentiation through autograd.Function: FP64 gradcheck, the FP32 loss
gradient against the oracle's analytic derivative, and the fused kernel."""
import math

import numpy as np
import pytest

import parity as P
from paper_2502_10831_gb300 import workloads

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def Fn():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_10831_gb300 import build, functional
    build.build()
    return functional


def _away(x, margin=1e-3):
    return workloads.away_from_nodes(x, margin)


@pytest.mark.parametrize("func", ["sin", "cos", "tan"])
def test_gradcheck_fp64(Fn, func):
    """4096 FP64 angles at least 1e-3 from every node and pole."""
    r = np.random.default_rng(5)
    x = r.uniform(-4 * math.pi, 4 * math.pi, 20000)
    x = x[_away(x)][:4096]
    xt = torch.from_numpy(x).cuda().requires_grad_(True)
    f = getattr(Fn, func)
    assert torch.autograd.gradcheck(f, (xt,), eps=1e-6, atol=1e-6, rtol=1e-5)


def _inputs(n, seed=0):
    x, w, v, u = workloads.autograd((n,), seed=workloads.SEED + seed)
    return x, w, v, u


def _oracle_grad(oracle, x, w, v, u, lo=-50.0, hi=50.0):
    xd = x.astype(np.float64)
    t = oracle.proposed("tan", xd)
    mask = (t >= lo) & (t <= hi)
    g = (w * oracle.derivative("sin", xd) + v * oracle.derivative("cos", xd)
         + u * oracle.derivative("tan", xd) * mask)
    loss = np.sum(w * oracle.proposed("sin", xd) + v * oracle.proposed("cos", xd) + u * np.clip(t, lo, hi))
    return g, loss, t


def _keep(oracle, x, t):
    u, *_ = oracle.reduce(x.astype(np.float64))
    keep = ~P.near_node(u)
    keep &= np.abs(oracle.proposed("cos", x.astype(np.float64))) >= 1e-3
    keep &= np.abs(np.abs(t) - 50.0) > 1e-2  # clamp edge: the mask may flip on rounding
    return keep


def test_fp32_loss_gradient_against_oracle(Fn, oracle):
    x, w, v, u = _inputs(1 << 20)
    xt = torch.from_numpy(x).cuda().requires_grad_(True)
    wt, vt, ut = (torch.from_numpy(a).cuda() for a in (w, v, u))
    loss = (wt * Fn.sin(xt) + vt * Fn.cos(xt) + ut * torch.clamp(Fn.tan(xt), -50, 50)).sum()
    loss.backward()
    g_ref, l_ref, t = _oracle_grad(oracle, x, w.astype(np.float64), v.astype(np.float64), u.astype(np.float64))
    keep = _keep(oracle, x, t)
    got = xt.grad.cpu().numpy().astype(np.float64)
    err = np.abs(got - g_ref)[keep] / np.maximum(1.0, np.abs(g_ref[keep]))
    assert err.max() <= 5e-5, err.max()
    assert abs(loss.item() - l_ref) <= 1e-4 * max(1.0, abs(l_ref)) + 1e-2


def test_fused_loss_matches_unfused_and_oracle(Fn, oracle):
    x, w, v, u = _inputs((1 << 20) + 3, seed=1)
    xt = torch.from_numpy(x).cuda().requires_grad_(True)
    wt, vt, ut = (torch.from_numpy(a).cuda() for a in (w, v, u))
    lf = Fn.sincostan_loss(xt, wt, vt, ut, -50.0, 50.0)
    lf.backward()
    gf = xt.grad.clone()
    xt.grad = None
    lu = (wt * Fn.sin(xt) + vt * Fn.cos(xt) + ut * torch.clamp(Fn.tan(xt), -50, 50)).sum()
    lu.backward()
    gu = xt.grad
    g_ref, l_ref, t = _oracle_grad(oracle, x, w.astype(np.float64), v.astype(np.float64), u.astype(np.float64))
    keep = _keep(oracle, x, t)
    gfn = gf.cpu().numpy().astype(np.float64)
    gun = gu.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(gfn - gun)[keep] / np.maximum(1.0, np.abs(gun[keep]))) <= 1e-5
    assert np.max(np.abs(gfn - g_ref)[keep] / np.maximum(1.0, np.abs(g_ref[keep]))) <= 5e-5
    assert abs(lf.item() - l_ref) <= 1e-5 * max(1.0, abs(l_ref)) + 1e-3
    assert abs(lf.item() - lu.item()) <= 1e-4 * max(1.0, abs(l_ref)) + 1e-2


def test_fused_loss_validation(Fn):
    from paper_2502_10831_gb300 import binding as B
    x = torch.zeros(8, device="cuda")
    loss = torch.zeros((), dtype=torch.float64, device="cuda")
    with pytest.raises(B.PtrigError):
        B.ptrig_sincostan_loss_f32(x, x, x, x, 1.0, -1.0, loss, x)
    with pytest.raises(B.PtrigError):
        B.ptrig_sincostan_loss_f32(x, x, x, x, -1.0, 1.0, None, x)
    B.ptrig_sincostan_loss_f32(x, x, x, x, -1.0, 1.0, loss, x, n=0)
    torch.cuda.synchronize()
    assert loss.item() == 0.0
