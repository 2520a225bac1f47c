"""Every launch configuration of the elementwise kernels gives the same
outputs.  Each kernel computes every element on its own, so the one-shot
whole-chunk kernels, the bounds-checked one-shot kernels, the persistent grids
and the 32-byte groups must agree bit for bit with the default launch (the one
the parity tests check against the oracle), on a ragged size that spans many
chunks of every shape, a partial chunk and a tail shorter than a vector, with
angles beyond the fast reduction range scattered through it so that the
full-reduction path runs inside every shape.  Needs a CUDA GPU; run with
-m gpu."""
import numpy as np
import pytest

from paper_2502_10831_gb300 import workloads

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

# (threads per block, vectors per thread (0: by size), blocks per SM; 0 = one-shot)
CONFIGS = [(64, 0, 0), (64, 1, 0), (64, 2, 0), (64, 4, 0), (64, 8, 0), (128, 2, 0), (128, 4, 0), (256, 4, 0),
           (512, 1, 0), (64, 4, 2), (256, 2, 8)]
N = 3 * 64 * 8 * 8 * 37 + 13


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_10831_gb300 import binding, build
    build.build()
    return binding


@pytest.fixture(scope="module")
def inputs():
    r = np.random.default_rng(23)
    x = workloads.bandwidth(N)
    idx = r.choice(N, N // 500, replace=False)
    x[idx] = (10.0 ** r.uniform(5.5, 37.5, idx.size) * r.choice([-1.0, 1.0], idx.size)).astype(np.float32)
    x[r.choice(N, 8, replace=False)] = np.array([np.nan, np.inf, -np.inf, 0.0, -0.0, 2.0 ** 19, -(2.0 ** 19), 65504.0],
                                                dtype=np.float32)
    xt = torch.from_numpy(x).cuda()
    h = torch.from_numpy(np.clip(workloads.bandwidth(N, seed=24), -60000, 60000).astype(np.float16)).cuda()
    return {"f32": xt, "gy": torch.from_numpy(r.standard_normal(N).astype(np.float32)).cuda(),
            "f16": h.view(torch.int16), "bf16": xt.to(torch.bfloat16).view(torch.int16)}


def _calls(B, inp):
    """(family, name, function returning the output tensors) for every
    elementwise entry point."""
    x, gy, h, b = inp["f32"], inp["gy"], inp["f16"], inp["bf16"]

    def unary(fn, xx):
        def run():
            y = torch.full_like(xx, 7)
            fn(xx, y)
            return (y,)
        return run

    def binary(fn, xx, extra=None):
        def run():
            y0 = torch.full_like(xx, 7) if extra is None else extra
            y1 = torch.full_like(xx, 7)
            fn(xx, y0, y1)
            return (y1,) if extra is not None else (y0, y1)
        return run

    out = []
    for f in ("sin", "cos", "tan"):
        out.append((B.FAMILY_F32, f"{f}_f32", unary(getattr(B, f"ptrig_{f}_f32"), x)))
        out.append((B.FAMILY_TAYLOR, f"taylor_{f}_f32", unary(getattr(B, f"ptrig_taylor_{f}_f32"), x)))
        out.append((B.FAMILY_BWD, f"{f}_bwd_f32", binary(getattr(B, f"ptrig_{f}_bwd_f32"), x, gy)))
    out.append((B.FAMILY_F32_SINCOS, "sincos_f32", binary(B.ptrig_sincos_f32, x)))
    for dt, xx, fam, famt, fams in (("f16", h, B.FAMILY_HALF, B.FAMILY_HALF_TAN, B.FAMILY_HALF_SINCOS),
                                    ("bf16", b, B.FAMILY_BF16, B.FAMILY_BF16_TAN, B.FAMILY_BF16_SINCOS)):
        for f in ("sin", "cos"):
            out.append((fam, f"{f}_{dt}", unary(getattr(B, f"ptrig_{f}_{dt}"), xx)))
        out.append((famt, f"tan_{dt}", unary(getattr(B, f"ptrig_tan_{dt}"), xx)))
        out.append((fams, f"sincos_{dt}", binary(getattr(B, f"ptrig_sincos_{dt}"), xx)))
    return out


def _bits(t):
    return t.view(torch.int32) if t.element_size() == 4 else t


def test_every_launch_configuration_matches_the_default(B, inputs):
    calls = _calls(B, inputs)
    ref = {name: [_bits(t).clone() for t in run()] for _, name, run in calls}
    torch.cuda.synchronize()
    for fam in sorted({c[0] for c in calls}):
        default = B.ptrig_get_launch_config(fam)
        try:
            for cfg in CONFIGS:
                B.ptrig_set_launch_config(fam, *cfg)
                for f2, name, run in calls:
                    if f2 != fam:
                        continue
                    got = run()
                    torch.cuda.synchronize()
                    for k, (g, want) in enumerate(zip(got, ref[name])):
                        g = _bits(g)
                        bad = int((g != want).sum())
                        assert bad == 0, (name, cfg, k, bad)
        finally:
            B.ptrig_set_launch_config(fam, *default)
