"""The C-ABI library builds, loads and exports every symbol include/ptrig.h
declares; host-side argument checks answer without touching a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ptrig.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ptrig_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2502_10831_gb300 import build
    build.build()
    from paper_2502_10831_gb300 import binding
    return binding.lib()


def test_header_declares_the_scope_entry_points():
    names = set(_declared())
    for fn in ("sin", "cos", "tan"):
        for dt in ("f32", "f16", "bf16", "f64"):
            assert f"ptrig_{fn}_{dt}" in names
        for dt in ("f32", "f64"):
            assert f"ptrig_{fn}_bwd_{dt}" in names
        assert f"ptrig_taylor_{fn}_f32" in names
    for dt in ("f32", "f16", "bf16"):
        assert f"ptrig_sincos_{dt}" in names
    for n in ("ptrig_batch_plan_create", "ptrig_batch_run", "ptrig_batch_plan_destroy", "ptrig_status_string"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_2502_10831_gb300 import binding
    assert sorted(binding.exported_symbols()) == _declared()


def test_status_strings(lib):
    from paper_2502_10831_gb300 import binding
    for s in range(5):
        assert binding.ptrig_status_string(s).startswith("PTRIG")
    assert "unknown" in binding.ptrig_status_string(99)


def test_host_validation_without_gpu(lib):
    """NULL pointers with n > 0 and bad selectors are rejected before any CUDA
    call; n == 0 is a no-op."""
    assert lib.ptrig_sin_f32(None, None, 0, None) == 0
    for name in ("ptrig_sin_f32", "ptrig_cos_f16", "ptrig_tan_bf16", "ptrig_sin_f64", "ptrig_taylor_tan_f32"):
        assert getattr(lib, name)(None, None, 4, None) == 1
    assert lib.ptrig_sincos_f32(1024, 2048, None, 4, None) == 1
    assert lib.ptrig_sin_bwd_f32(1024, None, 2048, 4, None) == 1
    assert lib.ptrig_taylor_n_f32(0, 6, 1024, 2048, 4, None) == 1
    assert lib.ptrig_taylor_n_f32(3, 5, 1024, 2048, 4, None) == 1
    assert lib.ptrig_cudamath_f32(4, 0, 1024, 2048, None, 4, None) == 1
    assert lib.ptrig_set_launch_config(0, 100, 4, 0) == 1
    assert lib.ptrig_set_launch_config(0, 256, 3, 0) == 1
    assert lib.ptrig_set_launch_config(11, 256, 4, 0) == 1
    assert lib.ptrig_set_launch_config(0, 256, 16, 0) == 1
    assert lib.ptrig_fp64_fma_probe(1024, 300, 10, None) == 1  # not a multiple of 256
    assert lib.ptrig_fp64_fma_probe(1024, 512, 0, None) == 1
    assert lib.ptrig_fp64_fma_probe(None, 512, 10, None) == 1
    assert lib.ptrig_fp64_fma_probe(None, 0, 10, None) == 0


def test_launch_config_roundtrip(lib):
    from paper_2502_10831_gb300 import binding as B
    old = B.ptrig_get_launch_config(B.FAMILY_TAYLOR)
    B.ptrig_set_launch_config(B.FAMILY_TAYLOR, 128, 2, 4)
    assert B.ptrig_get_launch_config(B.FAMILY_TAYLOR) == (128, 2, 4)
    B.ptrig_set_launch_config(B.FAMILY_TAYLOR, 256, 0, 0)  # loads in flight by size
    assert B.ptrig_get_launch_config(B.FAMILY_TAYLOR) == (256, 0, 0)
    B.ptrig_set_launch_config(B.FAMILY_TAYLOR, *old)


def test_default_launch_configs(lib):
    """The per-family defaults picked by the GB300 sweeps: one-shot 64-thread
    blocks (the whole-chunk kernel) with four 16-byte loads in flight (FP32
    sin, cos and tan by size: 0; two for the FP32 sincos), eight for bf16
    sin, cos and tan,
    128-thread blocks for the fp16 sincos and the derivatives; the CUDA-math
    comparison kernels persistent."""
    from paper_2502_10831_gb300 import binding as B
    want = {B.FAMILY_F32: (64, 0, 0), B.FAMILY_HALF: (64, 4, 0), B.FAMILY_TAYLOR: (64, 4, 0),
            B.FAMILY_BWD: (128, 2, 0), B.FAMILY_BF16: (64, 8, 0), B.FAMILY_CUDAMATH: (512, 2, 8),
            B.FAMILY_F32_SINCOS: (64, 2, 0), B.FAMILY_HALF_SINCOS: (128, 4, 0), B.FAMILY_BF16_SINCOS: (64, 4, 0),
            B.FAMILY_HALF_TAN: (64, 4, 0), B.FAMILY_BF16_TAN: (64, 8, 0)}
    assert len(want) == B.FAMILY_COUNT
    for fam, cfg in want.items():
        assert B.ptrig_get_launch_config(fam) == cfg, fam
    assert lib.ptrig_set_launch_config(B.FAMILY_COUNT, 64, 4, 0) == 1


def test_batch_plan_rejects_bad_descriptors(lib):
    from paper_2502_10831_gb300 import binding as B
    h = ctypes.c_void_p()
    bad = [
        B.ptrig_desc(1024, 2048, 0, 10, 7, 0),      # unknown func
        B.ptrig_desc(1024, 2048, 0, 10, 0, 1),      # reserved != 0
        B.ptrig_desc(0, 2048, 0, 10, 0, 0),         # NULL x
        B.ptrig_desc(1024, 2048, 0, 10, 3, 0),      # sincos without y1
    ]
    for d in bad:
        arr = (B.ptrig_desc * 1)(d)
        assert lib.ptrig_batch_plan_create(ctypes.byref(h), arr, 1, 0) == 1
        assert not h.value
    arr = (B.ptrig_desc * 1)(B.ptrig_desc(1024, 2048, 0, 10, 0, 0))
    assert lib.ptrig_batch_plan_create(ctypes.byref(h), arr, 1, 8) == 1  # unknown flag
    assert lib.ptrig_batch_plan_create(None, arr, 1, 0) == 1
    assert lib.ptrig_batch_plan_create(ctypes.byref(h), None, 3, 0) == 1
    lib.ptrig_batch_plan_destroy(None)


def test_product_path_does_not_reference_the_oracle():
    """The package never imports, loads or runs anything under oracle/, nor
    the CPU SIMD baseline under cpu_simd/ (no CPU fallback)."""
    pkg = os.path.join(ROOT, "paper_2502_10831_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                for pat in (r"\bimport\s+oracle", r"\bfrom\s+oracle\b", r"ptrig_oracle", r"ptro_",
                            r"cpu_simd", r"ptrig_cpu"):
                    assert not re.search(pat, src), (f, pat)


def test_cpu_baseline_does_not_reference_the_oracle():
    """cpu_simd/ is a third implementation: it shares nothing with oracle/."""
    d = os.path.join(ROOT, "cpu_simd")
    for f in os.listdir(d):
        if f.endswith((".py", ".c", ".h")):
            src = open(os.path.join(d, f)).read()
            for pat in (r"\bimport\s+oracle", r"\bfrom\s+oracle\b", r"ptrig_oracle", r"ptro_"):
                assert not re.search(pat, src), (f, pat)


def test_binding_refuses_mismatched_buffers_before_any_launch():
    """Tensors that are too small, of another element width or not contiguous
    are refused on the host (ValueError) before the library is called; so are
    CPU tensors that are not pinned."""
    torch = pytest.importorskip("torch")
    from paper_2502_10831_gb300 import binding as B

    x = torch.zeros(8, dtype=torch.float32)
    with pytest.raises(ValueError, match="CUDA tensors or pinned"):
        B.ptrig_sin_f32(x, torch.zeros(8, dtype=torch.float32))

    class Fake:  # stands in for CUDA tensors, so no device is needed
        def __init__(self, numel, esize, contiguous=True, device="cuda:0"):
            self._n, self._e, self._c, self.device = numel, esize, contiguous, device
            self.is_cuda, self.dtype = True, f"{esize}-byte"

        def numel(self):
            return self._n

        def element_size(self):
            return self._e

        def is_contiguous(self):
            return self._c

        def is_pinned(self):
            return False

        def data_ptr(self):
            raise AssertionError("the library was reached")

    cases = [
        ("ptrig_sin_f32", (Fake(8, 4), Fake(7, 4)), "fewer than"),
        ("ptrig_cos_f16", (Fake(8, 2), Fake(8, 4)), "2-byte"),
        ("ptrig_tan_f64", (Fake(8, 8), Fake(8, 8, contiguous=False)), "contiguous"),
        ("ptrig_sincos_bf16", (Fake(8, 2), Fake(8, 2), Fake(4, 2)), "fewer than"),
        ("ptrig_sin_bwd_f32", (Fake(8, 4), Fake(8, 4), Fake(8, 4, device="cuda:1")), "different devices"),
        ("ptrig_segment_f32", (Fake(8, 4), Fake(8, 4)), "1-byte"),
    ]
    for name, args, msg in cases:
        with pytest.raises(ValueError, match=msg):
            getattr(B, name)(*args)
    with pytest.raises(ValueError, match="descriptors need"):
        B.ptrig_batch_run_noalloc(Fake(10, 4), 2)  # 40 bytes for 2 descriptors (80 needed)


def test_functional_refuses_mismatched_out():
    torch = pytest.importorskip("torch")
    from paper_2502_10831_gb300 import functional as Fn

    x = torch.zeros(4, 4)
    for out in (torch.zeros(4, 3), torch.zeros(4, 4, dtype=torch.float64), torch.zeros(4, 8)[:, ::2]):
        with pytest.raises(ValueError):
            Fn._check_out(out, x)
    Fn._check_out(torch.zeros(4, 4), x)
