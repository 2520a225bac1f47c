"""The C ABI from a plain C99 program (tests/c_abi/use_ptrig.c): the headers
compile as C99 on the CPU; on a GPU the program links against libptrig.so and
the CUDA runtime, runs, and checks its results."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "c_abi", "use_ptrig.c")
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")


def _gcc():
    cc = shutil.which("gcc")
    if not cc:
        pytest.skip("no gcc")
    return cc


def test_headers_compile_as_c99(tmp_path):
    for hdr in ("ptrig.h", "ptrig_cpu.h"):
        src = tmp_path / "inc.c"
        src.write_text(f'#include "{hdr}"\nint main(void) {{ return 0; }}\n')
        r = subprocess.run([_gcc(), "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I",
                            os.path.join(ROOT, "include"), "-c", str(src), "-o", str(tmp_path / "inc.o")],
                           capture_output=True, text=True)
        assert r.returncode == 0, (hdr, r.stderr)


def test_c_client_object_compiles(tmp_path):
    if not os.path.exists(os.path.join(CUDA, "include", "cuda_runtime_api.h")):
        pytest.skip("no CUDA headers")
    r = subprocess.run([_gcc(), "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), "-I",
                        os.path.join(CUDA, "include"), "-c", SRC, "-o", str(tmp_path / "use.o")],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


@pytest.mark.gpu
def test_c_client_runs(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_10831_gb300 import build
    lib = build.build()
    libdir = os.path.dirname(lib)
    exe = tmp_path / "use_ptrig"
    r = subprocess.run([_gcc(), "-std=c99", "-O2", "-I", os.path.join(ROOT, "include"), "-I",
                        os.path.join(CUDA, "include"), SRC, "-o", str(exe), "-L", libdir, "-lptrig",
                        "-L", os.path.join(CUDA, "lib64"), "-lcudart", "-lm", f"-Wl,-rpath,{libdir}",
                        f"-Wl,-rpath,{os.path.join(CUDA, 'lib64')}"], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    run = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert run.returncode == 0 and run.stdout.startswith("ok"), (run.stdout, run.stderr)
