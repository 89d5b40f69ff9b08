"""The boundary is a C ABI: include/chemora.h compiles as plain C, and a C
program (tests/c_abi/wave_rk4.c: no Python, no C++) links libchemora.so and
the CUDA runtime and runs RK4 steps of the scalar wave on device memory it
allocates itself and through the host-buffer call (the -m gpu case runs it;
the two results must agree bit for bit and the discrete energy must not
grow)."""
import os
import shutil
import subprocess

import pytest

from paper_1410_1764_gb300 import _native as N

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")


def _lib():
    if not os.path.exists(N.LIB_PATH):
        import importlib.util
        spec = importlib.util.spec_from_file_location("b", os.path.join(ROOT, "paper_1410_1764_gb300", "build.py"))
        m = importlib.util.module_from_spec(spec)
        spec.loader.exec_module(m)
        m.build()
    return N.LIB_PATH


def test_header_is_plain_c():
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    r = subprocess.run([cc, "-std=c11", "-Wall", "-Wextra", "-Werror", "-fsyntax-only", "-x", "c",
                        os.path.join(ROOT, "include", "chemora.h")], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def _build_example(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None or not os.path.isdir(os.path.join(CUDA, "include")):
        pytest.skip("no C compiler or CUDA headers")
    lib = _lib()
    exe = str(tmp_path / "wave_rk4")
    libdir = os.path.dirname(lib)
    cmd = [cc, "-std=c11", "-O2", "-Wall", "-Werror", os.path.join(ROOT, "tests", "c_abi", "wave_rk4.c"),
           "-I", os.path.join(ROOT, "include"), "-I", os.path.join(CUDA, "include"),
           "-L", libdir, "-l:libchemora.so", "-Wl,-rpath," + libdir,
           "-L", os.path.join(CUDA, "lib64"), "-lcudart", "-Wl,-rpath," + os.path.join(CUDA, "lib64"), "-lm",
           "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe


def test_c_program_links(tmp_path):
    assert os.access(_build_example(tmp_path), os.X_OK)


@pytest.mark.gpu
def test_c_program_runs(tmp_path):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    exe = _build_example(tmp_path)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, (r.returncode, r.stdout, r.stderr)
    assert "max |device - host| = 0.000e+00" in r.stdout, r.stdout
