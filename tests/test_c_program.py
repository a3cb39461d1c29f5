"""The C ABI from a plain C program (tests/c/ppm_c_example.c): compiled as
C11 against include/ppm.h here (no GPU needed), and built, linked against
libppm.so and run on the GPU (-m gpu)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "c", "ppm_c_example.c")
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")


def _cc():
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    return cc


def test_c_example_compiles_against_the_header(tmp_path):
    obj = tmp_path / "ppm_c_example.o"
    r = subprocess.run([_cc(), "-std=c11", "-Wall", "-Wextra", "-Werror", "-c", SRC, "-o", str(obj),
                        "-I", os.path.join(ROOT, "include"), "-I", os.path.join(CUDA, "include")],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


@pytest.mark.gpu
def test_c_example_runs(tmp_path):
    import __graft_entry__
    __graft_entry__.build()
    libdir = os.path.join(ROOT, "paper_2504_04411_gb300")
    cudalib = os.path.join(CUDA, "lib64")
    exe = tmp_path / "ppm_c_example"
    r = subprocess.run([_cc(), "-std=c11", "-O2", SRC, "-o", str(exe),
                        "-I", os.path.join(ROOT, "include"), "-I", os.path.join(CUDA, "include"),
                        "-L", libdir, "-lppm", "-L", cudalib, "-lcudart", "-lm",
                        f"-Wl,-rpath,{libdir}", f"-Wl,-rpath,{cudalib}"], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.startswith("ok:"), r.stdout
    print(r.stdout)
