"""The C ABI from plain C: tests/c/round_example.c includes only include/ttround.h and the CUDA
runtime, links libttround, and rounds a small TT (the formal sum of two random TTs) adaptively.

* CPU: the header compiles as C11 with warnings on, and the program links against the library.
* GPU: the program runs; it checks the status, the left-orthonormality of the output cores and
  ||X - Y|| <= tol ||X|| against the dense tensor, and prints OK.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")


@pytest.fixture(scope="module")
def program(tmp_path_factory):
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc or not os.path.exists(os.path.join(CUDA, "include", "cuda_runtime.h")):
        pytest.skip("no C compiler or CUDA headers")
    from paper_2511_03598_gb300 import build
    lib = build.build()
    libdir = os.path.dirname(lib)
    exe = str(tmp_path_factory.mktemp("capi") / "round_example")
    cmd = [cc, "-std=c11", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
           "-I", os.path.join(CUDA, "include"), os.path.join(ROOT, "tests", "c", "round_example.c"),
           "-L", libdir, "-lttround", "-L", os.path.join(CUDA, "lib64"), "-lcudart", "-lm", "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    return exe, libdir


def test_c_program_compiles_and_links(program):
    exe, _ = program
    assert os.path.exists(exe)


@pytest.mark.gpu
def test_c_program_rounds_on_the_gpu(program):
    exe, libdir = program
    env = dict(os.environ)
    env["LD_LIBRARY_PATH"] = os.pathsep.join([libdir, os.path.join(CUDA, "lib64"), env.get("LD_LIBRARY_PATH", "")])
    r = subprocess.run([exe], capture_output=True, text=True, env=env, timeout=120)
    assert r.returncode == 0 and "OK" in r.stdout, r.stdout + r.stderr
