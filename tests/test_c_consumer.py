"""The C ABI from plain C: tests/native/closure_c.c includes include/semiring.h,
links libsemiring.so and the CUDA runtime, and closes a matrix read from a file
with cudaMemcpy in and out (no Python, no torch in that process).  Building it
needs no GPU; running it does, and its result is compared with the oracle's
Warshall closure (Section 2 Warshall, Section 3 Floyd)."""

import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "native", "closure_c.c")


@pytest.fixture(scope="module")
def program(tmp_path_factory):
    if not shutil.which("gcc"):
        pytest.skip("gcc not available")
    import __graft_entry__ as g
    g.build()
    cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    libdir = os.path.join(ROOT, "paper_1705_08743_gb300", "lib")
    exe = str(tmp_path_factory.mktemp("cabi") / "closure_c")
    cudalib = next((d for d in (os.path.join(cuda, "lib64"), os.path.join(cuda, "lib"),
                                os.path.join(cuda, "targets", "sbsa-linux", "lib"))
                    if os.path.exists(os.path.join(d, "libcudart.so"))), os.path.join(cuda, "lib64"))
    subprocess.run(["gcc", "-O1", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                    "-I", os.path.join(cuda, "include"), SRC, "-L", libdir, "-lsemiring", "-L", cudalib,
                    "-lcudart", f"-Wl,-rpath,{libdir}", f"-Wl,-rpath,{cudalib}", "-o", exe], check=True)
    return exe


def test_c_program_builds_against_the_header_and_library(program):
    assert os.access(program, os.X_OK)


@pytest.mark.gpu
@pytest.mark.parametrize("D", [300, 1500])
def test_c_program_closure_matches_oracle(program, tmp_path, D):
    W = synth.cfg2_antidist(D=D, p=0.02, wlo=1, whi=40, seed=4)
    A = oracle.encode_antidist(W, 255).astype(np.uint8)
    src, dst = tmp_path / "in.bin", tmp_path / "out.bin"
    A.tofile(src)
    r = subprocess.run([program, str(D), str(src), str(dst)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    assert r.stdout.startswith("ok")
    got = np.fromfile(dst, dtype=np.uint8).reshape(D, D)
    assert np.array_equal(got, oracle.warshall(A, 255))
