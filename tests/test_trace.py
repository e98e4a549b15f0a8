"""Tracing: every C-ABI call opens an NVTX range in the domain "semiring" and closes
it on return, failures included.  A small NVTX injection library (tests/native)
records the events; the calls below fail their argument checks before any CUDA
call, so no GPU is needed."""

import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "native", "nvtx_record.c")

CHILD = r"""
import ctypes, sys
from paper_1705_08743_gb300 import _capi as sr
L = sr.lib
assert L.antidist_closure(None, None, 4, 4, sr.SR_U8, None) == sr.SR_EINVAL
assert L.bool_mul(None, 16, 1, 16, 1, 16, 1, 4, 4, 4, sr.SR_BOOL_W32, 0, None) == sr.SR_EINVAL
assert L.antidist_mul(None, 1, 4, 1, 4, 2, 4, 4, 4, 4, 0, 0, None) == sr.SR_EINVAL
assert L.sr_cancel(None, 1) == sr.SR_EINVAL
assert L.sr_serve_start(None, None) == sr.SR_EINVAL
assert L.bool_closure_squaring_noalloc(None, 1, 4, sr.SR_U8, None) == sr.SR_EINVAL
assert L.sr_batch_create(None, None, 0, None) == sr.SR_EINVAL
assert L.sr_batched(None, None, 0, None) == sr.SR_EINVAL
rec = ctypes.CDLL(sys.argv[1])
rec.nvtx_record_log.restype = ctypes.c_char_p
sys.stdout.write(rec.nvtx_record_log().decode())
"""


@pytest.fixture(scope="module")
def recorder(tmp_path_factory):
    if not shutil.which("gcc"):
        pytest.skip("gcc not available")
    import __graft_entry__ as g
    g.build()
    so = str(tmp_path_factory.mktemp("nvtx") / "libnvtx_record.so")
    cuda_inc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")
    subprocess.run(["gcc", "-shared", "-fPIC", "-O1", "-I", cuda_inc, SRC, "-o", so], check=True)
    return so


def test_entry_points_open_and_close_ranges(recorder):
    env = dict(os.environ, NVTX_INJECTION64_PATH=recorder, PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "-c", CHILD, recorder], env=env, cwd=ROOT, capture_output=True,
                       text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    lines = [l.split(" ", 2) for l in r.stdout.strip().splitlines()]
    pushes = [l[2] for l in lines if l[0] == "push"]
    assert pushes == ["antidist_closure", "bool_mul", "antidist_mul", "sr_cancel", "sr_serve_start",
                      "bool_closure_squaring_noalloc", "sr_batch_create", "sr_batched", "sr_batch_create"]
    assert all(l[1] == "semiring" for l in lines)
    # strictly nested: each push is closed by the next pop, even on the error paths
    # sr_batched opens its own range around the nested sr_batch_create
    assert [l[0] for l in lines] == ["push", "pop"] * 7 + ["push", "push", "pop", "pop"]


GPU_CHILD = r"""
import ctypes, sys
import torch
from paper_1705_08743_gb300 import _capi as sr
D = 300
T = torch.zeros((D, D), dtype=torch.uint8, device="cuda")
sr.antidist_closure(None, T, D, D, sr.SR_U8)                 # stream schedule, three pivot blocks
ctx = sr.sr_create(workspace_bytes=sr.sr_workspace_query(sr.SR_OP_ANTIDIST_CLOSURE, sr.SR_U8, D))
sr.sr_set_option(ctx, sr.SR_OPT_CLOSURE_FUSED, 2)
T2 = torch.zeros((D, 304), dtype=torch.uint8, device="cuda")
sr.antidist_closure(ctx, T2, 304, D, sr.SR_U8)               # fused passes: block 0's launch, then three
B = torch.zeros((D, 10), dtype=torch.int32, device="cuda")
sr.bool_closure(None, B, 10, D, sr.SR_BOOL_W32, sr.SR_CLOSURE_WARSHALL)
torch.cuda.synchronize()
sr.sr_destroy(ctx)
rec = ctypes.CDLL(sys.argv[1])
rec.nvtx_record_log.restype = ctypes.c_char_p
sys.stdout.write(rec.nvtx_record_log().decode())
"""


@pytest.mark.gpu
def test_closure_schedules_open_a_range_per_pivot_block(recorder):
    """The closure schedules bracket each pivot block's launches in a range of its own
    (payload: the block index), nested in the call's range."""
    env = dict(os.environ, NVTX_INJECTION64_PATH=recorder, PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "-c", GPU_CHILD, recorder], env=env, cwd=ROOT, capture_output=True,
                       text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    ev = [l.split(" ", 2) for l in r.stdout.strip().splitlines()]
    ev = [(k, n) for k, d, *rest in ev for n in [rest[0] if rest else ""] if d == "semiring"]

    def call(name):
        """the events between the push of `name` and its matching pop"""
        i = next(j for j, (k, n) in enumerate(ev) if k == "push" and n == name)
        depth = 0
        for j in range(i, len(ev)):
            depth += 1 if ev[j][0] == "push" else -1
            if depth == 0:
                out = ev[i + 1:j]
                del ev[i:j + 1]
                return out
        raise AssertionError("unbalanced ranges")

    inner = call("antidist_closure")
    assert [n for k, n in inner if k == "push"] == [f"antidist_closure.block#{b}" for b in range(3)]
    inner = call("antidist_closure")
    assert [n for k, n in inner if k == "push"] == [f"antidist_closure.block#{b}" for b in range(-1, 3)]
    inner = call("bool_closure")
    blocks = [n for k, n in inner if k == "push"]
    assert blocks and all(n.startswith("bool_closure.block#") for n in blocks)
    assert [int(n.split("#")[1]) for n in blocks] == list(range(len(blocks)))
