"""The anti-distance closure's persistent schedule (SR_OPT_CLOSURE_PERSISTENT) on the
GPU, through the C ABI, against the CPU oracle's Warshall closure, bit for bit.

The schedule closes the whole matrix in one launch (work items in a dependency order,
bounded waits on per-block versions), so the checks also count launches: one kernel
per closure when the persistent schedule runs, several when the stream schedule does.
"""

import numpy as np
import pytest

import oracle
import synth
from gpu_util import to_dev, to_host, sr_dtype_of

pytestmark = pytest.mark.gpu

S_OF = {np.uint8: 255, np.uint16: 65535}


def rand_anti(rng, R, C, dt, density, lo=1):
    S = S_OF[dt]
    v = rng.integers(lo, S + 1, size=(R, C), dtype=np.int64)
    return np.where(rng.random((R, C)) < density, v, 0).astype(dt)


def _aligned_pad(D, dt):
    """Extra columns that make each row a multiple of 16 bytes (the schedule's vector path)."""
    per = 16 // np.dtype(dt).itemsize
    return (-D) % per


def _ctx(D, dt, mode=2, share=None):
    import paper_1705_08743_gb300 as sr
    ws = sr.sr_workspace_query(sr.SR_OP_ANTIDIST_CLOSURE, sr_dtype_of(dt), D)
    assert ws > 0
    ctx = sr.sr_create(workspace_bytes=ws)
    sr.sr_set_option(ctx, sr.SR_OPT_CLOSURE_PERSISTENT, mode)
    if share is not None:
        sr.sr_set_option(ctx, sr.SR_OPT_CLOSURE_PANEL_SHARE, share)
    return ctx


def _close(ctx, A, pad):
    import torch
    import paper_1705_08743_gb300 as sr
    dt = A.dtype.type
    D = A.shape[0]
    Td = to_dev(A, pad)
    torch.cuda.synchronize()
    n0 = sr.sr_kernel_launches()
    sr.antidist_closure(ctx, Td, Td.shape[1], D, sr_dtype_of(dt))
    torch.cuda.synchronize()
    launches = sr.sr_kernel_launches() - n0
    sr.sr_stream_status(ctx)
    out = to_host(Td, dt)
    if pad:
        assert (out[:, D:] == 0xA5).all(), "wrote past the row width"
    return out[:, :D], launches


@pytest.mark.parametrize("dt", [np.uint8, np.uint16])
@pytest.mark.parametrize("D", [256, 257, 300, 383, 513, 777, 1100, 2085])
def test_persistent_closure_random(dt, D):
    """Two to 17 pivot blocks, ragged last blocks and tiles, long sparse paths and
    saturating dense ones."""
    import paper_1705_08743_gb300 as sr
    rng = np.random.default_rng(D * 5 + 3)
    S = S_OF[dt]
    ctx = _ctx(D, dt)
    try:
        for dens, lo in [(2.0 / D, S - S // 10), (0.05, 1)]:
            A = rand_anti(rng, D, D, dt, dens, lo)
            got, launches = _close(ctx, A, _aligned_pad(D, dt))
            assert launches == 1, "persistent schedule not taken"
            assert np.array_equal(got, oracle.warshall(A, S)), (dens, lo)
    finally:
        sr.sr_destroy(ctx)


@pytest.mark.parametrize("share", [0, 64, 256])
def test_persistent_closure_panel_shares(share):
    import paper_1705_08743_gb300 as sr
    D, dt = 1000, np.uint8
    rng = np.random.default_rng(share)
    A = rand_anti(rng, D, D, dt, 3.0 / D, 200)
    ctx = _ctx(D, dt, share=share)
    try:
        got, launches = _close(ctx, A, _aligned_pad(D, dt))
        assert launches == 1
        assert np.array_equal(got, oracle.warshall(A, 255))
    finally:
        sr.sr_destroy(ctx)


def test_persistent_closure_falls_back_when_rows_are_unaligned_or_workspace_short():
    import paper_1705_08743_gb300 as sr
    D, dt = 300, np.uint8
    rng = np.random.default_rng(5)
    A = rand_anti(rng, D, D, dt, 0.02, 100)
    want = oracle.warshall(A, 255)
    ctx = _ctx(D, dt)
    try:
        got, launches = _close(ctx, A, 5)                    # rows of 305 bytes: no vector path
        assert launches > 1 and np.array_equal(got, want)
    finally:
        sr.sr_destroy(ctx)
    small = sr.sr_create(workspace_bytes=64)
    try:
        sr.sr_set_option(small, sr.SR_OPT_CLOSURE_PERSISTENT, 2)
        got, launches = _close(small, A, _aligned_pad(D, dt))
        assert launches > 1 and np.array_equal(got, want)
    finally:
        sr.sr_destroy(small)


def test_persistent_closure_timeout_then_rerun():
    """A spin limit of 0 makes the first wait that is not already met give up: the
    launch stops, sr_stream_status reports SR_ETIMEOUT once, and the context then
    closes the same input correctly."""
    import paper_1705_08743_gb300 as sr
    D, dt = 1100, np.uint8
    rng = np.random.default_rng(11)
    A = rand_anti(rng, D, D, dt, 3.0 / D, 220)
    ctx = _ctx(D, dt)
    try:
        sr.sr_set_option(ctx, sr.SR_OPT_SPIN_LIMIT, 0)
        Td = to_dev(A, _aligned_pad(D, dt))
        sr.antidist_closure(ctx, Td, Td.shape[1], D, sr.SR_U8)
        with pytest.raises(sr.SemiringError) as e:
            sr.sr_stream_status(ctx)
        assert e.value.status == sr.SR_ETIMEOUT
        sr.sr_stream_status(ctx)                              # the status word was cleared
        sr.sr_set_option(ctx, sr.SR_OPT_SPIN_LIMIT, 1 << 22)
        got, launches = _close(ctx, A, _aligned_pad(D, dt))
        assert launches == 1 and np.array_equal(got, oracle.warshall(A, 255))
    finally:
        sr.sr_destroy(ctx)


def test_persistent_closure_captured_in_cuda_graph():
    import torch
    import paper_1705_08743_gb300 as sr
    D, dt = 900, np.uint16
    rng = np.random.default_rng(9)
    A = rand_anti(rng, D, D, dt, 3.0 / D, 60000)
    want = oracle.warshall(A, 65535)
    ctx = _ctx(D, dt)
    try:
        src = to_dev(A, _aligned_pad(D, dt))
        T = torch.empty_like(src)
        ld = T.shape[1]
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            T.copy_(src)
            sr.antidist_closure(ctx, T, ld, D, sr.SR_U16, s.cuda_stream)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            T.copy_(src)
            sr.antidist_closure(ctx, T, ld, D, sr.SR_U16, s.cuda_stream)
        for _ in range(2):
            T.fill_(0)
            g.replay()
            torch.cuda.synchronize()
            assert np.array_equal(to_host(T, dt)[:, :D], want)
        sr.sr_stream_status(ctx)
    finally:
        sr.sr_destroy(ctx)


def test_persistent_distance_closure():
    """dist_closure (Section 4 dual) takes the same schedule through De Morgan."""
    import torch
    import paper_1705_08743_gb300 as sr
    D, dt = 520, np.uint8
    rng = np.random.default_rng(21)
    A = rand_anti(rng, D, D, dt, 0.01, 200)
    Dm = (255 - A).astype(np.uint8)                          # distances, 255 = none
    want = oracle.dist_closure(Dm, 255)
    ctx = _ctx(D, dt)
    try:
        Td = to_dev(Dm, _aligned_pad(D, dt))
        n0 = sr.sr_kernel_launches()
        sr.dist_closure(ctx, Td, Td.shape[1], D, sr.SR_U8)
        torch.cuda.synchronize()
        assert sr.sr_kernel_launches() - n0 == 3               # complement, closure, complement
        assert np.array_equal(to_host(Td, dt)[:, :D], want)
    finally:
        sr.sr_destroy(ctx)


@pytest.mark.slow
@pytest.mark.parametrize("D", [4096, 8192])
def test_cfg2_persistent_closure_full_size(D):
    """The config-2 generator (p = 0.05, w ~ U{1..31}, seed 1) at D = 4096 (every entry
    against the oracle's Warshall) and D = 8192 (sampled rows against the oracle's
    single-source path search, and T ⊗ T ⊕ T = T on every entry), as the benchmark
    runs it: a context with the schedule's workspace."""
    import torch
    import paper_1705_08743_gb300 as sr
    W = synth.cfg2_antidist(D=D, seed=1)
    Wd = to_dev(W)
    Td = torch.empty_like(Wd)
    ctx = _ctx(D, np.uint8, mode=2)
    try:
        sr.antidist_encode(None, Wd, D, Td, D, D, D, sr.SR_U8)
        torch.cuda.synchronize()
        n0 = sr.sr_kernel_launches()
        sr.antidist_closure(ctx, Td, D, D, sr.SR_U8)
        torch.cuda.synchronize()
        assert sr.sr_kernel_launches() - n0 == 1
        sr.sr_stream_status(ctx)
        got = to_host(Td, np.uint8)
        A = oracle.encode_antidist(W, 255)
        if D == 4096:
            assert np.array_equal(got, oracle.warshall(A, 255))
        else:
            for src in [0, 1, 2047, 4096, 5555, 8191]:
                assert np.array_equal(got[src], oracle.closure_row(A, src, 255)), src
            Cd = Td.clone()
            sr.antidist_mul(None, Td, D, Td.clone(), D, Cd, D, D, D, D, sr.SR_U8, 1)
            assert torch.equal(Cd, Td)
    finally:
        sr.sr_destroy(ctx)
