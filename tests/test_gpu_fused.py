"""The anti-distance closure's fused-pass schedule (SR_OPT_CLOSURE_FUSED) on the GPU,
through the C ABI, against the CPU oracle's Warshall closure (Section 2 Warshall,
Section 3 Floyd), bit for bit.

The schedule takes one launch per 128-wide pivot block plus one for block 0's phases
1-2; inside a launch the next block's closure, strips and panels are work items beside
phase 3, the panels waiting (bounded) for the first two.  The checks count launches too.
"""

import numpy as np
import pytest

import oracle
import synth
from gpu_util import to_dev, to_host, sr_dtype_of

pytestmark = pytest.mark.gpu

S_OF = {np.uint8: 255, np.uint16: 65535, np.uint32: 2 ** 32 - 1}


def rand_anti(rng, R, C, dt, density, lo=1):
    S = S_OF[dt]
    v = rng.integers(lo, S + 1, size=(R, C), dtype=np.int64)
    return np.where(rng.random((R, C)) < density, v, 0).astype(dt)


def _aligned_pad(D, dt):
    per = 16 // np.dtype(dt).itemsize
    return (-D) % per


def _ctx(D, dt, mode=2):
    import paper_1705_08743_gb300 as sr
    ws = sr.sr_workspace_query(sr.SR_OP_ANTIDIST_CLOSURE, sr_dtype_of(dt), D)
    ctx = sr.sr_create(workspace_bytes=max(ws, 1 << 16))
    sr.sr_set_option(ctx, sr.SR_OPT_CLOSURE_FUSED, mode)
    return ctx


def _close(ctx, A, pad, stream=None):
    import torch
    import paper_1705_08743_gb300 as sr
    dt = A.dtype.type
    D = A.shape[0]
    Td = to_dev(A, pad)
    torch.cuda.synchronize()
    n0 = sr.sr_kernel_launches()
    sr.antidist_closure(ctx, Td, Td.shape[1], D, sr_dtype_of(dt), stream)
    torch.cuda.synchronize()
    launches = sr.sr_kernel_launches() - n0
    sr.sr_stream_status(ctx)
    out = to_host(Td, dt)
    if pad:
        assert (out[:, D:] == 0xA5).all(), "wrote past the row width"
    return out[:, :D], launches


def _fused_launches(D):
    nb = (D + 127) // 128
    last_p3 = (D - (D - (nb - 1) * 128) + 127) // 128           # tiles per side of the last pass
    return 1 + (nb - 1) + (1 if last_p3 > 0 else 0)


@pytest.mark.parametrize("dt", [np.uint8, np.uint16])
@pytest.mark.parametrize("D", [1, 100, 128, 129, 300, 1000, 2085, 3600])
def test_fused_closure_random(dt, D):
    """Ragged last blocks (D = 129, 300, 1000, 2085, 3600), a single block (D <= 128),
    long sparse paths and dense input."""
    rng = np.random.default_rng(D * 3 + np.dtype(dt).itemsize)
    S = S_OF[dt]
    ctx = _ctx(D, dt)
    try:
        for dens, lo in [(3.0 / max(D, 1), S - S // 8), (0.05, 1)]:
            A = rand_anti(rng, D, D, dt, dens, lo)
            got, launches = _close(ctx, A, _aligned_pad(D, dt))
            assert launches == _fused_launches(D), (launches, D)
            assert np.array_equal(got, oracle.warshall(A, S)), (dens, lo)
    finally:
        import paper_1705_08743_gb300 as sr
        sr.sr_destroy(ctx)


def test_fused_closure_cfg2_4096_in_full():
    """The benchmark's workload (config-2 generator, D = 4096 u8) on every entry."""
    import paper_1705_08743_gb300 as sr
    D = 4096
    A = oracle.encode_antidist(synth.cfg2_antidist(D=D, seed=1, s_edge=0), 255).astype(np.uint8)
    ctx = _ctx(D, np.uint8)
    try:
        got, launches = _close(ctx, A, 0)
        assert launches == 33
        assert np.array_equal(got, oracle.warshall(A, 255))
    finally:
        sr.sr_destroy(ctx)


def test_fused_closure_follows_option_tuned_choice_and_falls_back():
    """Option 0 keeps the stream schedule; a recorded SR_TUNE_FUSED choice steers an
    automatic call; unaligned rows, a short workspace and u32 take the stream schedule
    with the same result."""
    import paper_1705_08743_gb300 as sr
    D, dt = 1000, np.uint8
    rng = np.random.default_rng(5)
    A = rand_anti(rng, D, D, dt, 3.0 / D, 220)
    want = oracle.warshall(A, 255)
    ctx = _ctx(D, dt, mode=0)
    try:
        got, n = _close(ctx, A, _aligned_pad(D, dt))
        assert n != _fused_launches(D) and np.array_equal(got, want)
        sr.sr_set_option(ctx, sr.SR_OPT_CLOSURE_FUSED, 1)
        sr.sr_set_option(ctx, sr.SR_OPT_CLOSURE_PERSISTENT, 0)
        sr.sr_tune_set(ctx, sr.SR_OP_ANTIDIST_CLOSURE, sr.SR_U8, D, sr.SR_TUNE_FUSED)
        got, n = _close(ctx, A, _aligned_pad(D, dt))
        assert n != _fused_launches(D)                      # persistent option not automatic: no record used
        sr.sr_set_option(ctx, sr.SR_OPT_CLOSURE_PERSISTENT, 1)
        got, n = _close(ctx, A, _aligned_pad(D, dt))
        assert n == _fused_launches(D) and np.array_equal(got, want)
        sr.sr_set_option(ctx, sr.SR_OPT_CLOSURE_FUSED, 2)
        got, n = _close(ctx, A, 3)                          # rows not 16-byte multiples
        assert n != _fused_launches(D) and np.array_equal(got, want)
        with pytest.raises(sr.SemiringError):
            sr.sr_tune_set(ctx, sr.SR_OP_ANTIDIST_CLOSURE, sr.SR_U32, D, sr.SR_TUNE_FUSED)
    finally:
        sr.sr_destroy(ctx)
    small = sr.sr_create(workspace_bytes=16)
    try:
        sr.sr_set_option(small, sr.SR_OPT_CLOSURE_FUSED, 2)
        got, n = _close(small, A, _aligned_pad(D, dt))
        assert n != _fused_launches(D) and np.array_equal(got, want)
    finally:
        sr.sr_destroy(small)
    A32 = rand_anti(rng, 300, 300, np.uint32, 0.02)
    ctx = _ctx(300, np.uint32)
    try:
        got, n = _close(ctx, A32, 0)
        assert np.array_equal(got, oracle.warshall(A32, 2 ** 32 - 1))
    finally:
        sr.sr_destroy(ctx)


def test_fused_closure_timeout_then_rerun():
    """A spin limit of 0 makes the panels' wait give up at its first unmet try: the
    launches end, sr_stream_status reports SR_ETIMEOUT once, and the context then closes
    the same input correctly."""
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
        assert launches == _fused_launches(D) and np.array_equal(got, oracle.warshall(A, 255))
    finally:
        sr.sr_destroy(ctx)


def test_fused_closure_captured_in_cuda_graph():
    """One stream, no events: the schedule captures into a CUDA graph whose replays close
    fresh input; the eager run is checked too."""
    import torch
    import paper_1705_08743_gb300 as sr
    D, dt = 1500, np.uint16
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
        assert np.array_equal(to_host(T, dt)[:, :D], want)
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
