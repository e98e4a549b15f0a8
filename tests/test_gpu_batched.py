"""Batched anti-distance closure (one persistent launch over many graphs)
against the oracle's Warshall closure of each graph; bit-exact."""

import numpy as np
import pytest

import oracle
import synth
from gpu_util import to_dev, to_host, sr_dtype_of

S_OF = {np.uint8: 255, np.uint16: 65535}


def rand_graph(rng, D, dt, lo_frac):
    S = S_OF[dt]
    p = min(1.0, 6.0 / D)
    lo = max(1, int(S * lo_frac))
    v = rng.integers(lo, S + 1, size=(D, D), dtype=np.int64)
    return np.where(rng.random((D, D)) < p, v, 0).astype(dt)


def make_batch(sizes, dt, seed):
    rng = np.random.default_rng(seed)
    return [rand_graph(rng, D, dt, 0.6 if i % 2 else 0.97) for i, D in enumerate(sizes)]


def run_batch(mats, tuning=None, use_graph=False, autotune=False, ctx=None, launches=1, pad=0, align=False):
    """align: pad every row to a multiple of 16 bytes (vector path for all graphs)."""
    from paper_1705_08743_gb300 import _capi as sr
    dt = mats[0].dtype.type
    per = 16 // np.dtype(dt).itemsize
    devs = [to_dev(M, (-M.shape[0]) % per if align else pad) for M in mats]
    descs = [sr.closure_desc(T, T.shape[1], M.shape[0], sr_dtype_of(dt)) for T, M in zip(devs, mats)]
    b = sr.sr_batch_create(ctx, descs)
    try:
        if tuning:
            sr.sr_batch_set_tuning(b, *tuning)
        if autotune:
            sr.sr_batch_autotune(ctx, b, reps=1)
        for _ in range(launches):
            sr.sr_batch_launch(b, use_graph)
        import torch
        torch.cuda.synchronize()
    finally:
        sr.sr_batch_destroy(b)
    return [to_host(T, dt)[:, :M.shape[0]] for T, M in zip(devs, mats)]


SIZES = [1, 5, 31, 32, 33, 64, 65, 100, 127, 128, 129, 200, 257, 300, 450, 513, 700]


@pytest.mark.gpu
@pytest.mark.parametrize("dt", [np.uint16, np.uint8])
@pytest.mark.parametrize("tuning", [(1, 1 << 30, 1), (2, 128, 2), (4, 256, 1), (4, 64, 2), (2, 1, 1), (0, 1, 1)])
@pytest.mark.parametrize("align", [False, True])
def test_batched_matches_oracle(dt, tuning, align):
    """Persistent kernel (clusters of 1, 2 or 4 CTAs, cooperative thresholds) and the
    grouped schedule (cluster 0: launches per pivot block over all graphs)."""
    mats = make_batch(SIZES, dt, seed=len(SIZES) + tuning[0] * 10 + tuning[1] % 97)
    got = run_batch(mats, tuning=tuning, align=align)
    S = S_OF[dt]
    for M, G in zip(mats, got):
        assert np.array_equal(G, oracle.warshall(M, S)), f"D={M.shape[0]}"


@pytest.mark.gpu
def test_batched_graph_replay_autotune_and_padding():
    from paper_1705_08743_gb300 import _capi as sr
    mats = make_batch([40, 300, 77, 640, 128, 9], np.uint16, seed=3)
    ctx = sr.sr_create()
    try:
        got = run_batch(mats, use_graph=True, launches=3, autotune=True, ctx=ctx, pad=5)
        for M, G in zip(mats, got):
            assert np.array_equal(G, oracle.warshall(M, 65535))
        # a second batch with the same signature reuses the recorded tuning
        got = run_batch(make_batch([40, 300, 77, 640, 128, 9], np.uint16, seed=4), autotune=True, ctx=ctx)
    finally:
        sr.sr_destroy(ctx)


@pytest.mark.gpu
def test_batched_grouped_schedule_in_cuda_graph():
    """The grouped schedule captured once into a CUDA graph and replayed on closed graphs
    (idempotent), with a mix of single-block and multi-block graphs and unaligned rows."""
    mats = make_batch([3, 128, 129, 600, 1000, 64, 257], np.uint16, seed=9)
    got = run_batch(mats, tuning=(0, 1, 1), use_graph=True, launches=2, pad=3)
    for M, G in zip(mats, got):
        assert np.array_equal(G, oracle.warshall(M, 65535)), f"D={M.shape[0]}"


@pytest.mark.gpu
@pytest.mark.parametrize("tuning", [(2, 256, 2), (0, 1, 1)])
@pytest.mark.parametrize("use_graph", [0, 1])
def test_batched_completion_times(tuning, use_graph):
    """Per-graph completion stamps (sr_batch_set_timing): every graph gets a time within
    the launch, the grouped schedule's graphs finish no earlier than the graphs with
    fewer pivot steps, the persistent kernel's graphs no later than the whole launch,
    and the results are unchanged."""
    import torch
    from paper_1705_08743_gb300 import _capi as sr
    sizes = [5, 64, 129, 300, 700, 1000, 33, 257]
    mats = make_batch(sizes, np.uint16, seed=17)
    devs = [to_dev(M) for M in mats]
    descs = [sr.closure_desc(T, T.shape[1], M.shape[0], sr.SR_U16) for T, M in zip(devs, mats)]
    b = sr.sr_batch_create(None, descs)
    try:
        sr.sr_batch_set_tuning(b, *tuning)
        with pytest.raises(sr.SemiringError):
            sr.sr_batch_completion_ms(b)                           # timing off
        sr.sr_batch_set_timing(b, True)
        s = torch.cuda.Stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(s):
            e0.record(s)
            sr.sr_batch_launch(b, use_graph, s.cuda_stream)
            e1.record(s)
        torch.cuda.synchronize()
        total = e0.elapsed_time(e1)
        ms = sr.sr_batch_completion_ms(b)
        assert len(ms) == len(sizes)
        assert all(0.0 <= t <= total + 0.05 for t in ms), (ms, total)
        if tuning[0] == 0:                                         # step ends are ordered by pivot steps
            steps = [(D + 127) // 128 for D in sizes]
            for i in range(len(sizes)):
                for j in range(len(sizes)):
                    if steps[i] < steps[j]:
                        assert ms[i] <= ms[j]
        sr.sr_batch_set_timing(b, False)
        sr.sr_batch_launch(b, use_graph, s.cuda_stream)
        torch.cuda.synchronize()
    finally:
        sr.sr_batch_destroy(b)
    for M, T in zip(mats, devs):
        assert np.array_equal(to_host(T, np.uint16), oracle.warshall(M, 65535))


@pytest.mark.gpu
def test_sr_batched_one_shot():
    from paper_1705_08743_gb300 import _capi as sr
    mats = make_batch([10, 90, 260], np.uint8, seed=5)
    devs = [to_dev(M) for M in mats]
    sr.sr_batched(None, [sr.closure_desc(T, T.shape[1], M.shape[0], sr.SR_U8) for T, M in zip(devs, mats)])
    for M, T in zip(mats, devs):
        assert np.array_equal(to_host(T, np.uint8), oracle.warshall(M, 255))


def test_batch_rejects_overlap_and_mixed_dtypes():
    from paper_1705_08743_gb300 import _capi as sr
    # validated before any device work: runs without a GPU
    a = sr.closure_desc(1 << 20, 100, 100, sr.SR_U16)
    b = sr.closure_desc((1 << 20) + 1000, 100, 100, sr.SR_U16)
    with pytest.raises(sr.SemiringError) as e:
        sr.sr_batch_create(None, [a, b])
    assert e.value.status == sr.SR_EINVAL and "overlap" in str(e.value)
    c = sr.closure_desc(1 << 24, 100, 100, sr.SR_U8)
    with pytest.raises(sr.SemiringError):
        sr.sr_batch_create(None, [a, c])
    d = sr.closure_desc(1 << 24, 100, 100, sr.SR_U32)      # the batched kernel has 16-bit lanes only
    with pytest.raises(sr.SemiringError) as e:
        sr.sr_batch_create(None, [d])
    assert e.value.status == sr.SR_EINVAL


@pytest.mark.gpu
@pytest.mark.slow
def test_cfg4_batched_full():
    """2000 graphs, D log-uniform in [32, 1024], u16, lengths U{1..4000}, p = 8/D, seed 3."""
    import torch
    from paper_1705_08743_gb300 import _capi as sr
    sizes, W = synth.cfg4_batched()
    mats = [oracle.encode_antidist(w, 65535).astype(np.uint16) for w in W]
    ctx = sr.sr_create()
    try:
        got = run_batch(mats, autotune=False, ctx=ctx, tuning=(4, 384, 1))
    finally:
        sr.sr_destroy(ctx)
    for M, G in zip(mats, got):
        assert np.array_equal(G, oracle.warshall(M, 65535)), f"D={M.shape[0]}"
