"""Anti-distance product and closure on the GPU (through the C ABI) against
the CPU oracle, element by element.  All arithmetic is integer: bit-exact."""

import numpy as np
import pytest

import oracle
import synth
from gpu_util import to_dev, to_host, sr_dtype_of

pytestmark = pytest.mark.gpu

S_OF = {np.uint8: 255, np.uint16: 65535, np.uint32: 2 ** 32 - 1}
DTS = [np.uint8, np.uint16, np.uint32]


def rand_anti(rng, R, C, dt, density, lo=1):
    S = S_OF[dt]
    v = rng.integers(lo, S + 1, size=(R, C), dtype=np.int64)
    return np.where(rng.random((R, C)) < density, v, 0).astype(dt)


def gpu_mul(A, B, C0=None, pad=(0, 0, 0)):
    import paper_1705_08743_gb300 as sr
    dt = A.dtype.type
    R, K = A.shape
    N = B.shape[1]
    Ad, Bd = to_dev(A, pad[0]), to_dev(B, pad[1])
    Cd = to_dev(np.zeros((R, N), dt) if C0 is None else C0, pad[2])
    sr.antidist_mul(None, Ad, Ad.shape[1], Bd, Bd.shape[1], Cd, Cd.shape[1], R, K, N, sr_dtype_of(dt),
                    0 if C0 is None else 1)
    out = to_host(Cd, dt)
    if pad[2]:
        assert (out[:, N:] == 0xA5).all(), "wrote past the row width"
    return out[:, :N]


def gpu_closure(A, pad=0):
    import paper_1705_08743_gb300 as sr
    dt = A.dtype.type
    D = A.shape[0]
    Td = to_dev(A, pad)
    sr.antidist_closure(None, Td, Td.shape[1], D, sr_dtype_of(dt))
    return to_host(Td, dt)[:, :D]


@pytest.mark.parametrize("dt", DTS)
@pytest.mark.parametrize("shape", [(1, 1, 1), (7, 13, 5), (128, 64, 128), (200, 300, 257),
                                   (129, 33, 130), (513, 77, 1000), (64, 1, 64)])
def test_mul_random(dt, shape):
    R, K, N = shape
    rng = np.random.default_rng(R * 7 + K * 3 + N)
    S = S_OF[dt]
    for dens, lo in [(0.5, 1), (0.9, S - S // 8)]:
        A, B = rand_anti(rng, R, K, dt, dens, lo), rand_anti(rng, K, N, dt, dens, lo)
        ref = oracle.mul(A, B, S)
        assert np.array_equal(gpu_mul(A, B), ref)
        C0 = rand_anti(rng, R, N, dt, 0.5)
        assert np.array_equal(gpu_mul(A, B, C0), oracle.mul(A, B, S, C=C0))


@pytest.mark.parametrize("dt", DTS)
def test_mul_unaligned_leading_dims(dt):
    rng = np.random.default_rng(3)
    A, B = rand_anti(rng, 70, 45, dt, 0.6), rand_anti(rng, 45, 99, dt, 0.6)
    S = S_OF[dt]
    assert np.array_equal(gpu_mul(A, B, pad=(3, 5, 7)), oracle.mul(A, B, S))
    C0 = rand_anti(rng, 70, 99, dt, 0.4)
    assert np.array_equal(gpu_mul(A, B, C0, pad=(16, 32, 9)), oracle.mul(A, B, S, C=C0))


@pytest.mark.parametrize("dt", DTS)
def test_mul_special_matrices(dt):
    S = S_OF[dt]
    rng = np.random.default_rng(4)
    n = 96
    I = (np.eye(n) * S).astype(dt)
    A = rand_anti(rng, n, n, dt, 0.5)
    assert np.array_equal(gpu_mul(I, A), A)                       # identity
    assert np.array_equal(gpu_mul(A, I), A)
    Z = np.zeros((n, n), dt)
    assert np.array_equal(gpu_mul(A, Z), Z)                       # zero absorbs
    F = np.full((n, n), S, dt)
    assert np.array_equal(gpu_mul(F, F), F)                       # all-S
    ones = np.ones((n, n), dt)                                    # lengths S-1: saturate
    assert np.array_equal(gpu_mul(ones, ones), oracle.mul(ones, ones, S))


@pytest.mark.parametrize("dt", [np.uint8, np.uint16])
def test_mul_more_than_one_wave(dt):
    """24 x 24 tiles of 128: more tiles than resident CTAs, a sparse last wave, ragged
    edges, accumulation and a padded C."""
    rng = np.random.default_rng(31)
    S = S_OF[dt]
    R, K, N = 3000, 40, 2990
    A, B = rand_anti(rng, R, K, dt, 0.5), rand_anti(rng, K, N, dt, 0.5)
    assert np.array_equal(gpu_mul(A, B), oracle.mul(A, B, S))
    C0 = rand_anti(rng, R, N, dt, 0.3)
    assert np.array_equal(gpu_mul(A, B, C0, pad=(0, 0, 8)), oracle.mul(A, B, S, C=C0))


@pytest.mark.parametrize("dt", [np.uint8, np.uint16])
@pytest.mark.parametrize("shape", [(1000, 1100, 1000), (2816, 1024, 2704)])
def test_mul_deep_last_wave_split_along_k(dt, shape):
    """Deep products (K >= 1024) whose last wave of CTAs is partial: its tiles are shared
    by thread-block clusters over slices of K and merged through distributed shared memory
    (64 tiles, all split two ways, ragged R, N and K; 22 x 22 tiles: for u8 one full wave
    of 456 CTAs plus a tail of 28 split four ways, for u16 a last wave of 180 tiles, too
    full to split).  Equal to the oracle with and without accumulation, and to the unsplit
    launch (SR_OPT_PRODUCT_SPLIT = 0), which takes one launch where the split takes two."""
    import torch
    import paper_1705_08743_gb300 as sr
    rng = np.random.default_rng(shape[0] + shape[1])
    S = S_OF[dt]
    R, K, N = shape
    A, B = rand_anti(rng, R, K, dt, 0.3), rand_anti(rng, K, N, dt, 0.3)
    C0 = rand_anti(rng, R, N, dt, 0.2)
    want0, want1 = oracle.mul(A, B, S), oracle.mul(A, B, S, C=C0)
    ctx = sr.sr_create()
    try:
        Ad, Bd = to_dev(A), to_dev(B)
        launches = {}
        for split in (1, 0):
            sr.sr_set_option(ctx, sr.SR_OPT_PRODUCT_SPLIT, split)
            for C_init, want in ((None, want0), (C0, want1)):
                Cd = to_dev(np.zeros((R, N), dt) if C_init is None else C_init)
                torch.cuda.synchronize()
                n0 = sr.sr_kernel_launches()
                sr.antidist_mul(ctx, Ad, Ad.shape[1], Bd, Bd.shape[1], Cd, Cd.shape[1], R, K, N,
                                sr_dtype_of(dt), 0 if C_init is None else 1)
                torch.cuda.synchronize()
                launches[split] = sr.sr_kernel_launches() - n0
                assert np.array_equal(to_host(Cd, dt)[:, :N], want), (split, C_init is None)
        tiles = ((R + 127) // 128) * ((N + 127) // 128)
        # resident CTAs per SM: u8 3 (registers), u16 2 (112 KB of shared memory each); the
        # tail splits at least two ways while that keeps one split CTA per SM
        sms = torch.cuda.get_device_properties(0).multi_processor_count
        slots = (3 if dt == np.uint8 else 2) * sms
        tail = tiles % slots
        assert launches[0] == 1
        assert launches[1] == (2 if tiles > slots and 0 < 2 * tail <= sms else 1)
        with pytest.raises(sr.SemiringError):
            sr.sr_set_option(ctx, sr.SR_OPT_PRODUCT_SPLIT, 2)
    finally:
        sr.sr_destroy(ctx)


@pytest.mark.parametrize("dt", [np.uint8, np.uint16])
def test_closure_24_pivot_blocks(dt):
    """D = 3072: 24 pivot blocks, each phase 3 more than one wave of 128x128 tiles, with
    the look-ahead chain of the next block running beside it on the side stream."""
    rng = np.random.default_rng(32)
    S = S_OF[dt]
    D = 3072
    A = rand_anti(rng, D, D, dt, 2.0 / D, S - S // 10)
    assert np.array_equal(gpu_closure(A), oracle.warshall(A, S))


def test_mul_u32_carry_edge():
    """u32: a ⊗ b = max(a + b − S, 0) with a + b up to 2^33 − 2.  Every pair of a set
    of values around the carry edge (a + b = S, S ± 1) and the extremes, as an outer
    product (K = 1) and summed over K = 40 with each pair once per k."""
    S = 2 ** 32 - 1
    rng = np.random.default_rng(12)
    v = np.concatenate([[0, 1, 2, 2 ** 31 - 1, 2 ** 31, 2 ** 31 + 1, 2 ** 32 - 2 ** 16, 2 ** 16, S - 1, S],
                        rng.integers(0, S + 1, 30, dtype=np.int64)]).astype(np.uint32)
    P = gpu_mul(v[:, None].copy(), v[None, :].copy())
    vi = v.astype(np.int64)
    assert np.array_equal(P.astype(np.int64), np.maximum(vi[:, None] + vi[None, :] - S, 0))
    A = np.tile(v[:, None], (1, 40))                               # row i: a_i in every k
    B = np.stack([np.roll(v, k) for k in range(40)])               # row k: v shifted by k
    assert np.array_equal(gpu_mul(A, B), oracle.mul(A, B, S))


@pytest.mark.parametrize("dt", DTS)
@pytest.mark.parametrize("D", [1, 2, 31, 33, 63, 64, 65, 127, 129, 200, 333])
def test_closure_random(dt, D):
    rng = np.random.default_rng(D)
    S = S_OF[dt]
    for dens, lo in [(min(1.0, 3.0 / D), S - S // 6), (0.3, 1), (min(1.0, 1.2 / D), S - 3)]:
        A = rand_anti(rng, D, D, dt, dens, lo)
        assert np.array_equal(gpu_closure(A), oracle.warshall(A, S)), (dens, lo)


@pytest.mark.parametrize("dt", DTS)
@pytest.mark.parametrize("D", [256, 257, 385, 640, 1100])
def test_closure_many_pivot_blocks(dt, D):
    """Several 128-wide pivot blocks: exercises the look-ahead (next pivot's panels
    on a second stream while the rest of phase 3 runs) and ragged last blocks."""
    rng = np.random.default_rng(D + 7)
    S = S_OF[dt]
    for dens, lo in [(2.0 / D, S - S // 10), (0.05, 1)]:
        A = rand_anti(rng, D, D, dt, dens, lo)
        assert np.array_equal(gpu_closure(A), oracle.warshall(A, S)), (dens, lo)


@pytest.mark.parametrize("D,dt", [(4700, np.uint8), (3700, np.uint16)])
def test_closure_phase3_on_two_main_streams(D, dt):
    """Look-ahead schedules with enough phase-3 work per pass that each pass is split at
    a tile-row boundary over the caller's stream and a peer stream (u8 D=4700: 35 x 35
    tiles a pass; u16 D=3700: 27 x 27 two-byte tiles), with a ragged last block: equal
    to the oracle's Warshall/Floyd closure, for long sparse paths and for dense input."""
    rng = np.random.default_rng(D)
    S = S_OF[dt]
    for dens, lo in [(3.0 / D, S - S // 8), (0.05, 1)]:
        A = rand_anti(rng, D, D, dt, dens, lo)
        assert np.array_equal(gpu_closure(A), oracle.warshall(A, S)), (dens, lo)


_WANT = {}


def _warshall_cached(A, S, key):
    if key not in _WANT:
        _WANT[key] = oracle.warshall(A, S)
    return _WANT[key]


@pytest.mark.parametrize("dt", DTS)
@pytest.mark.parametrize("width", [128, 256, 512])
@pytest.mark.parametrize("D", [100, 300, 777, 1100, 2000])
def test_closure_block_width(dt, width, D):
    """Every block width of the blocked closure (SR_OPT_CLOSURE_BLOCK): widths 256 and
    512 close each diagonal block by a nested 128-wide closure on the pivot side stream
    and run the look-ahead schedule at any size; one block, ragged last blocks, many
    blocks."""
    import paper_1705_08743_gb300 as sr
    rng = np.random.default_rng(D * 3 + 1)
    S = S_OF[dt]
    A = rand_anti(rng, D, D, dt, 2.0 / D, S - S // 10)
    want = _warshall_cached(A, S, (dt, D))
    ctx = sr.sr_create()
    try:
        sr.sr_set_option(ctx, sr.SR_OPT_CLOSURE_BLOCK, width)
        Td = to_dev(A, 3 if D == 777 else 0)
        sr.antidist_closure(ctx, Td, Td.shape[1], D, sr_dtype_of(dt))
        assert np.array_equal(to_host(Td, dt)[:, :D], want)
    finally:
        sr.sr_destroy(ctx)


def test_closure_block_width_rejects_other_values():
    import paper_1705_08743_gb300 as sr
    ctx = sr.sr_create()
    try:
        for bad in (-1, 64, 100, 1024):
            with pytest.raises(sr.SemiringError) as e:
                sr.sr_set_option(ctx, sr.SR_OPT_CLOSURE_BLOCK, bad)
            assert e.value.status == sr.SR_EINVAL
        sr.sr_set_option(ctx, sr.SR_OPT_CLOSURE_BLOCK, 0)
    finally:
        sr.sr_destroy(ctx)


@pytest.mark.parametrize("dt", DTS)
def test_closure_unaligned_ld(dt):
    rng = np.random.default_rng(8)
    A = rand_anti(rng, 150, 150, dt, 0.05, S_OF[dt] - 40)
    assert np.array_equal(gpu_closure(A, pad=5), oracle.warshall(A, S_OF[dt]))


@pytest.mark.parametrize("dt", DTS)
def test_closure_edge_cases(dt):
    S = S_OF[dt]
    D = 300
    Z = np.zeros((D, D), dt)
    assert np.array_equal(gpu_closure(Z), Z)
    F = np.full((D, D), S, dt)
    assert np.array_equal(gpu_closure(F), F)
    I = (np.eye(D) * S).astype(dt)
    assert np.array_equal(gpu_closure(I), I)
    # a single long chain 0 -> 1 -> ... -> D-1 -> 0 of length-1 edges: saturates for u8
    C = np.zeros((D, D), dt)
    for i in range(D):
        C[i, (i + 1) % D] = S - 1
    assert np.array_equal(gpu_closure(C), oracle.warshall(C, S))
    # reversed chain (pivot order stress)
    assert np.array_equal(gpu_closure(C.T.copy()), oracle.warshall(C.T.copy(), S))


@pytest.mark.parametrize("dt", DTS)
@pytest.mark.parametrize("shape", [(37, 101, 0), (40, 256, 0), (33, 100, -1), (5, 3, 13)])
def test_encode_matches_oracle(dt, shape):
    """Unaligned rows (scalar path), aligned rows (16-byte chunks), aligned rows with a
    ragged tail (pad -1: leading dimension rounded up to 16 bytes plus one chunk), and
    in place; the extremes 0, 1, S-1, S in every case."""
    import paper_1705_08743_gb300 as sr
    R, C, pad = shape
    S = S_OF[dt]
    if pad < 0:
        ch = 16 // np.dtype(dt).itemsize
        pad = (-C) % ch + ch
    rng = np.random.default_rng(C)
    W = rng.integers(0, S + 1, size=(R, C), dtype=np.int64).astype(dt)
    W[0, :min(4, C)] = [0, 1, S - 1, S][:min(4, C)]
    want = oracle.encode_antidist(W, S).astype(dt)
    Wd, Td = to_dev(W, pad), to_dev(np.zeros_like(W), pad)
    sr.antidist_encode(None, Wd, Wd.shape[1], Td, Td.shape[1], R, C, sr_dtype_of(dt))
    out = to_host(Td, dt)
    assert np.array_equal(out[:, :C], want)
    if pad:
        assert (out[:, C:] == 0xA5).all(), "wrote past the row width"
    sr.antidist_encode(None, Wd, Wd.shape[1], Wd, Wd.shape[1], R, C, sr_dtype_of(dt))     # in place
    assert np.array_equal(to_host(Wd, dt)[:, :C], want)


# ---------------------------------------------------------------- full size
@pytest.mark.slow
def test_cfg2_closure_full_4096():
    """Anti-distance closure D=4096 u8 (p=0.05, w ~ U{1..31}, seed 1): whole
    matrix against the oracle's Warshall, plus sampled rows against the
    oracle's single-source path search."""
    import torch
    import paper_1705_08743_gb300 as sr
    D = 4096
    W = synth.cfg2_antidist(D=D, seed=1)
    Wd = to_dev(W)
    Td = torch.empty_like(Wd)
    sr.antidist_encode(None, Wd, D, Td, D, D, D, sr.SR_U8)
    sr.antidist_closure(None, Td, D, D, sr.SR_U8)
    got = to_host(Td, np.uint8)
    A = oracle.encode_antidist(W, 255)
    ref = oracle.warshall(A, 255)
    assert np.array_equal(got, ref)
    for src in [0, 1, 777, 2048, 4095]:
        assert np.array_equal(got[src], oracle.closure_row(A, src, 255))


@pytest.mark.slow
def test_cfg2_product_full_4096():
    import torch
    import paper_1705_08743_gb300 as sr
    D = 4096
    A = oracle.encode_antidist(synth.cfg2_antidist(D=D, seed=1, s_edge=0), 255).astype(np.uint8)
    B = oracle.encode_antidist(synth.cfg2_antidist(D=D, seed=1, s_edge=3), 255).astype(np.uint8)
    Ad, Bd = to_dev(A), to_dev(B)
    Cd = torch.zeros((D, D), dtype=torch.uint8, device="cuda")
    sr.antidist_mul(None, Ad, D, Bd, D, Cd, D, D, D, D, sr.SR_U8, 0)
    got = to_host(Cd, np.uint8)
    ref = oracle.mul(A, B, 255)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("D,dt", [(700, np.uint8), (3600, np.uint16)])
def test_closure_captured_in_cuda_graph(D, dt):
    """The closure's side streams fork from and join back into the caller's stream, so
    it can be captured into a CUDA graph (two-stream schedule at D=700, look-ahead at
    D=3600 with 29 pivot blocks) and replayed; each replay closes fresh input."""
    import torch
    import paper_1705_08743_gb300 as sr
    S = S_OF[dt]
    rng = np.random.default_rng(D)
    A = rand_anti(rng, D, D, dt, 3.0 / D, S - S // 8)
    want = oracle.warshall(A, S)
    src = to_dev(A)
    T = torch.empty_like(src)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        T.copy_(src)
        sr.antidist_closure(None, T, D, D, sr_dtype_of(dt), s.cuda_stream)      # warm-up outside capture
    torch.cuda.synchronize()
    assert np.array_equal(to_host(T, dt), want)                                 # the eager run, too
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        T.copy_(src)
        sr.antidist_closure(None, T, D, D, sr_dtype_of(dt), s.cuda_stream)
    for _ in range(2):
        T.fill_(0)
        g.replay()
        torch.cuda.synchronize()
        assert np.array_equal(to_host(T, dt), want)


@pytest.mark.slow
def test_cfg2_closure_8192_sampled_rows_and_idempotence():
    """Closure D=8192 u8 (the same generator at twice the size), as the benchmark runs
    it: rows sampled across the matrix against the oracle's single-source path search,
    and on every entry the closure property T ⊗ T ⊕ T = T (checked with the product
    kernel, a different kernel from the closure's phase 3 launches)."""
    import torch
    import paper_1705_08743_gb300 as sr
    D = 8192
    W = synth.cfg2_antidist(D=D, seed=1)
    Wd = to_dev(W)
    Td = torch.empty_like(Wd)
    sr.antidist_encode(None, Wd, D, Td, D, D, D, sr.SR_U8)
    sr.antidist_closure(None, Td, D, D, sr.SR_U8)
    got = to_host(Td, np.uint8)
    A = oracle.encode_antidist(W, 255)
    for src in [0, 1, 2047, 4096, 5555, 8191]:
        assert np.array_equal(got[src], oracle.closure_row(A, src, 255)), src
    Cd = Td.clone()
    sr.antidist_mul(None, Td, D, Td.clone(), D, Cd, D, D, D, D, sr.SR_U8, 1)
    assert torch.equal(Cd, Td)


@pytest.mark.slow
def test_cfg2_product_8192_sampled_entries():
    """Product 8192^3 u8: 3000 entries sampled uniformly, each against the oracle's
    formula evaluated for that entry alone."""
    import torch
    import paper_1705_08743_gb300 as sr
    D = 8192
    A = oracle.encode_antidist(synth.cfg2_antidist(D=D, seed=1, s_edge=0), 255).astype(np.uint8)
    B = oracle.encode_antidist(synth.cfg2_antidist(D=D, seed=1, s_edge=3), 255).astype(np.uint8)
    Cd = torch.zeros((D, D), dtype=torch.uint8, device="cuda")
    sr.antidist_mul(None, to_dev(A), D, to_dev(B), D, Cd, D, D, D, D, sr.SR_U8, 0)
    got = to_host(Cd, np.uint8)
    rng = np.random.default_rng(8192)
    for i, j in zip(rng.integers(0, D, 3000), rng.integers(0, D, 3000)):
        assert got[i, j] == oracle.mul_entry(A, B, int(i), int(j), 255), (i, j)


@pytest.mark.slow
def test_u32_closure_4096_sampled_rows():
    """The u32 benchmark workload (D=4096, lengths 1..31, S = 2^32 - 1): sampled rows
    against single-source path search."""
    import torch
    import paper_1705_08743_gb300 as sr
    D, S = 4096, 2 ** 32 - 1
    W = synth.cfg2_antidist(D=D, seed=1, dtype=np.uint32)
    Wd = to_dev(W)
    Td = torch.empty_like(Wd)
    sr.antidist_encode(None, Wd, D, Td, D, D, D, sr.SR_U32)
    sr.antidist_closure(None, Td, D, D, sr.SR_U32)
    got = to_host(Td, np.uint32)
    A = oracle.encode_antidist(W, S)
    for src in [0, 777, 4095]:
        assert np.array_equal(got[src], oracle.closure_row(A, src, S)), src


def test_closures_from_two_host_threads():
    """Two host threads close different graphs at the same time, each on its own stream,
    with both schedules (two streams at D=1100, look-ahead at D=3600): the side streams
    are shared by every caller, the event pools are per thread, and every wait refers to
    work enqueued earlier, so the calls interleave without a cycle and stay bit-exact."""
    import threading
    import torch
    import paper_1705_08743_gb300 as sr
    cases = [(1100, np.uint8, 41), (3600, np.uint8, 42), (1100, np.uint16, 43), (3600, np.uint16, 44)]
    inputs = []
    for D, dt, seed in cases:
        rng = np.random.default_rng(seed)
        S = S_OF[dt]
        A = rand_anti(rng, D, D, dt, 3.0 / D, S - S // 8)
        inputs.append((D, dt, A, oracle.warshall(A, S)))
    errors = []

    def worker(items):
        try:
            s = torch.cuda.Stream()
            with torch.cuda.stream(s):
                for D, dt, A, want in items:
                    T = to_dev(A)
                    for _ in range(2):
                        sr.antidist_closure(None, T, D, D, sr_dtype_of(dt), s.cuda_stream)
                    s.synchronize()
                    if not np.array_equal(to_host(T, dt), want):
                        errors.append((D, dt))
        except Exception as e:          # reported below, on the main thread
            errors.append(repr(e))

    th = [threading.Thread(target=worker, args=(inputs[i::2],)) for i in range(2)]
    for t in th:
        t.start()
    for t in th:
        t.join(timeout=300)
    assert not any(t.is_alive() for t in th), "a worker did not finish"
    assert not errors, errors


@pytest.mark.parametrize("world", [2, 3])
def test_row_sharded_product_blocks(world):
    """The row-sharded product as each rank runs it (sr_shard_rows, then antidist_mul on
    its rows of A and C with all of B): the row blocks, computed as separate products on
    sub-matrix pointers, reassemble to the oracle's product (Section 2: rows of the
    product are independent)."""
    import torch
    import paper_1705_08743_gb300 as sr
    rng = np.random.default_rng(world)
    R, K, N = 1000, 300, 700
    A = rand_anti(rng, R, K, np.uint8, 0.3)
    B = rand_anti(rng, K, N, np.uint8, 0.3)
    Ad, Bd = to_dev(A), to_dev(B)
    Cd = torch.zeros((R, N), dtype=torch.uint8, device="cuda")
    for rank in range(world):
        r0, r1 = sr.sr_shard_rows(R, world, rank, 128)
        if r1 > r0:
            sr.antidist_mul(None, Ad[r0:r1], K, Bd, N, Cd[r0:r1], N, r1 - r0, K, N, sr.SR_U8, 0)
    assert np.array_equal(to_host(Cd, np.uint8), oracle.mul(A, B, 255))
