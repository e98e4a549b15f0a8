"""Boolean (bit-packed) product, packing and closure on the GPU through the C
ABI, against the CPU oracle; bit-exact."""

import numpy as np
import pytest

import oracle
import synth
from gpu_util import to_dev, to_host

pytestmark = pytest.mark.gpu


def rand_bool(rng, R, C, p):
    return (rng.random((R, C)) < p).astype(np.uint8)


def packed(dense, w):
    """Oracle packing into 64-bit words; a W32 matrix is the same bytes viewed as uint32."""
    M = oracle.pack_bits(dense)
    return M if w == 64 else M.view(np.uint32)


def unpacked(M, w, C):
    M64 = np.ascontiguousarray(M).view(np.uint64)
    return oracle.unpack_bits(M64, C)


def gpu_bool_mul(A, B, K, N, w, C0=None, pad=(0, 0, 0)):
    import paper_1705_08743_gb300 as sr
    dt = sr.SR_BOOL_W64 if w == 64 else sr.SR_BOOL_W32
    R = A.shape[0]
    Ad, Bd = to_dev(A, pad[0]), to_dev(B, pad[1])
    Cd = to_dev(np.zeros_like(packed(np.zeros((R, N), np.uint8), w)) if C0 is None else C0, pad[2])
    sr.bool_mul(None, Ad, Ad.shape[1], Bd, Bd.shape[1], Cd, Cd.shape[1], R, K, N, dt, 0 if C0 is None else 1)
    out = to_host(Cd, np.uint64 if w == 64 else np.uint32)
    return out[:, :A.shape[1] if False else out.shape[1] - pad[2]]


@pytest.mark.parametrize("w", [32, 64])
@pytest.mark.parametrize("shape", [(1, 1, 1), (5, 70, 129), (64, 64, 64), (33, 200, 65), (300, 517, 1000),
                                   (129, 4096, 96)])
def test_bool_mul_random(w, shape):
    R, K, N = shape
    rng = np.random.default_rng(R + K + N)
    for p in [0.02, 0.3]:
        A, B = rand_bool(rng, R, K, p), rand_bool(rng, K, N, p)
        got = gpu_bool_mul(packed(A, w), packed(B, w), K, N, w)
        assert np.array_equal(unpacked(got, w, N), oracle.mul(A, B, 1))
        C0 = rand_bool(rng, R, N, 0.1)
        got = gpu_bool_mul(packed(A, w), packed(B, w), K, N, w, C0=packed(C0, w))
        assert np.array_equal(unpacked(got, w, N), np.maximum(C0, oracle.mul(A, B, 1)))
        # pad bits written zero
        if N % 64:
            g64 = np.ascontiguousarray(got).view(np.uint64)
            assert int((g64[:, -1] >> np.uint64(N % 64)).sum()) == 0


@pytest.mark.parametrize("w", [32, 64])
def test_bool_mul_garbage_pad_bits_and_unaligned(w):
    rng = np.random.default_rng(5)
    R, K, N = 77, 100, 90
    A, B = rand_bool(rng, R, K, 0.1), rand_bool(rng, K, N, 0.1)
    Ap, Bp = packed(A, w).copy(), packed(B, w).copy()
    # set every pad bit of A and B: the product must ignore them
    for M, n in [(Ap, K), (Bp, N)]:
        M64 = M.view(np.uint64)
        if n % 64:
            M64[:, -1] |= ~np.uint64((1 << (n % 64)) - 1)
    got = gpu_bool_mul(Ap, Bp, K, N, w, pad=(1, 3, 2))
    assert np.array_equal(unpacked(got, w, N), oracle.mul(A, B, 1))


@pytest.mark.parametrize("w", [32, 64])
@pytest.mark.parametrize("shape", [(40, 3000, 90), (260, 1500, 700), (7, 9000, 33), (512, 512, 512)])
def test_bool_mul_split_k(w, shape):
    """Small output, long K: the product is split along K across CTAs whose partial
    results are ORed together.  Garbage pad bits in C must come out zero, with and
    without accumulation, exactly as in the unsplit product."""
    R, K, N = shape
    rng = np.random.default_rng(K)
    A, B = rand_bool(rng, R, K, 0.01), rand_bool(rng, K, N, 0.01)
    ref = oracle.mul(A, B, 1)
    C0 = rand_bool(rng, R, N, 0.05)
    Cp = packed(C0, w).copy()
    dt = np.uint64 if w == 64 else np.uint32
    last, nb = (N - 1) // w, N % w                   # the row's last word and its valid bits
    if nb:
        Cp[:, last] |= ~dt((1 << nb) - 1)
    for acc in (False, True):
        got = gpu_bool_mul(packed(A, w), packed(B, w), K, N, w, C0=Cp if acc else None, pad=(0, 1, 1))
        assert np.array_equal(unpacked(got, w, N), np.maximum(C0, ref) if acc else ref)
        if nb:
            assert int((got[:, last] >> dt(nb)).sum()) == 0


@pytest.mark.parametrize("w", [32, 64])
def test_pack_unpack(w):
    import torch
    import paper_1705_08743_gb300 as sr
    dt = sr.SR_BOOL_W64 if w == 64 else sr.SR_BOOL_W32
    rng = np.random.default_rng(6)
    for (R, C) in [(1, 1), (3, 31), (5, 64), (17, 65), (40, 1000), (7, 1008), (9, 1024), (3, 4096)]:
        d = rand_bool(rng, R, C, 0.4)
        d[d == 1] = rng.integers(1, 256, size=int(d.sum()))        # any nonzero byte is 1
        dd = to_dev(d)
        ref = packed((d != 0).astype(np.uint8), w)
        Md = torch.zeros(ref.shape, dtype=torch.int64 if w == 64 else torch.int32, device="cuda")
        sr.bool_pack(None, dd, C, Md, ref.shape[1], R, C, dt)
        assert np.array_equal(to_host(Md, ref.dtype), ref)
        back = torch.zeros((R, C), dtype=torch.uint8, device="cuda")
        sr.bool_unpack(None, Md, ref.shape[1], back, C, R, C, dt)
        assert np.array_equal(back.cpu().numpy(), (d != 0).astype(np.uint8))


def gpu_bool_closure(dense, w, method, pad=0, ctx=None):
    import paper_1705_08743_gb300 as sr
    dt = sr.SR_BOOL_W64 if w == 64 else sr.SR_BOOL_W32
    D = dense.shape[0]
    Md = to_dev(packed(dense, w), pad)
    sr.bool_closure(ctx, Md, Md.shape[1], D, dt, method)
    out = to_host(Md, np.uint64 if w == 64 else np.uint32)
    return out[:, :out.shape[1] - pad] if pad else out


@pytest.fixture(scope="module")
def sq_ctx():
    import paper_1705_08743_gb300 as sr
    ctx = sr.sr_create(workspace_bytes=64 << 20)
    yield ctx
    sr.sr_destroy(ctx)


@pytest.mark.parametrize("w", [32, 64])
@pytest.mark.parametrize("D", [1, 5, 31, 32, 33, 64, 65, 127, 128, 129, 130, 200, 256, 300, 385, 513, 700])
def test_bool_closure(w, D, sq_ctx):
    import paper_1705_08743_gb300 as sr
    rng = np.random.default_rng(D * 3 + w)
    for p in [1.5 / D, 0.5 / D, 4.0 / D]:
        A = rand_bool(rng, D, D, min(1.0, p))
        ref = oracle.warshall(A, 1)
        for method in (sr.SR_CLOSURE_WARSHALL, sr.SR_CLOSURE_SQUARING):
            got = gpu_bool_closure(A, w, method, ctx=sq_ctx)
            assert np.array_equal(unpacked(got, w, D), ref), (p, method)


@pytest.mark.parametrize("w,D", [(64, 2500), (32, 2333)])
def test_bool_closure_four_russians_phase3(w, D):
    """From D = 2304 on, phase 3 runs on the Four Russians tables with the rows and words
    of the two pivot blocks left out by remapping; Warshall form, every word compared."""
    import paper_1705_08743_gb300 as sr
    dense = synth.bool_dag_union(D, seed=D)
    got = gpu_bool_closure(dense, w, sr.SR_CLOSURE_WARSHALL)
    want = oracle.bool_warshall_w64(oracle.pack_bits(dense))
    assert np.array_equal(np.ascontiguousarray(got).view(np.uint64), want)


@pytest.mark.parametrize("w,D,pad", [(64, 2500, 0), (32, 2333, 3), (64, 4500, 0), (32, 4200, 0)])
def test_bool_closure_wide_tensor_blocks(w, D, pad):
    """Warshall form with 2048-bit blocks, panels and phase 3 on the tensor cores (forced
    below its default size): two and three blocks, ragged last blocks, W32 and W64, an
    unaligned leading dimension; every word compared with the oracle's packed Warshall."""
    import paper_1705_08743_gb300 as sr
    dt = sr.SR_BOOL_W64 if w == 64 else sr.SR_BOOL_W32
    dense = synth.bool_dag_union(D, seed=D + 1)
    ctx = sr.sr_create(workspace_bytes=sr.sr_workspace_query(sr.SR_OP_BOOL_CLOSURE, dt, D, sr.SR_CLOSURE_WARSHALL))
    try:
        sr.sr_set_option(ctx, sr.SR_OPT_BOOL_TENSOR, 2)
        got = gpu_bool_closure(dense, w, sr.SR_CLOSURE_WARSHALL, pad=pad, ctx=ctx)
        sr.sr_stream_status(ctx)
    finally:
        sr.sr_destroy(ctx)
    want = oracle.bool_warshall_w64(oracle.pack_bits(dense))
    assert np.array_equal(unpacked(got, w, D), unpacked(want, 64, D))


def test_bool_closure_default_takes_tensor_schedule_from_4096():
    """With the default options and a context holding the Warshall workspace, D = 4096 and
    D = 4100 (one ragged block) take the tensor-core schedule; D = 4095 keeps the 128-bit
    word schedule.  Every word against the oracle, and the kernel launch count tells the
    schedules apart."""
    import paper_1705_08743_gb300 as sr
    launches = {}
    for D in (4095, 4096, 4100):
        dense = synth.bool_dag_union(D, seed=D)
        ctx = sr.sr_create(workspace_bytes=sr.sr_workspace_query(sr.SR_OP_BOOL_CLOSURE, sr.SR_BOOL_W64, D,
                                                                  sr.SR_CLOSURE_WARSHALL))
        try:
            n0 = sr.sr_kernel_launches()
            got = gpu_bool_closure(dense, 64, sr.SR_CLOSURE_WARSHALL, ctx=ctx)
            launches[D] = sr.sr_kernel_launches() - n0
            sr.sr_stream_status(ctx)
        finally:
            sr.sr_destroy(ctx)
        want = oracle.bool_warshall_w64(oracle.pack_bits(dense))
        assert np.array_equal(np.ascontiguousarray(got).view(np.uint64), want), D
    # GB300: 122 launches for two 2048-bit blocks (each diagonal block: 12 tensor-core
    # products with their operand expansions and 11 convergence checks), 148 with a third,
    # 4-bit block, against 191 for 32 blocks of 128 bits
    assert launches[4096] < launches[4095] and launches[4100] < launches[4095], launches


@pytest.mark.parametrize("kind", ["chain", "dense", "two_chains"])
def test_bool_squaring_tensor_path_stops_early_only_when_converged(kind):
    """Squaring form on the tensor cores, which skips the squarings after the first one that
    leaves I ⊕ A's power unchanged: a 1500-node chain (every squaring changes it), a dense
    random graph (converges after a few), and two chains of different lengths (the short one
    converges first, the long one must not be cut short); every word against the oracle."""
    import paper_1705_08743_gb300 as sr
    D = 1500
    rng = np.random.default_rng(1500)
    dense = np.zeros((D, D), np.uint8)
    if kind == "chain":
        dense[np.arange(D - 1), np.arange(1, D)] = 1
    elif kind == "dense":
        dense = rand_bool(rng, D, D, 12.0 / D)
    else:
        dense[np.arange(99), np.arange(1, 100)] = 1                     # 0 -> 1 -> ... -> 99
        dense[np.arange(100, D - 1), np.arange(101, D)] = 1             # 100 -> ... -> 1499
    ctx = sr.sr_create(workspace_bytes=sr.sr_workspace_query(sr.SR_OP_BOOL_CLOSURE, sr.SR_BOOL_W64, D,
                                                              sr.SR_CLOSURE_SQUARING))
    try:
        sr.sr_set_option(ctx, sr.SR_OPT_BOOL_TENSOR, 2)
        got = gpu_bool_closure(dense, 64, sr.SR_CLOSURE_SQUARING, ctx=ctx)
        sr.sr_stream_status(ctx)
    finally:
        sr.sr_destroy(ctx)
    want = oracle.bool_warshall_w64(oracle.pack_bits(dense))
    assert np.array_equal(np.ascontiguousarray(got).view(np.uint64), want)


def test_bool_closure_pad_and_unaligned(sq_ctx):
    import paper_1705_08743_gb300 as sr
    rng = np.random.default_rng(9)
    D = 250
    A = synth.bool_dag_union(D, seed=4)
    ref = oracle.warshall(A, 1)
    for w in (32, 64):
        got = gpu_bool_closure(A, w, sr.SR_CLOSURE_WARSHALL, pad=3)
        assert np.array_equal(unpacked(got, w, D), ref)


def test_bool_squaring_needs_workspace():
    import paper_1705_08743_gb300 as sr
    A = np.zeros((40, 40), np.uint8)
    with pytest.raises(sr.SemiringError) as e:
        gpu_bool_closure(A, 64, sr.SR_CLOSURE_SQUARING, ctx=None)
    assert e.value.status == sr.SR_EINVAL


# ---------------------------------------------------------------- full size
def test_cfg1_bool_product_512():
    """512x512x512, Bernoulli(0.02), seed 0, 32 columns per word."""
    A, B = synth.cfg1_bool_product()
    got = gpu_bool_mul(packed(A, 32), packed(B, 32), 512, 512, 32)
    ref = oracle.mul(A, B, 1)
    assert np.array_equal(unpacked(got, 32, 512), ref)
    assert 0.1 < ref.mean() < 0.3


@pytest.mark.slow
def test_cfg3_bool_closure_full_16384(sq_ctx):
    """D=16384 W64 DAG-union graph, seed 2: Warshall form vs the oracle's
    packed Warshall, and sampled rows by BFS; the squaring form on the same
    input must agree (needs 2*32 MiB workspace)."""
    import paper_1705_08743_gb300 as sr
    D = 16384
    G = synth.cfg3_bool_closure(D)
    Gp = oracle.pack_bits(G)
    ref = oracle.bool_warshall_w64(Gp)
    got = gpu_bool_closure(G, 64, sr.SR_CLOSURE_WARSHALL)
    assert np.array_equal(got, ref)
    for src in [0, 5, 8191, 16383]:
        assert np.array_equal(got[src], oracle.bool_closure_row_w64(Gp, src))
    ctx = sr.sr_create(workspace_bytes=sr.sr_workspace_query(sr.SR_OP_BOOL_CLOSURE, sr.SR_BOOL_W64, D,
                                                              sr.SR_CLOSURE_SQUARING))
    try:
        got2 = gpu_bool_closure(G, 64, sr.SR_CLOSURE_SQUARING, ctx=ctx)
    finally:
        sr.sr_destroy(ctx)
    assert np.array_equal(got2, ref)
    # with a workspace for 2048-deep tensor-core products the Warshall form takes wide blocks
    ctx = sr.sr_create(workspace_bytes=sr.sr_workspace_query(sr.SR_OP_BOOL_CLOSURE, sr.SR_BOOL_W64, D,
                                                              sr.SR_CLOSURE_WARSHALL))
    try:
        got3 = gpu_bool_closure(G, 64, sr.SR_CLOSURE_WARSHALL, ctx=ctx)
        sr.sr_stream_status(ctx)
    finally:
        sr.sr_destroy(ctx)
    assert np.array_equal(got3, ref)


# ---------------------------------------------------------------- tensor-core path
@pytest.mark.parametrize("w", [32, 64])
def test_bool_mul_tensor_path_many_tiles_per_cta(w):
    """More output tiles (16 x 20) than SMs, so each persistent CTA walks several and
    alternates its two accumulators; ragged in every dimension, with and without
    accumulation, against the oracle's packed product."""
    import paper_1705_08743_gb300 as sr
    R, K, N = 2000, 1100, 5000
    rng = np.random.default_rng(2024 + w)
    dt = sr.SR_BOOL_W64 if w == 64 else sr.SR_BOOL_W32
    ctx = sr.sr_create(workspace_bytes=sr.sr_workspace_query(sr.SR_OP_BOOL_MUL, sr.SR_BOOL_W64, max(R, K, N)))
    sr.sr_set_option(ctx, sr.SR_OPT_BOOL_TENSOR, 2)
    try:
        A, B, C0 = rand_bool(rng, R, K, 0.02), rand_bool(rng, K, N, 0.02), rand_bool(rng, R, N, 0.05)
        Ad, Bd = to_dev(packed(A, w)), to_dev(packed(B, w))
        for acc in (0, 1):
            Cd = to_dev(packed(C0, w)) if acc else to_dev(np.zeros_like(packed(C0, w)))
            sr.bool_mul(ctx, Ad, Ad.shape[1], Bd, Bd.shape[1], Cd, Cd.shape[1], R, K, N, dt, acc)
            sr.sr_stream_status(ctx)
            got = unpacked(to_host(Cd, np.uint64 if w == 64 else np.uint32), w, N)
            want = oracle.unpack_bits(oracle.bool_mul_w64(oracle.pack_bits(A), oracle.pack_bits(B), N,
                                                          C=oracle.pack_bits(C0) if acc else None), N)
            assert np.array_equal(got, want), acc
            assert 0.05 < want.mean() < 0.95
    finally:
        sr.sr_destroy(ctx)


@pytest.mark.parametrize("shape", [(128, 128, 256), (128, 1024, 256), (200, 300, 257), (333, 2100, 700),
                                   (1, 64, 1), (1000, 4096, 1000)])
@pytest.mark.parametrize("w", [32, 64])
def test_bool_mul_tensor_path(shape, w):
    """Count on the tensor cores, then test > 0: bit-exact against the oracle,
    with and without accumulation, forced on for every shape."""
    import paper_1705_08743_gb300 as sr
    R, K, N = shape
    rng = np.random.default_rng(R * 31 + K + N)
    ctx = sr.sr_create(workspace_bytes=sr.sr_workspace_query(sr.SR_OP_BOOL_MUL, sr.SR_BOOL_W64, max(R, K, N)) + 4096)
    sr.sr_set_option(ctx, sr.SR_OPT_BOOL_TENSOR, 2)
    dt = sr.SR_BOOL_W64 if w == 64 else sr.SR_BOOL_W32
    try:
        for p in [0.01, 0.2]:
            A, B = rand_bool(rng, R, K, p), rand_bool(rng, K, N, p)
            Ad, Bd = to_dev(packed(A, w)), to_dev(packed(B, w))
            C0 = rand_bool(rng, R, N, 0.1)
            for acc in (0, 1):
                Cd = to_dev(packed(C0, w)) if acc else to_dev(np.zeros_like(packed(C0, w)))
                sr.bool_mul(ctx, Ad, Ad.shape[1], Bd, Bd.shape[1], Cd, Cd.shape[1], R, K, N, dt, acc)
                sr.sr_stream_status(ctx)
                got = unpacked(to_host(Cd, np.uint64 if w == 64 else np.uint32), w, N)
                want = oracle.mul(A, B, 1)
                if acc:
                    want = np.maximum(C0, want)
                assert np.array_equal(got, want), (p, acc)
    finally:
        sr.sr_destroy(ctx)


# ---------------------------------------------------------------- Four Russians
@pytest.mark.parametrize("shape", [(1, 1, 1), (5, 7, 33), (512, 512, 1024), (513, 300, 1030), (700, 1029, 2100),
                                   (1100, 4100, 70), (64, 9, 4096)])
@pytest.mark.parametrize("w", [32, 64])
def test_bool_mul_four_russians(shape, w):
    """Table-lookup product (8-bit groups of K) forced on for every shape: K not a
    multiple of 8 or 32, ragged row tiles and word windows, garbage pad bits in A, B and
    C, unaligned leading dimensions; with and without accumulation."""
    import paper_1705_08743_gb300 as sr
    R, K, N = shape
    rng = np.random.default_rng(R * 17 + K * 5 + N)
    ctx = sr.sr_create()
    sr.sr_set_option(ctx, sr.SR_OPT_BOOL_TENSOR, 0)
    sr.sr_set_option(ctx, sr.SR_OPT_BOOL_FOUR_RUSSIANS, 2)
    dt = sr.SR_BOOL_W64 if w == 64 else sr.SR_BOOL_W32
    hdt = np.uint64 if w == 64 else np.uint32
    try:
        for p in [0.01, 0.3]:
            A, B = rand_bool(rng, R, K, p), rand_bool(rng, K, N, p)
            Ap, Bp = packed(A, w).copy(), packed(B, w).copy()
            for M, n in [(Ap, K), (Bp, N)]:                    # set every pad bit
                last, nb = (n - 1) // w, n % w
                if nb:
                    M[:, last] |= ~hdt((1 << nb) - 1)
            Ad, Bd = to_dev(Ap, 1), to_dev(Bp, 3)
            C0 = rand_bool(rng, R, N, 0.1)
            for acc in (0, 1):
                Cd = to_dev(packed(C0, w) if acc else np.zeros_like(packed(C0, w)), 2)
                sr.bool_mul(ctx, Ad, Ad.shape[1], Bd, Bd.shape[1], Cd, Cd.shape[1], R, K, N, dt, acc)
                out = to_host(Cd, hdt)[:, :-2]
                want = oracle.mul(A, B, 1)
                if acc:
                    want = np.maximum(C0, want)
                assert np.array_equal(unpacked(out, w, N), want), (p, acc)
                if N % w:
                    assert int((out[:, (N - 1) // w] >> hdt(N % w)).sum()) == 0
    finally:
        sr.sr_destroy(ctx)


def test_bool_mul_four_russians_default_large():
    """Default (auto) mode at a size where the table path is selected (8192 x 1024 x
    8192: 256 CTAs of 256 rows x 32 words); compared with the oracle's packed product."""
    R, K, N = 8192, 1024, 8192
    rng = np.random.default_rng(77)
    A, B = rand_bool(rng, R, K, 0.002), rand_bool(rng, K, N, 0.002)
    A64, B64 = oracle.pack_bits(A), oracle.pack_bits(B)
    got = gpu_bool_mul(A64.view(np.uint32), B64.view(np.uint32), K, N, 32)
    want = oracle.bool_mul_w64(A64, B64, N)
    assert np.array_equal(np.ascontiguousarray(got).view(np.uint64), want)
    assert want.any()


def test_tensor_path_bounded_wait_gives_up_and_recovers():
    """Fault injection without a GPU fault: with a spin limit of 0 every mbarrier wait of
    the tensor-core pipeline gives up at once; each CTA drains the copies and MMAs it
    started, frees its tensor memory and returns, and the context's status word reports
    SR_ETIMEOUT.  The same context then computes the right product with the limit back."""
    import paper_1705_08743_gb300 as sr
    R = K = N = 1024
    rng = np.random.default_rng(1024)
    A, B = rand_bool(rng, R, K, 0.01), rand_bool(rng, K, N, 0.01)
    ctx = sr.sr_create(workspace_bytes=sr.sr_workspace_query(sr.SR_OP_BOOL_MUL, sr.SR_BOOL_W64, R) + 4096)
    try:
        sr.sr_set_option(ctx, sr.SR_OPT_BOOL_TENSOR, 2)
        Ad, Bd = to_dev(packed(A, 64)), to_dev(packed(B, 64))
        Cd = to_dev(np.zeros_like(packed(np.zeros((R, N), np.uint8), 64)))
        sr.sr_set_option(ctx, sr.SR_OPT_SPIN_LIMIT, 0)
        sr.bool_mul(ctx, Ad, Ad.shape[1], Bd, Bd.shape[1], Cd, Cd.shape[1], R, K, N, sr.SR_BOOL_W64, 0)
        with pytest.raises(sr.SemiringError) as e:
            sr.sr_stream_status(ctx)
        assert e.value.status == sr.SR_ETIMEOUT
        sr.sr_stream_status(ctx)                          # reading the status cleared it
        sr.sr_set_option(ctx, sr.SR_OPT_SPIN_LIMIT, 1 << 22)
        sr.bool_mul(ctx, Ad, Ad.shape[1], Bd, Bd.shape[1], Cd, Cd.shape[1], R, K, N, sr.SR_BOOL_W64, 0)
        sr.sr_stream_status(ctx)
        got = unpacked(to_host(Cd, np.uint64), 64, N)
        assert np.array_equal(got, oracle.mul(A, B, 1))
    finally:
        sr.sr_destroy(ctx)
