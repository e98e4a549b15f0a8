"""Distance form (Section 4 dual; dransclose), entrywise operators and the
reflexive closure on the GPU through the C ABI, against the oracle; bit-exact."""

import numpy as np
import pytest

import oracle
from gpu_util import to_dev, to_host, sr_dtype_of

pytestmark = pytest.mark.gpu
S_OF = {np.uint8: 255, np.uint16: 65535, np.uint32: 2 ** 32 - 1}
DTS = [np.uint8, np.uint16, np.uint32]


def rand_dist(rng, R, C, dt, p=0.4):
    S = S_OF[dt]
    v = rng.integers(0, S, size=(R, C), dtype=np.int64)
    return np.where(rng.random((R, C)) < p, v, S).astype(dt)     # S = no edge


@pytest.mark.parametrize("dt", DTS)
@pytest.mark.parametrize("shape", [(1, 1, 1), (50, 70, 90), (129, 33, 257), (300, 300, 300)])
def test_dist_mul(dt, shape):
    import paper_1705_08743_gb300 as sr
    R, K, N = shape
    S = S_OF[dt]
    rng = np.random.default_rng(R + K + N)
    A, B = rand_dist(rng, R, K, dt), rand_dist(rng, K, N, dt)
    ctx = sr.sr_create(workspace_bytes=sr.sr_workspace_query(sr.SR_OP_DIST_MUL, sr_dtype_of(dt), max(shape)))
    try:
        for acc in (0, 1):
            C0 = rand_dist(rng, R, N, dt, p=0.7)
            Ad, Bd, Cd = to_dev(A, 3), to_dev(B), to_dev(C0 if acc else np.zeros((R, N), dt))
            sr.dist_mul(ctx, Ad, Ad.shape[1], Bd, N, Cd, N, R, K, N, sr_dtype_of(dt), acc)
            want = oracle.dist_mul(A, B, S, Z=C0 if acc else None)
            assert np.array_equal(to_host(Cd, dt), want)
    finally:
        sr.sr_destroy(ctx)


@pytest.mark.parametrize("dt", DTS)
@pytest.mark.parametrize("D", [1, 7, 130, 300])
def test_dist_closure(dt, D):
    import paper_1705_08743_gb300 as sr
    S = S_OF[dt]
    rng = np.random.default_rng(D)
    A = rand_dist(rng, D, D, dt, p=min(1.0, 3.0 / D))
    Td = to_dev(A)
    sr.dist_closure(None, Td, D, D, sr_dtype_of(dt))
    assert np.array_equal(to_host(Td, dt), oracle.dist_closure(A, S))


@pytest.mark.parametrize("dt", DTS)
def test_entrywise_anti(dt):
    import paper_1705_08743_gb300 as sr
    S = S_OF[dt]
    rng = np.random.default_rng(4)
    A = rng.integers(0, S + 1, size=(37, 101), dtype=np.int64).astype(dt)
    B = rng.integers(0, S + 1, size=(37, 101), dtype=np.int64).astype(dt)
    for name, op in [("and", sr.SR_EW_AND), ("or", sr.SR_EW_OR), ("xor", sr.SR_EW_XOR), ("not", sr.SR_EW_NOT)]:
        Ad, Bd, Cd = to_dev(A), to_dev(B), to_dev(np.zeros_like(A))
        sr.sr_entrywise(None, op, Ad, 101, Bd, 101, Cd, 101, 37, 101, sr_dtype_of(dt))
        want = oracle.entrywise(name, A, None if name == "not" else B, S=S).astype(dt)
        assert np.array_equal(to_host(Cd, dt), want), name


@pytest.mark.parametrize("w", [32, 64])
def test_entrywise_bits_and_reflexive(w):
    import paper_1705_08743_gb300 as sr
    dt = sr.SR_BOOL_W64 if w == 64 else sr.SR_BOOL_W32
    rng = np.random.default_rng(5)
    R, N = 20, 100
    a = (rng.random((R, N)) < 0.5).astype(np.uint8)
    b = (rng.random((R, N)) < 0.5).astype(np.uint8)
    Pa, Pb = oracle.pack_bits(a), oracle.pack_bits(b)
    if w == 32:
        Pa, Pb = Pa.view(np.uint32), Pb.view(np.uint32)
    for name, op in [("and", sr.SR_EW_AND), ("or", sr.SR_EW_OR), ("xor", sr.SR_EW_XOR), ("not", sr.SR_EW_NOT)]:
        Ad, Bd, Cd = to_dev(Pa), to_dev(Pb), to_dev(np.zeros_like(Pa))
        sr.sr_entrywise(None, op, Ad, Pa.shape[1], Bd, Pb.shape[1], Cd, Pa.shape[1], R, N, dt)
        got = oracle.unpack_bits(np.ascontiguousarray(to_host(Cd, Pa.dtype)).view(np.uint64), N)
        want = oracle.entrywise(name, a, None if name == "not" else b, S=1).astype(np.uint8)
        assert np.array_equal(got, want), name
    D = 100
    T = (rng.random((D, D)) < 0.1).astype(np.uint8)
    P = oracle.pack_bits(T)
    if w == 32:
        P = P.view(np.uint32)
    Td = to_dev(P)
    sr.sr_reflexive(None, Td, P.shape[1], D, dt)
    got = oracle.unpack_bits(np.ascontiguousarray(to_host(Td, P.dtype)).view(np.uint64), D)
    want = T.copy()
    np.fill_diagonal(want, 1)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("dt", DTS)
def test_reflexive_anti_is_identity_join(dt):
    import paper_1705_08743_gb300 as sr
    S = S_OF[dt]
    rng = np.random.default_rng(6)
    A = rng.integers(0, S + 1, size=(64, 64), dtype=np.int64).astype(dt)
    Td = to_dev(A)
    sr.sr_reflexive(None, Td, 64, 64, sr_dtype_of(dt))
    want = np.maximum(A, (np.eye(64, dtype=np.int64) * S).astype(dt))      # I ⊕ A
    assert np.array_equal(to_host(Td, dt), want)
