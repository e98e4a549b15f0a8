"""Pins for the CPU oracle: checks against what the paper and the mathematics
fix, not against the oracle itself.

- hand-worked fixtures (tests/golden, Sections 2-3 graph reading);
- brute-force enumeration of simple paths/cycles on graphs with D <= 7;
- scipy's Floyd-Warshall on lengths S - a (a library route to the same
  reflexive closure);
- the identities of Section 2 (closure = A ⊗ (I ⊕ A)^(D'-1); reflexive and
  non-reflexive closures related by adding I and multiplying by A), closure
  idempotence, associativity and distributivity (Section 3);
- De Morgan duality with the distance (min, saturating +) form (Section 4);
- the Boolean <-> anti-distance embedding 1 -> S, 0 -> 0 (Section 3);
- the semantics of ⊗ through distances: S - (a ⊗ b) = min((S-a) + (S-b), S).
"""

import itertools

import numpy as np
import pytest

import oracle
import synth
from golden_io import all_fixtures, load

S32 = 2 ** 32 - 1                    # the u32 anti-distance type (Section 4)
SS = [1, 255, 65535, S32]


def rand_mat(rng, R, C, S, density=0.5, lo=None):
    """Random matrix over {0..S} with given density of nonzeros."""
    if S == 1:
        return (rng.random((R, C)) < density).astype(np.uint32)
    lo = 1 if lo is None else lo
    v = rng.integers(lo, S + 1, size=(R, C), dtype=np.int64)
    return np.where(rng.random((R, C)) < density, v, 0).astype(np.uint32)


def ident(D, S):
    return (np.eye(D, dtype=np.uint32) * S).astype(np.uint32)


# ------------------------------------------------------------------ brute force

def brute_closure(A, S):
    """max over paths with >= 1 edge of max(S - length, 0), enumerating simple
    paths (i != j) and simple cycles (i == j); lengths are S - a >= 0, so a
    best walk is always simple."""
    A = np.asarray(A, dtype=np.int64)
    D = A.shape[0]
    T = np.zeros((D, D), dtype=np.int64)

    def dfs(src, v, length, seen):
        for u in range(D):
            a = A[v, u]
            if a == 0:
                continue
            L = length + (S - a)
            val = max(S - L, 0)
            if u == src:
                T[src, src] = max(T[src, src], val)
            elif u not in seen:
                T[src, u] = max(T[src, u], val)
                dfs(src, u, L, seen | {u})

    for i in range(D):
        dfs(i, i, 0, {i})
    return T.astype(np.uint32)


def brute_product(A, B, S):
    """(A ⊗ B)_ij over all k, from the distance reading: the two-edge path
    i -> k -> j has length (S - A_ik) + (S - B_kj); value max(S - length, 0);
    for S = 1 the path exists iff both edges exist."""
    R, K = A.shape
    N = B.shape[1]
    P = np.zeros((R, N), np.int64)
    for i in range(R):
        for j in range(N):
            best = 0
            for k in range(K):
                a, b = int(A[i, k]), int(B[k, j])
                if a == 0 or b == 0:
                    continue
                if S == 1:
                    best = 1
                else:
                    best = max(best, max(S - ((S - a) + (S - b)), 0))
            P[i, j] = best
    return P.astype(np.uint32)


def minplus_sat(X, Y, S):
    """Distance-matrix product (Section 4): min over k of X_ik + Y_kj, sums
    saturating at S."""
    X = X.astype(np.int64)
    Y = Y.astype(np.int64)
    Z = np.min(X[:, :, None] + Y[None, :, :], axis=1)
    return np.minimum(Z, S).astype(np.uint32)


# ------------------------------------------------------------------ fixtures

@pytest.mark.parametrize("name", all_fixtures())
def test_golden_fixture(name):
    fx = load(name)
    S, A, T = fx["S"], fx["A"], fx["T"]
    assert np.array_equal(oracle.warshall(A, S), T)
    assert np.array_equal(oracle.closure_squaring(A, S), T)
    for i in range(A.shape[0]):
        assert np.array_equal(oracle.closure_row(A, i, S), T[i])
    if "A2" in fx:
        assert np.array_equal(oracle.mul(A, A, S), fx["A2"])
    assert np.array_equal(brute_closure(A, S), T)


# ------------------------------------------------------------------ ⊗ semantics

def test_times_table_u8_by_distances():
    S = 255
    a = np.arange(S + 1, dtype=np.uint32)
    P = oracle.mul(a[:, None], a[None, :], S)           # 256 x 256 outer product
    da, db = (S - a.astype(np.int64))[:, None], (S - a.astype(np.int64))[None, :]
    assert np.array_equal(S - P.astype(np.int64), np.minimum(da + db, S))


def test_times_table_u16_sampled_by_distances():
    S = 65535
    rng = np.random.default_rng(5)
    a = np.concatenate([np.array([0, 1, 2, S - 1, S, 32767, 32768]),
                        rng.integers(0, S + 1, 500)]).astype(np.uint32)
    P = oracle.mul(a[:, None], a[None, :], S)
    d = S - a.astype(np.int64)
    assert np.array_equal(S - P.astype(np.int64), np.minimum(d[:, None] + d[None, :], S))


def test_times_table_u32_sampled_by_distances():
    """S = 2^32 − 1: a + b − S needs 33 bits; the closed form through distances
    (computed here in Python integers) fixes every entry, including the carry edge
    a + b = S, S + 1 and the extremes 0 and S."""
    S = S32
    rng = np.random.default_rng(9)
    a = np.concatenate([np.array([0, 1, 2, S - 1, S, 2 ** 31 - 1, 2 ** 31, 2 ** 31 + 1, 2 ** 16, 2 ** 32 - 2 ** 16]),
                        rng.integers(0, S + 1, 300, dtype=np.int64)]).astype(np.uint32)
    P = oracle.mul(a[:, None], a[None, :], S)
    d = S - a.astype(np.int64)
    assert np.array_equal(S - P.astype(np.int64), np.minimum(d[:, None] + d[None, :], S))
    ai = [int(x) for x in a[:10]]
    for i, x in enumerate(ai):
        for j, y in enumerate(ai):
            assert int(P[i, j]) == max(x + y - S, 0)


def test_u32_closure_is_u16_closure_shifted_when_paths_are_short():
    """With edge lengths <= 31 and D = 50 every path is shorter than 2^16 − 1, so
    no value saturates in either type and each reachable entry is S − length:
    the u32 closure equals the u16 one plus (2^32 − 1) − (2^16 − 1) where nonzero."""
    rng = np.random.default_rng(13)
    D = 50
    W = np.where(rng.random((D, D)) < 0.08, rng.integers(1, 32, (D, D)), 0).astype(np.uint32)
    T16 = oracle.warshall(oracle.encode_antidist(W, 65535), 65535).astype(np.int64)
    T32 = oracle.warshall(oracle.encode_antidist(W, S32), S32).astype(np.int64)
    assert np.array_equal(T32, np.where(T16 > 0, T16 + (S32 - 65535), 0))
    assert (T16 > 0).sum() > D                                # the graph has long paths


def test_times_boolean_truth_table():
    a = np.array([0, 1], np.uint32)
    P = oracle.mul(a[:, None], a[None, :], 1)
    assert P.tolist() == [[0, 0], [0, 1]]               # AND


def test_mul_entry_matches_loop_form():
    rng = np.random.default_rng(0)
    for S in SS:
        A, B = rand_mat(rng, 13, 17, S), rand_mat(rng, 17, 11, S)
        P = oracle.mul(A, B, S)
        for i, j in itertools.product(range(13), range(11)):
            assert P[i, j] == oracle.mul_entry(A, B, i, j, S)


@pytest.mark.parametrize("S", SS)
def test_product_brute_force(S):
    rng = np.random.default_rng(S)
    A, B = rand_mat(rng, 6, 9, S, lo=S // 2), rand_mat(rng, 9, 7, S, lo=S // 2)
    assert np.array_equal(oracle.mul(A, B, S), brute_product(A, B, S))
    C = rand_mat(rng, 6, 7, S)
    assert np.array_equal(oracle.mul(A, B, S, C=C), np.maximum(C, brute_product(A, B, S)))


# ------------------------------------------------------------------ closure

@pytest.mark.parametrize("S", SS)
@pytest.mark.parametrize("D", [1, 2, 3, 5, 7])
def test_closure_brute_force(S, D):
    rng = np.random.default_rng(100 * D + S % 97)
    for trial in range(4):
        lo = max(1, S - S // 3) if trial % 2 else 1            # long paths vs saturation
        A = rand_mat(rng, D, D, S, density=0.45, lo=lo)
        T = brute_closure(A, S)
        assert np.array_equal(oracle.warshall(A, S), T)
        assert np.array_equal(oracle.closure_squaring(A, S), T)
        for i in range(D):
            assert np.array_equal(oracle.closure_row(A, i, S), T[i])


@pytest.mark.parametrize("S", [255, 65535, S32])
def test_closure_vs_scipy_floyd_warshall(S):
    sp = pytest.importorskip("scipy.sparse.csgraph")
    rng = np.random.default_rng(7)
    D = 60
    A = rand_mat(rng, D, D, S, density=0.08, lo=S - S // 8)
    A = np.minimum(A, S - 1)        # scipy's dense input reads a 0 length as "no edge"
    T = oracle.warshall(A, S)
    L = np.where(A > 0, S - A.astype(np.float64), np.inf)
    dist = sp.floyd_warshall(L, directed=True)              # diagonal 0: reflexive
    ref = np.where(np.isfinite(dist), np.maximum(S - dist, 0), 0).astype(np.uint32)
    R = np.maximum(T, ident(D, S))                          # I ⊕ T
    assert np.array_equal(R, ref)


@pytest.mark.parametrize("S", SS)
def test_closure_identities(S):
    rng = np.random.default_rng(11 + S)
    D = 40
    A = rand_mat(rng, D, D, S, density=0.06 if S == 1 else 0.1, lo=(S * 3) // 4 or 1)
    T = oracle.warshall(A, S)
    I = ident(D, S)
    R = np.maximum(I, T)
    assert np.array_equal(oracle.mul(T, T, S, C=T), T)              # T ⊗ T ⊕ T = T
    assert np.array_equal(np.maximum(A, oracle.mul(A, T, S)), T)     # T = A ⊕ A ⊗ T
    assert np.array_equal(np.maximum(A, oracle.mul(T, A, S)), T)     # T = A ⊕ T ⊗ A
    assert np.array_equal(oracle.mul(R, R, S), R)                    # R ⊗ R = R
    assert np.array_equal(oracle.mul(A, R, S), T)                    # T = A ⊗ R
    assert np.array_equal(oracle.mul(R, A, S), T)                    # T = R ⊗ A
    # the finite sum A ⊕ A^2 ⊕ ... ⊕ A^D written out (Section 2)
    acc, P = A.copy(), A.copy()
    for _ in range(D - 1):
        P = oracle.mul(P, A, S)
        acc = np.maximum(acc, P)
    assert np.array_equal(acc, T)


@pytest.mark.parametrize("S", SS)
def test_identity_is_neutral_and_zero_absorbs(S):
    rng = np.random.default_rng(3)
    A = rand_mat(rng, 9, 9, S)
    I = ident(9, S)
    Z = np.zeros((9, 9), np.uint32)
    assert np.array_equal(oracle.mul(I, A, S), A)
    assert np.array_equal(oracle.mul(A, I, S), A)
    assert np.array_equal(oracle.mul(A, Z, S), Z)
    assert np.array_equal(oracle.warshall(Z, S), Z)


# ------------------------------------------------------------------ algebra

@pytest.mark.parametrize("S", SS)
def test_associativity_distributivity(S):
    rng = np.random.default_rng(21 + S)
    A, B, C = rand_mat(rng, 8, 10, S), rand_mat(rng, 10, 12, S), rand_mat(rng, 12, 9, S)
    assert np.array_equal(oracle.mul(oracle.mul(A, B, S), C, S), oracle.mul(A, oracle.mul(B, C, S), S))
    B2 = rand_mat(rng, 10, 12, S)
    assert np.array_equal(oracle.mul(A, np.maximum(B, B2), S),
                          np.maximum(oracle.mul(A, B, S), oracle.mul(A, B2, S)))
    A2 = rand_mat(rng, 8, 10, S)
    assert np.array_equal(oracle.mul(np.maximum(A, A2), B, S),
                          np.maximum(oracle.mul(A, B, S), oracle.mul(A2, B, S)))


@pytest.mark.parametrize("S", [255, 65535, S32])
def test_de_morgan_duality(S):
    rng = np.random.default_rng(31)
    A, B = rand_mat(rng, 11, 14, S, density=0.7), rand_mat(rng, 14, 9, S, density=0.7)
    nA, nB = (S - A.astype(np.int64)), (S - B.astype(np.int64))
    assert np.array_equal(S - oracle.mul(A, B, S).astype(np.int64), minplus_sat(nA, nB, S))


@pytest.mark.parametrize("S", [255, 65535, S32])
def test_boolean_embedding(S):
    rng = np.random.default_rng(41)
    A = rand_mat(rng, 30, 30, 1, density=0.07)
    B = rand_mat(rng, 30, 30, 1, density=0.2)
    assert np.array_equal(oracle.mul(A * S, B * S, S), oracle.mul(A, B, 1) * S)
    assert np.array_equal(oracle.warshall(A * S, S), oracle.warshall(A, 1) * S)


# ------------------------------------------------------------------ packed Boolean

def test_pack_bit_position():
    # entry (r, c) is bit (c & 7) of byte (c >> 3) of row r (Section 4 listing),
    # i.e. bit c % 64 of word c // 64 on a little-endian machine
    for c in [0, 1, 7, 8, 31, 32, 63, 64, 65, 99]:
        d = np.zeros((2, 100), np.uint8)
        d[1, c] = 1
        M = oracle.pack_bits(d)
        assert M.shape == (2, 2)
        assert int(M[0].sum()) == 0
        assert int(M[1, c // 64]) == 1 << (c % 64)
        assert int(M[1, 1 - c // 64]) == 0


def test_pack_roundtrip_and_padding():
    rng = np.random.default_rng(2)
    d = (rng.random((7, 130)) < 0.5).astype(np.uint8)
    M = oracle.pack_bits(d, ldw=4)
    assert np.array_equal(oracle.unpack_bits(M, 130), d)
    assert int(M[:, 3].sum()) == 0                                # extra word untouched
    assert int((M[:, 2] >> np.uint64(2)).sum()) == 0              # pad bits zero


def test_bool_packed_matches_dense():
    rng = np.random.default_rng(9)
    for (R, K, N) in [(5, 70, 129), (64, 64, 64), (33, 200, 65)]:
        A = rand_mat(rng, R, K, 1, density=0.05)
        B = rand_mat(rng, K, N, 1, density=0.1)
        P = oracle.bool_mul_w64(oracle.pack_bits(A), oracle.pack_bits(B), N)
        assert np.array_equal(oracle.unpack_bits(P, N), oracle.mul(A, B, 1))
        C = rand_mat(rng, R, N, 1, density=0.1)
        P2 = oracle.bool_mul_w64(oracle.pack_bits(A), oracle.pack_bits(B), N, C=oracle.pack_bits(C))
        assert np.array_equal(oracle.unpack_bits(P2, N), np.maximum(C, oracle.mul(A, B, 1)))


def test_bool_packed_closure_matches_dense_and_bfs():
    rng = np.random.default_rng(10)
    for D in [1, 5, 64, 65, 150]:
        A = rand_mat(rng, D, D, 1, density=1.5 / D)
        T = oracle.warshall(A, 1)
        Tp = oracle.bool_warshall_w64(oracle.pack_bits(A))
        assert np.array_equal(oracle.unpack_bits(Tp, D), T)
        Ap = oracle.pack_bits(A)
        for i in range(0, D, max(1, D // 7)):
            row = oracle.bool_closure_row_w64(Ap, i)
            assert np.array_equal(oracle.unpack_bits(row[None, :], D)[0], T[i])


def test_bool_closure_brute_force_small():
    rng = np.random.default_rng(12)
    for D in [3, 6]:
        A = rand_mat(rng, D, D, 1, density=0.3)
        T = brute_closure(A, 1)
        assert np.array_equal(oracle.unpack_bits(oracle.bool_warshall_w64(oracle.pack_bits(A)), D), T)


# ------------------------------------------------------------------ encoding

def test_encode_antidist():
    W = np.array([[0, 1, 30], [254, 255, 300]], np.uint32)
    assert oracle.encode_antidist(W, 255).tolist() == [[0, 254, 225], [1, 0, 0]]
    # a path of two encoded edges has the value of its summed length (Section 3)
    a, b = oracle.encode_antidist(np.array([[12, 40]], np.uint32), 255)[0]
    assert oracle.mul(np.array([[a]]), np.array([[b]]), 255)[0, 0] == 255 - 52


# ------------------------------------------------------------------ generator

def test_generator_deterministic_and_pointwise():
    A = synth.bernoulli(40, 50, 0.3, seed=4, s=0)
    assert np.array_equal(A, synth.bernoulli(40, 50, 0.3, seed=4, s=0))
    thr = synth.threshold(0.3)
    for (i, j) in [(0, 0), (3, 17), (39, 49)]:
        assert A[i, j] == (synth.h_int(4, 0, i, j) < thr)
    W = synth.weighted_graph(30, 30, 0.5, 1, 31, seed=1, s_edge=0)
    assert W.diagonal().sum() == 0 and W.max() <= 31
    nz = W[W > 0]
    assert nz.min() >= 1


def test_generator_density():
    A = synth.bernoulli(512, 512, 0.02, seed=0, s=0)
    assert abs(A.mean() - 0.02) < 0.002
    sizes = synth.log_uniform_sizes(2000, 32, 1024, seed=3)
    assert min(sizes) >= 32 and max(sizes) <= 1024
    mean_cube = np.mean(np.array(sizes, dtype=np.float64) ** 3)
    assert 0.8 < mean_cube / synth.expected_log_uniform_cube(32, 1024) < 1.25


# ------------------------------------------------------------------ distance form (f1) and entrywise (f3)

def brute_dist_closure(Dm, S):
    """min over simple paths (i != j) / simple cycles (i == j) of min(length, S);
    entries >= S are no edge."""
    Dm = np.asarray(Dm, dtype=np.int64)
    n = Dm.shape[0]
    T = np.full((n, n), S, dtype=np.int64)

    def dfs(src, v, length, seen):
        for u in range(n):
            w = Dm[v, u]
            if w >= S:
                continue
            L = min(length + w, S)
            if u == src:
                T[src, src] = min(T[src, src], L)
            elif u not in seen:
                T[src, u] = min(T[src, u], L)
                dfs(src, u, L, seen | {u})

    for i in range(n):
        dfs(i, i, 0, {i})
    return T.astype(np.uint32)


@pytest.mark.parametrize("S", [255, 65535, S32])
def test_dist_mul_by_de_morgan_and_brute_force(S):
    rng = np.random.default_rng(51)
    A, B = rand_mat(rng, 9, 13, S, density=0.6), rand_mat(rng, 13, 7, S, density=0.6)
    dA, dB = (S - A.astype(np.int64)).astype(np.uint32), (S - B.astype(np.int64)).astype(np.uint32)
    # De Morgan (Section 4): S − (A ⊗ B) = (S − A) + (S − B) in the distance form
    assert np.array_equal(oracle.dist_mul(dA, dB, S), (S - oracle.mul(A, B, S).astype(np.int64)).astype(np.uint32))
    assert np.array_equal(oracle.dist_mul(dA, dB, S), minplus_sat(dA, dB, S))
    Z = rand_mat(rng, 9, 7, S, density=0.9)
    assert np.array_equal(oracle.dist_mul(dA, dB, S, Z=Z), np.minimum(Z, minplus_sat(dA, dB, S)))


@pytest.mark.parametrize("S", [255, 65535, S32])
@pytest.mark.parametrize("D", [1, 4, 7])
def test_dist_closure_brute_force_and_de_morgan(S, D):
    rng = np.random.default_rng(60 + D)
    A = rand_mat(rng, D, D, S, density=0.5, lo=S - S // 3)
    dA = (S - A.astype(np.int64)).astype(np.uint32)        # absent edge (a = 0) -> S = infinity
    T = oracle.dist_closure(dA, S)
    assert np.array_equal(T, brute_dist_closure(dA, S))
    assert np.array_equal(T, (S - oracle.warshall(A, S).astype(np.int64)).astype(np.uint32))


def test_entrywise_table():
    # Conclusion table: & = min, | = max, ^ = |a − b|, ~ = S − a
    a = np.array([[0, 5, 255, 100]], np.uint32)
    b = np.array([[7, 5, 0, 200]], np.uint32)
    assert oracle.entrywise("and", a, b).tolist() == [[0, 5, 0, 100]]
    assert oracle.entrywise("or", a, b).tolist() == [[7, 5, 255, 200]]
    assert oracle.entrywise("xor", a, b).tolist() == [[7, 0, 255, 100]]
    assert oracle.entrywise("not", a, S=255).tolist() == [[255, 250, 0, 155]]
    bits_a, bits_b = np.array([[0, 0, 1, 1]], np.uint32), np.array([[0, 1, 0, 1]], np.uint32)
    assert oracle.entrywise("and", bits_a, bits_b, S=1).tolist() == [[0, 0, 0, 1]]
    assert oracle.entrywise("or", bits_a, bits_b, S=1).tolist() == [[0, 1, 1, 1]]
    assert oracle.entrywise("xor", bits_a, bits_b, S=1).tolist() == [[0, 1, 1, 0]]
    assert oracle.entrywise("not", bits_a, S=1).tolist() == [[1, 1, 0, 0]]
