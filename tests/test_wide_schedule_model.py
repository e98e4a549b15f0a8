"""The Boolean closure's wide-block schedule (the tensor-core Warshall schedule), run as
a host model with numpy and compared with the oracle's Warshall closure (Section 2).

Per pivot block kb the schedule makes both panels of kb, each over the whole row or
column; then phase 3 covers every tile except block row kb, block column kb and the next
diagonal block (kb+1, kb+1). Beside phase 3, the next diagonal block takes its update from
kb and is closed by repeated squaring (Section 2's A ⊗ (I ⊕ A)^(2^m) identity).
Phase 3 leaves block row and column kb out because it would not change them once the
panels are made: T_kj ⊕ T_kk ⊗ T_kj = T_kj when T_kk is closed, and the same holds down
the column.
These tests execute exactly those steps on small matrices with narrow blocks. The
result must equal the oracle's closure. A variant that also skips a band phase 3 does
need must fail, so the tests can tell the skips apart.
"""

import numpy as np
import pytest

import oracle


def _mm(X, Y):
    return (X.astype(np.int64) @ Y.astype(np.int64)) > 0


def _squaring_closure(A):
    """Non-reflexive closure A ⊗ (I ⊕ A)^(2^m), m = ceil(log2(n - 1)), by squaring."""
    n = A.shape[0]
    M = A | np.eye(n, dtype=bool)
    m = 0
    while (1 << m) < max(n - 1, 1):
        m += 1
    for _ in range(m):
        M = _mm(M, M)
    return _mm(A, M)


def wide_schedule(A, W, skip_panels=True, extra_skip=None):
    T = A.astype(bool).copy()
    D = T.shape[0]
    nb = (D + W - 1) // W

    def blk(b):
        return slice(b * W, min(D, (b + 1) * W))

    T[blk(0), blk(0)] = _squaring_closure(T[blk(0), blk(0)])
    for kb in range(nb):
        k = blk(kb)
        Tkk = T[k, k].copy()
        T[k, :] |= _mm(Tkk, T[k, :])                        # row panel, every word
        T[:, k] |= _mm(T[:, k], Tkk)                        # column panel, every row
        upd = _mm(T[:, k], T[k, :])                         # phase 3's products
        keep = np.ones((D, D), dtype=bool)
        if skip_panels:
            keep[k, :] = False
            keep[:, k] = False
        if kb + 1 < nb:
            k1 = blk(kb + 1)
            keep[k1, k1] = False
            # the next diagonal block beside phase 3: its update from kb, then its closure
            T[k1, k1] |= _mm(T[k1, k], T[k, k1])
            T[k1, k1] = _squaring_closure(T[k1, k1])
            if extra_skip is not None:
                keep[extra_skip(kb, D, W)] = False
        T |= upd & keep
    return T


def _graph(rng, D, kind):
    if kind == "sparse":
        return rng.random((D, D)) < 1.5 / max(D, 1)
    if kind == "chain":                       # a long path through every block, in a shuffled order
        p = rng.permutation(D)
        A = np.zeros((D, D), dtype=bool)
        A[p[:-1], p[1:]] = True
        return A
    return rng.random((D, D)) < 0.08


@pytest.mark.parametrize("D", [1, 2, 7, 16, 17, 33, 64, 70, 101])
@pytest.mark.parametrize("W", [4, 8, 16, 32])
@pytest.mark.parametrize("kind", ["sparse", "chain", "dense"])
def test_wide_schedule_with_panels_skipped_gives_the_closure(D, W, kind):
    rng = np.random.default_rng(D * 131 + W * 7 + len(kind))
    A = _graph(rng, D, kind)
    want = oracle.warshall(A.astype(np.uint8), 1).astype(bool)
    assert np.array_equal(wide_schedule(A, W), want)
    assert np.array_equal(wide_schedule(A, W, skip_panels=False), want)


def test_skipping_a_needed_band_is_detected():
    """Skipping block row kb+1 outside the diagonal block (which phase 3 must update) gives
    a wrong closure on a chain, so the tests above would catch a band chosen wrongly."""
    rng = np.random.default_rng(5)
    D, W = 64, 8
    A = _graph(rng, D, "chain")
    want = oracle.warshall(A.astype(np.uint8), 1).astype(bool)

    def next_row_band(kb, D, W):
        return (slice((kb + 1) * W, min(D, (kb + 2) * W)), slice(None))

    assert not np.array_equal(wide_schedule(A, W, extra_skip=next_row_band), want)
