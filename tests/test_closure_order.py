"""The persistent closure's work order (sr_closure_order), checked on the host.

The persistent anti-distance closure runs the blocked Warshall/Floyd loop
(Section 2 Warshall, Section 3 Floyd) as work items that CTAs take in one fixed
order, each waiting for per-block versions.  Two properties make it correct and
free of deadlock, and both are properties of the order alone:

* every item's dependencies come earlier in the order (so the earliest unfinished
  item can always run), and each 64x64 block is updated exactly once per pivot
  block, in pivot order;
* the items, run in any order that respects those dependencies, compute the
  closure: checked by executing them with numpy in random dependency-respecting
  orders and comparing with the oracle's Warshall closure.
"""

import random

import numpy as np
import pytest

import oracle
import synth

PW, TT = 128, 128          # pivot block width, phase-3 tile side
BPT = TT // PW


def _blocks(item, nb):
    """(written blocks, operand blocks and the version each needs) of an item, from
    the definitions: tile (i, j) of pivot block s lies on the grid of pivot-width blocks
    without block row and column s, BPT grid blocks per tile side."""
    typ, s, i, j, j2 = item
    nbc = nb - 1

    def two(t):
        return [x if x < s else x + 1 for x in range(BPT * t, BPT * t + BPT) if x < nbc]

    if typ == 3:
        return [(s, s)], []
    if typ == 0:
        rows, cols = two(i), two(j) + (two(j2) if j2 >= 0 else [])
        return [(r, c) for r in rows for c in cols], [(r, s) for r in rows] + [(s, c) for c in cols]
    if typ == 1:
        return [(s, c) for c in two(j)], [(s, s)]
    return [(r, s) for r in two(i)], [(s, s)]


@pytest.mark.parametrize("D", [256, 257, 383, 384, 400, 513, 640, 1000, 1024, 1500, 2085, 4096, 8192])
@pytest.mark.parametrize("share", [0, 128, 256])
def test_order_respects_dependencies_and_covers_every_block(D, share):
    from paper_1705_08743_gb300 import _capi as sr
    order = sr.sr_closure_order(D, share)
    nb = (D + PW - 1) // PW
    ver = np.zeros((nb, nb), np.int64)
    for q, item in enumerate(order):
        typ, s, i, j, j2 = item
        bw = min(PW, D - PW * s)
        T = -(-(D - bw) // TT)                         # tiles per side of pivot block s's grid
        if typ == 0:
            assert 0 <= i < T and 0 <= j < T and (j2 == -1 or j < j2 < T), item
        elif typ in (1, 2):
            assert 0 <= (j if typ == 1 else i) < T, item
        w, rd = _blocks(item, nb)
        assert w, f"item {q} {item} writes nothing"
        for b in w:
            assert ver[b] == s, f"item {q} {item}: block {b} at version {ver[b]}, expected {s}"
        for b in rd:
            assert ver[b] >= s + 1, f"item {q} {item}: operand {b} not ready (version {ver[b]})"
        for b in w:
            ver[b] = s + 1
    assert (ver == nb).all(), "some block missed a pivot step"
    # per pivot block: one diagonal item, and phase 3 covers every block outside row/col s once
    assert sum(1 for it in order if it[0] == 3) == nb


def test_order_rejects_sizes_outside_its_range():
    from paper_1705_08743_gb300 import _capi as sr
    assert sr.lib.sr_closure_order(255, 128, None, 0) == -1
    assert sr.lib.sr_closure_order(256, 128, None, 0) > 0
    assert sr.lib.sr_closure_order(32769, 128, None, 0) == -1
    assert sr.lib.sr_closure_order(32768, 128, None, 0) > 0


def _mul(A, B, S):
    """max over k of max(A_ik + B_kj - S, 0) (Section 3 ⊗, Section 2 product), int64."""
    out = np.zeros((A.shape[0], B.shape[1]), np.int64)
    for k in range(A.shape[1]):
        out = np.maximum(out, np.maximum(A[:, k:k + 1] + B[k:k + 1, :] - S, 0))
    return out


def _run_item(T, item, D, S):
    typ, s, i, j, j2 = item
    k0 = s * PW
    bw = min(PW, D - k0)
    ks = slice(k0, k0 + bw)
    keep = np.r_[0:k0, k0 + bw:D]                  # rows/columns outside block s
    if typ == 3:
        Tk = T[ks, ks]
        for k in range(bw):                        # plain Floyd on the block
            Tk[:, :] = np.maximum(Tk, np.maximum(Tk[:, k:k + 1] + Tk[k:k + 1, :] - S, 0))
        return
    if typ == 0:
        rows = keep[i * TT:(i + 1) * TT]
        for jj in [j] + ([j2] if j2 >= 0 else []):
            cols = keep[jj * TT:(jj + 1) * TT]
            T[np.ix_(rows, cols)] = np.maximum(T[np.ix_(rows, cols)], _mul(T[rows][:, ks], T[ks][:, cols], S))
    elif typ == 1:
        cols = keep[j * TT:(j + 1) * TT]
        T[ks, cols] = np.maximum(T[ks, cols], _mul(T[ks, ks], T[ks, cols], S))
    else:
        rows = keep[i * TT:(i + 1) * TT]
        T[rows, ks] = np.maximum(T[rows, ks], _mul(T[rows, ks], T[ks, ks], S))


@pytest.mark.parametrize("D,seed", [(300, 0), (401, 1), (520, 2)])
def test_items_in_random_dependency_orders_give_the_closure(D, seed):
    """Execute the items with numpy, each time picking at random one of the next few
    items of the order whose dependencies are met (as concurrent CTAs might finish
    them), and compare with the oracle's Warshall closure."""
    from paper_1705_08743_gb300 import _capi as sr
    S = 255
    W = synth.cfg2_antidist(D=D, p=0.02, wlo=1, whi=60, seed=seed, s_edge=0, dtype=np.uint8)
    A = oracle.encode_antidist(W, S).astype(np.int64)
    want = oracle.warshall(A.astype(np.uint8), S).astype(np.int64)
    order = sr.sr_closure_order(D, 128)
    nb = (D + PW - 1) // PW
    rng = random.Random(seed)
    for trial in range(2):
        T = A.copy()
        ver = np.zeros((nb, nb), np.int64)
        pending = list(order)
        while pending:
            window = pending[:24]
            ready = [it for it in window
                     if all(ver[b] == it[1] for b in _blocks(it, nb)[0])
                     and all(ver[b] >= it[1] + 1 for b in _blocks(it, nb)[1])]
            assert ready, "no item of the window can run"
            it = rng.choice(ready)
            pending.remove(it)
            _run_item(T, it, D, S)
            for b in _blocks(it, nb)[0]:
                ver[b] = it[1] + 1
        assert np.array_equal(T, want), f"trial {trial}: closure differs"
