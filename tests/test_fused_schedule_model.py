"""The anti-distance closure's fused-pass schedule (one launch per pivot block), run as a
host model with numpy and compared with the oracle's Warshall closure (Section 2
Warshall, Section 3 Floyd ⊕ = max, a ⊗ b = max(a + b − S, 0)).

The launch for pivot block kb starts with block kb closed and its panels made (a first
launch, kb = -1, closes block 0 and makes its panels). Its work items are:

1. block kb+1's update from kb, T[kb+1, kb+1] ⊕= T[kb+1, kb] ⊗ T[kb, kb+1];
2. the strips: kb's update of block row and column kb+1 outside blocks kb and kb+1;
3. block kb+1's closure, after item 1;
4. phase 3 of kb on every block outside block rows and columns kb and kb+1;
5. block kb+1's panels, its row outside block kb+1 and its column outside it, after
   items 2 and 3.

CTAs take the items in any order the two waits allow, and items run side by side. These
tests run each launch's items one at a time, in random orders that respect the waits.
Blocks are a few entries wide and D is ragged. Every order must give the oracle's closure,
and a schedule with item 2 left out must fail.
"""

import random

import numpy as np
import pytest

import oracle

S = 255


def _mul(X, Y):
    """X ⊗ Y over the anti-distance semiring (entries 0..S)."""
    if X.shape[1] == 0:
        return np.zeros((X.shape[0], Y.shape[1]), dtype=np.int64)
    return np.maximum((X[:, :, None] + Y[None, :, :] - S).max(axis=1), 0)


def _close_block(T, b):
    """In-place Warshall/Floyd closure of the diagonal block b (slice) of T."""
    for k in range(b.start, b.stop):
        T[b, b] = np.maximum(T[b, b], _mul(T[b, k:k + 1], T[k:k + 1, b]))


def _launch_items(nb, kb):
    """(name, args, waits) of the launch for pivot block kb."""
    items = []
    nxt = kb + 1 < nb
    if nxt:
        items.append(("upd", (), ()))
        items += [("strip_row", (j,), ()) for j in range(nb) if j not in (kb, kb + 1)]
        items += [("strip_col", (i,), ()) for i in range(nb) if i not in (kb, kb + 1)]
        items.append(("close", (), ("upd",)))
    items += [("p3", (i, j), ()) for i in range(nb) for j in range(nb)
              if i not in (kb, kb + 1) and j not in (kb, kb + 1)]
    if nxt:
        items += [("row_panel", (j,), ("close", "strip")) for j in range(nb) if j != kb + 1]
        items += [("col_panel", (i,), ("close", "strip")) for i in range(nb) if i != kb + 1]
    return items


def _order(items, rng):
    """A random order in which every item comes after all items of the kinds it waits for."""
    left = list(items)
    out = []
    while left:
        ready = [it for it in left
                 if not any(o is not it and o[0].startswith(w) for w in it[2] for o in left)]
        it = rng.choice(ready)
        left.remove(it)
        out.append(it)
    return out


def fused_schedule(A, B, rng, drop=()):
    T = A.astype(np.int64).copy()
    D = T.shape[0]
    nb = (D + B - 1) // B

    def blk(b):
        return slice(b * B, min(D, (b + 1) * B))

    def panels(b):
        for j in range(nb):
            if j != b:
                T[blk(b), blk(j)] = np.maximum(T[blk(b), blk(j)], _mul(T[blk(b), blk(b)], T[blk(b), blk(j)]))
        for i in range(nb):
            if i != b:
                T[blk(i), blk(b)] = np.maximum(T[blk(i), blk(b)], _mul(T[blk(i), blk(b)], T[blk(b), blk(b)]))

    _close_block(T, blk(0))                                # the launch with kb = -1
    panels(0)
    for kb in range(nb):
        k, k1 = blk(kb), blk(kb + 1) if kb + 1 < nb else None
        for name, args, _ in _order(_launch_items(nb, kb), rng):
            if name in drop:
                continue
            if name == "upd":
                T[k1, k1] = np.maximum(T[k1, k1], _mul(T[k1, k], T[k, k1]))
            elif name == "strip_row":
                j = blk(args[0])
                T[k1, j] = np.maximum(T[k1, j], _mul(T[k1, k], T[k, j]))
            elif name == "strip_col":
                i = blk(args[0])
                T[i, k1] = np.maximum(T[i, k1], _mul(T[i, k], T[k, k1]))
            elif name == "close":
                _close_block(T, k1)
            elif name == "p3":
                i, j = blk(args[0]), blk(args[1])
                T[i, j] = np.maximum(T[i, j], _mul(T[i, k], T[k, j]))
            elif name == "row_panel":
                j = blk(args[0])
                T[k1, j] = np.maximum(T[k1, j], _mul(T[k1, k1], T[k1, j]))
            elif name == "col_panel":
                i = blk(args[0])
                T[i, k1] = np.maximum(T[i, k1], _mul(T[i, k1], T[k1, k1]))
    return T


def _graph(rng, D, kind):
    v = rng.integers(1, S + 1, size=(D, D))
    if kind == "long":                      # strong edges on a shuffled path, weak elsewhere
        p = rng.permutation(D)
        A = np.where(rng.random((D, D)) < 2.0 / max(D, 1), rng.integers(1, S // 2, size=(D, D)), 0)
        A[p[:-1], p[1:]] = rng.integers(S - 8, S + 1, size=D - 1)
        return A
    return np.where(rng.random((D, D)) < 0.15, v, 0)


@pytest.mark.parametrize("D", [1, 3, 8, 9, 20, 33, 40])
@pytest.mark.parametrize("B", [2, 4, 8])
@pytest.mark.parametrize("kind", ["long", "dense"])
def test_fused_schedule_items_in_any_allowed_order_give_the_closure(D, B, kind):
    rng = np.random.default_rng(D * 97 + B * 5 + len(kind))
    A = _graph(rng, D, kind)
    want = oracle.warshall(A.astype(np.uint8), S).astype(np.int64)
    for seed in range(3):
        got = fused_schedule(A, B, random.Random(seed))
        assert np.array_equal(got, want), seed


def test_schedule_without_the_strips_fails():
    """Leaving out item 2 leaves block row and column kb+1 without kb's update: on a long
    path the closure comes out wrong, so the test above would notice missing strips."""
    rng = np.random.default_rng(3)
    A = _graph(rng, 32, "long")
    want = oracle.warshall(A.astype(np.uint8), S).astype(np.int64)
    got = fused_schedule(A, 4, random.Random(0), drop=("strip_row", "strip_col"))
    assert not np.array_equal(got, want)
