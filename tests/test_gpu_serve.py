"""Served request loop: mixed closure/product requests of every semiring admitted
concurrently under a device-memory budget.  Each result must equal the oracle
and the same request run alone through the direct C-ABI calls (all integer
arithmetic: bit-exact)."""

import numpy as np
import pytest

import oracle
from gpu_util import to_dev, to_host

pytestmark = pytest.mark.gpu


def _sr():
    from paper_1705_08743_gb300 import _capi as sr
    return sr


def pinned(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).pin_memory()


def rand_anti(rng, R, C, S, p=0.3, lo_frac=0.7):
    lo = max(1, int(S * lo_frac))
    v = rng.integers(lo, S + 1, size=(R, C), dtype=np.int64)
    return np.where(rng.random((R, C)) < p, v, 0).astype({255: np.uint8, 65535: np.uint16}.get(S, np.uint32))


def words(dense, w):
    """Dense rows of w-bit words (row width ceil(C/w) words), from the oracle's packing."""
    M = oracle.pack_bits(dense)
    if w == 64:
        return M
    return np.ascontiguousarray(M.view(np.uint32)[:, :(dense.shape[1] + 31) // 32])


def rand_bool_words(rng, R, C, p, w):
    d = (rng.random((R, C)) < p).astype(np.uint8)
    return d, words(d, w)


def build_requests(rng):
    """(kind, request fields, host inputs, expected result) for every semiring."""
    sr = _sr()
    reqs = []
    for D in [17, 100, 300, 640]:                           # anti-distance closures (small u8/u16 ones batch)
        for S, dt in [(255, sr.SR_U8), (65535, sr.SR_U16), (2 ** 32 - 1, sr.SR_U32)]:
            A = rand_anti(rng, D, D, S, p=min(1.0, 4.0 / D))
            reqs.append(dict(op=sr.SR_OP_ANTIDIST_CLOSURE, dtype=dt, R=D, A=A, B=None,
                             want=oracle.warshall(A, S).astype(A.dtype), cols=D))
    for (R, K, N) in [(50, 70, 90), (256, 130, 300)]:      # anti-distance products
        for S, dt in [(255, sr.SR_U8), (65535, sr.SR_U16), (2 ** 32 - 1, sr.SR_U32)]:
            A, B = rand_anti(rng, R, K, S, p=0.5), rand_anti(rng, K, N, S, p=0.5)
            reqs.append(dict(op=sr.SR_OP_ANTIDIST_MUL, dtype=dt, R=R, K=K, N=N, A=A, B=B,
                             want=oracle.mul(A, B, S).astype(A.dtype), cols=N))
    for D, w, method in [(200, 64, 0), (333, 32, 1), (1000, 64, 0), (129, 32, 0)]:   # Boolean closures
        d, M = rand_bool_words(rng, D, D, 1.5 / D, w)
        want = words(oracle.warshall(d, 1).astype(np.uint8), w)
        reqs.append(dict(op=sr.SR_OP_BOOL_CLOSURE, dtype=sr.SR_BOOL_W64 if w == 64 else sr.SR_BOOL_W32, R=D,
                         A=M, B=None, method=method, want=want, cols=D))
    for (R, K, N, w) in [(70, 200, 90, 32), (300, 64, 500, 64)]:                     # Boolean products
        da, A = rand_bool_words(rng, R, K, 0.05, w)
        db, B = rand_bool_words(rng, K, N, 0.05, w)
        want = words(oracle.mul(da, db, 1).astype(np.uint8), w)
        reqs.append(dict(op=sr.SR_OP_BOOL_MUL, dtype=sr.SR_BOOL_W64 if w == 64 else sr.SR_BOOL_W32, R=R, K=K,
                         N=N, A=A, B=B, want=want, cols=N))
    return reqs


def run_alone(q):
    """The same request through the direct entry points, one call at a time."""
    import torch
    sr = _sr()
    if q["op"] in (sr.SR_OP_ANTIDIST_CLOSURE, sr.SR_OP_BOOL_CLOSURE):
        T = to_dev(q["A"])
        if q["op"] == sr.SR_OP_ANTIDIST_CLOSURE:
            sr.antidist_closure(None, T, T.shape[1], q["R"], q["dtype"])
        else:
            ctx = sr.sr_create(workspace_bytes=sr.sr_workspace_query(sr.SR_OP_BOOL_CLOSURE, q["dtype"], q["R"], 1))
            sr.bool_closure(ctx, T, T.shape[1], q["R"], q["dtype"], q.get("method", 0))
            torch.cuda.synchronize()
            sr.sr_destroy(ctx)
        return to_host(T, q["A"].dtype)
    A, B = to_dev(q["A"]), to_dev(q["B"])
    C = torch.zeros((q["R"], q["want"].shape[1]), dtype=A.dtype, device="cuda")
    fn = sr.antidist_mul if q["op"] == sr.SR_OP_ANTIDIST_MUL else sr.bool_mul
    fn(None, A, A.shape[1], B, B.shape[1], C, C.shape[1], q["R"], q["K"], q["N"], q["dtype"], 0)
    return to_host(C, q["A"].dtype)


def submit_all(ctx, reqs):
    sr = _sr()
    tickets, outs, keep = [], [], []
    for q in reqs:
        A, B = pinned(q["A"]), (pinned(q["B"]) if q["B"] is not None else None)
        out = pinned(np.zeros_like(q["want"]))
        keep.append((A, B, out))
        r = sr.make_request(q["op"], q["dtype"], q["R"], q.get("K", 0), q.get("N", 0), A=A, B=B, out=out,
                            method=q.get("method", 0))
        tickets.append(sr.sr_submit(ctx, r))
        outs.append(out)
    return tickets, outs, keep


def test_mixed_requests_match_alone_and_oracle():
    sr = _sr()
    rng = np.random.default_rng(0)
    reqs = build_requests(rng)
    ctx = sr.sr_create()
    try:
        sr.sr_serve_start(ctx, arena_bytes=256 << 20, slots=4)
        tickets, outs, _keep = submit_all(ctx, reqs)
        for t in tickets:
            sr.sr_wait(ctx, t, 60000)
        stats = sr.sr_serve_stats(ctx)
        for q, t, out in zip(reqs, tickets, outs):
            got = out.numpy()
            assert np.array_equal(got, q["want"]), (q["op"], q["dtype"], q["R"])
            assert np.array_equal(got, run_alone(q)), "differs from the same request run alone"
            info = sr.sr_result(ctx, t)
            assert info.status == 0 and info.latency_ms >= info.queue_ms >= 0
            sr.sr_release(ctx, t)
        assert stats["completed"] == len(reqs) and stats["failed"] == 0
        assert stats["batches"] >= 1
    finally:
        sr.sr_destroy(ctx)


def test_admission_under_small_arena():
    """Arena for ~3 requests at a time: everything completes, peak use within budget."""
    sr = _sr()
    rng = np.random.default_rng(1)
    D = 700
    reqs = []
    for i in range(12):
        A = rand_anti(rng, D, D, 65535, p=4.0 / D)
        reqs.append(dict(op=sr.SR_OP_ANTIDIST_CLOSURE, dtype=sr.SR_U16, R=D, A=A, B=None,
                         want=oracle.warshall(A, 65535).astype(np.uint16)))
    budget = 3 * (D * (D + 8) * 2 + 4096)
    ctx = sr.sr_create()
    try:
        sr.sr_serve_start(ctx, arena_bytes=budget, slots=8, batch_max_d=256)
        tickets, outs, _k = submit_all(ctx, reqs)
        for t in tickets:
            sr.sr_wait(ctx, t, 60000)
        for q, out in zip(reqs, outs):
            assert np.array_equal(out.numpy(), q["want"])
        st = sr.sr_serve_stats(ctx)
        assert st["arena_peak_bytes"] <= budget and st["completed"] == 12
        assert st["arena_in_use"] == 0
        # larger than the whole arena: refused at submission
        big = pinned(np.zeros((2000, 2000), np.uint16))
        with pytest.raises(sr.SemiringError) as e:
            sr.sr_submit(ctx, sr.make_request(sr.SR_OP_ANTIDIST_CLOSURE, sr.SR_U16, 2000, A=big, out=big))
        assert e.value.status == sr.SR_ENOMEM
    finally:
        sr.sr_destroy(ctx)


def test_resident_matrices_and_kept_results():
    sr = _sr()
    rng = np.random.default_rng(2)
    D = 300
    A = rand_anti(rng, D, D, 255, p=3.0 / D)
    B = rand_anti(rng, D, D, 255, p=0.2)
    ctx = sr.sr_create()
    try:
        sr.sr_serve_start(ctx, arena_bytes=64 << 20)
        hB = sr.sr_resident_put(ctx, pinned(B), D, D, sr.SR_U8)
        # closure kept resident, then used as the left operand of a product with resident B
        t1 = sr.sr_submit(ctx, sr.make_request(sr.SR_OP_ANTIDIST_CLOSURE, sr.SR_U8, D, A=pinned(A), keep=1))
        sr.sr_wait(ctx, t1)
        hT = sr.sr_result(ctx, t1).resident
        assert hT != 0
        out = pinned(np.zeros((D, D), np.uint8))
        t2 = sr.sr_submit(ctx, sr.make_request(sr.SR_OP_ANTIDIST_MUL, sr.SR_U8, D, D, D, rA=hT, rB=hB, out=out))
        sr.sr_wait(ctx, t2)
        T = oracle.warshall(A, 255)
        assert np.array_equal(out.numpy(), oracle.mul(T, B, 255))
        back = pinned(np.zeros((D, D), np.uint8))
        sr.sr_resident_get(ctx, hT, back)
        assert np.array_equal(back.numpy(), T)
        sr.sr_resident_free(ctx, hT)
        sr.sr_resident_free(ctx, hB)
        with pytest.raises(sr.SemiringError) as e:
            sr.sr_submit(ctx, sr.make_request(sr.SR_OP_ANTIDIST_MUL, sr.SR_U8, D, D, D, rA=hT, rB=hB, out=out))
        assert e.value.status == sr.SR_ENOTFOUND
    finally:
        sr.sr_destroy(ctx)


def test_wait_timeout_and_bad_requests():
    sr = _sr()
    rng = np.random.default_rng(3)
    ctx = sr.sr_create()
    try:
        sr.sr_serve_start(ctx, arena_bytes=512 << 20, slots=1)
        D = 3000
        A = pinned(rand_anti(rng, D, D, 65535, p=4.0 / D))
        out = pinned(np.zeros((D, D), np.uint16))
        t = sr.sr_submit(ctx, sr.make_request(sr.SR_OP_ANTIDIST_CLOSURE, sr.SR_U16, D, A=A, out=out))
        with pytest.raises(sr.SemiringError) as e:
            sr.sr_wait(ctx, t, 0)                      # a host-side wait with no time to wait
        assert e.value.status == sr.SR_ETIMEOUT
        try:
            sr.sr_result(ctx, t)                         # finished already, or SR_EBUSY
        except sr.SemiringError as e:
            assert e.status == sr.SR_EBUSY
        sr.sr_wait(ctx, t, 120000)
        with pytest.raises(sr.SemiringError) as e:     # op / dtype mismatch
            sr.sr_submit(ctx, sr.make_request(sr.SR_OP_BOOL_MUL, sr.SR_U8, 10, A=A, B=A, out=out))
        assert e.value.status == sr.SR_EINVAL
        with pytest.raises(sr.SemiringError) as e:
            sr.sr_poll(ctx, 123456789)
        assert e.value.status == sr.SR_ENOTFOUND
    finally:
        sr.sr_destroy(ctx)


def test_cancel_waiting_request():
    """A request withdrawn while it waits never runs: its output stays untouched and
    sr_wait reports SR_ECANCELED; the requests around it still match the oracle."""
    sr = _sr()
    rng = np.random.default_rng(5)
    ctx = sr.sr_create()
    try:
        sr.sr_serve_start(ctx, arena_bytes=512 << 20, slots=1)
        D = 1200                                     # the closure holds the one slot while the rest queue
        A0 = pinned(rand_anti(rng, D, D, 65535, p=4.0 / D))
        out0 = pinned(np.zeros((D, D), np.uint16))
        prods = []
        for i in range(4):                           # products queue behind it (products never group)
            A, B = rand_anti(rng, 200, 150, 255, p=0.5), rand_anti(rng, 150, 230, 255, p=0.5)
            prods.append([None, pinned(np.full((200, 230), 7, np.uint8)), oracle.mul(A, B, 255).astype(np.uint8),
                          (pinned(A), pinned(B))])
        t0 = sr.sr_submit(ctx, sr.make_request(sr.SR_OP_ANTIDIST_CLOSURE, sr.SR_U16, D, A=A0, out=out0))
        for p in prods:
            p[0] = sr.sr_submit(ctx, sr.make_request(sr.SR_OP_ANTIDIST_MUL, sr.SR_U8, 200, 150, 230, A=p[3][0],
                                                     B=p[3][1], out=p[1]))
        victim = prods[-1][0]                        # last in line: waits until the four before it finish
        sr.sr_cancel(ctx, victim)
        sr.sr_cancel(ctx, victim)                    # a second cancel changes nothing
        with pytest.raises(sr.SemiringError) as e:
            sr.sr_wait(ctx, victim, 1000)
        assert e.value.status == sr.SR_ECANCELED
        assert sr.sr_result(ctx, victim).status == sr.SR_ECANCELED
        sr.sr_wait(ctx, t0, 120000)
        assert np.array_equal(out0.numpy(), oracle.warshall(A0.numpy(), 65535).astype(np.uint16))
        for t, out, want, _ in prods[:-1]:
            sr.sr_wait(ctx, t, 60000)
            assert np.array_equal(out.numpy(), want)
        assert (prods[-1][1].numpy() == 7).all()     # never written
        with pytest.raises(sr.SemiringError) as e:
            sr.sr_cancel(ctx, 987654321)
        assert e.value.status == sr.SR_ENOTFOUND
        sr.sr_cancel(ctx, t0)                        # finished: no effect
        assert sr.sr_result(ctx, t0).status == sr.SR_OK
        st = sr.sr_serve_stats(ctx)
        assert st["cancelled"] == 1 and st["pending"] == 0 and st["arena_in_use"] == 0
        for t in [t0, victim] + [p[0] for p in prods[:-1]]:
            sr.sr_release(ctx, t)
    finally:
        sr.sr_destroy(ctx)
