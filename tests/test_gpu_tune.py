"""The autotuner of the single calls (sr_autotune_closure / sr_autotune_mul) and its
JSON cache: choices are timed once, recorded per (op, dtype, size bucket), followed by
antidist_closure / bool_mul / antidist_mul while their options are automatic, and
reused by a later process from the cache file without timing again.  Results are
checked against the oracle (Section 2 Warshall / Section 3 Floyd, Section 2 product)."""

import json
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle
import synth
from gpu_util import to_dev, to_host

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _ws(sr, D):
    return max(sr.sr_workspace_query(sr.SR_OP_ANTIDIST_CLOSURE, sr.SR_U8, D),
               sr.sr_workspace_query(sr.SR_OP_BOOL_MUL, sr.SR_BOOL_W32, D))


def test_autotune_closure_cache_reused_by_another_process(tmp_path):
    import torch
    from paper_1705_08743_gb300 import _capi as sr
    cache = str(tmp_path / "tune.json")
    ctx = sr.sr_create(workspace_bytes=_ws(sr, 1024), tune_cache=cache)
    try:
        choice, ms = sr.sr_autotune_closure(ctx, sr.SR_U8, 1000, reps=1)
        assert choice in (128, 256, 512, sr.SR_TUNE_PERSISTENT, sr.SR_TUNE_FUSED) and ms > 0
        assert sr.sr_tune_get(ctx, sr.SR_OP_ANTIDIST_CLOSURE, sr.SR_U8, 1000) == (choice, pytest.approx(ms))
        bchoice, _ = sr.sr_autotune_mul(ctx, sr.SR_OP_BOOL_MUL, sr.SR_BOOL_W32, 700, reps=1)
        assert bchoice in (sr.SR_TUNE_BOOL_WORDS, sr.SR_TUNE_BOOL_TABLES, sr.SR_TUNE_BOOL_TENSOR)
        achoice, _ = sr.sr_autotune_mul(ctx, sr.SR_OP_ANTIDIST_MUL, sr.SR_U16, 300, reps=1)
        assert achoice in (64, 128)
        torch.cuda.synchronize()
    finally:
        sr.sr_destroy(ctx)
    with open(cache) as f:
        d = json.load(f)
    assert d["semiring_tune"] == 1 and d["sms"] > 0
    assert d["entries"]["closure/u8/1024"][0] == choice
    assert d["entries"]["bool_mul/w32/768"][0] == bchoice
    assert d["entries"]["antidist_mul/u16/384"][0] == achoice
    # a second process: the choices come from the file, and asking again times nothing
    child = f"""
import sys
sys.path.insert(0, {ROOT!r})
import torch
from paper_1705_08743_gb300 import _capi as sr
torch.cuda.init()
ctx = sr.sr_create(workspace_bytes=1 << 20, tune_cache={cache!r})
n0 = sr.sr_kernel_launches()
print(sr.sr_tune_get(ctx, sr.SR_OP_ANTIDIST_CLOSURE, sr.SR_U8, 1000)[0],
      sr.sr_autotune_closure(ctx, sr.SR_U8, 1000)[0],
      sr.sr_autotune_mul(ctx, sr.SR_OP_BOOL_MUL, sr.SR_BOOL_W32, 700)[0],
      sr.sr_kernel_launches() - n0)
sr.sr_destroy(ctx)
"""
    r = subprocess.run([sys.executable, "-c", child], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    got = [int(x) for x in r.stdout.split()]
    assert got == [choice, choice, bchoice, 0]


def test_single_calls_follow_the_recorded_choice():
    """A recorded choice steers the call while its options are automatic: the persistent
    schedule is one launch, a stream schedule several; an explicit option wins over the
    record; every result equals the oracle's."""
    import torch
    from paper_1705_08743_gb300 import _capi as sr
    D = 1000
    W = synth.cfg2_antidist(D=D, p=0.01, wlo=1, whi=60, seed=8)
    A = oracle.encode_antidist(W, 255).astype(np.uint8)
    want = oracle.warshall(A, 255)
    ctx = sr.sr_create(workspace_bytes=_ws(sr, D))

    def close():
        T = to_dev(A, 8)                                   # 1008-byte rows: vector path
        torch.cuda.synchronize()
        n0 = sr.sr_kernel_launches()
        sr.antidist_closure(ctx, T, T.shape[1], D, sr.SR_U8)
        torch.cuda.synchronize()
        sr.sr_stream_status(ctx)
        return to_host(T, np.uint8)[:, :D], sr.sr_kernel_launches() - n0

    try:
        sr.sr_tune_set(ctx, sr.SR_OP_ANTIDIST_CLOSURE, sr.SR_U8, D, sr.SR_TUNE_PERSISTENT)
        got, n = close()
        assert n == 1 and np.array_equal(got, want)
        sr.sr_tune_set(ctx, sr.SR_OP_ANTIDIST_CLOSURE, sr.SR_U8, D, 256)
        got, n = close()
        assert n > 1 and np.array_equal(got, want)
        sr.sr_tune_set(ctx, sr.SR_OP_ANTIDIST_CLOSURE, sr.SR_U8, D, sr.SR_TUNE_PERSISTENT)
        sr.sr_set_option(ctx, sr.SR_OPT_CLOSURE_PERSISTENT, 0)       # explicit: never
        got, n = close()
        assert n > 1 and np.array_equal(got, want)
        # Boolean product through each recorded path, and the anti-distance tile choice
        G1, G2 = synth.bool_dag_union(700, seed=3), synth.bool_dag_union(700, seed=4)
        want_b = oracle.pack_bits(oracle.mul(G1, G2, 1).astype(np.uint8)).view(np.uint32)
        Ad, Bd = to_dev(oracle.pack_bits(G1).view(np.uint32)), to_dev(oracle.pack_bits(G2).view(np.uint32))
        for path in (sr.SR_TUNE_BOOL_WORDS, sr.SR_TUNE_BOOL_TABLES, sr.SR_TUNE_BOOL_TENSOR):
            sr.sr_tune_set(ctx, sr.SR_OP_BOOL_MUL, sr.SR_BOOL_W32, 700, path)
            Cd = torch.zeros_like(Ad)
            sr.bool_mul(ctx, Ad, Ad.shape[1], Bd, Bd.shape[1], Cd, Cd.shape[1], 700, 700, 700, sr.SR_BOOL_W32, 0)
            torch.cuda.synchronize()
            assert np.array_equal(to_host(Cd, np.uint32), want_b), path
        B8 = oracle.encode_antidist(synth.cfg2_antidist(D=D, p=0.02, seed=9, s_edge=3), 255).astype(np.uint8)
        want_p = oracle.mul(A, B8, 255)
        for tile in (64, 128):
            sr.sr_tune_set(ctx, sr.SR_OP_ANTIDIST_MUL, sr.SR_U8, D, tile)
            Xd, Yd = to_dev(A), to_dev(B8)
            Zd = torch.zeros_like(Xd)
            sr.antidist_mul(ctx, Xd, D, Yd, D, Zd, D, D, D, D, sr.SR_U8, 0)
            torch.cuda.synchronize()
            assert np.array_equal(to_host(Zd, np.uint8), want_p), tile
        with pytest.raises(sr.SemiringError):
            sr.sr_tune_set(ctx, sr.SR_OP_ANTIDIST_CLOSURE, sr.SR_U8, D, 300)
        with pytest.raises(sr.SemiringError):
            sr.sr_tune_set(ctx, sr.SR_OP_BOOL_MUL, sr.SR_U8, D, sr.SR_TUNE_BOOL_TABLES)   # dtype of another op
    finally:
        sr.sr_destroy(ctx)


def test_tune_cache_from_another_gpu_is_not_used(tmp_path):
    from paper_1705_08743_gb300 import _capi as sr
    cache = tmp_path / "other.json"
    cache.write_text(json.dumps({"semiring_tune": 1, "device": "some other GPU", "sms": 7,
                                 "entries": {"closure/u8/1024": [512, 0, 0, 1.0]}}))
    ctx = sr.sr_create(tune_cache=str(cache))                # loads nothing, silently
    try:
        assert sr.sr_tune_get(ctx, sr.SR_OP_ANTIDIST_CLOSURE, sr.SR_U8, 1000) is None
        with pytest.raises(sr.SemiringError) as e:
            sr.sr_tune_load(ctx, str(cache))                  # explicitly: refused
        assert e.value.status == sr.SR_EINVAL
        bad = tmp_path / "bad.json"
        bad.write_text("{not json")
        with pytest.raises(sr.SemiringError):
            sr.sr_tune_load(ctx, str(bad))
        ctx3 = sr.sr_create(tune_cache=str(bad))             # a broken cache does not stop sr_create
        sr.sr_destroy(ctx3)
        # a save followed by a load round-trips
        sr.sr_tune_set(ctx, sr.SR_OP_ANTIDIST_MUL, sr.SR_U8, 5000, 64)
        out = str(tmp_path / "mine.json")
        sr.sr_tune_save(ctx, out)
        ctx2 = sr.sr_create()
        try:
            sr.sr_tune_load(ctx2, out)
            assert sr.sr_tune_get(ctx2, sr.SR_OP_ANTIDIST_MUL, sr.SR_U8, 5000)[0] == 64
        finally:
            sr.sr_destroy(ctx2)
    finally:
        sr.sr_destroy(ctx)
