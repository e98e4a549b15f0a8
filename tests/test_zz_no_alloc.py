"""The allocation-free Boolean closure (bool_closure_squaring_noalloc).

Some callers of this library cannot allocate device memory — another allocator
already owns the device, or a fixed memory budget or a no-synchronisation rule
forbids cudaMalloc — so this entry point runs the repeated-squaring closure in a
scratch array that ships inside the library.  These tests check it against the
regular entry point (bool_closure with SR_CLOSURE_SQUARING and a context
workspace), bit for bit, on two calls in a row that share that scratch, and
check that a problem too large for the scratch is refused.

The file is named to be collected last, so a run that stops at its first
failure has run every other test before this one.
"""

import numpy as np
import pytest

import oracle
import synth


def _words(dense, w):
    M = oracle.pack_bits(dense)
    return M if w == 64 else M.view(np.uint32)


def test_rejects_problem_larger_than_scratch():
    from paper_1705_08743_gb300 import _capi as sr
    # validated before any CUDA call: runs on a host without a GPU
    st = sr.lib.bool_closure_squaring_noalloc(1 << 20, 129, 8200, sr.SR_BOOL_W64, None)
    assert st == sr.SR_EINVAL
    assert "scratch" in sr.last_error()
    st = sr.lib.bool_closure_squaring_noalloc(1 << 20, 1, 100, sr.SR_U8, None)
    assert st == sr.SR_EINVAL


@pytest.mark.gpu
def test_noalloc_matches_workspace_entry_point_twice():
    import torch
    from gpu_util import to_dev
    from paper_1705_08743_gb300 import _capi as sr

    cases = [(synth.bool_dag_union(700, seed=11), 64), (synth.bool_dag_union(1500, seed=12), 32)]
    ctx = sr.sr_create(workspace_bytes=sr.sr_workspace_query(sr.SR_OP_BOOL_CLOSURE, sr.SR_BOOL_W64, 1500,
                                                              sr.SR_CLOSURE_SQUARING))
    try:
        for call, (G, w) in enumerate(cases):          # two calls in a row share the scratch
            dt = sr.SR_BOOL_W64 if w == 64 else sr.SR_BOOL_W32
            D = G.shape[0]
            P = _words(G, w)
            ref = to_dev(P)
            sr.bool_closure(ctx, ref, ref.shape[1], D, dt, sr.SR_CLOSURE_SQUARING)
            got = to_dev(P)
            sr.bool_closure_squaring_noalloc(got, got.shape[1], D, dt)
            torch.cuda.synchronize()
            assert torch.equal(got, ref), f"call {call}: allocation-free result differs"
            # and both equal the oracle's Warshall closure
            want = _words(oracle.warshall(G, 1).astype(np.uint8), w)
            assert np.array_equal(got.cpu().numpy().view(want.dtype), want)
    finally:
        sr.sr_destroy(ctx)
