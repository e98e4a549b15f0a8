"""The allocation-free Boolean closure (bool_closure_squaring_noalloc).

Some callers of this library cannot allocate device memory: another allocator
already owns the device, or a fixed memory budget or a no-synchronisation rule
forbids cudaMalloc.  This entry point runs the repeated-squaring closure in a
scratch array that ships inside the library.  These tests check it against the
regular entry point (bool_closure with SR_CLOSURE_SQUARING and a context
workspace), bit for bit, on calls in a row that share that scratch (a large
problem before a small one, so the small call runs over scratch the large one
filled), check that the calls after the first change the device's free memory
by nothing, and check that a problem too large for the scratch is refused.

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
    # one above the largest size that fits (8192 rows of 128 words, twice = 16 MiB)
    st = sr.lib.bool_closure_squaring_noalloc(1 << 20, 129, 8193, sr.SR_BOOL_W64, None)
    assert st == sr.SR_EINVAL and "scratch" in sr.last_error()
    # a leading dimension whose extent overflows the 2^46-word bound of every entry point
    st = sr.lib.bool_closure_squaring_noalloc(1 << 20, 1 << 41, 100, sr.SR_BOOL_W64, None)
    assert st == sr.SR_EINVAL and "too large" in sr.last_error()


def _garbage_pad(P, D, w):
    """Set every pad bit (columns D.. of the last word of each row)."""
    P = P.copy()
    r = D % w
    if r:
        mask = (~((1 << r) - 1)) & ((1 << w) - 1)
        P[:, -1] |= P.dtype.type(mask)
    return P


@pytest.mark.gpu
def test_noalloc_matches_workspace_entry_point_in_a_row():
    import torch
    from gpu_util import to_dev
    from paper_1705_08743_gb300 import _capi as sr

    # large, then small (reuses scratch the large call filled), then the largest that fits
    cases = [(synth.bool_dag_union(1500, seed=12), 32, 0, True),
             (synth.bool_dag_union(700, seed=11), 64, 2, True),
             (synth.bool_dag_union(8192, seed=13), 64, 0, False)]
    ctx = sr.sr_create(workspace_bytes=sr.sr_workspace_query(sr.SR_OP_BOOL_CLOSURE, sr.SR_BOOL_W64, 8192,
                                                              sr.SR_CLOSURE_SQUARING))
    try:
        # the first call on the device loads the library's scratch array
        one = to_dev(np.ones((1, 1), np.uint64))
        sr.bool_closure_squaring_noalloc(one, 1, 1, sr.SR_BOOL_W64)
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        for call, (G, w, pad, check_oracle) in enumerate(cases):
            dt = sr.SR_BOOL_W64 if w == 64 else sr.SR_BOOL_W32
            D = G.shape[0]
            P = _words(G, w)
            ref = to_dev(P, pad)
            sr.bool_closure(ctx, ref, ref.shape[1], D, dt, sr.SR_CLOSURE_SQUARING)
            # W64 input with every pad bit set: the result must ignore them and write them zero
            Pin = _garbage_pad(P, D, w) if w == 64 else P
            got = to_dev(Pin, pad)
            torch.cuda.synchronize()
            free1 = torch.cuda.mem_get_info()[0]
            sr.bool_closure_squaring_noalloc(got, got.shape[1], D, dt)
            torch.cuda.synchronize()
            assert torch.cuda.mem_get_info()[0] == free1, f"call {call}: device free memory changed"
            n = P.shape[1]
            assert torch.equal(got[:, :n], ref[:, :n]), f"call {call}: allocation-free result differs"
            if check_oracle:           # both equal the oracle's Warshall closure
                want = _words(oracle.warshall(G, 1).astype(np.uint8), w)
                assert np.array_equal(got[:, :n].cpu().numpy().view(want.dtype), want)
            del ref, got
        torch.cuda.synchronize()
        assert free0 > 0
    finally:
        sr.sr_destroy(ctx)


@pytest.mark.gpu
def test_noalloc_refuses_8193_on_a_device_buffer():
    import torch
    from paper_1705_08743_gb300 import _capi as sr
    T = torch.zeros((8193, 129), dtype=torch.int64, device="cuda")
    st = sr.lib.bool_closure_squaring_noalloc(T.data_ptr(), 129, 8193, sr.SR_BOOL_W64, None)
    assert st == sr.SR_EINVAL and "scratch" in sr.last_error()
    torch.cuda.synchronize()
    assert int(T.abs().sum().item()) == 0          # nothing was queued
