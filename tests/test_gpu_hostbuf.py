"""Pinned host buffers as operands (sr_host_mapped): on a device that addresses pinned
host memory at the same pointer, antidist_encode reads its input and antidist_mul its
operands from host memory, and a product writes its result there, over the host link.
Results equal the device-buffer calls' and the oracle's (Section 3 encoding, Section 2
product).  Every host-memory call is made only after sr_host_mapped confirmed the
mapping."""

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def test_host_mapped_query():
    import torch
    import paper_1705_08743_gb300 as sr
    dev = torch.zeros(64, dtype=torch.uint8, device="cuda")
    pinned = torch.zeros(64, dtype=torch.uint8).pin_memory()
    pageable = np.zeros(64, np.uint8)
    assert not sr.sr_host_mapped(dev)
    assert not sr.sr_host_mapped(pageable.ctypes.data)
    assert not sr.sr_host_mapped(0)
    assert sr.sr_host_mapped(pinned)           # GB300 with unified addressing


@pytest.mark.parametrize("D", [300, 1000])
def test_encode_and_product_on_pinned_host_buffers(D):
    import torch
    import paper_1705_08743_gb300 as sr
    W = synth.cfg2_antidist(D=D, seed=5)
    W2 = synth.cfg2_antidist(D=D, seed=5, s_edge=3)
    hW = torch.from_numpy(W).pin_memory()
    hW2 = torch.from_numpy(W2).pin_memory()
    hC = torch.full((D, D), 7, dtype=torch.uint8).pin_memory()
    if not (sr.sr_host_mapped(hW) and sr.sr_host_mapped(hW2) and sr.sr_host_mapped(hC)):
        pytest.skip("pinned host memory is not mapped into the device address space")
    A = oracle.encode_antidist(W, 255).astype(np.uint8)
    B = oracle.encode_antidist(W2, 255).astype(np.uint8)
    # encode straight from host memory into a device matrix
    T = torch.empty((D, D), dtype=torch.uint8, device="cuda")
    sr.antidist_encode(None, hW, D, T, D, D, D, sr.SR_U8)
    torch.cuda.synchronize()
    assert np.array_equal(T.cpu().numpy(), A)
    # product: A from host memory, B on the device, C written into host memory
    hA = torch.from_numpy(A).pin_memory()
    Bd = torch.from_numpy(B).cuda()
    sr.antidist_mul(None, hA, D, Bd, D, hC, D, D, D, D, sr.SR_U8, 0)
    torch.cuda.synchronize()
    want = oracle.mul(A, B, 255)
    assert np.array_equal(hC.numpy(), want)
    Cd = torch.empty((D, D), dtype=torch.uint8, device="cuda")
    sr.antidist_mul(None, torch.from_numpy(A).cuda(), D, Bd, D, Cd, D, D, D, D, sr.SR_U8, 0)
    torch.cuda.synchronize()
    assert np.array_equal(Cd.cpu().numpy(), hC.numpy())


def test_pack_from_pinned_host_input():
    """bool_pack reads a dense 0/1 matrix in pinned host memory (the Boolean workloads'
    zero-copy input path): the same words as packing the device copy, and the oracle's
    bit layout (Section 4 matBool)."""
    import torch
    import paper_1705_08743_gb300 as sr
    D = 1000
    dense = synth.bool_dag_union(D, seed=7).astype(np.uint8)
    h = torch.from_numpy(dense).pin_memory()
    if not sr.sr_host_mapped(h):
        pytest.skip("pinned host memory is not mapped into the device address space")
    nw = (D + 31) // 32
    out_h = torch.zeros((D, nw), dtype=torch.int32, device="cuda")
    out_d = torch.zeros_like(out_h)
    sr.bool_pack(None, h, D, out_h, nw, D, D, sr.SR_BOOL_W32)
    sr.bool_pack(None, torch.from_numpy(dense).cuda(), D, out_d, nw, D, D, sr.SR_BOOL_W32)
    torch.cuda.synchronize()
    assert torch.equal(out_h, out_d)
    assert np.array_equal(out_h.cpu().numpy().view(np.uint32), oracle.pack_bits(dense).view(np.uint32))
