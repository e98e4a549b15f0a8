"""Shape-inferring wrappers over the C ABI for contiguous torch tensors.

Anti-distance matrices are uint8 (S = 255), uint16-valued (S = 65535, stored as
torch.uint16 or int16 bit patterns) or uint32-valued tensors (S = 2^32 − 1, stored
as torch.uint32 or int32 bit patterns); Boolean matrices are int32/int64 tensors
of packed words (32/64 columns per word).  Each helper reads shapes and leading
dimensions off the tensor and calls the C function of the same role.
"""

from __future__ import annotations

import torch

from . import _capi as C


def anti_dtype(t: torch.Tensor) -> int:
    if t.dtype == torch.uint8:
        return C.SR_U8
    if t.dtype in (torch.int16, getattr(torch, "uint16", torch.int16)):
        return C.SR_U16
    if t.dtype in (torch.int32, getattr(torch, "uint32", torch.int32)):
        return C.SR_U32
    raise TypeError(f"anti-distance tensors are uint8, 16-bit or 32-bit, got {t.dtype}")


def bool_dtype(t: torch.Tensor) -> int:
    if t.dtype in (torch.int32, getattr(torch, "uint32", torch.int32)):
        return C.SR_BOOL_W32
    if t.dtype in (torch.int64, getattr(torch, "uint64", torch.int64)):
        return C.SR_BOOL_W64
    raise TypeError(f"Boolean tensors hold 32- or 64-bit words, got {t.dtype}")


def _ld(t: torch.Tensor) -> int:
    assert t.dim() == 2 and t.stride(1) == 1, "row-major 2-D tensor with unit column stride expected"
    return t.stride(0)


def antidist_mul(A, B, C_out=None, accumulate=False, ctx=None, stream=None):
    R, K = A.shape
    N = B.shape[1]
    if C_out is None:
        C_out = torch.zeros((R, N), dtype=A.dtype, device=A.device)
    C.antidist_mul(ctx, A, _ld(A), B, _ld(B), C_out, _ld(C_out), R, K, N, anti_dtype(A), int(accumulate), stream)
    return C_out


def antidist_closure(T, ctx=None, stream=None):
    D = T.shape[0]
    C.antidist_closure(ctx, T, _ld(T), D, anti_dtype(T), stream)
    return T


def bool_mul(A, B, N: int, K: int, C_out=None, accumulate=False, ctx=None, stream=None):
    R = A.shape[0]
    dt = bool_dtype(A)
    if C_out is None:
        w = 32 if dt == C.SR_BOOL_W32 else 64
        C_out = torch.zeros((R, (N + w - 1) // w), dtype=A.dtype, device=A.device)
    C.bool_mul(ctx, A, _ld(A), B, _ld(B), C_out, _ld(C_out), R, K, N, dt, int(accumulate), stream)
    return C_out


def bool_closure(T, D: int, method=C.SR_CLOSURE_WARSHALL, ctx=None, stream=None):
    C.bool_closure(ctx, T, _ld(T), D, bool_dtype(T), method, stream)
    return T
