"""Helpers for the GPU tests: numpy <-> CUDA tensors holding the library's
encodings (u8, u16 as int16 bit patterns, Boolean words as int32/int64)."""

import numpy as np

_VIEW = {np.dtype(np.uint8): np.uint8, np.dtype(np.uint16): np.int16,
         np.dtype(np.uint32): np.int32, np.dtype(np.uint64): np.int64}


def to_dev(a, pad_cols: int = 0):
    """Copy a 2-D numpy array to cuda:0; pad_cols extra columns (nonzero
    garbage) give a leading dimension larger than the row width."""
    import torch
    a = np.ascontiguousarray(a)
    if pad_cols:
        g = np.full((a.shape[0], a.shape[1] + pad_cols), 0xA5, dtype=a.dtype)
        g[:, :a.shape[1]] = a
        a = g
    v = a.view(_VIEW[a.dtype])
    return torch.from_numpy(v.copy()).cuda()


def to_host(t, dtype, cols=None):
    a = t.cpu().numpy().view(dtype)
    return a if cols is None else a[:, :cols]


def sr_dtype_of(npdt):
    import paper_1705_08743_gb300 as sr
    return {np.dtype(np.uint8): sr.SR_U8, np.dtype(np.uint16): sr.SR_U16,
            np.dtype(np.uint32): sr.SR_U32}[np.dtype(npdt)]
