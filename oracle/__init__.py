"""CPU oracle for the semiring product and closure (arXiv 1705.08743).

TEST INFRASTRUCTURE ONLY: tests, the smoke check and the benchmark's CPU
baseline may import this package; the library under
``paper_1705_08743_gb300`` never does, and the two share no code.

The arithmetic lives in ``oracle.c`` (plain C, OpenMP over independent rows);
this module compiles it with gcc on first use and wraps it for numpy arrays.
Entries are integers in {0..S}: S = 1 is the Boolean semiring of Section 2,
S = 255 / 65535 / 2^32 − 1 the anti-distance matrices of Sections 3-4 (all
sums are formed in 64 bits, so the u32 type needs no special case).

Parity status of each function is recorded in the tests that pin it
(``tests/test_oracle_pins.py``): every function here is pinned against
something other than itself (closed forms, brute-force path enumeration,
scipy's Floyd-Warshall, the paper's identities).
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

_i64 = ctypes.c_int64
_u32 = ctypes.c_uint32
_p = ctypes.c_void_p


def build(force: bool = False) -> str:
    """Compile oracle.c into _build/liboracle.so (gcc -O3 -fopenmp)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O3", "-std=c11", "-fopenmp", "-fPIC", "-shared", _SRC, "-o", tmp]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            sig = {
                "or_num_threads": (ctypes.c_int, []),
                "or_set_num_threads": (None, [ctypes.c_int]),
                "or_mul": (None, [_p, _p, _p, _i64, _i64, _i64, _u32, ctypes.c_int]),
                "or_mul_entry": (_u32, [_p, _p, _i64, _i64, _i64, _i64, _u32]),
                "or_warshall": (None, [_p, _i64, _u32]),
                "or_closure_squaring": (None, [_p, _p, _i64, _u32, _p]),
                "or_closure_row": (None, [_p, _i64, _u32, _i64, _p]),
                "or_pack_bits": (None, [_p, _i64, _i64, _p, _i64]),
                "or_unpack_bits": (None, [_p, _i64, _i64, _i64, _p]),
                "or_bool_mul_w64": (None, [_p, _i64, _p, _i64, _p, _i64, _i64, _i64, _i64, ctypes.c_int]),
                "or_bool_warshall_w64": (None, [_p, _i64, _i64]),
                "or_bool_closure_row_w64": (None, [_p, _i64, _i64, _i64, _p]),
                "or_encode_antidist": (None, [_p, _i64, _u32, _p]),
                "or_dist_mul": (None, [_p, _p, _p, _i64, _i64, _i64, _u32, ctypes.c_int]),
                "or_dist_closure": (None, [_p, _i64, _u32]),
                "or_entrywise": (None, [ctypes.c_int, _p, _p, _p, _i64, _u32]),
            }
            for name, (res, args) in sig.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def _u32c(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.uint32)


def num_threads() -> int:
    return _load().or_num_threads()


def set_num_threads(n: int) -> None:
    _load().or_set_num_threads(int(n))


# ---------------------------------------------------------------- dense {0..S}

def mul(A, B, S: int, C=None) -> np.ndarray:
    """(C if given else 0) ⊕ A ⊗ B over {0..S}; returns a new uint32 array."""
    A, B = _u32c(A), _u32c(B)
    R, K = A.shape
    K2, N = B.shape
    assert K == K2
    out = np.zeros((R, N), np.uint32) if C is None else _u32c(C).copy()
    _load().or_mul(_ptr(A), _ptr(B), _ptr(out), R, K, N, S, 0 if C is None else 1)
    return out


def mul_entry(A, B, i: int, j: int, S: int) -> int:
    A, B = _u32c(A), _u32c(B)
    return int(_load().or_mul_entry(_ptr(A), _ptr(B), A.shape[1], B.shape[1], i, j, S))


def warshall(A, S: int) -> np.ndarray:
    """Non-reflexive closure A ⊕ A² ⊕ ... by Warshall/Floyd, in a copy."""
    T = _u32c(A).copy()
    D = T.shape[0]
    assert T.shape == (D, D)
    _load().or_warshall(_ptr(T), D, S)
    return T


def closure_squaring(A, S: int) -> np.ndarray:
    """Non-reflexive closure by A ⊗ (I ⊕ A)^(2^m), m = ceil(log2(max(D-1,1)))."""
    A = _u32c(A)
    D = A.shape[0]
    T = np.zeros_like(A)
    work = np.zeros((2, D, D), np.uint32)
    _load().or_closure_squaring(_ptr(A), _ptr(T), D, S, _ptr(work))
    return T


def closure_row(A, src: int, S: int) -> np.ndarray:
    """Row src of the non-reflexive closure, by single-source shortest paths."""
    A = _u32c(A)
    D = A.shape[0]
    row = np.zeros(D, np.uint32)
    _load().or_closure_row(_ptr(A), D, S, src, _ptr(row))
    return row


def encode_antidist(W, S: int) -> np.ndarray:
    """Weights (0 = no edge) -> anti-distance entries S - w (0 if w >= S)."""
    W = _u32c(W)
    out = np.zeros_like(W)
    _load().or_encode_antidist(_ptr(W), W.size, S, _ptr(out))
    return out


# ------------------------------------------------------------ Boolean, packed

def words64(C: int) -> int:
    return (C + 63) // 64


def pack_bits(dense, ldw: int | None = None) -> np.ndarray:
    """Dense 0/1 (R x C) -> (R x ldw) uint64 bit rows, LSB-first, pad bits 0."""
    dense = np.ascontiguousarray(dense, dtype=np.uint8)
    R, C = dense.shape
    ldw = words64(C) if ldw is None else ldw
    M = np.zeros((R, ldw), np.uint64)
    _load().or_pack_bits(_ptr(dense), R, C, _ptr(M), ldw)
    return M


def unpack_bits(M, C: int) -> np.ndarray:
    M = np.ascontiguousarray(M, dtype=np.uint64)
    R, ldw = M.shape
    dense = np.zeros((R, C), np.uint8)
    _load().or_unpack_bits(_ptr(M), ldw, R, C, _ptr(dense))
    return dense


def bool_mul_w64(A, B, N: int, C=None) -> np.ndarray:
    """Packed Boolean product; A (R x ceil(K/64)) words, B (K x ceil(N/64)) words."""
    A = np.ascontiguousarray(A, dtype=np.uint64)
    B = np.ascontiguousarray(B, dtype=np.uint64)
    R, lda = A.shape
    K, ldb = B.shape
    nw = words64(N)
    out = np.zeros((R, nw), np.uint64) if C is None else np.ascontiguousarray(C, np.uint64).copy()
    _load().or_bool_mul_w64(_ptr(A), lda, _ptr(B), ldb, _ptr(out), out.shape[1], R, K, nw,
                            0 if C is None else 1)
    return out


def bool_warshall_w64(A) -> np.ndarray:
    T = np.ascontiguousarray(A, dtype=np.uint64).copy()
    D = T.shape[0]
    _load().or_bool_warshall_w64(_ptr(T), T.shape[1], D)
    return T


def bool_closure_row_w64(A, src: int) -> np.ndarray:
    A = np.ascontiguousarray(A, dtype=np.uint64)
    D = A.shape[0]
    row = np.zeros(words64(D), np.uint64)
    _load().or_bool_closure_row_w64(_ptr(A), A.shape[1], D, src, _ptr(row))
    return row


# ------------------------------------------------------------ distance form

def dist_mul(X, Y, S: int, Z=None) -> np.ndarray:
    """(Z if given else all-S) ∧ (X + Y) with min and saturating addition at S."""
    X, Y = _u32c(X), _u32c(Y)
    R, K = X.shape
    N = Y.shape[1]
    out = np.full((R, N), S, np.uint32) if Z is None else _u32c(Z).copy()
    _load().or_dist_mul(_ptr(X), _ptr(Y), _ptr(out), R, K, N, S, 0 if Z is None else 1)
    return out


def dist_closure(A, S: int) -> np.ndarray:
    """Floyd on saturating distances, diagonal = shortest cycle (not reset to 0)."""
    T = _u32c(A).copy()
    _load().or_dist_closure(_ptr(T), T.shape[0], S)
    return T


ENTRYWISE = {"and": 0, "or": 1, "xor": 2, "not": 3}


def entrywise(op: str, A, B=None, S: int = 255) -> np.ndarray:
    A = _u32c(A)
    Bc = None if B is None else _u32c(B)
    out = np.zeros_like(A)
    _load().or_entrywise(ENTRYWISE[op], _ptr(A), None if Bc is None else _ptr(Bc), _ptr(out), A.size, S)
    return out
