"""The C-ABI library loads and exports every function include/semiring.h
declares (no GPU needed: nothing is called)."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "semiring.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w]*\s*\**\s*([A-Za-z_]\w*)\s*\([^;{]*\)\s*;", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    from paper_1705_08743_gb300 import _capi
    return _capi


def test_header_parses():
    names = declared_functions()
    for must in ["antidist_mul", "antidist_closure", "bool_mul", "bool_closure", "sr_create"]:
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    cdll = ctypes.CDLL(lib.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(cdll, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if n not in lib.exported_symbols()]
    assert not missing, missing


def test_errors_without_device(lib):
    # argument checks run before any CUDA call: a bad dtype is rejected on any host
    st = lib.lib.antidist_mul(None, 1, 4, 1, 4, 2, 4, 4, 4, 4, 0, 0, None)
    assert st == lib.SR_EINVAL
    assert "dtype" in lib.last_error()
    st = lib.lib.antidist_closure(None, None, 4, 4, lib.SR_U8, None)
    assert st == lib.SR_EINVAL and "NULL" in lib.last_error()
    st = lib.lib.bool_mul(None, 16, 1, 16, 1, 16, 1, 4, 4, 4, lib.SR_BOOL_W32, 0, None)
    assert st == lib.SR_EINVAL and "overlap" in lib.last_error()
    assert lib.lib.sr_cancel(None, 1) == lib.SR_EINVAL and "not serving" in lib.last_error()


def test_workspace_query_without_device(lib):
    # host arithmetic only: the Warshall form of bool_closure asks for tensor-core operand
    # space once it has two 2048-bit blocks, the squaring form always needs its matrices
    W = lib.SR_CLOSURE_WARSHALL
    assert lib.sr_workspace_query(lib.SR_OP_BOOL_CLOSURE, lib.SR_BOOL_W64, 2048, W) == 0
    small = lib.sr_workspace_query(lib.SR_OP_BOOL_CLOSURE, lib.SR_BOOL_W64, 2049, W)
    big = lib.sr_workspace_query(lib.SR_OP_BOOL_CLOSURE, lib.SR_BOOL_W64, 16384, W)
    assert 0 < small < big
    assert 2 * 16384 * 2048 < big < 4 * 16384 * 2048 + (64 << 20)     # phase 3's fp8 operands dominate
    sq = lib.sr_workspace_query(lib.SR_OP_BOOL_CLOSURE, lib.SR_BOOL_W64, 1000, lib.SR_CLOSURE_SQUARING)
    assert sq >= 2 * 1000 * 32 * 4
    # the anti-distance closure's persistent schedule (a version per pivot-block pair, D in
    # [128, 32768]) and fused-pass schedule (four counters per launch, D <= 32768): u8/u16 only
    pc = lib.sr_workspace_query(lib.SR_OP_ANTIDIST_CLOSURE, lib.SR_U8, 4096, 0)
    assert pc >= 4 * (4096 // 128) ** 2
    assert lib.sr_workspace_query(lib.SR_OP_ANTIDIST_CLOSURE, lib.SR_U32, 4096, 0) == 0
    assert lib.sr_workspace_query(lib.SR_OP_ANTIDIST_CLOSURE, lib.SR_U8, 100, 0) == 2 * 4 * 4   # two launches
    assert lib.sr_workspace_query(lib.SR_OP_ANTIDIST_CLOSURE, lib.SR_U16, 40000, 0) == 0
