"""CPU checks of the boundary: the C-ABI library builds, loads, and exports
every function include/ppst.h declares (no compute calls: no GPU here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "ppst.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ppst_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libppst():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2508_12093_gb300 import _lib
    return ctypes.CDLL(_lib.LIB_PATH)


def test_every_declared_symbol_is_exported(libppst):
    names = declared_functions()
    assert len(names) >= 30
    missing = [n for n in names if not hasattr(libppst, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    from paper_2508_12093_gb300 import _lib
    assert set(declared_functions()) == set(_lib.SIGNATURES)


def test_statistic_ids_match_the_header():
    """The binding's statistic ids are the header's ppst_stat values."""
    from paper_2508_12093_gb300 import _lib, STATS
    src = open(os.path.join(ROOT, "include", "ppst.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    body = re.search(r"typedef enum \{([^}]*)\} ppst_stat;", src).group(1)
    enum = {k: int(v) for k, v in re.findall(r"(PPST_[A-Z_]+)\s*=\s*(\d+)", body)}
    assert enum == {k: getattr(_lib, k) for k in enum}
    assert sorted(STATS.values()) == sorted(enum.values())


def test_null_and_bad_handles_are_rejected(libppst):
    # argument checks that run before any CUDA call
    from paper_2508_12093_gb300 import _lib
    lib = _lib.lib
    out = ctypes.c_void_p()
    assert lib.ppst_ctx_create(None, None, None, ctypes.byref(out)) == -1
    bad = _lib.ppst_params(30, 2, 1, 1, 60, 50, 60, 50.0, 0.0, 0)   # log_n out of range
    assert lib.ppst_ctx_create(ctypes.byref(bad), None, None, ctypes.byref(out)) == -1
    assert out.value is None
    assert lib.ppst_sync(None) == -1
    assert lib.ppst_last_error(None) == b"invalid context"
    junk = (ctypes.c_uint32 * 8)(1, 2, 3, 4, 5, 6, 7, 8)
    assert lib.ppst_ct_level(ctypes.cast(junk, ctypes.c_void_p), None, None) == -1
    lib.ppst_free(None)


def test_oracle_library_builds():
    from oracle import _clib
    assert os.path.exists(_clib.build())
