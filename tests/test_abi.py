"""The C-ABI library builds for sm_103a, loads, and exports every function
that include/*.h declares.  No GPU needed: only calls that do not touch a
device are made."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^\s*[A-Za-z_][\w\s\*]*?\b(\w+)\s*\([^;{]*\)\s*;", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2408_09399_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("tmfg_create", "tmfg_destroy", "tmfg_build", "tmfg_apsp",
                     "tmfg_sync_status", "tmfg_strerror", "tmfg_row_sort", "dbht_cluster"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_host_only_calls(lib):
    lib.tmfg_max_n.restype = ctypes.c_int64
    lib.tmfg_max_n.argtypes = [ctypes.c_int]
    assert lib.tmfg_max_n(0) >= 20000      # the n=20000 workload fits
    assert lib.tmfg_max_n(1) >= 200
    assert lib.tmfg_max_n(7) == 0
    lib.tmfg_workspace_bytes.restype = ctypes.c_size_t
    lib.tmfg_workspace_bytes.argtypes = [ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    n = 20000
    assert lib.tmfg_workspace_bytes(n, 0, 0, 0) >= 2 * n * (n - 1)
    assert lib.tmfg_workspace_bytes(n, 0, 2, 0) > lib.tmfg_workspace_bytes(n, 0, 1, 0)
    # DBHT: the three levels' distance matrices dominate (n^2 floats)
    assert lib.tmfg_workspace_bytes(n, 0, 3, 0) >= 4 * n * n
    lib.tmfg_strerror.restype = ctypes.c_char_p
    assert lib.tmfg_strerror(0) == b"ok"
    assert b"symmetric" in lib.tmfg_strerror(4)


def test_argument_errors_need_no_device(lib):
    P = ctypes.c_void_p
    lib.tmfg_build.argtypes = [P, P, ctypes.c_int64, ctypes.c_int64, P, P, P, P, P, P]
    assert lib.tmfg_build(None, None, 3, 3, None, None, None, None, None, None) == 1
    lib.tmfg_sync_status.argtypes = [P, P]
    assert lib.tmfg_sync_status(None, None) == 1
    i64 = ctypes.c_int64
    lib.dbht_cluster.argtypes = [P, P, i64, i64, ctypes.c_int32, P, P, P, P, P, i64, P, P]
    assert lib.dbht_cluster(None, None, 10, 10, 0, None, None, None, None, None, 10, None,
                            None) == 1
    lib.tmfg_memory_latency.argtypes = [P, i64, ctypes.c_int32, ctypes.c_int32, P]
    ns = ctypes.c_double()
    assert lib.tmfg_memory_latency(None, 1 << 20, 10, 0, ctypes.byref(ns)) == 1
    lib.tmfg_cluster_exchange_latency.argtypes = [P, ctypes.c_int32, ctypes.c_int32, P]
    assert lib.tmfg_cluster_exchange_latency(None, 8, 10, ctypes.byref(ns)) == 1


def test_package_fails_loudly_without_a_device():
    import torch
    import paper_2408_09399_gb300 as T
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    with pytest.raises(RuntimeError):
        T.tmfg_create(0)
