"""CPU oracle for the TMFG-DBHT hot path (arXiv 2408.09399).

TEST INFRASTRUCTURE ONLY: imported by the tests, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``.  The product path (the CUDA
library and its binding) never imports this package.

The arithmetic lives in ``tmfg_oracle.c`` (plain C, one function per step of
the paper's Algorithms 1 and 2, the APSP of Section 2, the approximate APSP
of Section 4.3, the DBHT of Section 2 and the ARI of Section 5); this module
only marshals numpy arrays into it.  Every function here returns numpy
arrays; sizes follow the C comments.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tmfg_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

F32, F64 = 0, 1
CORR, HEAP, EXACT_GREEDY = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile ``tmfg_oracle.c`` into ``liboracle.so`` with gcc (OpenMP on,
    no FMA contraction, no fast-math).  Returns the library path."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    compile_library(_SRC, tmp)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def compile_library(src: str, out: str) -> str:
    """gcc flags of the oracle: OpenMP on, no FMA contraction, no fast-math."""
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared", "-o", out, src, "-lm"]
    subprocess.run(cmd, check=True)
    return out


def _bind(lib):
    """Declare the argument and result types of every entry point."""
    P = ctypes.c_void_p
    i64 = ctypes.c_int64
    ci = ctypes.c_int
    lib.oracle_set_threads.argtypes = [ci]
    lib.oracle_set_threads.restype = ci
    lib.oracle_quantize.argtypes = [ctypes.c_double]
    lib.oracle_quantize.restype = i64
    lib.oracle_rowsums.argtypes = [P, i64, i64, ci, P]
    lib.oracle_rowsums.restype = None
    lib.oracle_rowsort.argtypes = [P, i64, i64, ci, P]
    lib.oracle_rowsort.restype = ci
    lib.oracle_tmfg.argtypes = [P, i64, i64, ci, ci, i64, ci, P, P, P, P, P, P, P, P]
    lib.oracle_tmfg.restype = ci
    lib.oracle_apsp_exact.argtypes = [P, i64, i64, ci, P, i64, ci, P]
    lib.oracle_apsp_exact.restype = ci
    lib.oracle_sssp_rows.argtypes = [P, i64, i64, ci, P, i64, ci, P, i64, P]
    lib.oracle_sssp_rows.restype = ci
    lib.oracle_sssp_bounded_rows.argtypes = [P, i64, i64, ci, P, i64, ci, P, P, i64, P]
    lib.oracle_sssp_bounded_rows.restype = ci
    lib.oracle_rowsort_rows.argtypes = [P, i64, i64, ci, P, i64, P]
    lib.oracle_rowsort_rows.restype = ci
    lib.oracle_hubs.argtypes = [i64, P, i64, i64, P]
    lib.oracle_hubs.restype = ci
    lib.oracle_apsp_approx.argtypes = [P, i64, i64, ci, P, i64, i64, ctypes.c_double, ci,
                                       P, P, P, P]
    lib.oracle_apsp_approx.restype = ci
    lib.oracle_apsp_approx_rows.argtypes = [P, i64, i64, ci, P, i64, i64, ctypes.c_double, ci,
                                            P, i64, P]
    lib.oracle_apsp_approx_rows.restype = ci
    lib.oracle_complete_linkage.argtypes = [P, i64, P]
    lib.oracle_complete_linkage.restype = ci
    lib.oracle_dbht.argtypes = [P, i64, i64, ci, P, P, P, P, P, P, P, P, P, P]
    lib.oracle_dbht.restype = ci
    lib.oracle_cut.argtypes = [P, i64, i64, P]
    lib.oracle_cut.restype = ci
    lib.oracle_ari.argtypes = [P, P, i64]
    lib.oracle_ari.restype = ctypes.c_double
    lib.oracle_pearson.argtypes = [P, i64, i64, ci, P]
    lib.oracle_pearson.restype = ci
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = _bind(ctypes.CDLL(_LIB_PATH))
    return _lib


class use_library:
    """Context manager for the oracle's own tests: route every call of this
    module through another build of the oracle (a library compiled from a
    copy of ``tmfg_oracle.c`` with one planted mistake), then restore."""

    def __init__(self, path: str):
        self.lib = _bind(ctypes.CDLL(path))

    def __enter__(self):
        global _lib
        _load()
        with _lock:
            self.saved, _lib = _lib, self.lib
        return self

    def __exit__(self, *exc):
        global _lib
        with _lock:
            _lib = self.saved


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _check(rc, what):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


def _mat(S):
    S = np.ascontiguousarray(S)
    if S.dtype == np.float32:
        return S, F32
    if S.dtype == np.float64:
        return S, F64
    raise TypeError("S must be float32 or float64")


def set_threads(k: int = 0) -> int:
    """Host threads for the oracle's parallel loops (k < 1: unchanged);
    returns the number in use."""
    return int(_load().oracle_set_threads(int(k)))


def quantize(x: float) -> int:
    """q(x) = x * 2^40 rounded to the nearest integer, ties to even."""
    return int(_load().oracle_quantize(float(x)))


def rowsums(S):
    S, dt = _mat(S)
    n = S.shape[0]
    out = np.empty(n, np.int64)
    _load().oracle_rowsums(_ptr(S), n, S.shape[1], dt, _ptr(out))
    return out


def rowsort(S):
    """Every row v of S sorted by (S[v,u] desc, u asc) over u != v: (n, n-1) int32."""
    S, dt = _mat(S)
    n = S.shape[0]
    out = np.empty((n, n - 1), np.int32)
    _check(_load().oracle_rowsort(_ptr(S), n, S.shape[1], dt, _ptr(out)), "rowsort")
    return out


def tmfg(S, mode: str = "heap", prefix: int = 1, maxcorrs_bruteforce: bool = False):
    """TMFG by corr-tmfg (Algorithm 1), heap-tmfg (Algorithm 2) or the exact
    greedy ('exact').  Returns a dict of numpy arrays: order (n), edges
    (3n-6, 2), ins_face (n-4, 3), parent (n-3), ins_gain (n-4), rowsum (n),
    faces (2n-4, 3) and stats {face_evals, stale_pops, and the wall time in ns of
    the row sums + clique, the row sort and the insertion loop}."""
    S, dt = _mat(S)
    n = S.shape[0]
    m = {"corr": CORR, "heap": HEAP, "exact": EXACT_GREEDY}[mode]
    order = np.empty(n, np.int32)
    edges = np.empty((3 * n - 6, 2), np.int32)
    ins_face = np.empty((n - 4, 3), np.int32)
    parent = np.empty(n - 3, np.int32)
    ins_gain = np.empty(n - 4, np.float64)
    rs = np.empty(n, np.int64)
    faces = np.empty((2 * n - 4, 3), np.int32)
    stats = np.zeros(5, np.int64)
    rc = _load().oracle_tmfg(_ptr(S), n, S.shape[1], dt, m, int(prefix),
                             1 if maxcorrs_bruteforce else 0, _ptr(order), _ptr(edges),
                             _ptr(ins_face), _ptr(parent), _ptr(ins_gain), _ptr(rs),
                             _ptr(faces), _ptr(stats))
    _check(rc, "tmfg")
    return {"order": order, "edges": edges, "ins_face": ins_face, "parent": parent,
            "ins_gain": ins_gain, "rowsum": rs, "faces": faces,
            "stats": {"face_evals": int(stats[0]), "stale_pops": int(stats[1]),
                      "ns_rowsums_clique": int(stats[2]), "ns_rowsort": int(stats[3]),
                      "ns_loop": int(stats[4])}}


def apsp_exact(S, edges, prec: int = 64):
    """All-pairs shortest paths over the TMFG, one Dijkstra per source.
    prec=64: double arithmetic; prec=32: the float path-sum arithmetic."""
    S, dt = _mat(S)
    n = S.shape[0]
    edges = np.ascontiguousarray(edges, np.int32)
    D = np.empty((n, n), np.float64)
    _check(_load().oracle_apsp_exact(_ptr(S), n, S.shape[1], dt, _ptr(edges), edges.shape[0],
                                     prec, _ptr(D)), "apsp_exact")
    return D


def sssp_rows(S, edges, sources, prec: int = 64):
    """Exact shortest-path rows for the given sources only: (len(sources), n)."""
    S, dt = _mat(S)
    n = S.shape[0]
    edges = np.ascontiguousarray(edges, np.int32)
    src = np.ascontiguousarray(sources, np.int32)
    D = np.empty((src.shape[0], n), np.float64)
    _check(_load().oracle_sssp_rows(_ptr(S), n, S.shape[1], dt, _ptr(edges), edges.shape[0],
                                    prec, _ptr(src), src.shape[0], _ptr(D)), "sssp_rows")
    return D


def sssp_bounded_rows(S, edges, sources, bounds, prec: int = 32):
    """Radius-bounded searches from the given sources (Section 4.3)."""
    S, dt = _mat(S)
    n = S.shape[0]
    edges = np.ascontiguousarray(edges, np.int32)
    src = np.ascontiguousarray(sources, np.int32)
    b = np.ascontiguousarray(bounds, np.float64)
    D = np.empty((src.shape[0], n), np.float64)
    _check(_load().oracle_sssp_bounded_rows(_ptr(S), n, S.shape[1], dt, _ptr(edges),
                                            edges.shape[0], prec, _ptr(src), _ptr(b),
                                            src.shape[0], _ptr(D)), "sssp_bounded_rows")
    return D


def rowsort_rows(S, rows):
    """Sorted rows (R3) for the listed rows only: (len(rows), n-1) int32."""
    S, dt = _mat(S)
    n = S.shape[0]
    r = np.ascontiguousarray(rows, np.int32)
    out = np.empty((r.shape[0], n - 1), np.int32)
    _check(_load().oracle_rowsort_rows(_ptr(S), n, S.shape[1], dt, _ptr(r), r.shape[0],
                                       _ptr(out)), "rowsort_rows")
    return out


def hubs(n, edges, h):
    edges = np.ascontiguousarray(edges, np.int32)
    out = np.empty(h, np.int32)
    _check(_load().oracle_hubs(n, _ptr(edges), edges.shape[0], h, _ptr(out)), "hubs")
    return out


def apsp_approx(S, edges, n_hubs: int = 0, radius_factor: float = 2.0, prec: int = 32):
    """Hub-based approximate APSP (Section 4.3).  Returns (D, info) where
    info holds hubs, nearest hub rank per vertex and the distance to it."""
    S, dt = _mat(S)
    n = S.shape[0]
    edges = np.ascontiguousarray(edges, np.int32)
    h = n_hubs if n_hubs > 0 else int(np.ceil(np.sqrt(n)))
    h = min(h, n)
    D = np.empty((n, n), np.float64)
    hb = np.empty(h, np.int32)
    near = np.empty(n, np.int32)
    dnear = np.empty(n, np.float64)
    _check(_load().oracle_apsp_approx(_ptr(S), n, S.shape[1], dt, _ptr(edges), edges.shape[0],
                                      h, float(radius_factor), prec, _ptr(D), _ptr(hb),
                                      _ptr(near), _ptr(dnear)), "apsp_approx")
    return D, {"hubs": hb, "nearest": near, "dnear": dnear}


def apsp_approx_rows(S, edges, sources, n_hubs: int = 0, radius_factor: float = 2.0,
                     prec: int = 32):
    """Rows ``sources`` of apsp_approx (same arguments) without its n x n
    work matrix: (len(sources), n) float64."""
    S, dt = _mat(S)
    n = S.shape[0]
    e = np.ascontiguousarray(edges, np.int32)
    src = np.ascontiguousarray(sources, np.int32)
    D = np.empty((len(src), n), np.float64)
    _check(_load().oracle_apsp_approx_rows(_ptr(S), n, S.shape[1], dt, _ptr(e), e.shape[0],
                                           int(n_hubs), float(radius_factor), prec, _ptr(src),
                                           len(src), _ptr(D)), "apsp_approx_rows")
    return D


def complete_linkage(D):
    D = np.ascontiguousarray(D, np.float64)
    n = D.shape[0]
    Z = np.empty((n - 1, 4), np.float64)
    _check(_load().oracle_complete_linkage(_ptr(D), n, _ptr(Z)), "complete_linkage")
    return Z


def dbht(S, t, D):
    """DBHT dendrogram from a TMFG result dict ``t`` (as returned by tmfg)
    and a distance matrix D (n x n, float64).  Returns (Z, info)."""
    S, dt = _mat(S)
    n = S.shape[0]
    D = np.ascontiguousarray(D, np.float64)
    Z = np.empty((n - 1, 4), np.float64)
    direction = np.empty(n - 4, np.int32)
    conv = np.empty(n - 3, np.int32)
    group = np.empty(n, np.int32)
    bub = np.empty(n, np.int32)
    args = [np.ascontiguousarray(t[k], np.int32) for k in ("order", "edges", "ins_face", "parent")]
    rc = _load().oracle_dbht(_ptr(S), n, S.shape[1], dt, *[_ptr(a) for a in args], _ptr(D),
                             _ptr(Z), _ptr(direction), _ptr(conv), _ptr(group), _ptr(bub))
    _check(rc, "dbht")
    return Z, {"direction": direction, "converging": conv, "group": group, "bubble": bub}


def cut(Z, k):
    Z = np.ascontiguousarray(Z, np.float64)
    n = Z.shape[0] + 1
    labels = np.empty(n, np.int32)
    _check(_load().oracle_cut(_ptr(Z), n, int(k), _ptr(labels)), "cut")
    return labels


def ari(truth, pred) -> float:
    a = np.ascontiguousarray(truth, np.int32)
    b = np.ascontiguousarray(pred, np.int32)
    return float(_load().oracle_ari(_ptr(a), _ptr(b), a.shape[0]))


def pearson(X):
    X = np.ascontiguousarray(X)
    dt = F32 if X.dtype == np.float32 else F64
    if X.dtype not in (np.float32, np.float64):
        raise TypeError("X must be float32 or float64")
    n, T = X.shape
    S = np.empty((n, n), np.float64)
    _check(_load().oracle_pearson(_ptr(X), n, T, dt, _ptr(S)), "pearson")
    return S
