"""GB300-native TMFG construction and APSP over the TMFG (arXiv 2408.09399).

A thin ctypes binding over ``libtmfg.so`` (C ABI in ``include/tmfg.h``).
Each function has the name of the C entry point it calls and only marshals
arguments: torch CUDA tensors become device pointers, the current (or given)
torch stream becomes the cudaStream_t.  Every step of the computation runs in
the library's CUDA kernels; there is no CPU path.  Importing this package
does not load the library; the first call does, and raises if it is missing
or no CUDA device is present.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtmfg.so")

TMFG_F32, TMFG_F64 = 0, 1
TMFG_CORR, TMFG_HEAP = 0, 1
TMFG_CHECK_SYMMETRY = 1
SIM_PRECISIONS = {"f64": 0, "f32": 1, "bf16x3": 2, "tf32x3": 3}
ERRORS = {0: "TMFG_OK", 1: "TMFG_EINVAL", 2: "TMFG_ENOMEM", 3: "TMFG_ENONFINITE",
          4: "TMFG_EASYMMETRIC", 5: "TMFG_ETIMEOUT", 6: "TMFG_ECUDA", 7: "TMFG_ERANGE",
          8: "TMFG_ETOOBIG", 9: "TMFG_EINTERNAL"}

_lock = threading.Lock()
_lib = None


class TmfgError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {ERRORS.get(code, code)} ({_strerror(code)})")


class _Params(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("prefix", ctypes.c_int32), ("dtype", ctypes.c_int32),
                ("flags", ctypes.c_uint32)]


class _Job(ctypes.Structure):
    _fields_ = [("S", ctypes.c_void_p), ("n", ctypes.c_int64), ("ld", ctypes.c_int64),
                ("order", ctypes.c_void_p), ("edges", ctypes.c_void_p),
                ("ins_face", ctypes.c_void_p), ("bubble_parent", ctypes.c_void_p),
                ("D", ctypes.c_void_p), ("ldd", ctypes.c_int64)]


class _LoopShape(ctypes.Structure):
    _fields_ = [("threads", ctypes.c_int32), ("probe_lanes", ctypes.c_int32),
                ("stage_groups", ctypes.c_int32), ("kernel", ctypes.c_int32),
                ("cluster", ctypes.c_int32)]


class _BatchConfig(ctypes.Structure):
    _fields_ = [("sssp_threads", ctypes.c_int32), ("loop", _LoopShape)]


class _DbhtOutputs(ctypes.Structure):
    _fields_ = [("direction", ctypes.c_void_p), ("converging", ctypes.c_void_p),
                ("group", ctypes.c_void_p), ("bubble", ctypes.c_void_p)]


class _ServeConfig(ctypes.Structure):
    _fields_ = [("lanes", ctypes.c_int32), ("max_batch", ctypes.c_int32),
                ("lane_bytes", ctypes.c_size_t), ("params", _Params),
                ("apsp", ctypes.c_int32), ("sssp_threads", ctypes.c_int32),
                ("pipeline", ctypes.c_int32), ("precision", ctypes.c_int32)]


class _PipelineJob(ctypes.Structure):
    _fields_ = [("X", ctypes.c_void_p), ("n", ctypes.c_int64), ("T", ctypes.c_int64),
                ("ldx", ctypes.c_int64), ("S", ctypes.c_void_p), ("order", ctypes.c_void_p),
                ("edges", ctypes.c_void_p), ("ins_face", ctypes.c_void_p),
                ("bubble_parent", ctypes.c_void_p), ("D", ctypes.c_void_p),
                ("Z", ctypes.c_void_p), ("k", ctypes.c_int32), ("labels", ctypes.c_void_p)]


class _PipelineParams(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("tmfg", _Params)]


class _ServeResult(ctypes.Structure):
    _fields_ = [("id", ctypes.c_int64), ("status", ctypes.c_int32), ("batch", ctypes.c_int32),
                ("batch_size", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("t_submit_ns", ctypes.c_int64), ("t_launch_ns", ctypes.c_int64),
                ("t_done_ns", ctypes.c_int64)]


class _SolveParams(ctypes.Structure):
    _fields_ = [("n_hubs", ctypes.c_int32), ("radius_factor", ctypes.c_float),
                ("row_blocks", ctypes.c_int32)]


class _ApspParams(ctypes.Structure):
    _fields_ = [("approx", ctypes.c_int32), ("n_hubs", ctypes.c_int32),
                ("radius_factor", ctypes.c_float)]


def load_library():
    """Load libtmfg.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libtmfg.so not built ({LIB_PATH}); run "
                               "paper_2408_09399_gb300.build.build() first")
        lib = ctypes.CDLL(LIB_PATH)
        P, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
        lib.tmfg_create.argtypes = [ctypes.POINTER(P), ctypes.c_int, ctypes.c_size_t]
        lib.tmfg_create.restype = ctypes.c_int
        lib.tmfg_destroy.argtypes = [P]
        lib.tmfg_destroy.restype = None
        lib.tmfg_max_n.argtypes = [ctypes.c_int]
        lib.tmfg_max_n.restype = i64
        lib.tmfg_max_n_mode.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int]
        lib.tmfg_max_n_mode.restype = i64
        lib.tmfg_workspace_bytes.argtypes = [i64, ctypes.c_int, ctypes.c_int, ctypes.c_int]
        lib.tmfg_workspace_bytes.restype = ctypes.c_size_t
        lib.tmfg_build.argtypes = [P, P, i64, i64, ctypes.POINTER(_Params), P, P, P, P, P]
        lib.tmfg_build.restype = ctypes.c_int
        lib.tmfg_row_sort.argtypes = [P, P, i64, i64, i32, P, i64, P, P]
        lib.tmfg_row_sort.restype = ctypes.c_int
        lib.tmfg_apsp.argtypes = [P, P, i64, i64, i32, P, ctypes.POINTER(_ApspParams), P, i64, P]
        lib.tmfg_apsp.restype = ctypes.c_int
        lib.tmfg_batch_run.argtypes = [P, ctypes.POINTER(_Job), ctypes.c_int32,
                                       ctypes.POINTER(_Params), ctypes.POINTER(_BatchConfig), P]
        lib.tmfg_batch_run.restype = ctypes.c_int
        lib.tmfg_pipeline_run.argtypes = [P, ctypes.POINTER(_PipelineJob), i32,
                                          ctypes.POINTER(_PipelineParams),
                                          ctypes.POINTER(_BatchConfig), P]
        lib.tmfg_pipeline_run.restype = ctypes.c_int
        lib.tmfg_pipeline_request_bytes.argtypes = [i64, i64, i32]
        lib.tmfg_pipeline_request_bytes.restype = ctypes.c_size_t
        lib.tmfg_cut_labels.argtypes = [P, P, i64, i32, P, P]
        lib.tmfg_cut_labels.restype = ctypes.c_int
        lib.tmfg_serve_submit_pipeline.argtypes = [P, ctypes.POINTER(_PipelineJob), P]
        lib.tmfg_serve_submit_pipeline.restype = i64
        lib.tmfg_solve_host_stages.argtypes = [P, P, i32]
        lib.tmfg_solve_host_stages.restype = ctypes.c_int
        lib.tmfg_set_loop_shape.argtypes = [P, ctypes.POINTER(_LoopShape)]
        lib.tmfg_set_loop_shape.restype = ctypes.c_int
        lib.dbht_cluster.argtypes = [P, P, i64, i64, i32, P, P, P, P, P, i64, P, P]
        lib.dbht_cluster.restype = ctypes.c_int
        lib.dbht_cluster_detail.argtypes = [P, P, i64, i64, i32, P, P, P, P, P, i64, P,
                                            ctypes.POINTER(_DbhtOutputs), P]
        lib.dbht_cluster_detail.restype = ctypes.c_int
        lib.tmfg_solve_host.argtypes = [P, P, i64, i64, ctypes.POINTER(_Params),
                                        ctypes.POINTER(_SolveParams), P, P, P, P, P, P, i64, P]
        lib.tmfg_solve_host.restype = ctypes.c_int
        lib.tmfg_similarity.argtypes = [P, P, i64, i64, i32, P, i64, P]
        lib.tmfg_similarity.restype = ctypes.c_int
        lib.tmfg_serve_start.argtypes = [ctypes.POINTER(P), ctypes.c_int,
                                         ctypes.POINTER(_ServeConfig)]
        lib.tmfg_serve_start.restype = ctypes.c_int
        lib.tmfg_serve_submit.argtypes = [P, ctypes.POINTER(_Job), P]
        lib.tmfg_serve_submit.restype = i64
        lib.tmfg_serve_poll.argtypes = [P, ctypes.POINTER(_ServeResult), i32, i32]
        lib.tmfg_serve_poll.restype = ctypes.c_int
        lib.tmfg_serve_stop.argtypes = [P]
        lib.tmfg_serve_stop.restype = ctypes.c_int
        lib.tmfg_serve_now_ns.argtypes = []
        lib.tmfg_serve_now_ns.restype = i64
        lib.tmfg_serve_request_bytes.argtypes = [i64, i32]
        lib.tmfg_serve_request_bytes.restype = ctypes.c_size_t
        lib.tmfg_serve_plan.argtypes = [P, i32, i32, i32, ctypes.c_size_t, P]
        lib.tmfg_serve_plan.restype = ctypes.c_int
        lib.tmfg_sync_status.argtypes = [P, P]
        lib.tmfg_sync_status.restype = ctypes.c_int
        lib.tmfg_last_stats.argtypes = [P, P, ctypes.c_int]
        lib.tmfg_last_stats.restype = ctypes.c_int
        lib.tmfg_memory_latency.argtypes = [P, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, P]
        lib.tmfg_memory_latency.restype = ctypes.c_int
        lib.tmfg_cluster_exchange_latency.argtypes = [P, ctypes.c_int32, ctypes.c_int32, P]
        lib.tmfg_cluster_exchange_latency.restype = ctypes.c_int
        lib.tmfg_strerror.argtypes = [ctypes.c_int]
        lib.tmfg_strerror.restype = ctypes.c_char_p
        _lib = lib
        return lib


def _strerror(code: int) -> str:
    try:
        return load_library().tmfg_strerror(int(code)).decode()
    except Exception:  # library not loadable: keep the numeric code
        return str(code)


def _check(code: int, where: str):
    if code != 0:
        raise TmfgError(code, where)


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("libtmfg needs a CUDA device; none is available")
    return torch


def _stream_handle(stream):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dev_ptr(t, dtype=None, what="tensor"):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError(f"{what} must be a CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{what} must have dtype {dtype}, got {t.dtype}")
    return ctypes.c_void_p(t.data_ptr())


def _mat_dtype(S):
    torch = _torch()
    if S.dim() != 2 or S.shape[0] != S.shape[1]:
        raise ValueError("S must be a square matrix")
    if S.stride(1) != 1:
        raise ValueError("S must be row-major with unit column stride")
    if S.dtype == torch.float32:
        return TMFG_F32
    if S.dtype == torch.float64:
        return TMFG_F64
    raise TypeError("S must be float32 or float64")


class Context:
    """Owns a tmfg_ctx (device status word + workspace)."""

    def __init__(self, device: int = 0, workspace_budget_bytes: int = 0):
        lib = load_library()
        _torch()
        h = ctypes.c_void_p()
        _check(lib.tmfg_create(ctypes.byref(h), int(device), int(workspace_budget_bytes)),
               "tmfg_create")
        self.handle = h
        self.device = device

    def close(self):
        if getattr(self, "handle", None):
            load_library().tmfg_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tmfg_create(device: int = 0, workspace_budget_bytes: int = 0) -> Context:
    return Context(device, workspace_budget_bytes)


def tmfg_destroy(ctx: Context):
    ctx.close()


def tmfg_max_n(dtype: int = TMFG_F32, mode: str = "corr", prefix: int = 1) -> int:
    """Largest n tmfg_build takes for this dtype, mode and prefix."""
    m = {"corr": TMFG_CORR, "heap": TMFG_HEAP}[mode]
    return int(load_library().tmfg_max_n_mode(int(dtype), m, int(prefix)))


def tmfg_workspace_bytes(n: int, dtype: int = TMFG_F32, what: int = 0, n_hubs: int = 0) -> int:
    return int(load_library().tmfg_workspace_bytes(int(n), int(dtype), int(what), int(n_hubs)))


def tmfg_build(ctx: Context, S, mode: str = "heap", prefix: int = 1, check_symmetry: bool = False,
               out=None, stream=None):
    """TMFG of S (a square CUDA tensor).  Returns dict of int32 CUDA tensors
    order (n), edges (3n-6, 2), ins_face (n-4, 3), bubble_parent (n-3).
    Asynchronous: call tmfg_sync_status to wait and read data errors."""
    torch = _torch()
    n = S.shape[0]
    dt = _mat_dtype(S)
    if out is None:
        dev = S.device
        out = {"order": torch.empty(n, dtype=torch.int32, device=dev),
               "edges": torch.empty((max(3 * n - 6, 0), 2), dtype=torch.int32, device=dev),
               "ins_face": torch.empty((max(n - 4, 0), 3), dtype=torch.int32, device=dev),
               "bubble_parent": torch.empty(max(n - 3, 0), dtype=torch.int32, device=dev)}
    p = _Params({"corr": TMFG_CORR, "heap": TMFG_HEAP}[mode], int(prefix), dt,
                TMFG_CHECK_SYMMETRY if check_symmetry else 0)
    i32 = torch.int32
    rc = load_library().tmfg_build(ctx.handle, _dev_ptr(S), n, S.stride(0), ctypes.byref(p),
                                   _dev_ptr(out["order"], i32), _dev_ptr(out["edges"], i32),
                                   _dev_ptr(out["ins_face"], i32) if n > 4 else None,
                                   _dev_ptr(out["bubble_parent"], i32), _stream_handle(stream))
    _check(rc, "tmfg_build")
    return out


def tmfg_row_sort(ctx: Context, S, idx=None, rowsum=None, stream=None):
    """Sorted index rows (uint16 stored in an int16 tensor, n x ldi) and int64
    row sums of S.  Returns (idx, rowsum)."""
    torch = _torch()
    n = S.shape[0]
    dt = _mat_dtype(S)
    if idx is None:
        ldi = ((n - 1) + 7) // 8 * 8
        idx = torch.empty((n, ldi), dtype=torch.int16, device=S.device)
    if rowsum is None:
        rowsum = torch.empty(n, dtype=torch.int64, device=S.device)
    rc = load_library().tmfg_row_sort(ctx.handle, _dev_ptr(S), n, S.stride(0), dt,
                                      _dev_ptr(idx, torch.int16), idx.stride(0),
                                      _dev_ptr(rowsum, torch.int64), _stream_handle(stream))
    _check(rc, "tmfg_row_sort")
    return idx, rowsum


def tmfg_apsp(ctx: Context, S, edges, approx: bool = False, n_hubs: int = 0,
              radius_factor: float = 0.0, D=None, stream=None):
    """Shortest-path distances over the TMFG given by ``edges`` (int32 CUDA
    tensor, 3n-6 x 2).  Returns D (float32 CUDA tensor, n x n)."""
    torch = _torch()
    n = S.shape[0]
    dt = _mat_dtype(S)
    if D is None:
        D = torch.empty((n, n), dtype=torch.float32, device=S.device)
    p = _ApspParams(1 if approx else 0, int(n_hubs), float(radius_factor))
    rc = load_library().tmfg_apsp(ctx.handle, _dev_ptr(S), n, S.stride(0), dt,
                                  _dev_ptr(edges.contiguous(), torch.int32), ctypes.byref(p),
                                  _dev_ptr(D, torch.float32), D.stride(0), _stream_handle(stream))
    _check(rc, "tmfg_apsp")
    return D


def tmfg_solve_host(ctx: Context, S, mode: str = "corr", prefix: int = 1, exact: bool = True,
                    approx: bool = True, n_hubs: int = 0, radius_factor: float = 0.0,
                    row_blocks: int = 0, check_symmetry: bool = False, out=None, stream=None):
    """The whole step from host memory (see tmfg_solve_host in include/tmfg.h):
    S is a CPU tensor (page-locked for overlapped copies); returns a dict of
    CPU tensors order, edges, ins_face, bubble_parent and, when asked, D and
    D_approx (float32, n x n).  Asynchronous: call tmfg_sync_status before
    reading them."""
    torch = _torch()
    if S.is_cuda or S.dim() != 2 or S.shape[0] != S.shape[1] or S.stride(1) != 1:
        raise ValueError("S must be a square row-major CPU matrix")
    if S.dtype not in (torch.float32, torch.float64):
        raise TypeError("S must be float32 or float64")
    n = S.shape[0]
    dt = TMFG_F32 if S.dtype == torch.float32 else TMFG_F64
    if out is None:
        pin = S.is_pinned()
        out = {"order": torch.empty(n, dtype=torch.int32, pin_memory=pin),
               "edges": torch.empty((3 * n - 6, 2), dtype=torch.int32, pin_memory=pin),
               "ins_face": torch.empty((max(n - 4, 0), 3), dtype=torch.int32, pin_memory=pin),
               "bubble_parent": torch.empty(n - 3, dtype=torch.int32, pin_memory=pin)}
        if exact:
            out["D"] = torch.empty((n, n), dtype=torch.float32, pin_memory=pin)
        if approx:
            out["D_approx"] = torch.empty((n, n), dtype=torch.float32, pin_memory=pin)
    for k, v in out.items():
        if v.is_cuda:
            raise ValueError(f"{k} must be a CPU tensor")
    D, Da = out.get("D"), out.get("D_approx")
    ldd = (D if D is not None else Da).stride(0) if (D is not None or Da is not None) else n
    p = _Params({"corr": TMFG_CORR, "heap": TMFG_HEAP}[mode], int(prefix), dt,
                TMFG_CHECK_SYMMETRY if check_symmetry else 0)
    sp = _SolveParams(int(n_hubs), float(radius_factor), int(row_blocks))
    ptr = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None  # noqa: E731
    rc = load_library().tmfg_solve_host(
        ctx.handle, ptr(S), n, S.stride(0), ctypes.byref(p), ctypes.byref(sp), ptr(out["order"]),
        ptr(out["edges"]), ptr(out["ins_face"]) if n > 4 else None, ptr(out["bubble_parent"]),
        ptr(D), ptr(Da), ldd, _stream_handle(stream))
    _check(rc, "tmfg_solve_host")
    return out


def tmfg_similarity(ctx: Context, X, precision: str = "bf16x3", S=None, stream=None):
    """Pearson similarity of the rows of X (float32 CUDA tensor, n x T,
    contiguous) in the given precision ('f64', 'f32', 'bf16x3', 'tf32x3').
    Returns S (float32, n x n)."""
    torch = _torch()
    if X.dim() != 2 or X.dtype != torch.float32 or not X.is_contiguous():
        raise TypeError("X must be a contiguous float32 matrix")
    n, T = X.shape
    if S is None:
        S = torch.empty((n, n), dtype=torch.float32, device=X.device)
    rc = load_library().tmfg_similarity(ctx.handle, _dev_ptr(X), n, T, SIM_PRECISIONS[precision],
                                        _dev_ptr(S, torch.float32), S.stride(0),
                                        _stream_handle(stream))
    _check(rc, "tmfg_similarity")
    return S


def _dbht_args(ctx, S, t, D):
    torch = _torch()
    n = S.shape[0]
    dt = _mat_dtype(S)
    if D.dtype != torch.float32 or D.dim() != 2 or D.stride(1) != 1:
        raise TypeError("D must be a row-major float32 matrix")
    i32 = torch.int32
    return [ctx.handle, _dev_ptr(S), n, S.stride(0), dt,
            _dev_ptr(t["order"], i32), _dev_ptr(t["edges"].contiguous(), i32),
            _dev_ptr(t["ins_face"].contiguous(), i32) if n > 4 else None,
            _dev_ptr(t["bubble_parent"], i32), _dev_ptr(D, torch.float32), D.stride(0)]


def dbht_cluster(ctx: Context, S, t, D, linkage=None, stream=None):
    """DBHT dendrogram of the TMFG ``t`` (the dict tmfg_build returns) with
    distances D (float32, n x n).  Returns the (n-1) x 4 float64 linkage
    (scipy layout) as a CUDA tensor."""
    torch = _torch()
    n = S.shape[0]
    if linkage is None:
        linkage = torch.empty((n - 1, 4), dtype=torch.float64, device=S.device)
    rc = load_library().dbht_cluster(*_dbht_args(ctx, S, t, D),
                                     _dev_ptr(linkage, torch.float64), _stream_handle(stream))
    _check(rc, "dbht_cluster")
    return linkage


def dbht_cluster_detail(ctx: Context, S, t, D, linkage=None, stream=None):
    """dbht_cluster that also returns the bubble-edge directions (n-4), the
    converging-bubble flags (n-3), each vertex's group (converging bubble)
    and bubble (n each), as int32 CUDA tensors.  Returns (linkage, info)."""
    torch = _torch()
    n = S.shape[0]
    dev = S.device
    if linkage is None:
        linkage = torch.empty((n - 1, 4), dtype=torch.float64, device=dev)
    info = {"direction": torch.zeros(max(n - 4, 1), dtype=torch.int32, device=dev),
            "converging": torch.empty(n - 3, dtype=torch.int32, device=dev),
            "group": torch.empty(n, dtype=torch.int32, device=dev),
            "bubble": torch.empty(n, dtype=torch.int32, device=dev)}
    outs = _DbhtOutputs(*[info[k].data_ptr() for k in ("direction", "converging", "group",
                                                        "bubble")])
    rc = load_library().dbht_cluster_detail(*_dbht_args(ctx, S, t, D),
                                            _dev_ptr(linkage, torch.float64), ctypes.byref(outs),
                                            _stream_handle(stream))
    _check(rc, "dbht_cluster_detail")
    info["direction"] = info["direction"][: max(n - 4, 0)]
    return linkage, info


def tmfg_solve_host_stages(ctx: Context) -> dict:
    """Stage times (ms from its start) of the last tmfg_solve_host on ctx."""
    buf = (ctypes.c_float * 8)()
    _check(load_library().tmfg_solve_host_stages(ctx.handle, buf, 8), "tmfg_solve_host_stages")
    names = ["start", "uploads_done", "tmfg_done", "exact_piece1_down", "exact_piece2_down",
             "exact_piece3_down", "exact_piece4_down", "approx_down"]
    return {k: round(float(v), 3) for k, v in zip(names, buf) if v >= 0}


def _loop_shape(shape) -> "_LoopShape":
    shape = shape or {}
    return _LoopShape(int(shape.get("threads", 0)), int(shape.get("probe_lanes", 0)),
                      int(shape.get("stage_groups", 0)), int(shape.get("kernel", 0)),
                      int(shape.get("cluster", 0)))


def tmfg_set_loop_shape(ctx: Context, shape=None) -> None:
    """Shape of the corr-tmfg prefix-1 insertion loop for this context's later
    builds: a dict with threads (256/512), probe_lanes (4/8/16),
    stage_groups (0 default, -1 none), kernel (0 automatic, 1 the prefix-1
    kernel, 2 the general one, 3 the cluster kernel) and cluster (8 or 16
    CTAs); None restores the defaults.  Every shape gives the same TMFG."""
    _check(load_library().tmfg_set_loop_shape(ctx.handle, ctypes.byref(_loop_shape(shape))),
           "tmfg_set_loop_shape")


def tmfg_batch_run(ctx: Context, mats, mode: str = "corr", prefix: int = 1, apsp: bool = True,
                   sssp_threads: int = 0, outs=None, stream=None, loop_shape=None):
    """TMFG (and exact APSP when ``apsp``) of every matrix in ``mats`` (CUDA
    tensors of one dtype) with one launch per stage.  Returns a list of dicts
    like tmfg_build's, plus "D" when ``apsp``.  Asynchronous."""
    torch = _torch()
    if not mats:
        return []
    dt = _mat_dtype(mats[0])
    if outs is None:
        outs = []
        for S in mats:
            n = S.shape[0]
            o = {"order": torch.empty(n, dtype=torch.int32, device=S.device),
                 "edges": torch.empty((3 * n - 6, 2), dtype=torch.int32, device=S.device),
                 "ins_face": torch.empty((max(n - 4, 1), 3), dtype=torch.int32, device=S.device),
                 "bubble_parent": torch.empty(n - 3, dtype=torch.int32, device=S.device)}
            if apsp:
                o["D"] = torch.empty((n, n), dtype=torch.float32, device=S.device)
            outs.append(o)
    jobs = (_Job * len(mats))()
    for i, (S, o) in enumerate(zip(mats, outs)):
        if _mat_dtype(S) != dt:
            raise TypeError("all matrices of a batch must have the same dtype")
        n = S.shape[0]
        D = o.get("D") if apsp else None
        jobs[i] = _Job(S.data_ptr(), n, S.stride(0), o["order"].data_ptr(), o["edges"].data_ptr(),
                       o["ins_face"].data_ptr(), o["bubble_parent"].data_ptr(),
                       D.data_ptr() if D is not None else None, D.stride(0) if D is not None else 0)
    p = _Params({"corr": TMFG_CORR, "heap": TMFG_HEAP}[mode], int(prefix), dt, 0)
    cfg = _BatchConfig(int(sssp_threads), _loop_shape(loop_shape))
    rc = load_library().tmfg_batch_run(ctx.handle, jobs, len(mats), ctypes.byref(p),
                                       ctypes.byref(cfg), _stream_handle(stream))
    _check(rc, "tmfg_batch_run")
    return outs


_SIM = {"f64": 0, "f32": 1, "bf16x3": 2, "tf32x3": 3}


def _pipeline_outputs(n, dev):
    torch = _torch()
    return {"S": torch.empty((n, n), dtype=torch.float32, device=dev),
            "order": torch.empty(n, dtype=torch.int32, device=dev),
            "edges": torch.empty((3 * n - 6, 2), dtype=torch.int32, device=dev),
            "ins_face": torch.empty((max(n - 4, 1), 3), dtype=torch.int32, device=dev),
            "bubble_parent": torch.empty(n - 3, dtype=torch.int32, device=dev),
            "D": torch.empty((n, n), dtype=torch.float32, device=dev),
            "Z": torch.empty((n - 1, 4), dtype=torch.float64, device=dev),
            "labels": torch.empty(n, dtype=torch.int32, device=dev)}


def _pipeline_job(X, k, o):
    torch = _torch()
    if X.dtype != torch.float32 or X.dim() != 2 or X.stride(1) != 1:
        raise TypeError("X must be a row-major float32 matrix (series x length)")
    n, T = X.shape
    return _PipelineJob(X.data_ptr(), n, T, X.stride(0), o["S"].data_ptr(), o["order"].data_ptr(),
                        o["edges"].data_ptr(), o["ins_face"].data_ptr(),
                        o["bubble_parent"].data_ptr(), o["D"].data_ptr(), o["Z"].data_ptr(),
                        int(k), o["labels"].data_ptr() if k > 0 else None)


def tmfg_pipeline_run(ctx: Context, series, ks, precision: str = "bf16x3", mode: str = "corr",
                      prefix: int = 1, outs=None, stream=None, sssp_threads: int = 0,
                      loop_shape=None):
    """The whole clustering of every instance: similarity of its series (a
    float32 CUDA tensor, series x length), TMFG and exact APSP (batched), DBHT
    linkage and the labels of its cut at k (ks[i]; 0 = no cut).  Returns a
    list of dicts with S, the TMFG arrays, D, Z and labels.  Asynchronous."""
    if not series:
        return []
    if outs is None:
        outs = [_pipeline_outputs(X.shape[0], X.device) for X in series]
    jobs = (_PipelineJob * len(series))()
    for i, (X, k, o) in enumerate(zip(series, ks, outs)):
        jobs[i] = _pipeline_job(X, k, o)
    pp = _PipelineParams(_SIM[precision],
                         _Params({"corr": TMFG_CORR, "heap": TMFG_HEAP}[mode], int(prefix),
                                 TMFG_F32, 0))
    cfg = _BatchConfig(int(sssp_threads), _loop_shape(loop_shape))
    _check(load_library().tmfg_pipeline_run(ctx.handle, jobs, len(series), ctypes.byref(pp),
                                            ctypes.byref(cfg), _stream_handle(stream)),
           "tmfg_pipeline_run")
    return outs


def tmfg_pipeline_request_bytes(n: int, T: int, precision: str = "bf16x3") -> int:
    return int(load_library().tmfg_pipeline_request_bytes(int(n), int(T), _SIM[precision]))


def tmfg_cut_labels(ctx: Context, Z, k: int, labels=None, stream=None):
    """Labels (int32 CUDA tensor) of the cut of linkage Z at k clusters."""
    torch = _torch()
    n = Z.shape[0] + 1
    if labels is None:
        labels = torch.empty(n, dtype=torch.int32, device=Z.device)
    _check(load_library().tmfg_cut_labels(ctx.handle, _dev_ptr(Z, torch.float64), n, int(k),
                                          _dev_ptr(labels, torch.int32), _stream_handle(stream)),
           "tmfg_cut_labels")
    return labels


class Server:
    """Owns a tmfg_server (continuous-batching request server) and keeps each
    request's tensors alive until its result has been polled."""

    def __init__(self, device, cfg):
        lib = load_library()
        _torch()
        h = ctypes.c_void_p()
        _check(lib.tmfg_serve_start(ctypes.byref(h), int(device), ctypes.byref(cfg)),
               "tmfg_serve_start")
        self.handle = h
        self.device = device
        self.apsp = bool(cfg.apsp)
        self.live = {}

    def close(self):
        if getattr(self, "handle", None):
            rc = load_library().tmfg_serve_stop(self.handle)
            self.handle = None
            self.live.clear()
            _check(rc, "tmfg_serve_stop")

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tmfg_serve_start(device: int = 0, lanes: int = 0, max_batch: int = 0, lane_bytes: int = 0,
                     mode: str = "corr", prefix: int = 1, dtype: int = TMFG_F32,
                     apsp: bool = True, sssp_threads: int = 0, pipeline: bool = False,
                     precision: str = "bf16x3") -> Server:
    """Start a request server (see tmfg_serve_start in include/tmfg.h); with
    ``pipeline`` its jobs are whole clusterings from raw series
    (tmfg_serve_submit_pipeline)."""
    cfg = _ServeConfig(int(lanes), int(max_batch), int(lane_bytes),
                       _Params({"corr": TMFG_CORR, "heap": TMFG_HEAP}[mode], int(prefix),
                               int(dtype), 0),
                       1 if apsp else 0, int(sssp_threads), 1 if pipeline else 0,
                       _SIM[precision])
    return Server(device, cfg)


def tmfg_serve_submit_pipeline(server: Server, X, k: int, out=None, stream=None) -> int:
    """Queue the whole clustering of series X (float32 CUDA, series x length)
    with its cut at k; returns the request id.  Outputs as tmfg_pipeline_run's."""
    if out is None:
        out = _pipeline_outputs(X.shape[0], X.device)
    job = _pipeline_job(X, k, out)
    rid = load_library().tmfg_serve_submit_pipeline(server.handle, ctypes.byref(job),
                                                    _stream_handle(stream))
    if rid < 0:
        raise TmfgError(int(-rid), "tmfg_serve_submit_pipeline")
    server.live[int(rid)] = (X, out)
    return int(rid)


def tmfg_serve_submit(server: Server, S, out=None, stream=None) -> int:
    """Queue the TMFG (and exact APSP) of S; returns the request id.  The
    outputs (dict as from tmfg_build, plus D when the server runs APSP) are
    allocated here unless given, and come back with the result."""
    torch = _torch()
    n = S.shape[0]
    _mat_dtype(S)
    if out is None:
        dev = S.device
        out = {"order": torch.empty(n, dtype=torch.int32, device=dev),
               "edges": torch.empty((max(3 * n - 6, 0), 2), dtype=torch.int32, device=dev),
               "ins_face": torch.empty((max(n - 4, 0), 3), dtype=torch.int32, device=dev),
               "bubble_parent": torch.empty(max(n - 3, 0), dtype=torch.int32, device=dev)}
        if server.apsp:
            out["D"] = torch.empty((n, n), dtype=torch.float32, device=dev)
    D = out.get("D")
    job = _Job(S.data_ptr(), n, S.stride(0), out["order"].data_ptr(), out["edges"].data_ptr(),
               out["ins_face"].data_ptr() if n > 4 else None, out["bubble_parent"].data_ptr(),
               D.data_ptr() if D is not None else None, D.stride(0) if D is not None else 0)
    rid = load_library().tmfg_serve_submit(server.handle, ctypes.byref(job),
                                           _stream_handle(stream))
    if rid < 0:
        raise TmfgError(int(-rid), "tmfg_serve_submit")
    server.live[int(rid)] = (S, out)
    return int(rid)


def tmfg_serve_poll(server: Server, max_results: int = 1024, wait_us: int = 0) -> list:
    """Finished requests: dicts with id, status, batch, batch_size, the three
    timestamps (ns) and the request's outputs."""
    buf = (_ServeResult * max(1, int(max_results)))()
    c = load_library().tmfg_serve_poll(server.handle, buf, int(max_results), int(wait_us))
    if c < 0:
        raise TmfgError(int(-c), "tmfg_serve_poll")
    res = []
    for i in range(c):
        r = buf[i]
        S, out = server.live.pop(int(r.id))
        res.append({"id": int(r.id), "status": int(r.status), "batch": int(r.batch),
                    "batch_size": int(r.batch_size), "t_submit_ns": int(r.t_submit_ns),
                    "t_launch_ns": int(r.t_launch_ns), "t_done_ns": int(r.t_done_ns),
                    "S": S, "out": out})
    return res


def tmfg_serve_stop(server: Server):
    server.close()


def tmfg_serve_now_ns() -> int:
    return int(load_library().tmfg_serve_now_ns())


def tmfg_serve_request_bytes(n: int, apsp: bool = True) -> int:
    return int(load_library().tmfg_serve_request_bytes(int(n), 1 if apsp else 0))


def tmfg_serve_plan(ns, apsp: bool = True, max_batch: int = 256, lane_bytes: int = 4 << 30):
    """Batch index of each queued request under the admission rule (host
    only; no device needed)."""
    import numpy as np
    n = np.ascontiguousarray(ns, np.int64)
    out = np.empty(len(n), np.int32)
    rc = load_library().tmfg_serve_plan(n.ctypes.data_as(ctypes.c_void_p), len(n),
                                        1 if apsp else 0, int(max_batch), int(lane_bytes),
                                        out.ctypes.data_as(ctypes.c_void_p))
    _check(rc, "tmfg_serve_plan")
    return out


def tmfg_sync_status(ctx: Context, stream=None, raise_on_error: bool = True) -> int:
    """Wait for the stream, then return (or raise) the recorded status."""
    code = load_library().tmfg_sync_status(ctx.handle, _stream_handle(stream))
    if raise_on_error:
        _check(code, "device status")
    return int(code)


def tmfg_last_stats(ctx: Context) -> dict:
    arr = (ctypes.c_int64 * 16)()
    _check(load_library().tmfg_last_stats(ctx.handle, arr, 16), "tmfg_last_stats")
    keys = ["face_evals", "stale_pops", "scan_chunks", "rounds", "loop_ns", "cycles_recompute",
            "cycles_index", "cycles_select", "cycles_push", "cycles_refresh", "cycles_gains",
            "cycles_extract", "cycles_validate", "cycles_resolve", "cycles_stale_scan",
            "epoch_iters"]
    return {k: int(arr[i]) for i, k in enumerate(keys)}


def tmfg_memory_latency(ctx: Context, nbytes: int, hops: int = 20000, warm: int = 0) -> float:
    """Nanoseconds per dependent load over a scattered cycle of 128-byte
    lines in a fresh buffer of ``nbytes`` (see tmfg_memory_latency in
    include/tmfg.h): a buffer inside L2 with ``warm`` = its line count gives
    the L2 hit latency, a cold multi-gigabyte one the DRAM miss latency."""
    ns = ctypes.c_double()
    _check(load_library().tmfg_memory_latency(ctx.handle, int(nbytes), int(hops), int(warm),
                                              ctypes.byref(ns)), "tmfg_memory_latency")
    return ns.value


def tmfg_cluster_exchange_latency(ctx: Context, cluster: int = 8, iters: int = 20000) -> float:
    """Nanoseconds per exchange of a cluster of ``cluster`` CTAs: every CTA
    stores a 16-byte record into every CTA's shared memory, then a cluster
    barrier (the per-insertion step of the cluster loop kernel; see
    tmfg_cluster_exchange_latency in include/tmfg.h)."""
    ns = ctypes.c_double()
    _check(load_library().tmfg_cluster_exchange_latency(ctx.handle, int(cluster), int(iters),
                                                        ctypes.byref(ns)),
           "tmfg_cluster_exchange_latency")
    return ns.value


def tmfg_strerror(code: int) -> str:
    return _strerror(code)
