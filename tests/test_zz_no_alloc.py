"""The allocation-free exact APSP entry point, tmfg_apsp_exact_noalloc.

It exists for callers that cannot allocate device memory (their device
memory belongs to their own pool or caching allocator, or the calling path
must not take an allocator's locks and synchronisation).  Its scratch is a
static device array shared by all calls, so this test calls it twice in a
row, with different n, and checks each result bit for bit against the
context-based tmfg_apsp, the tolerance the APSP parity tests use; a third
case runs at the largest n the array admits.  It also checks the size
limit.  Collected last so that a failure here comes after every other test
has run; it also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

from paper_2408_09399_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

NOALLOC_MAX_N = 21581  # TMFG_NOALLOC_MAX_N in include/tmfg.h


@pytest.fixture(scope="module")
def T():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_09399_gb300 import build
    build.build()
    import paper_2408_09399_gb300 as T
    lib = T.load_library()
    P = ctypes.c_void_p
    lib.tmfg_apsp_exact_noalloc.argtypes = [P, ctypes.c_int64, ctypes.c_int64, ctypes.c_int32, P,
                                            P, ctypes.c_int64, P, P]
    lib.tmfg_apsp_exact_noalloc.restype = ctypes.c_int
    return T


@pytest.fixture
def ctx(T):
    c = T.tmfg_create(0)
    try:
        yield c
    finally:
        c.close()


def noalloc(T, S, edges, D, status):
    stream = torch.cuda.current_stream()
    dt = 0 if S.dtype == torch.float32 else 1
    return T.load_library().tmfg_apsp_exact_noalloc(
        ctypes.c_void_p(S.data_ptr()), S.shape[0], S.stride(0), dt,
        ctypes.c_void_p(edges.data_ptr()), ctypes.c_void_p(D.data_ptr()), D.stride(0),
        ctypes.c_void_p(status.data_ptr()), ctypes.c_void_p(stream.cuda_stream))


def device_similarity(n, seed):
    """A symmetric U(-1, 1) matrix with unit diagonal made on the device
    (the largest case would take minutes to make on the host)."""
    g = torch.Generator(device="cuda:0")
    g.manual_seed(seed)
    S = torch.rand((n, n), generator=g, device="cuda:0") * 2 - 1
    S = torch.triu(S, 1)
    S = S + S.T
    S.fill_diagonal_(1.0)
    return S


def random_tmfg_edges(n, seed):
    """Edges of a random TMFG-shaped planar graph (3n - 6 edges): the
    4-clique 0..3, then vertex k joined to the three corners of a face drawn
    at random, that face replaced by the three it splits into."""
    rng = np.random.default_rng(seed)
    faces = [(0, 1, 2), (0, 1, 3), (0, 2, 3), (1, 2, 3)]
    edges = [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]
    for k in range(4, n):
        i = int(rng.integers(len(faces)))
        x, y, z = faces[i]
        edges += [(k, x), (k, y), (k, z)]
        faces[i] = (k, x, y)
        faces += [(k, y, z), (k, x, z)]
    return torch.tensor(edges, dtype=torch.int32, device="cuda:0")


def check_against_context_path(T, ctx, S, mode, status):
    n = S.shape[0]
    if mode == "given":
        edges = random_tmfg_edges(n, 5)
    else:
        edges = T.tmfg_build(ctx, S, mode)["edges"]
    ref = T.tmfg_apsp(ctx, S, edges)
    T.tmfg_sync_status(ctx)
    D = torch.full((n, n), float("nan"), dtype=torch.float32, device="cuda:0")
    assert noalloc(T, S, edges, D, status) == 0
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    assert torch.equal(D, ref), f"n={n}"


def test_noalloc_matches_context_entry_point_twice(T, ctx):
    status = torch.full((1,), -7, dtype=torch.int32, device="cuda:0")
    for n, dtype, seed in [(1500, np.float32, 1), (700, np.float64, 2)]:
        S = torch.as_tensor(W.random_similarity(seed, n, dtype), device="cuda:0")
        check_against_context_path(T, ctx, S, "heap", status)


def test_noalloc_at_the_largest_size(T, ctx):
    """The CSR carve at n = TMFG_NOALLOC_MAX_N must fit the static array
    exactly; a larger exact-path workspace would overrun it.  The graph is a
    random TMFG-shaped one (the APSP takes any 3n - 6 edges), so the case
    does not depend on the largest n the TMFG build accepts."""
    status = torch.full((1,), -7, dtype=torch.int32, device="cuda:0")
    S = device_similarity(NOALLOC_MAX_N, 3)
    check_against_context_path(T, ctx, S, "given", status)
    del S
    torch.cuda.empty_cache()


def test_noalloc_rejects_sizes_beyond_the_limit(T):
    n = NOALLOC_MAX_N + 1
    S = torch.zeros((4, 4), dtype=torch.float32, device="cuda:0")
    edges = torch.zeros((6, 2), dtype=torch.int32, device="cuda:0")
    D = torch.zeros((4, 4), dtype=torch.float32, device="cuda:0")
    status = torch.zeros(1, dtype=torch.int32, device="cuda:0")
    lib = T.load_library()
    rc = lib.tmfg_apsp_exact_noalloc(ctypes.c_void_p(S.data_ptr()), n, n, 0,
                                     ctypes.c_void_p(edges.data_ptr()),
                                     ctypes.c_void_p(D.data_ptr()), n,
                                     ctypes.c_void_p(status.data_ptr()), None)
    assert rc == 8  # TMFG_ETOOBIG, returned before any device work
