"""Batched runs (many instances per launch) give every instance exactly the
result it gets alone: the same TMFG bit for bit as tmfg_build and the oracle,
and the same exact APSP as tmfg_apsp."""
import numpy as np
import pytest

import oracle
from paper_2408_09399_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def T():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_09399_gb300 import build
    build.build()
    import paper_2408_09399_gb300 as T
    return T


@pytest.fixture(scope="module")
def ctx(T):
    c = T.tmfg_create(0)
    yield c
    c.close()


def sizes(seed, k, lo=4, hi=700):
    u = W.uniform(seed, "sizes", k)
    return [int(round(np.exp(np.log(lo) + x * (np.log(hi) - np.log(lo))))) for x in u]


@pytest.mark.parametrize("mode,P", [("corr", 1), ("corr", 10), ("heap", 1)])
def test_batch_equals_single_and_oracle(T, ctx, mode, P):
    ns = sizes(7, 24) + [4, 5, 6]
    mats_np = [W.random_similarity(100 + i, n, np.float32, "uniform" if i % 3 else "quantized")
               for i, n in enumerate(ns)]
    mats = [torch.as_tensor(S, device="cuda:0") for S in mats_np]
    outs = T.tmfg_batch_run(ctx, mats, mode, P, apsp=True)
    T.tmfg_sync_status(ctx)
    for S_np, S, o in zip(mats_np, mats, outs):
        n = S.shape[0]
        ref = oracle.tmfg(S_np, mode, P)
        assert np.array_equal(o["order"].cpu().numpy(), ref["order"]), n
        assert np.array_equal(o["edges"].cpu().numpy(), ref["edges"]), n
        if n > 4:
            assert np.array_equal(o["ins_face"].cpu().numpy(), ref["ins_face"]), n
        assert np.array_equal(o["bubble_parent"].cpu().numpy(), ref["parent"]), n
        D1 = T.tmfg_apsp(ctx, S, o["edges"])
        T.tmfg_sync_status(ctx)
        assert torch.equal(o["D"], D1), n


def test_batch_float64_and_no_apsp(T, ctx):
    ns = [200, 5, 64, 333]
    mats_np = [W.random_similarity(300 + i, n, np.float64) for i, n in enumerate(ns)]
    mats = [torch.as_tensor(S, device="cuda:0") for S in mats_np]
    outs = T.tmfg_batch_run(ctx, mats, "heap", 1, apsp=False)
    T.tmfg_sync_status(ctx)
    for S_np, o in zip(mats_np, outs):
        ref = oracle.tmfg(S_np, "heap")
        assert np.array_equal(o["edges"].cpu().numpy(), ref["edges"])
        assert "D" not in o


def test_batch_twice_reuses_staging(T, ctx):
    mats = [torch.as_tensor(W.random_similarity(400 + i, 150 + i, np.float32), device="cuda:0")
            for i in range(6)]
    a = T.tmfg_batch_run(ctx, mats, "corr", 1)
    b = T.tmfg_batch_run(ctx, list(reversed(mats)), "corr", 1)
    T.tmfg_sync_status(ctx)
    for x, y in zip(a, reversed(b)):
        assert torch.equal(x["edges"], y["edges"]) and torch.equal(x["D"], y["D"])



@pytest.mark.parametrize("threads", [256, 512])
def test_batch_search_shapes_equal_single_and_oracle(T, ctx, threads):
    """Both CTA sizes of the batched exact search give tmfg_apsp's distances,
    which equal the oracle's float path sums: ragged sizes from 4 to 4096,
    ties from quantized S."""
    ns = [4, 5, 33, 250, 1100, 4096] + sizes(11, 6, 6, 900)
    mats_np = [W.random_similarity(700 + i, n, np.float32, "quantized" if i % 2 else "uniform")
               for i, n in enumerate(ns)]
    mats = [torch.as_tensor(S, device="cuda:0") for S in mats_np]
    outs = T.tmfg_batch_run(ctx, mats, "corr", 1, apsp=True, sssp_threads=threads)
    T.tmfg_sync_status(ctx)
    for S_np, S, o in zip(mats_np, mats, outs):
        n = S.shape[0]
        D1 = T.tmfg_apsp(ctx, S, o["edges"])
        T.tmfg_sync_status(ctx)
        assert torch.equal(o["D"], D1), (n, threads)
        if n <= 300:
            ref = oracle.apsp_exact(S_np, o["edges"].cpu().numpy(), prec=32)
            assert np.array_equal(o["D"].cpu().numpy().astype(np.float64), ref), (n, threads)
