"""Sizes past one CTA's shared memory and every launch shape of the
corr-tmfg prefix-1 loop, against the oracle.

- Rows longer than the one-pass sort holds (n > 21575 for float, > 10788
  for double) are sorted as two halves and merged: the sorted ids must equal
  the oracle's (S desc, u asc) order bit for bit on sampled rows, with ties,
  and the exact row sums must match on every row.
- corr-tmfg with prefix 1 at n = 30000 (the pointers then live in global
  memory) must give the oracle's TMFG bit for bit, and its exact and
  approximate APSP the oracle's rows.
- Every loop shape (threads, lanes per row refresh, copied index groups,
  and the general kernel) gives the same TMFG, single and batched.
"""
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
    T.tmfg_set_loop_shape(c, None)
    c.close()


def device_similarity(n, seed, dtype=torch.float32, quantized=False):
    """Symmetric U(-1, 1) (or quantized to 1/8, many ties) with unit diagonal,
    made on the device."""
    g = torch.Generator(device="cuda:0")
    g.manual_seed(seed)
    S = torch.rand((n, n), generator=g, device="cuda:0", dtype=torch.float64) * 2 - 1
    if quantized:
        S = torch.floor((S + 1) * 8.5) / 8 - 1
    S = torch.triu(S, 1)
    S = S + S.T
    S.fill_diagonal_(1.0)
    return S.to(dtype)


def sampled_rows(n, seed, k=48):
    rng = np.random.default_rng(seed)
    return np.unique(np.concatenate([[0, n - 1, n // 2], rng.integers(0, n, k)])).astype(np.int32)


@pytest.mark.slow
@pytest.mark.parametrize("n,dtype,quantized", [(21576, torch.float32, False),
                                               (30001, torch.float32, True),
                                               (10789, torch.float64, False),
                                               (14000, torch.float64, True)])
def test_row_sort_long_rows(T, ctx, n, dtype, quantized):
    S = device_similarity(n, 11 + n, dtype, quantized)
    idx, rs = T.tmfg_row_sort(ctx, S)
    T.tmfg_sync_status(ctx)
    Sn = S.cpu().numpy()
    rows = sampled_rows(n, n)
    got = idx[torch.as_tensor(rows, device="cuda:0")].cpu().numpy().view(np.uint16)
    assert np.array_equal(got[:, : n - 1].astype(np.int32), oracle.rowsort_rows(Sn, rows))
    assert np.all(got[:, n - 1:] == 0xFFFF)
    assert np.array_equal(rs.cpu().numpy(), oracle.rowsums(Sn))


@pytest.mark.slow
def test_tmfg_n30000_matches_oracle(T, ctx):
    n = 30000
    assert T.tmfg_max_n(0) >= n
    S = device_similarity(n, 5)
    T.tmfg_set_loop_shape(ctx, None)
    out = T.tmfg_build(ctx, S, "corr", 1)
    D = T.tmfg_apsp(ctx, S, out["edges"])
    Da = T.tmfg_apsp(ctx, S, out["edges"], approx=True)
    T.tmfg_sync_status(ctx)
    Sn = S.cpu().numpy()
    ref = oracle.tmfg(Sn, "corr", 1)
    assert np.array_equal(out["order"].cpu().numpy(), ref["order"])
    assert np.array_equal(out["edges"].cpu().numpy(), ref["edges"])
    assert np.array_equal(out["ins_face"].cpu().numpy(), ref["ins_face"])
    assert np.array_equal(out["bubble_parent"].cpu().numpy(), ref["parent"])
    src = sampled_rows(n, 3, 16)
    sd = torch.as_tensor(src, device="cuda:0")
    assert np.array_equal(D[sd].cpu().numpy().astype(np.float64),
                          oracle.sssp_rows(Sn, ref["edges"], src, prec=32))
    assert np.array_equal(Da[sd].cpu().numpy().astype(np.float64),
                          oracle.apsp_approx_rows(Sn, ref["edges"], src, 0, 2.0, prec=32))


SHAPES = [dict(kernel=1), dict(kernel=1, probe_lanes=4), dict(kernel=1, probe_lanes=16),
          dict(kernel=1, threads=512), dict(kernel=1, threads=512, probe_lanes=16),
          dict(kernel=1, stage_groups=-1), dict(kernel=1, stage_groups=3), dict(kernel=2)]


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "-".join(f"{k}{v}" for k, v in s.items()))
def test_loop_shapes_match_oracle(T, ctx, shape):
    T.tmfg_set_loop_shape(ctx, shape)
    try:
        for n, dtype, kind in [(4, np.float32, "uniform"), (9, np.float64, "quantized"),
                               (300, np.float32, "quantized"), (1500, np.float32, "uniform"),
                               (2100, np.float64, "uniform")]:
            S = W.random_similarity(4400 + n, n, dtype, kind)
            out = T.tmfg_build(ctx, torch.as_tensor(S, device="cuda:0"), "corr", 1)
            T.tmfg_sync_status(ctx)
            ref = oracle.tmfg(S, "corr", 1)
            assert np.array_equal(out["order"].cpu().numpy(), ref["order"]), (n, shape)
            assert np.array_equal(out["edges"].cpu().numpy(), ref["edges"]), (n, shape)
            assert np.array_equal(out["bubble_parent"].cpu().numpy(), ref["parent"]), (n, shape)
    finally:
        T.tmfg_set_loop_shape(ctx, None)


@pytest.mark.parametrize("shape", [dict(kernel=1), dict(kernel=1, threads=512, probe_lanes=16),
                                   dict(kernel=2)], ids=["p1", "p1-512-16", "general"])
def test_batched_loop_shapes_match_oracle(T, ctx, shape):
    ns = [4, 5, 37, 250, 900, 1200]
    mats_np = [W.random_similarity(500 + i, n, np.float32, "quantized" if i % 2 else "uniform")
               for i, n in enumerate(ns)]
    mats = [torch.as_tensor(S, device="cuda:0") for S in mats_np]
    outs = T.tmfg_batch_run(ctx, mats, "corr", 1, apsp=False, loop_shape=shape)
    T.tmfg_sync_status(ctx)
    for S_np, o in zip(mats_np, outs):
        ref = oracle.tmfg(S_np, "corr", 1)
        assert np.array_equal(o["edges"].cpu().numpy(), ref["edges"]), S_np.shape[0]
        assert np.array_equal(o["order"].cpu().numpy(), ref["order"]), S_np.shape[0]
