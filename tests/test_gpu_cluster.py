"""The corr-tmfg prefix-1 insertion loop on a thread-block cluster (kernel 3
of tmfg_loop_shape), against the oracle.

The cluster kernel splits the faces over 8 or 16 CTAs and keeps a replica of
the sorted-row pointers in each; whatever the split, the TMFG must be the
oracle's bit for bit: order, edges, faces used and bubble parents.  Sizes
cover n = 4 (no insertion), n below the cluster size (CTAs that own no face),
ragged face counts, ties (quantized S), double input, builds that run in
segments with the rows compacted between them (n >= 1024), the benchmark's
n = 20000 workload and n = 30000.
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


def assert_same(out, ref, tag):
    assert np.array_equal(out["order"].cpu().numpy(), ref["order"]), tag
    assert np.array_equal(out["edges"].cpu().numpy(), ref["edges"]), tag
    assert np.array_equal(out["ins_face"].cpu().numpy(), ref["ins_face"]), tag
    assert np.array_equal(out["bubble_parent"].cpu().numpy(), ref["parent"]), tag


@pytest.mark.parametrize("C", [8, 16])
def test_cluster_kernel_matches_oracle(T, ctx, C):
    T.tmfg_set_loop_shape(ctx, dict(kernel=3, cluster=C))
    try:
        for n, dtype, kind in [(4, np.float32, "uniform"), (5, np.float32, "uniform"),
                               (9, np.float64, "quantized"), (13, np.float32, "constant"),
                               (300, np.float32, "quantized"), (1025, np.float32, "uniform"),
                               (1500, np.float32, "quantized"), (2100, np.float64, "uniform")]:
            S = W.random_similarity(8800 + n, n, dtype, kind)
            out = T.tmfg_build(ctx, torch.as_tensor(S, device="cuda:0"), "corr", 1)
            T.tmfg_sync_status(ctx)
            assert_same(out, oracle.tmfg(S, "corr", 1), (n, C, kind))
    finally:
        T.tmfg_set_loop_shape(ctx, None)


def test_cluster_kernel_config2(T, ctx):
    """n = 5000, T = 1000, 20 planted clusters (six segments, five row
    compactions), both cluster sizes."""
    S, _ = W.config_similarity(2)
    ref = oracle.tmfg(S, "corr", 1)
    try:
        for C in (8, 16):
            T.tmfg_set_loop_shape(ctx, dict(kernel=3, cluster=C))
            out = T.tmfg_build(ctx, torch.as_tensor(S, device="cuda:0"), "corr", 1)
            T.tmfg_sync_status(ctx)
            assert_same(out, ref, C)
    finally:
        T.tmfg_set_loop_shape(ctx, None)


@pytest.mark.slow
def test_cluster_kernel_full_size(T, ctx):
    """The benchmark's workload (n = 20000, 50 planted clusters, Student-t(4)
    noise, float32) on both cluster sizes equals the oracle."""
    S, _ = W.config_similarity(3, device="cuda")
    ref = oracle.tmfg(S.cpu().numpy(), "corr", 1)
    try:
        for C in (8, 16):
            T.tmfg_set_loop_shape(ctx, dict(kernel=3, cluster=C))
            out = T.tmfg_build(ctx, S, "corr", 1)
            T.tmfg_sync_status(ctx)
            assert_same(out, ref, C)
    finally:
        T.tmfg_set_loop_shape(ctx, None)


@pytest.mark.slow
def test_cluster_kernel_n30000(T, ctx):
    """n = 30000 (only the 16-CTA split fits shared memory) on a symmetric
    U(-1, 1) matrix made on the device."""
    n = 30000
    g = torch.Generator(device="cuda:0")
    g.manual_seed(5)
    S = torch.rand((n, n), generator=g, device="cuda:0", dtype=torch.float64) * 2 - 1
    S = torch.triu(S, 1)
    S = (S + S.T).fill_diagonal_(1.0).to(torch.float32)
    ref = oracle.tmfg(S.cpu().numpy(), "corr", 1)
    try:
        T.tmfg_set_loop_shape(ctx, dict(kernel=3, cluster=16))
        out = T.tmfg_build(ctx, S, "corr", 1)
        T.tmfg_sync_status(ctx)
        assert_same(out, ref, 16)
    finally:
        T.tmfg_set_loop_shape(ctx, None)


def test_cluster_kernel_rejected_in_batch(T, ctx):
    mats = [torch.as_tensor(W.random_similarity(3, 40, np.float32), device="cuda:0")]
    with pytest.raises(T.TmfgError) as e:
        T.tmfg_batch_run(ctx, mats, "corr", 1, apsp=False, loop_shape=dict(kernel=3))
    assert e.value.code == 1
