"""The latency diagnostics behind the loop's latency bound: an L2-resident
pointer chain must be faster than a cold multi-gigabyte one, both in a
physically sensible range, and a cluster exchange (stores into every CTA's
shared memory, then a cluster barrier) must take between 50 ns and 20 us."""
import pytest

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


def test_l2_hit_faster_than_dram_miss(T):
    ctx = T.tmfg_create(0)
    try:
        l2 = T.tmfg_memory_latency(ctx, 16 << 20, hops=5000, warm=(16 << 20) // 128)
        dram = T.tmfg_memory_latency(ctx, 1 << 30, hops=5000)
    finally:
        ctx.close()
    assert 20.0 < l2 < 3000.0, l2
    assert l2 < dram < 20000.0, (l2, dram)


def test_bad_arguments(T):
    ctx = T.tmfg_create(0)
    try:
        for args in ((100, 10, 0), (1 << 20, 0, 0), (1 << 20, 10, -1)):
            with pytest.raises(T.TmfgError):
                T.tmfg_memory_latency(ctx, *args)
    finally:
        ctx.close()


def test_cluster_exchange_latency(T):
    ctx = T.tmfg_create(0)
    try:
        for c in (8, 16):
            ns = T.tmfg_cluster_exchange_latency(ctx, c, iters=2000)
            assert 50.0 < ns < 20000.0, (c, ns)
        for c, it in ((4, 10), (8, 0)):
            with pytest.raises(T.TmfgError):
                T.tmfg_cluster_exchange_latency(ctx, c, iters=it)
    finally:
        ctx.close()
