"""The memory-latency diagnostic (pointer chasing) behind the loop's latency
bound: an L2-resident chain must be faster than a cold multi-gigabyte one,
and both must fall in a physically sensible range."""
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
