"""Host-side rules of the request server, no GPU needed: a request's memory
need, and how queued requests are grouped into batches (first come first
served, bounded by the batch cap and the lane's memory)."""
import ctypes

import numpy as np
import pytest


@pytest.fixture(scope="module")
def T():
    from paper_2408_09399_gb300 import build
    build.build()
    import paper_2408_09399_gb300 as T
    return T


def test_request_bytes_grow_with_n(T):
    b = [T.tmfg_serve_request_bytes(n) for n in (4, 64, 1000, 4000)]
    assert all(x < y for x, y in zip(b, b[1:]))
    # the sorted index rows (uint16, n x round8(n-1)) dominate large requests
    assert b[-1] >= 2 * 4000 * 4000
    assert T.tmfg_serve_request_bytes(1000, apsp=False) < T.tmfg_serve_request_bytes(1000)


def test_plan_respects_the_batch_cap(T):
    plan = T.tmfg_serve_plan([64] * 300, max_batch=256, lane_bytes=8 << 30)
    assert (plan[:256] == 0).all() and (plan[256:] == 1).all()


def test_plan_respects_lane_memory_and_order(T):
    rng = np.random.default_rng(3)
    ns = np.round(np.exp(rng.uniform(np.log(64), np.log(4000), 500))).astype(np.int64)
    lane = 256 << 20
    plan = T.tmfg_serve_plan(ns, max_batch=64, lane_bytes=lane)
    assert (np.diff(plan) >= 0).all()                  # first come, first served
    assert plan[0] == 0 and (np.diff(plan) <= 1).all()  # batches numbered densely
    need = np.array([T.tmfg_serve_request_bytes(int(n)) for n in ns])
    for b in range(plan.max() + 1):
        members = np.flatnonzero(plan == b)
        assert len(members) <= 64
        assert need[members].sum() <= lane
        nxt = members[-1] + 1
        if nxt < len(ns) and len(members) < 64:
            # the batch closed because the next request did not fit (the
            # descriptor tables add well under 1 MB)
            assert need[members].sum() + need[nxt] > lane - (1 << 20)


def test_plan_refuses_requests_larger_than_a_lane(T):
    lane = T.tmfg_serve_request_bytes(1000)
    with pytest.raises(T.TmfgError) as e:
        T.tmfg_serve_plan([100, 5000], lane_bytes=lane)
    assert e.value.code == 2
    with pytest.raises(T.TmfgError):
        T.tmfg_serve_plan([3])


def test_server_needs_a_device(T):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    with pytest.raises(RuntimeError):
        T.tmfg_serve_start(0)
