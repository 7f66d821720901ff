"""The continuous-batching request server: every request's result is the
same, bit for bit, whether it is served alone or in a mix with others (and
equals the oracle); batches respect the admission limits and overlap on the
device; data errors stay with their batch; refusals and shutdown are clean."""
import time

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


def sizes(seed, k, lo=4, hi=700):
    u = W.uniform(seed, "serve_sizes", k)
    return [int(round(np.exp(np.log(lo) + x * (np.log(hi) - np.log(lo))))) for x in u]


def requests(seed=11, k=40):
    ns = sizes(seed, k) + [4, 5, 6]
    mats = [W.random_similarity(500 + i, n, np.float32, "uniform" if i % 4 else "quantized")
            for i, n in enumerate(ns)]
    return mats


def collect(T, srv, count, timeout_s=120.0):
    got = {}
    t_end = time.time() + timeout_s
    while len(got) < count:
        assert time.time() < t_end, "server did not finish in time"
        for r in T.tmfg_serve_poll(srv, 1024, 20000):
            got[r["id"]] = r
    return got


def host(out):
    return {k: v.cpu().numpy() for k, v in out.items()}


def test_alone_equals_mix_equals_oracle(T):
    mats_np = requests()
    mats = [torch.as_tensor(S, device="cuda:0") for S in mats_np]
    sizes_b = [T.tmfg_serve_request_bytes(S.shape[0]) for S in mats]
    # lanes small enough that memory, not only max_batch, splits batches
    lane = 3 * max(sizes_b) + (1 << 20)
    srv = T.tmfg_serve_start(0, lanes=2, max_batch=8, lane_bytes=lane)
    ids = [T.tmfg_serve_submit(srv, S) for S in mats]
    mix = collect(T, srv, len(ids))
    T.tmfg_serve_stop(srv)
    for i in ids:
        assert mix[i]["status"] == 0
        assert 1 <= mix[i]["batch_size"] <= 8
    # the batches of the mix respected the lane memory
    by_batch = {}
    for i in ids:
        by_batch.setdefault(mix[i]["batch"], []).append(i)
    for b, members in by_batch.items():
        assert sum(sizes_b[i] for i in members) <= lane
    assert len(by_batch) >= 6
    # two lanes: some batch launched while another was still running
    spans = sorted({(mix[m[0]]["t_launch_ns"], mix[m[0]]["t_done_ns"]) for m in by_batch.values()})
    assert any(spans[j + 1][0] < spans[j][1] for j in range(len(spans) - 1))

    srv = T.tmfg_serve_start(0, lanes=1, max_batch=1)
    for i, S in zip(ids, mats):
        rid = T.tmfg_serve_submit(srv, S)
        alone = collect(T, srv, 1)[rid]
        assert alone["status"] == 0 and alone["batch_size"] == 1
        a, m = host(alone["out"]), host(mix[i]["out"])
        for k in a:
            assert np.array_equal(a[k], m[k]), (S.shape[0], k)
    T.tmfg_serve_stop(srv)

    for i, S_np in zip(ids, mats_np):
        n = S_np.shape[0]
        ref = oracle.tmfg(S_np, "corr", 1)
        o = host(mix[i]["out"])
        assert np.array_equal(o["order"], ref["order"]), n
        assert np.array_equal(o["edges"], ref["edges"]), n
        assert np.array_equal(o["bubble_parent"], ref["parent"]), n
        if n <= 300:
            assert np.array_equal(o["D"], oracle.apsp_exact(S_np, ref["edges"], 32).astype(np.float32)), n


def test_inputs_produced_on_another_stream(T):
    """A request's matrix written on the submitter's stream just before the
    submission is read only after that write (the server waits for it)."""
    srv = T.tmfg_serve_start(0, lanes=2)
    side = torch.cuda.Stream()
    n = 600
    S_np = W.random_similarity(77, n, np.float32)
    src = torch.as_tensor(S_np, device="cuda:0")
    ids = []
    outs = []
    with torch.cuda.stream(side):
        for _ in range(4):
            S = torch.empty_like(src)
            torch.cuda._sleep(2_000_000)  # delay the write on the side stream
            S.copy_(src)
            ids.append(T.tmfg_serve_submit(srv, S, stream=side))
            outs.append(S)
    got = collect(T, srv, len(ids))
    T.tmfg_serve_stop(srv)
    ref = oracle.tmfg(S_np, "corr", 1)
    for i in ids:
        assert np.array_equal(got[i]["out"]["edges"].cpu().numpy(), ref["edges"])


def test_data_error_stays_with_its_batch(T):
    srv = T.tmfg_serve_start(0, lanes=1, max_batch=1)
    good = torch.as_tensor(W.random_similarity(3, 50, np.float32), device="cuda:0")
    bad_np = W.random_similarity(4, 50, np.float32)
    bad_np[3, 7] = bad_np[7, 3] = np.nan
    bad = torch.as_tensor(bad_np, device="cuda:0")
    ids = [T.tmfg_serve_submit(srv, S) for S in (good, bad, good)]
    got = collect(T, srv, 3)
    T.tmfg_serve_stop(srv)
    assert [got[i]["status"] for i in ids] == [0, 3, 0]


def test_refusals_and_shutdown(T):
    big = torch.as_tensor(W.random_similarity(5, 2000, np.float32), device="cuda:0")
    small = torch.as_tensor(W.random_similarity(6, 100, np.float32), device="cuda:0")
    lane = T.tmfg_serve_request_bytes(1000) + (1 << 20)
    srv = T.tmfg_serve_start(0, lanes=2, lane_bytes=lane)
    with pytest.raises(T.TmfgError) as e:
        T.tmfg_serve_submit(srv, big)
    assert e.value.code == 2
    # stop with work still queued and running: finishes it, no hang
    for _ in range(30):
        T.tmfg_serve_submit(srv, small)
    t0 = time.time()
    T.tmfg_serve_stop(srv)
    assert time.time() - t0 < 60
    with pytest.raises(Exception):
        T.tmfg_serve_start(0, lanes=99)
