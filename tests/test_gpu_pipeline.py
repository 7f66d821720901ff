"""The whole clustering from raw series (tmfg_pipeline_run and the request
server in pipeline mode): every request's similarity, TMFG, distances,
dendrogram and labels equal, bit for bit, what the single calls give it
(tmfg_similarity, tmfg_build, tmfg_apsp, dbht_cluster, tmfg_cut_labels) and
what the oracle gives from the same similarity matrix; the result is the
same alone and in a mix of served requests."""
import time

import numpy as np
import pytest

import oracle
from paper_2408_09399_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

KEYS = ("S", "order", "edges", "bubble_parent", "D", "Z", "labels")


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


def reqs(seed, count, hi=700):
    return W.serving_requests(seed, count, device="cuda:0", n_range=(4, hi), T_range=(64, 400),
                              k_range=(1, 12), similarity=False)


def single(T, ctx, X, k, precision):
    S = T.tmfg_similarity(ctx, X, precision)
    t = T.tmfg_build(ctx, S, "corr", 1)
    D = T.tmfg_apsp(ctx, S, t["edges"])
    Z = T.dbht_cluster(ctx, S, t, D)
    lab = T.tmfg_cut_labels(ctx, Z, k) if k > 0 else None
    T.tmfg_sync_status(ctx)
    return {"S": S, "order": t["order"], "edges": t["edges"],
            "bubble_parent": t["bubble_parent"], "D": D, "Z": Z, "labels": lab}


def check_oracle(o, k):
    S = o["S"].cpu().numpy()
    ref = oracle.tmfg(S, "corr", 1)
    assert np.array_equal(o["edges"].cpu().numpy(), ref["edges"])
    D = oracle.apsp_exact(S, ref["edges"], prec=32)
    assert np.array_equal(o["D"].cpu().numpy().astype(np.float64), D)
    Z, _ = oracle.dbht(S, ref, D)
    assert np.array_equal(o["Z"].cpu().numpy(), Z)
    if k > 0:
        assert np.array_equal(o["labels"].cpu().numpy(), oracle.cut(Z, k))


@pytest.mark.parametrize("precision", ["bf16x3", "f32"])
def test_pipeline_equals_single_calls_and_oracle(T, ctx, precision):
    rs = reqs(31, 12)
    rs[0]["k"] = 0  # no cut
    outs = T.tmfg_pipeline_run(ctx, [r["X"] for r in rs], [r["k"] for r in rs], precision)
    T.tmfg_sync_status(ctx)
    for r, o in zip(rs, outs):
        s = single(T, ctx, r["X"], r["k"], precision)
        for key in KEYS:
            if key == "labels" and r["k"] == 0:
                continue
            assert torch.equal(o[key], s[key]), (r["n"], key)
        check_oracle(o, r["k"])


def test_cut_labels_matches_oracle(T, ctx):
    rng = np.random.default_rng(5)
    for n in (2, 3, 17, 400):
        X = rng.normal(size=(n, 3))
        D = np.sqrt(((X[:, None] - X[None]) ** 2).sum(-1))
        Z = oracle.complete_linkage(D)
        Zd = torch.as_tensor(Z, device="cuda:0")
        for k in sorted({1, 2, min(n, 5), n}):
            lab = T.tmfg_cut_labels(ctx, Zd, k)
            T.tmfg_sync_status(ctx)
            assert np.array_equal(lab.cpu().numpy(), oracle.cut(Z, k)), (n, k)


def collect(T, srv, count, timeout_s=180.0):
    got = {}
    t_end = time.time() + timeout_s
    while len(got) < count:
        assert time.time() < t_end, "server did not finish in time"
        for r in T.tmfg_serve_poll(srv, 1024, 20000):
            got[r["id"]] = r
    return got


def test_served_pipeline_alone_equals_mix_equals_oracle(T, ctx):
    rs = reqs(37, 16)
    need = [T.tmfg_pipeline_request_bytes(r["n"], r["T"]) for r in rs]
    lane = 3 * max(need) + (1 << 20)
    srv = T.tmfg_serve_start(0, lanes=2, max_batch=4, lane_bytes=lane, pipeline=True)
    ids = [T.tmfg_serve_submit_pipeline(srv, r["X"], r["k"]) for r in rs]
    mix = collect(T, srv, len(ids))
    T.tmfg_serve_stop(srv)
    assert all(mix[i]["status"] == 0 for i in ids)
    assert len({mix[i]["batch"] for i in ids}) >= 4
    srv = T.tmfg_serve_start(0, lanes=1, max_batch=1, pipeline=True)
    for i, r in zip(ids, rs):
        rid = T.tmfg_serve_submit_pipeline(srv, r["X"], r["k"])
        alone = collect(T, srv, 1)[rid]
        assert alone["status"] == 0
        for key in KEYS:
            assert torch.equal(alone["out"][key], mix[i]["out"][key]), (r["n"], key)
    T.tmfg_serve_stop(srv)
    for i, r in list(zip(ids, rs))[::3]:
        check_oracle(mix[i]["out"], r["k"])
