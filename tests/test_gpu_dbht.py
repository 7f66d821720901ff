"""Parity of the device DBHT (dbht_cluster, through the C ABI) with the CPU
oracle: the linkage matrix, the bubble-edge directions, the converging
bubbles and every vertex's group and bubble must match exactly, on the
TMFG and distances the CUDA path computed (the oracle is given the same
TMFG and the same float32 distances, widened to double)."""
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


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda:0")


def gpu_pipeline(T, ctx, S, mode="corr", P=1, approx=False):
    dS = dev(S)
    t = T.tmfg_build(ctx, dS, mode, P)
    D = T.tmfg_apsp(ctx, dS, t["edges"], approx=approx)
    Z, info = T.dbht_cluster_detail(ctx, dS, t, D)
    T.tmfg_sync_status(ctx)
    th = {"order": t["order"].cpu().numpy(), "edges": t["edges"].cpu().numpy(),
          "ins_face": t["ins_face"].cpu().numpy(), "parent": t["bubble_parent"].cpu().numpy()}
    return th, D.cpu().numpy(), Z.cpu().numpy(), {k: v.cpu().numpy() for k, v in info.items()}


def assert_matches_oracle(S, th, D, Z, info, tag=""):
    Zr, ref = oracle.dbht(S, th, D.astype(np.float64))
    assert np.array_equal(info["direction"], ref["direction"]), f"direction {tag}"
    assert np.array_equal(info["converging"], ref["converging"]), f"converging {tag}"
    assert np.array_equal(info["group"], ref["group"]), f"group {tag}"
    assert np.array_equal(info["bubble"], ref["bubble"]), f"bubble {tag}"
    assert np.array_equal(Z, Zr), f"linkage {tag}: first diff row " + str(
        np.flatnonzero(np.any(Z != Zr, axis=1))[:3])


def check_linkage(Z, n):
    """Valid scipy-layout dendrogram: every id used once, sizes add up."""
    assert Z.shape == (n - 1, 4)
    size = np.ones(2 * n - 1, np.int64)
    used = np.zeros(2 * n - 1, bool)
    for r, (a, b, h, s) in enumerate(Z):
        a, b = int(a), int(b)
        assert a < b < n + r and not used[a] and not used[b]
        used[a] = used[b] = True
        size[n + r] = size[a] + size[b]
        assert size[n + r] == int(s) and h >= 0
    assert size[-1] == n


@pytest.mark.parametrize("n", [4, 5, 6, 10, 37, 120, 513])
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("kind", ["uniform", "quantized", "constant"])
def test_dbht_random_matches_oracle(T, ctx, n, dtype, kind):
    S = W.random_similarity(4000 + n, n, dtype, kind)
    th, D, Z, info = gpu_pipeline(T, ctx, S)
    check_linkage(Z, n)
    assert_matches_oracle(S, th, D, Z, info, f"n={n} {kind}")


@pytest.mark.parametrize("mode,P,approx", [("corr", 1, False), ("heap", 1, False),
                                           ("corr", 10, True)])
def test_dbht_config1(T, ctx, mode, P, approx):
    S, _ = W.config_similarity(1)
    th, D, Z, info = gpu_pipeline(T, ctx, S, mode, P, approx)
    assert_matches_oracle(S, th, D, Z, info, f"{mode} P={P} approx={approx}")


@pytest.mark.parametrize("n", [1000, 2000])
def test_dbht_config2_shapes(T, ctx, n):
    """Planted Dirichlet clusters at sizes where groups hold hundreds of
    cells (the level-2 linkage spans many warps and re-scan rounds)."""
    S, _ = W.config_similarity(2, n=n)
    th, D, Z, info = gpu_pipeline(T, ctx, S)
    assert_matches_oracle(S, th, D, Z, info, f"n={n}")


def test_dbht_ties_in_large_groups(T, ctx):
    """Planted clusters with S rounded to multiples of 1/16: groups of
    hundreds of cells whose distances tie often, so the merge order of the
    nearest-neighbour chain rests on the representative tie-break; the
    dendrogram must still be the oracle's sequential smallest-key one."""
    S, _ = W.config_similarity(2, n=1500)
    S = (np.round(np.asarray(S, np.float64) * 16.0) / 16.0).astype(np.float32)
    th, D, Z, info = gpu_pipeline(T, ctx, S)
    check_linkage(Z, S.shape[0])
    assert len(np.unique(Z[:, 2])) < len(Z) // 2  # many tied merge heights
    assert_matches_oracle(S, th, D, Z, info, "quantized n=1500")


def test_dbht_planted_clusters_recovered(T, ctx):
    """Section 5: on clean planted inputs the cut at the true k recovers the
    clusters exactly (ARI = 1), from the device dendrogram."""
    n, Tlen, k = 120, 2000, 4
    for seed in (3, 4):
        X, lab = W.factor_series(seed, n, Tlen, k, "equal", (0.7, 0.9), "normal")
        S = W.pearson_similarity(X, np.float64)
        _, _, Z, _ = gpu_pipeline(T, ctx, S, "heap")
        assert oracle.ari(lab, oracle.cut(Z, k)) == 1.0


def test_dbht_deterministic(T, ctx):
    S, _ = W.config_similarity(2, n=700)
    a = gpu_pipeline(T, ctx, S)[2]
    b = gpu_pipeline(T, ctx, S)[2]
    assert np.array_equal(a, b)


def test_dbht_rejects_bad_tmfg(T, ctx):
    n = 50
    S = W.random_similarity(5, n, np.float32)
    dS = dev(S)
    t = T.tmfg_build(ctx, dS, "corr", 1)
    D = T.tmfg_apsp(ctx, dS, t["edges"])
    T.tmfg_sync_status(ctx)
    bad = dict(t)
    bad["bubble_parent"] = t["bubble_parent"].clone()
    bad["bubble_parent"][7] = 9            # a parent must precede its child
    T.dbht_cluster(ctx, dS, bad, D)
    with pytest.raises(T.TmfgError) as e:
        T.tmfg_sync_status(ctx)
    assert e.value.code == 1
    bad = dict(t)
    bad["order"] = t["order"].clone()
    bad["order"][3] = bad["order"][4]      # not a permutation
    T.dbht_cluster(ctx, dS, bad, D)
    with pytest.raises(T.TmfgError) as e:
        T.tmfg_sync_status(ctx)
    assert e.value.code == 1
    # the context is usable afterwards
    Z = T.dbht_cluster(ctx, dS, t, D)
    T.tmfg_sync_status(ctx)
    check_linkage(Z.cpu().numpy(), n)


def test_dbht_argument_errors(T, ctx):
    S = W.random_similarity(6, 20, np.float32)
    dS = dev(S)
    t = T.tmfg_build(ctx, dS, "corr", 1)
    D = T.tmfg_apsp(ctx, dS, t["edges"])
    T.tmfg_sync_status(ctx)
    with pytest.raises(TypeError):
        T.dbht_cluster(ctx, dS, t, D.double())
    lib = T.load_library()
    import ctypes
    Z = torch.empty((19, 4), dtype=torch.float64, device="cuda:0")
    args = [ctx.handle, ctypes.c_void_p(dS.data_ptr()), 20, 20, 0,
            ctypes.c_void_p(t["order"].data_ptr()), ctypes.c_void_p(t["edges"].data_ptr()),
            ctypes.c_void_p(t["ins_face"].data_ptr()),
            ctypes.c_void_p(t["bubble_parent"].data_ptr()), ctypes.c_void_p(D.data_ptr()), 20,
            ctypes.c_void_p(Z.data_ptr()), None]
    assert lib.dbht_cluster(*args) == 0
    T.tmfg_sync_status(ctx)
    bad = list(args)
    bad[3] = 19                       # ld < n
    assert lib.dbht_cluster(*bad) == 1
    bad = list(args)
    bad[2], bad[3], bad[10] = 30000, 30000, 30000
    assert lib.dbht_cluster(*bad) == 8  # above DBHT_MAX_N
    bad = list(args)
    bad[9] = None
    assert lib.dbht_cluster(*bad) == 1


@pytest.mark.slow
def test_dbht_config2_full(T, ctx):
    S, lab = W.config_similarity(2)
    th, D, Z, info = gpu_pipeline(T, ctx, S)
    assert_matches_oracle(S, th, D, Z, info, "config 2")


@pytest.mark.slow
def test_dbht_full_size_n20000(T, ctx):
    """n = 20000 (the bench workload): too large for the oracle's level-2
    linkage, so the checks are properties: a valid dendrogram, every group a
    subtree of it, and the group and bubble of sampled vertices equal to the
    least mean distance rule evaluated directly in double."""
    S, lab = W.config_similarity(3, device="cuda:0")
    n = S.shape[0]
    t = T.tmfg_build(ctx, S, "corr", 1)
    D = T.tmfg_apsp(ctx, S, t["edges"])
    Z, info = T.dbht_cluster_detail(ctx, S, t, D)
    T.tmfg_sync_status(ctx)
    Z = Z.cpu().numpy()
    check_linkage(Z, n)
    group = info["group"].cpu().numpy()
    bub = info["bubble"].cpu().numpy()
    conv = np.flatnonzero(info["converging"].cpu().numpy())
    order = t["order"].cpu().numpy()
    face = t["ins_face"].cpu().numpy()
    bv = np.concatenate([order[None, :4], np.concatenate([order[4:, None], face], axis=1)])
    Dh = D.cpu().numpy().astype(np.float64)

    def mean4(v, b):
        s = 0.0
        for u in bv[b]:
            s = s + (Dh[min(v, u), max(v, u)])
        return s / 4.0

    rng = np.random.default_rng(0)
    for v in rng.choice(n, 64, replace=False):
        m = [mean4(v, c) for c in conv]
        assert group[v] == conv[int(np.argmin(m))]
    # the first n - ngroups merges stay inside groups and end with exactly
    # one cluster per group (the levels of the three-level linkage)
    ng = len(np.unique(group))
    parent = np.arange(2 * n - 1)

    def find(x):
        while parent[x] != x:
            parent[x] = parent[parent[x]]
            x = parent[x]
        return x

    for r in range(n - ng):
        a, b = int(Z[r, 0]), int(Z[r, 1])
        parent[find(a)] = n + r
        parent[find(b)] = n + r
    roots = np.array([find(v) for v in range(n)])
    for g in np.unique(group):
        assert len(np.unique(roots[group == g])) == 1
    assert len(np.unique(roots)) == ng


def test_dbht_hand_traced_case(T, ctx):
    """The hand-traced DBHT case (given TMFG, S on its edges, integer D):
    directions, converging bubbles, groups, bubbles and linkage on the
    device equal the values worked out by hand, as they do in the oracle."""
    import json
    import os
    case = json.load(open(os.path.join(os.path.dirname(__file__), "golden",
                                       "hand_traced_dbht.json")))
    n = case["n"]
    S = np.eye(n, dtype=np.float32)
    for key, val in case["S_edges_64ths"].items():
        i, j = map(int, key.split(","))
        S[i, j] = S[j, i] = val / 64.0
    D = np.zeros((n, n), np.float32)
    for key, val in case["D_upper"].items():
        i, j = map(int, key.split(","))
        D[i, j] = D[j, i] = val
    tg = {"order": case["tmfg"]["order"], "edges": case["tmfg"]["edges"],
          "ins_face": case["tmfg"]["ins_face"], "bubble_parent": case["tmfg"]["parent"]}
    td = {k: torch.tensor(v, dtype=torch.int32, device="cuda:0") for k, v in tg.items()}
    Z, info = T.dbht_cluster_detail(ctx, dev(S), td, dev(D))
    assert T.tmfg_sync_status(ctx) == 0
    e = case["expect"]
    assert info["direction"].cpu().tolist() == e["direction"]
    assert info["converging"].cpu().tolist() == e["converging"]
    assert info["group"].cpu().tolist() == e["group"]
    assert info["bubble"].cpu().tolist() == e["bubble"]
    assert Z.cpu().tolist() == [[float(x) for x in row] for row in e["linkage"]]
