"""Pins for the DBHT, linkage, dendrogram cut, ARI and Pearson parts of the
oracle (Section 2 DBHT sketch; Section 5 evaluation) against scipy/sklearn,
a hand trace, an independent planar-separation formulation and the planted
truth of clean inputs."""
import json
import os

import numpy as np
import pytest
from scipy.cluster.hierarchy import fcluster, linkage
from scipy.spatial.distance import squareform

import oracle
from paper_2408_09399_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hand_traced_tmfg.json")


def partitions_of(Z, n):
    """Set of leaf sets created by the merges of a linkage matrix."""
    members = {i: frozenset([i]) for i in range(n)}
    out = set()
    for r, (a, b, _, size) in enumerate(Z):
        m = members[int(a)] | members[int(b)]
        assert len(m) == int(size)
        members[n + r] = m
        out.add(m)
    return out


@pytest.mark.parametrize("seed,n", [(1, 10), (2, 40), (3, 90)])
def test_complete_linkage_matches_scipy(seed, n):
    adjusted_rand_score = pytest.importorskip("sklearn.metrics").adjusted_rand_score
    X = W.normal(seed, "pts", n * 3).reshape(n, 3)
    D = np.sqrt(((X[:, None, :] - X[None, :, :]) ** 2).sum(-1))
    Z = oracle.complete_linkage(D)
    Zs = linkage(squareform(D, checks=False), method="complete")
    np.testing.assert_allclose(np.sort(Z[:, 2]), np.sort(Zs[:, 2]), rtol=1e-12)
    assert partitions_of(Z, n) == partitions_of(Zs, n)
    for k in (2, 3, 5):
        a = oracle.cut(Z, k)
        b = fcluster(Zs, k, criterion="maxclust")
        assert len(set(a.tolist())) == k
        assert adjusted_rand_score(a, b) == 1.0


def test_ari_matches_sklearn():
    adjusted_rand_score = pytest.importorskip("sklearn.metrics").adjusted_rand_score
    for seed in range(5):
        a = (W.u64(seed, "a", 300) % np.uint64(7)).astype(np.int32)
        b = (W.u64(seed, "b", 300) % np.uint64(5)).astype(np.int32)
        b[:100] = a[:100]
        assert abs(oracle.ari(a, b) - adjusted_rand_score(a, b)) < 1e-12
    a = np.array([0, 0, 1, 1, 2], np.int32)
    assert oracle.ari(a, a) == 1.0


def test_pearson_matches_numpy():
    X = W.normal(4, "x", 30 * 50).reshape(30, 50)
    np.testing.assert_allclose(oracle.pearson(X), np.corrcoef(X), rtol=1e-12, atol=1e-12)


def test_directions_hand_traced():
    case = [c for c in json.load(open(GOLDEN))["cases"] if c["name"] == "B_n7"][0]
    S = np.eye(7)
    for key, val in case["upper_64ths"].items():
        i, j = map(int, key.split(","))
        S[i, j] = S[j, i] = val / 64.0
    t = oracle.tmfg(S, "corr", 1)
    D = oracle.apsp_exact(S, t["edges"], 64)
    _, info = oracle.dbht(S, t, D)
    assert info["direction"].tolist() == case["dbht_direction"]["direction"]
    assert info["converging"].tolist() == case["dbht_direction"]["converging"]


def separated_side(n, edges, tri, v):
    """Vertices reachable from v in the TMFG with the triangle removed."""
    adj = [[] for _ in range(n)]
    for a, b in edges:
        adj[a].append(b)
        adj[b].append(a)
    seen, stack = {v}, [v]
    while stack:
        for w in adj[stack.pop()]:
            if w not in seen and w not in tri:
                seen.add(w)
                stack.append(w)
    return seen


def test_directions_by_planar_separation():
    """The inside of separating triangle t_k is the component of G - t_k that
    holds v_k (a topological definition, independent of the bubble tree)."""
    for seed, n, kind in [(11, 25, "uniform"), (12, 60, "uniform"), (13, 30, "constant"),
                          (14, 40, "quantized")]:
        S = W.random_similarity(seed, n, np.float32, kind)
        t = oracle.tmfg(S, "heap")
        D = oracle.apsp_exact(S, t["edges"], 64)
        _, info = oracle.dbht(S, t, D)
        E = t["edges"].tolist()
        for k in range(1, n - 3):
            tri = set(t["ins_face"][k - 1].tolist())
            inside = separated_side(n, E, tri, int(t["order"][3 + k]))
            w_in = w_out = 0
            for a, b in E:
                if (a in tri) == (b in tri):
                    continue
                j = b if a in tri else a
                q = oracle.quantize(float(S[a, b]))
                if j in inside:
                    w_in += q
                else:
                    w_out += q
            assert info["direction"][k - 1] == (1 if w_in > w_out else 0)


def check_linkage(Z, n):
    assert Z.shape == (n - 1, 4)
    used = set()
    for r, (a, b, h, size) in enumerate(Z):
        a, b = int(a), int(b)
        assert a < b < n + r and a not in used and b not in used
        used |= {a, b}
        assert h >= 0
    assert Z[-1, 3] == n
    partitions_of(Z, n)


def test_dbht_structure_and_groups():
    S, _ = W.config_similarity(1)
    t = oracle.tmfg(S, "heap")
    D = oracle.apsp_exact(S, t["edges"], 64)
    Z, info = oracle.dbht(S, t, D)
    n = S.shape[0]
    check_linkage(Z, n)
    conv = np.flatnonzero(info["converging"])
    assert len(conv) >= 1
    assert set(info["group"].tolist()) <= set(conv.tolist())
    # every group is one subtree of the dendrogram
    parts = partitions_of(Z, n)
    for g in set(info["group"].tolist()):
        assert frozenset(np.flatnonzero(info["group"] == g).tolist()) in parts | {
            frozenset([int(np.flatnonzero(info["group"] == g)[0])])}


@pytest.mark.parametrize("seed", [3, 4])
def test_planted_clusters_recovered(seed):
    """Section 5: TMFG-DBHT recovers clusters; on clean planted inputs
    (strong loadings, long series) the cut at the true k gives ARI = 1."""
    n, T, k = 120, 2000, 4
    X, lab = W.factor_series(seed, n, T, k, "equal", (0.7, 0.9), "normal")
    S = W.pearson_similarity(X, np.float64)
    for mode in ("corr", "heap"):
        t = oracle.tmfg(S, mode)
        D = oracle.apsp_exact(S, t["edges"], 64)
        Z, _ = oracle.dbht(S, t, D)
        assert oracle.ari(lab, oracle.cut(Z, k)) == 1.0


def test_direction_tie_points_to_parent():
    """n=5 with constant S: the inserted vertex and the fourth clique vertex
    each have three edges to the separating triangle, so w_in == w_out and the
    edge points toward the parent (reading of the DBHT direction rule)."""
    S = np.full((5, 5), 0.25)
    np.fill_diagonal(S, 1.0)
    t = oracle.tmfg(S, "heap")
    _, info = oracle.dbht(S, t, oracle.apsp_exact(S, t["edges"], 64))
    assert info["direction"].tolist() == [0]
    assert info["converging"].tolist() == [1, 0]


GOLDEN_DBHT = os.path.join(os.path.dirname(__file__), "golden", "hand_traced_dbht.json")


def load_dbht_case():
    """The hand-traced DBHT case: S on the TMFG edges (1/64ths), the TMFG
    itself and an integer distance matrix D, all given explicitly."""
    case = json.load(open(GOLDEN_DBHT))
    n = case["n"]
    S = np.eye(n)
    for key, val in case["S_edges_64ths"].items():
        i, j = map(int, key.split(","))
        S[i, j] = S[j, i] = val / 64.0
    D = np.zeros((n, n))
    for key, val in case["D_upper"].items():
        i, j = map(int, key.split(","))
        D[i, j] = D[j, i] = float(val)
    t = {k: np.array(v, np.int32) for k, v in case["tmfg"].items()}
    return case, S, t, D


def test_dbht_assignment_rules_hand_traced():
    """Rules (d) group of a vertex, (e) home of a bubble and (f) bubble of a
    vertex of the DBHT reading, each decided once by a margin and once by a
    tie in the hand trace, and the linkage rows that follow from them."""
    case, S, t, D = load_dbht_case()
    Z, info = oracle.dbht(S, t, D)
    e = case["expect"]
    assert info["direction"].tolist() == e["direction"]
    assert info["converging"].tolist() == e["converging"]
    assert info["group"].tolist() == e["group"]
    assert info["bubble"].tolist() == e["bubble"]
    # the home of each bubble shows in which group its vertices landed
    for v, b in enumerate(e["bubble"]):
        assert e["home"][b] == e["group"][v]
    assert Z.tolist() == [[float(x) for x in row] for row in e["linkage"]]


def _section(src, marker):
    """Offset of the code following a comment marker in the oracle source."""
    i = src.index(marker)
    return i + len(marker)


# Planted mistakes in the assignment rules of oracle_dbht: (marker of the
# rule's block, text in that block, its replacement).  Each must make the
# hand-traced case fail.
DBHT_MUTATIONS = {
    "d_argmax": ("/* (d) group of each vertex */", "s < bm", "s > bm"),
    "d_tie_to_larger": ("/* (d) group of each vertex */", "s < bm", "s <= bm"),
    "e_argmax": ("/* (e) home of each bubble */", "s < bm", "s > bm"),
    "e_tie_to_larger": ("/* (e) home of each bubble */", "s < bm", "s <= bm"),
    "f_argmax": ("/* (f) bubble of each vertex */", "s < bm", "s > bm"),
    "f_tie_to_larger": ("/* (f) bubble of each vertex */", "s < bm", "s <= bm"),
}


@pytest.fixture(scope="module")
def oracle_source():
    return open(os.path.join(os.path.dirname(oracle.__file__), "tmfg_oracle.c")).read()


def test_unmutated_copy_passes(tmp_path, oracle_source):
    """Control for the mutation test: an unchanged copy built the same way
    reproduces the hand trace."""
    src = tmp_path / "copy.c"
    src.write_text(oracle_source)
    lib = oracle.compile_library(str(src), str(tmp_path / "copy.so"))
    with oracle.use_library(lib):
        test_dbht_assignment_rules_hand_traced()


@pytest.mark.parametrize("name", sorted(DBHT_MUTATIONS))
def test_planted_assignment_mistake_fails_the_hand_trace(tmp_path, oracle_source, name):
    marker, old, new = DBHT_MUTATIONS[name]
    at = _section(oracle_source, marker)
    k = oracle_source.index(old, at)
    assert k - at < 1200, "the pattern must lie in the rule's own block"
    mutated = oracle_source[:k] + new + oracle_source[k + len(old):]
    src = tmp_path / f"{name}.c"
    src.write_text(mutated)
    lib = oracle.compile_library(str(src), str(tmp_path / f"{name}.so"))
    with oracle.use_library(lib):
        with pytest.raises(AssertionError):
            test_dbht_assignment_rules_hand_traced()
