"""Pins for the TMFG oracle (Algorithms 1 and 2 of Section 4).

Nothing here compares the oracle with itself: each test checks it against a
hand trace (tests/golden), a library routine, a closed-form special case, the
structural invariants of a TMFG (Section 2: a maximal planar graph built from
4-cliques), or a brute-force reformulation.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2408_09399_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hand_traced_tmfg.json")


def golden_cases():
    with open(GOLDEN) as f:
        return json.load(f)["cases"]


def golden_matrix(case, dtype):
    n = case["n"]
    S = np.eye(n)
    if "constant_64ths" in case:
        S[:] = case["constant_64ths"] / 64.0
        np.fill_diagonal(S, 1.0)
    else:
        for key, val in case["upper_64ths"].items():
            i, j = map(int, key.split(","))
            S[i, j] = S[j, i] = val / 64.0
    return S.astype(dtype)


# ---------------------------------------------------------------- invariants

def replay_faces(n, order, ins_face):
    """Rebuild the face list from the insertion record (Algorithm 1, line of
    F = F + 3 new faces - t) independently of the oracle's bookkeeping."""
    c = order[:4]
    faces = {frozenset((c[0], c[1], c[2])), frozenset((c[0], c[1], c[3])),
             frozenset((c[0], c[2], c[3])), frozenset((c[1], c[2], c[3]))}
    for k in range(n - 4):
        v = int(order[4 + k])
        x, y, z = (int(a) for a in ins_face[k])
        t = frozenset((x, y, z))
        assert t in faces, f"insertion {k} uses a face that is not live"
        faces.remove(t)
        faces |= {frozenset((v, x, y)), frozenset((v, y, z)), frozenset((v, x, z))}
    return faces


def check_tmfg_invariants(n, r):
    order, edges, ins_face, parent = r["order"], r["edges"], r["ins_face"], r["parent"]
    # every vertex exactly once
    assert sorted(order.tolist()) == list(range(n))
    # 3n-6 distinct edges, no self loops
    E = {frozenset(map(int, e)) for e in edges}
    assert len(E) == 3 * n - 6 == edges.shape[0]
    assert all(len(e) == 2 for e in E)
    adj = {v: set() for v in range(n)}
    for a, b in edges:
        adj[int(a)].add(int(b))
        adj[int(b)].add(int(a))
    # every insertion forms a 4-clique with a live face
    faces = replay_faces(n, order, ins_face)
    inserted = set(order[:4].tolist())
    for k in range(n - 4):
        v = int(order[4 + k])
        x, y, z = (int(a) for a in ins_face[k])
        assert x < y < z and {x, y, z} <= inserted and v not in inserted
        assert {x, y, z} <= adj[v]
        assert y in adj[x] and z in adj[x] and z in adj[y]
        assert [int(a) for a in edges[6 + 3 * k]] == [v, x]
        inserted.add(v)
    # 2n-4 triangular faces; every edge on exactly two faces; Euler: V-E+F=2
    assert len(faces) == 2 * n - 4
    assert n - len(E) + len(faces) == 2
    count = {}
    for f in faces:
        fl = sorted(f)
        for e in ((fl[0], fl[1]), (fl[0], fl[2]), (fl[1], fl[2])):
            count[frozenset(e)] = count.get(frozenset(e), 0) + 1
            assert frozenset(e) in E
    assert set(count) == E and set(count.values()) == {2}
    # the faces around every vertex form one cycle: a triangulated sphere,
    # hence a (maximal) planar graph
    for v in range(n):
        around = [sorted(set(f) - {v}) for f in faces if v in f]
        link = {}
        for a, b in around:
            link.setdefault(a, []).append(b)
            link.setdefault(b, []).append(a)
        assert all(len(x) == 2 for x in link.values())
        # a 2-regular graph is a union of cycles; connected means one cycle
        start = next(iter(link))
        seen, stack = {start}, [start]
        while stack:
            for w in link[stack.pop()]:
                if w not in seen:
                    seen.add(w)
                    stack.append(w)
        assert len(seen) == len(link) == len(adj[v])
    # bubble tree: n-3 nodes, n-4 edges, parents are earlier bubbles, and the
    # face used by insertion k belongs to (was created by) its parent bubble
    assert parent[0] == -1 and parent.shape[0] == n - 3
    bubble_vertices = [set(order[:4].tolist())]
    for k in range(1, n - 3):
        p = int(parent[k])
        assert 0 <= p < k
        assert set(ins_face[k - 1].tolist()) <= bubble_vertices[p]
        bubble_vertices.append(set(ins_face[k - 1].tolist()) | {int(order[3 + k])})


def test_invariants_random_all_modes():
    for seed, n, dtype in [(1, 5, np.float32), (2, 9, np.float64), (3, 40, np.float32),
                           (4, 97, np.float64), (5, 150, np.float32)]:
        S = W.random_similarity(seed, n, dtype)
        for mode, P in [("corr", 1), ("corr", 3), ("corr", 10), ("heap", 1), ("exact", 1)]:
            r = oracle.tmfg(S, mode, P)
            check_tmfg_invariants(n, r)


def test_invariants_planted_clusters():
    S, _ = W.config_similarity(1)
    for mode, P in [("corr", 1), ("corr", 10), ("heap", 1)]:
        check_tmfg_invariants(S.shape[0], oracle.tmfg(S, mode, P))


def test_n4_and_n5():
    S = W.random_similarity(11, 4, np.float64)
    r = oracle.tmfg(S, "heap")
    rs = [sum(Fraction(float(S[v, u])) for u in range(4) if u != v) for v in range(4)]
    assert r["order"].tolist() == sorted(range(4), key=lambda v: (-rs[v], v))
    assert r["ins_face"].shape == (0, 3) and r["parent"].tolist() == [-1]
    # n=5: the only remaining vertex goes to the face of largest gain
    S = W.random_similarity(12, 5, np.float64)
    r = oracle.tmfg(S, "corr")
    c = r["order"][:4]
    v = int(r["order"][4])
    faces = [(c[0], c[1], c[2]), (c[0], c[1], c[3]), (c[0], c[2], c[3]), (c[1], c[2], c[3])]
    gains = [sum(S[a, v] for a in f) for f in faces]
    assert tuple(sorted(r["ins_face"][0])) == tuple(sorted(faces[int(np.argmax(gains))]))


# ---------------------------------------------------------------- hand traces

@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_hand_traced_cases(dtype):
    for case in golden_cases():
        S = golden_matrix(case, dtype)
        for key, exp in case["expect"].items():
            mode = {"corr1": ("corr", 1), "corr2": ("corr", 2), "heap": ("heap", 1),
                    "exact": ("exact", 1)}[key]
            r = oracle.tmfg(S, *mode)
            assert r["order"].tolist() == exp["order"], (case["name"], key)
            assert r["ins_face"].tolist() == exp["ins_face"], (case["name"], key)
            assert r["parent"].tolist() == exp["parent"], (case["name"], key)
            if "edges" in exp:
                assert r["edges"].tolist() == exp["edges"], (case["name"], key)
            if "ins_gain_64ths" in exp:
                assert (r["ins_gain"] * 64).tolist() == exp["ins_gain_64ths"]
            if "stale_pops" in exp:
                assert r["stats"]["stale_pops"] == exp["stale_pops"], (case["name"], key)


# ---------------------------------------------------------------- special cases

@pytest.mark.parametrize("n", [6, 9, 13, 24])
def test_additive_matrix_equals_exact_greedy(n):
    """S[i,j] = a_i + a_j (dyadic, exact in float): every MaxCorrs is the
    uninserted vertex of largest a, which is also every face's best vertex,
    so corr-tmfg (any P=1) and heap-tmfg must make the exact greedy choices
    of the Massara algorithm, including tie-breaks."""
    for dtype in (np.float32, np.float64):
        S = W.random_similarity(100 + n, n, dtype, kind="dyadic_additive")
        ex = oracle.tmfg(S, "exact")
        for mode in ("corr", "heap"):
            r = oracle.tmfg(S, mode)
            for k in ("order", "edges", "ins_face", "parent"):
                assert np.array_equal(r[k], ex[k]), (n, mode, k)


def test_pointer_equals_bruteforce_argmax():
    """The lazily advanced sorted-row pointer (Section 4.3) must give the same
    MaxCorrs as a fresh argmax over the uninserted vertices (Algorithm 1)."""
    for seed, n, kind in [(21, 30, "uniform"), (22, 45, "quantized"), (23, 25, "constant"),
                          (24, 60, "uniform")]:
        S = W.random_similarity(seed, n, np.float32, kind)
        for mode, P in [("corr", 1), ("corr", 4), ("heap", 1)]:
            a = oracle.tmfg(S, mode, P)
            b = oracle.tmfg(S, mode, P, maxcorrs_bruteforce=True)
            for k in ("order", "edges", "ins_face", "parent"):
                assert np.array_equal(a[k], b[k]), (seed, mode, P, k)


def test_negative_zero_is_zero():
    S = W.random_similarity(31, 40, np.float32, "quantized")
    assert np.any(np.signbit(S) & (S == 0))
    S2 = S.copy()
    S2[S2 == 0] = 0.0
    for mode, P in [("corr", 1), ("corr", 5), ("heap", 1)]:
        a, b = oracle.tmfg(S, mode, P), oracle.tmfg(S2, mode, P)
        for k in ("order", "edges", "ins_face", "parent"):
            assert np.array_equal(a[k], b[k])


def test_corr_prefix_larger_than_remaining():
    S = W.random_similarity(41, 12, np.float64)
    r = oracle.tmfg(S, "corr", 1000)
    check_tmfg_invariants(12, r)


# ---------------------------------------------------------------- sort and sums

def test_rowsort_matches_lexsort():
    for seed, kind in [(51, "uniform"), (52, "quantized"), (53, "constant")]:
        for dtype in (np.float32, np.float64):
            S = W.random_similarity(seed, 37, dtype, kind)
            idx = oracle.rowsort(S)
            n = S.shape[0]
            for v in range(n):
                us = np.array([u for u in range(n) if u != v])
                vals = S[v, us].astype(np.float64) + 0.0  # -0.0 -> +0.0
                ref = us[np.lexsort((us, -vals))]
                assert np.array_equal(idx[v], ref)


def test_quantize_round_half_even():
    ulp = 2.0 ** -40
    assert oracle.quantize(0.5 * ulp) == 0
    assert oracle.quantize(1.5 * ulp) == 2
    assert oracle.quantize(2.5 * ulp) == 2
    assert oracle.quantize(-2.5 * ulp) == -2
    assert oracle.quantize(0.7) == round(Fraction(0.7) * 2 ** 40)


def test_rowsums_exact_and_clique_by_exact_sum():
    S = W.random_similarity(61, 50, np.float32)
    rs = oracle.rowsums(S)
    for v in range(50):
        exact = sum(round(Fraction(float(S[v, u])) * 2 ** 40) for u in range(50) if u != v)
        assert rs[v] == exact
    # clique = top four by the true (rational) row sums when no near-ties
    true = [sum(Fraction(float(S[v, u])) for u in range(50) if u != v) for v in range(50)]
    top = sorted(range(50), key=lambda v: (-true[v], v))[:4]
    gaps = sorted(true, reverse=True)
    assert min(gaps[i] - gaps[i + 1] for i in range(4)) > Fraction(50, 2 ** 40)
    assert oracle.tmfg(S, "heap")["order"][:4].tolist() == top


# ---------------------------------------------------------------- quality (soft)

def test_edge_sum_close_to_exact_greedy():
    """Section 5 (edge sums): heap-tmfg edge sums were within 1% of the
    prefix-1 exact-greedy TMFG.  A soft check on planted-cluster inputs."""
    S, _ = W.config_similarity(1)
    ex = oracle.tmfg(S, "exact")

    def esum(r):
        return float(sum(S[a, b] for a, b in r["edges"]))
    base = esum(ex)
    for mode in ("corr", "heap"):
        assert esum(oracle.tmfg(S, mode)) >= base * (1 - 0.02)
    # a larger prefix makes the graph no better in this case
    assert esum(oracle.tmfg(S, "corr", 10)) <= base * (1 + 1e-9) + 1e-9


def test_insertion_gains_are_face_sums():
    S = W.random_similarity(71, 30, np.float64)
    r = oracle.tmfg(S, "heap")
    for k in range(26):
        v = int(r["order"][4 + k])
        x, y, z = (int(a) for a in r["ins_face"][k])
        assert math.isclose(r["ins_gain"][k], S[x, v] + S[y, v] + S[z, v], rel_tol=0, abs_tol=1e-12)


def test_gain_summation_order_float32():
    """The gain of face {a<b<c} for u is (S[a,u] + S[b,u]) + S[c,u] rounded
    in float32 at each step (the fixed order of the reading R1), not in
    wider precision and not in another association."""
    S = W.random_similarity(81, 120, np.float32)
    r = oracle.tmfg(S, "heap")
    f32 = np.float32
    other_order_differs = 0
    for k in range(116):
        v = int(r["order"][4 + k])
        x, y, z = (int(a) for a in r["ins_face"][k])
        a, b, c = f32(S[x, v]), f32(S[y, v]), f32(S[z, v])
        assert r["ins_gain"][k] == float(f32(f32(a + b) + c))
        other_order_differs += float(f32(a + f32(b + c))) != r["ins_gain"][k]
    assert other_order_differs > 0
