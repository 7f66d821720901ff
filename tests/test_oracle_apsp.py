"""Pins for the APSP oracle (Section 2: one Dijkstra per source over the TMFG;
Section 4.3: hub-based approximate APSP) against library routines, closed
forms, an independent Bellman-Ford and the approximation's bounds."""
import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.csgraph import dijkstra

import oracle
from paper_2408_09399_gb300 import workloads as W


def tmfg_case(seed, n, dtype=np.float32, mode="heap"):
    S = W.random_similarity(seed, n, dtype)
    return S, oracle.tmfg(S, mode)["edges"]


def scipy_apsp(S, edges):
    n = S.shape[0]
    a, b = edges[:, 0], edges[:, 1]
    w = np.sqrt(np.maximum(0.0, 2.0 * (1.0 - S[a, b].astype(np.float64))))
    G = sp.coo_matrix((w, (a, b)), shape=(n, n)).tocsr()
    return dijkstra(G, directed=False)


@pytest.mark.parametrize("seed,n", [(1, 12), (2, 60), (3, 200)])
def test_exact_matches_scipy_dijkstra(seed, n):
    S, edges = tmfg_case(seed, n, np.float64)
    D = oracle.apsp_exact(S, edges, prec=64)
    np.testing.assert_allclose(D, scipy_apsp(S, edges), rtol=1e-13, atol=1e-14)


def test_path_and_star_closed_forms():
    n = 9
    # path 0-1-...-8 with S = 1/2 on its edges: every length is 1
    S = np.eye(n)
    edges = np.array([[i, i + 1] for i in range(n - 1)], np.int32)
    for i in range(n - 1):
        S[i, i + 1] = S[i + 1, i] = 0.5
    for prec in (32, 64):
        D = oracle.apsp_exact(S.astype(np.float32), edges, prec)
        assert np.array_equal(D, np.abs(np.arange(n)[:, None] - np.arange(n)[None, :]).astype(float))
    # star around 0 with lengths a_i: S[0,i] = 1 - a_i^2/2 (exact dyadic)
    a = np.array([0.0, 0.25, 0.5, 0.75, 1.0, 1.25, 0.125, 1.5, 0.375])
    S = np.eye(n)
    edges = np.array([[0, i] for i in range(1, n)], np.int32)
    for i in range(1, n):
        S[0, i] = S[i, 0] = 1.0 - a[i] ** 2 / 2.0
    expect = a[:, None] + a[None, :]
    np.fill_diagonal(expect, 0.0)
    expect[0, :] = a
    expect[:, 0] = a
    for prec in (32, 64):
        assert np.array_equal(oracle.apsp_exact(S.astype(np.float32), edges, prec), expect)


def bellman_ford_f32(S, edges):
    """Float32 path-sum fixpoint by plain Bellman-Ford sweeps (a different
    algorithm from Dijkstra, same definition: the minimum over paths of the
    left-to-right float32 sum of the edge lengths)."""
    n = S.shape[0]
    f32 = np.float32
    arcs = []
    for a, b in edges:
        s = f32(S[a, b])
        t = f32(f32(1.0) - s)
        t = f32(f32(2.0) * t)
        l = f32(np.sqrt(max(t, f32(0.0)), dtype=np.float32))
        arcs += [(a, b, l), (b, a, l)]
    src = np.array([x[0] for x in arcs])
    dst = np.array([x[1] for x in arcs])
    ln = np.array([x[2] for x in arcs], np.float32)
    D = np.full((n, n), np.inf, np.float32)
    np.fill_diagonal(D, 0)
    while True:
        cand = (D[:, src] + ln[None, :]).astype(np.float32)
        new = D.copy()
        np.minimum.at(new.T, dst, cand.T)
        if np.array_equal(new, D):
            return D
        D = new


def test_f32_mode_is_the_float_path_fixpoint():
    for seed, n in [(5, 30), (6, 80)]:
        S, edges = tmfg_case(seed, n)
        D32 = oracle.apsp_exact(S, edges, prec=32)
        assert np.array_equal(D32.astype(np.float32), bellman_ford_f32(S, edges))
        D64 = oracle.apsp_exact(S, edges, prec=64)
        np.testing.assert_allclose(D32, D64, rtol=1e-5, atol=1e-7)


def test_sssp_rows_match_full():
    S, edges = tmfg_case(7, 50)
    D = oracle.apsp_exact(S, edges, prec=32)
    src = [0, 7, 49, 13]
    assert np.array_equal(oracle.sssp_rows(S, edges, src, prec=32), D[src])


def test_hubs_are_top_degree():
    S, edges = tmfg_case(8, 100)
    deg = np.bincount(edges.ravel(), minlength=100)
    ref = np.lexsort((np.arange(100), -deg))[:10]
    assert oracle.hubs(100, edges, 10).tolist() == ref.tolist()


@pytest.mark.parametrize("prec", [32, 64])
def test_approx_bounds(prec):
    """Section 4.3: exact distances from the hubs, exact distances inside the
    radius, and otherwise the path through the nearest hub; the triangle
    inequality bounds the estimate by d(s,t) + 2 d_s."""
    S, _ = W.config_similarity(1)
    edges = oracle.tmfg(S, "heap")["edges"]
    n = S.shape[0]
    Dx = oracle.apsp_exact(S, edges, prec=prec)
    Da, info = oracle.apsp_approx(S, edges, 0, 2.0, prec=prec)
    hubs, near, dn = info["hubs"], info["nearest"], info["dnear"]
    assert len(hubs) == int(np.ceil(np.sqrt(n)))
    tol = 1e-5 if prec == 32 else 1e-12
    assert np.array_equal(Da, Da.T)
    assert np.all(Da >= Dx * (1 - tol) - tol)
    assert np.all(Da <= Dx + 2 * dn[:, None] + tol * (1 + Dx))
    for i, h in enumerate(hubs):          # hub rows are exact
        np.testing.assert_allclose(Da[h], Dx[h], rtol=tol, atol=tol)
        assert dn[h] == 0
    # nearest hub: the smallest hub distance, ties to the lower hub rank
    HD = Dx[hubs]
    assert np.all(dn == HD.min(axis=0))
    assert np.all(near == np.argmin(HD, axis=0))
    # inside the radius the estimate is the exact distance
    inside = Dx <= (2.0 * dn[:, None]) * (1 - 1e-6)
    np.testing.assert_allclose(Da[inside], Dx[inside], rtol=tol, atol=tol)
    # and the approximation is not trivial here
    assert np.any(Da > Dx * (1 + 1e-6))


def test_approx_all_hubs_is_exact():
    S, edges = tmfg_case(9, 40, np.float64)
    Dx = oracle.apsp_exact(S, edges, prec=64)
    Da, _ = oracle.apsp_approx(S, edges, 40, 2.0, prec=64)
    np.testing.assert_allclose(Da, np.minimum(Dx, Dx.T), rtol=1e-14, atol=1e-14)


def test_approx_ties_constant_lengths():
    """Constant S: every edge has the same length, so hop counts decide and
    ties between hubs are everywhere; the nearest hub is the lowest rank."""
    S = W.random_similarity(10, 50, np.float32, "constant")
    edges = oracle.tmfg(S, "heap")["edges"]
    for prec in (32, 64):
        Dx = oracle.apsp_exact(S, edges, prec=prec)
        Da, info = oracle.apsp_approx(S, edges, 0, 2.0, prec=prec)
        HD = Dx[info["hubs"]]
        assert np.any((HD == HD.min(axis=0)).sum(axis=0) > 1)
        assert np.all(info["nearest"] == np.argmin(HD, axis=0))
        assert np.all(Da >= Dx - 1e-6)


def test_sampled_oracle_rows_match_full():
    S, edges = tmfg_case(12, 70)
    D = oracle.apsp_exact(S, edges, prec=32)
    src = [3, 0, 69]
    b = oracle.sssp_bounded_rows(S, edges, src, [np.inf, np.inf, np.inf])
    assert np.array_equal(b, D[src])
    b = oracle.sssp_bounded_rows(S, edges, src, [0.5, 1.0, 2.0])
    for i, s in enumerate(src):
        within = D[s] <= [0.5, 1.0, 2.0][i]
        assert np.array_equal(b[i][within], D[s][within])
    assert np.array_equal(oracle.rowsort_rows(S, [5, 0, 69]), oracle.rowsort(S)[[5, 0, 69]])


@pytest.mark.parametrize("seed,n,h,rf,prec", [(13, 90, 0, 2.0, 32), (14, 150, 5, 1.5, 32),
                                             (15, 120, 0, 3.0, 64), (16, 64, 64, 2.0, 32)])
def test_approx_rows_match_full_approx(seed, n, h, rf, prec):
    """The row-sampled approximate APSP (used at sizes where the full n x n
    oracle does not fit) gives exactly the rows of the full one."""
    S, edges = tmfg_case(seed, n)
    D, _ = oracle.apsp_approx(S, edges, h, rf, prec)
    src = np.array([0, n - 1, n // 2, 7, 7], np.int32)
    R = oracle.apsp_approx_rows(S, edges, src, h, rf, prec)
    assert np.array_equal(R, D[src])
