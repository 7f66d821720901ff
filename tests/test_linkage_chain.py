"""The device runs levels 2 and 3 of DBHT's complete linkage by the
nearest-neighbour chain, then sorts the chain's merges by key and replays
them.  That this reproduces the oracle's sequential smallest-key linkage row
for row (ties included) rests on an argument: complete linkage is reducible
and the keys (distance, then the smaller and the larger representative)
order all pairs strictly.  These host tests check the argument itself: a
plain restatement of the chain procedure, on tie-heavy and continuous
random inputs, against the oracle's sequential linkage."""
import numpy as np
import pytest

import oracle


def nn_chain_linkage(D):
    n = D.shape[0]
    dm = D.astype(np.float64).copy()
    alive = np.ones(n, bool)
    rep = list(range(n))

    def key(i, j):
        return (dm[i, j], min(rep[i], rep[j]), max(rep[i], rep[j]))

    chain, merges = [0], []
    while len(merges) < n - 1:
        x = chain[-1]
        y = min((j for j in range(n) if alive[j] and j != x), key=lambda j: key(x, j))
        if len(chain) >= 2 and chain[-2] == y:
            a, b = min(x, y), max(x, y)
            merges.append((key(a, b), a, b))
            for k in range(n):
                if alive[k] and k != a and k != b:
                    dm[a, k] = dm[k, a] = max(dm[a, k], dm[b, k])
            rep[a] = min(rep[a], rep[b])
            alive[b] = False
            chain = chain[:-2]
            if not chain:
                chain = [int(np.flatnonzero(alive)[0])]
        else:
            assert y not in chain, "a chain that revisits an item: not reducible"
            chain.append(y)
    merges.sort()
    keys = [m[0] for m in merges]
    assert all(k1 < k2 for k1, k2 in zip(keys, keys[1:])), "merge keys must increase strictly"
    ids, sz, Z = list(range(n)), [1] * n, []
    for r, (k, a, b) in enumerate(merges):
        Z.append((min(ids[a], ids[b]), max(ids[a], ids[b]), k[0], sz[a] + sz[b]))
        ids[a] = n + r
        sz[a] += sz[b]
    return np.array(Z, np.float64)


def sym(rng, n, levels):
    A = rng.integers(0, levels, (n, n)).astype(np.float64) if levels else rng.random((n, n))
    A = np.triu(A, 1)
    return A + A.T


@pytest.mark.parametrize("levels", [2, 3, 5, 0])
@pytest.mark.parametrize("n", [2, 3, 7, 20, 45])
def test_chain_matches_sequential_linkage(n, levels):
    rng = np.random.default_rng(1000 * n + levels)
    for _ in range(6):
        D = sym(rng, n, levels)
        assert np.array_equal(nn_chain_linkage(D), oracle.complete_linkage(D))


def test_chain_matches_on_path_sums():
    """Distances shaped like DBHT's: shortest-path sums on a planted graph."""
    rng = np.random.default_rng(7)
    n = 40
    W = np.round(rng.random((n, n)) * 4) / 4 + 0.25
    W = np.triu(W, 1)
    W = W + W.T
    D = W.copy()
    for k in range(n):  # Floyd-Warshall
        D = np.minimum(D, D[:, [k]] + D[[k], :])
    np.fill_diagonal(D, 0.0)
    assert np.array_equal(nn_chain_linkage(D), oracle.complete_linkage(D))
