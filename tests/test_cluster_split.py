"""The cluster loop kernel splits corr-tmfg (prefix 1) over C CTAs: face f
belongs to CTA f mod C and row w to CTA w mod C.  Every CTA keeps a replica of
every row's pointer word (ptr, Mc).  At each insertion of v the owner of a row
refreshes it if its Mc is v (or, for v's own row, if its Mc was inserted
earlier) and stores the new word into every replica.  A CTA that evaluates a
face whose vertex's word is still stale in its replica waits for the owner's
store, and refreshes its replica itself if the wait runs out.  The CTAs run
unsynchronised between the cluster barriers, so an owner's store may land
before a read, after it, or between a timed-out wait and the local refresh.

That any such interleaving still gives the oracle's TMFG rests on every word
being valid at all times (Mc is the id at position ptr and every id before ptr
is inserted), and on the local refresh checking the word it reads again before
it scans on from ptr + 1.  These host tests restate the split procedure in
plain Python, deliver the owners' stores at seeded random times, and check it
against the oracle; a local refresh that skips the second check must fail.
"""
import numpy as np
import pytest

import oracle
from paper_2408_09399_gb300 import workloads as W

NONE = 0xFFFF


def split_tmfg(S, C, seed, recheck=True):
    n = S.shape[0]
    mlen = n - 1
    rows = oracle.rowsort(S)
    rs = oracle.rowsums(S)
    rng = np.random.default_rng(seed)
    nl = (2 * n - 4 + C - 1) // C
    ins = set()
    pm = [[(0, int(rows[w][0])) for w in range(n)] for _ in range(C)]
    frec = [[None] * nl for _ in range(C)]
    fv = [[NONE] * nl for _ in range(C)]
    leaf = [[None] * nl for _ in range(C)]
    clique = sorted(range(n), key=lambda v: (-int(rs[v]), v))[:4]
    order, parent = list(clique), [-1]

    def stale(word):
        return word[1] != NONE and word[1] in ins

    def scan_on(word, w):  # first uninserted id after position ptr of row w
        q = word[0] + 1
        while q < mlen:
            e = int(rows[w][q])
            if e not in ins:
                return (q, e)
            q += 1
        return (mlen, NONE)

    def gain(x, c):
        if S.dtype == np.float32:
            return np.float32(np.float32(S[x[0], c] + S[x[1], c]) + S[x[2], c])
        return (S[x[0], c] + S[x[1], c]) + S[x[2], c]

    def cluster_round(face_lists, row_lists):
        # C: the owners' new words, each store to a replica pending
        pending = {}
        for r in range(C):
            for w in row_lists[r]:
                word = scan_on(pm[r][w], w)
                pm[r][w] = word
                for j in range(C):
                    if j != r:
                        pending[(j, w)] = word
        # some stores land before the evaluations
        for key in list(pending):
            if rng.random() < 0.5:
                j, w = key
                pm[j][w] = pending.pop(key)
        # D: every face with the fresh Mc of its vertices
        for r in rng.permutation(C):
            for lf in face_lists[r]:
                x = frec[r][lf][:3]
                cs = []
                for w in x:
                    if stale(pm[r][w]):
                        # the wait ran out; the owner's store may land now
                        if (r, w) in pending and rng.random() < 0.5:
                            pm[r][w] = pending.pop((r, w))
                        word = pm[r][w]
                        if not recheck or stale(word):
                            word = scan_on(word, w)
                        pm[r][w] = max(pm[r][w], word)
                    assert not stale(pm[r][w]), "a stale MaxCorrs reached a face"
                    cs.append(pm[r][w][1])
                bv, bg = -1, None
                for c in cs:
                    if c == NONE:
                        continue
                    g = gain(x, c)
                    if bv < 0 or g > bg or (g == bg and c < bv):
                        bv, bg = c, g
                f = lf * C + r
                leaf[r][lf] = None if bv < 0 else (bg, -bv, -f)
                fv[r][lf] = NONE if bv < 0 else bv
        # the rest land before the cluster barrier
        for (j, w), word in pending.items():
            pm[j][w] = word

    tri = [(0, 1, 2), (0, 1, 3), (0, 2, 3), (1, 2, 3)]
    ins.update(clique)
    face_lists = [[] for _ in range(C)]
    row_lists = [[c for c in clique if c % C == r and stale(pm[r][c])] for r in range(C)]
    for f in range(4):
        frec[f % C][f // C] = tuple(sorted(clique[i] for i in tri[f])) + (0,)
        face_lists[f % C].append(f // C)
    cluster_round(face_lists, row_lists)
    for k in range(n - 4):
        best = max((x for r in range(C) for x in leaf[r] if x is not None), default=None)
        assert best is not None
        v, t = -best[1], -best[2]
        fx, fy, fz, tb = frec[t % C][t // C]
        order.append(v)
        parent.append(tb)
        nf = 4 + 2 * k
        face_lists = [[] for _ in range(C)]
        row_lists = [[] for _ in range(C)]
        for r in range(C):
            if v % C == r and stale(pm[r][v]):
                row_lists[r].append(v)
            row_lists[r] += [w for w in range(r, n, C) if w in ins and pm[r][w][1] == v]
            for f, face in ((t, (v, fx, fy)), (nf, (v, fy, fz)), (nf + 1, (v, fx, fz))):
                if f % C == r:
                    frec[r][f // C] = tuple(sorted(face)) + (k + 1,)
                    face_lists[r].append(f // C)
            cur = (nf - 1 - r) // C + 1 if r < nf else 0
            face_lists[r] += [lf for lf in range(cur)
                              if fv[r][lf] == v and not (t % C == r and lf == t // C)]
        ins.add(v)
        cluster_round(face_lists, row_lists)
    return np.array(order), np.array(parent)


CASES = [(13, "constant", np.float32), (40, "quantized", np.float32), (120, "uniform", np.float32),
         (9, "quantized", np.float64), (200, "quantized", np.float64)]


@pytest.mark.parametrize("n,kind,dtype", CASES)
@pytest.mark.parametrize("C", [2, 8, 16])
def test_split_equals_oracle(n, kind, dtype, C):
    S = W.random_similarity(8800 + n, n, dtype, kind)
    ref = oracle.tmfg(S, "corr", 1)
    for seed in range(3):
        order, parent = split_tmfg(S, C, seed)
        assert np.array_equal(order, ref["order"]), (n, kind, C, seed)
        assert np.array_equal(parent, ref["parent"]), (n, kind, C, seed)


def test_local_refresh_without_recheck_fails():
    """Scanning on from ptr + 1 of a word that the owner's store has just
    made fresh skips that uninserted Mc: the planted mistake must be caught."""
    bad = 0
    for n, kind in [(13, "constant"), (40, "quantized")]:
        S = W.random_similarity(8800 + n, n, np.float32, kind)
        ref = oracle.tmfg(S, "corr", 1)
        for seed in range(3):
            try:
                order, parent = split_tmfg(S, 8, seed, recheck=False)
                bad += not (np.array_equal(order, ref["order"])
                            and np.array_equal(parent, ref["parent"]))
            except AssertionError:
                bad += 1
    assert bad > 0
