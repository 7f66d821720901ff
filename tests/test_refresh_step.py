"""The lazy MaxCorrs pointer (Algorithm 1, the sorted-row pointer of each
vertex) is refreshed on the GPU by a group of PL lanes that reads the next
PL * 8 sorted ids from ptr + 1 rounded down to a multiple of 8: lane l holds
the ids at positions base + 8 l ... base + 8 l + 7, turns them into an 8-bit
mask (bit t: position base + 8 l + t is at or after ptr + 1 and is either the
row's end or an uninserted id), and the group takes the lowest lane with a
set bit and that lane's lowest bit.  A step that finds nothing moves base on
by PL * 8.

These host tests restate that step in plain Python and check that it lands
where the plain definition does: the first position after ptr whose id is
not inserted, or the end of the row (position n - 1, or the end marker of a
compacted row).  A restatement that let the highest lane win must fail.
"""
import numpy as np
import pytest

import oracle
from paper_2408_09399_gb300 import workloads as W

NONE = 0xFFFF


def first_free(row, inserted, ptr, mlen):
    """The plain definition: first q > ptr with an uninserted id, else the end."""
    for q in range(ptr + 1, mlen):
        e = int(row[q])
        if e == NONE:
            return q, NONE
        if not inserted[e]:
            return q, e
    return mlen, NONE


def group_refresh(row, inserted, ptr, mlen, n, PL, lowest=True):
    """The lanes' masks, one ballot, one shuffle per step."""
    ldi = len(row)
    p = ptr + 1
    while p < mlen:
        base = p & ~7
        masks = []
        for lane in range(PL):
            q0 = base + 8 * lane
            m = 0
            for t in range(8):
                q = q0 + t
                e = int(row[q]) if q < ldi else NONE
                stop = q >= mlen or e >= n
                if q >= p and (stop or not inserted[e]):
                    m |= 1 << t
            masks.append(m)
        hits = [lane for lane in range(PL) if masks[lane]]
        if hits:
            lane = min(hits) if lowest else max(hits)
            m = masks[lane]
            t = (m & -m).bit_length() - 1
            q = base + 8 * lane + t
            e = int(row[q]) if q < ldi else NONE
            if q >= mlen or e >= n:
                return min(q, mlen), NONE
            return q, e
        p = base + PL * 8
    return mlen, NONE


def rows_with_padding(S):
    """Sorted rows padded with end markers past a multiple of 8 (the device
    layout keeps every 16-byte load of a row inside the row)."""
    rows = oracle.rowsort(S)
    n = S.shape[0]
    ldi = (n - 1 + 7) // 8 * 8 + 8
    out = np.full((n, ldi), NONE, np.int64)
    out[:, :n - 1] = rows
    return out


@pytest.mark.parametrize("PL", [8, 16, 32])
@pytest.mark.parametrize("n", [9, 40, 300])
def test_group_refresh_equals_definition(PL, n):
    S = W.random_similarity(4100 + n, n, np.float32, "quantized")
    rows = rows_with_padding(S)
    rng = np.random.default_rng(n * 7 + PL)
    mlen = n - 1
    for trial in range(60):
        inserted = rng.random(n) < rng.choice([0.1, 0.5, 0.9, 0.99])
        w = int(rng.integers(n))
        row = rows[w].copy()
        if trial % 3 == 0:
            # a compacted row: inserted ids dropped, then the end marker
            keep = [int(e) for e in row[:mlen] if not inserted[e] or rng.random() < 0.3]
            row[:] = NONE
            row[:len(keep)] = keep
        ptr = int(rng.integers(-1, mlen))
        got = group_refresh(row, inserted, ptr, mlen, n, PL)
        assert got == first_free(row, inserted, ptr, mlen), (n, PL, trial)


def test_highest_lane_restatement_fails():
    """The planted mistake (the highest lane with a hit wins) must be caught."""
    n = 300
    S = W.random_similarity(4400, n, np.float32, "uniform")
    rows = rows_with_padding(S)
    rng = np.random.default_rng(3)
    bad = 0
    for trial in range(40):
        inserted = rng.random(n) < 0.2
        w = int(rng.integers(n))
        ptr = int(rng.integers(-1, 100))
        if group_refresh(rows[w], inserted, ptr, n - 1, n, 32, lowest=False) != \
                first_free(rows[w], inserted, ptr, n - 1):
            bad += 1
    assert bad > 0
