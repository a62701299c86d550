"""Host-side check of the arithmetic the fused merge's per-pair barrier rests on.

After the exchange levels, each group of 2^F consecutive pairs (diagonals
d_k = floor(k n / 2^G), exact splits i_k) owns the region [d_k0, d_k0+2^F): A's slices of
the group first, then B's.  The two-pairs kernel lets pair k store its output
[d_k, d_k+1) once every element there has been staged by its reader; readers count
their slices in at the pairs whose output ranges they overlap, the pair of position x
being the last k with d_k <= x, i.e. floor(((x + 1) 2^G - 1) / n).  This test checks,
on oracle splits of ragged inputs (empty pairs included), that the members' slices tile
each group region exactly, that the formula names the right pair and stays inside the
group, and that every pair's count equals its output length.  No GPU is involved.
"""
import numpy as np
import pytest

import oracle as orc
import workloads as W


def _slices(split, n, G, F, k):
    """Positions of pair k's A and B slices in its group's region, and their lengths."""
    d = lambda q: (q * n) >> G
    k0 = (k >> F) << F
    k1 = k0 + (1 << F)
    dlo, ilo, ihi = d(k0), split[k0], split[k1]
    i0, i1, d0, d1 = split[k], split[k + 1], d(k), d(k + 1)
    pos_a = dlo + (i0 - ilo)
    pos_b = dlo + (ihi - ilo) + ((d0 - i0) - (dlo - ilo))
    return (pos_a, i1 - i0), (pos_b, (d1 - d0) - (i1 - i0))


@pytest.mark.parametrize("la, lb, G, F, dist", [
    (1000, 1000, 6, 3, "uniform"), (5000, 77, 7, 4, "uniform"), (3, 9000, 8, 8, "uniform"),
    (4096, 4096, 9, 5, "dup16"), (12345, 6789, 10, 9, "alternation"),
    (100, 100, 9, 9, "uniform"), (7, 5, 4, 2, "uniform"), (2000, 2000, 5, 1, "disjoint"),
    (2000, 2000, 5, 5, "revdisjoint")])
def test_member_slices_tile_the_group_and_counts_cover_each_output(la, lb, G, F, dist):
    a, b = W.make_pair(dist, np.int32, la, lb, seed=la ^ lb)
    n, P = la + lb, 1 << G
    d = lambda q: (q * n) >> G
    split = [orc.split_bsearch(a, b, d(k)) for k in range(P + 1)]
    cnt = np.zeros(P, dtype=np.int64)
    for g0 in range(0, P, 1 << F):
        covered = np.zeros(d(g0 + (1 << F)) - d(g0), dtype=np.int64)
        for k in range(g0, g0 + (1 << F)):
            for s, ln in _slices(split, n, G, F, k):
                covered[s - d(g0):s - d(g0) + ln] += 1
                x = s
                while x < s + ln:
                    w = (((x + 1) << G) - 1) // n
                    assert d(w) <= x < d(w + 1)
                    assert w >> F == k >> F, "a slice counted outside its group"
                    y = min(d(w + 1), s + ln)
                    cnt[w] += y - x
                    x = y
        assert np.all(covered == 1), "the members' slices do not tile the group region"
    assert np.array_equal(cnt, [d(k + 1) - d(k) for k in range(P)])
