"""Pins for oracle/tree.py: the interaction lists partition all panel pairs.

Every ordered pair of panels (k, l) must be handled exactly once: either
its two leaves are U-list neighbours, or there is exactly one level at
which the ancestor of l is in the V-list of the ancestor of k."""
import numpy as np
import pytest

import meshgen
from oracle import tree


@pytest.mark.parametrize("target,ws", [(4, 1), (16, 1), (4, 2), (16, 2)])
def test_lists_cover_every_pair_once(target, ws):
    m = meshgen.bar(length=4e-3, n_w=3, n_h=3, n_l=20, seed=9)
    t = tree.build(m.xyz, m.tri, leaf_target=target, ws=ws)
    L = t["L"]
    N = m.n_tri
    rank = np.empty(N, np.int64)
    rank[t["perm"]] = np.arange(N)
    sk = t["keys"][t["perm"]]
    # box index of every panel (by Morton rank) at every level
    box = {lev: np.searchsorted(t["levels"][lev], sk >> np.uint64(3 * (21 - lev))) for lev in range(L + 1)}
    count = np.zeros((N, N), np.int64)
    leaf = box[L]
    for a in range(N):
        for b in t["U"][leaf[a]]:
            count[a, leaf == b] += 1
    for lev in range(2, L + 1):
        for bx, lst in enumerate(t["V"][lev]):
            tg = np.flatnonzero(box[lev] == bx)
            for s in lst:
                src = np.flatnonzero(box[lev] == s)
                count[np.ix_(tg, src)] += 1
    assert count.min() == 1 and count.max() == 1
    # U symmetric
    for i, lst in enumerate(t["U"]):
        for j in lst:
            assert i in t["U"][j]


def test_keys_and_order_are_morton():
    m = meshgen.bar(length=4e-3, n_w=3, n_h=3, n_l=20, seed=9)
    k = tree.keys(m.xyz, m.tri)
    q = tree.decode(k)
    assert np.array_equal(tree.morton(q), k)
    c = tree.centroids(m.xyz, m.tri)
    # cells are monotone in the coordinates
    for a in range(3):
        o = np.argsort(c[:, a], kind="stable")
        assert np.all(np.diff(q[o, a]) >= 0)
