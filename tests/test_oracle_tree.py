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


def _coverage(t, N):
    L = t["L"]
    sk = t["keys"][t["perm"]]
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
    return count, box


@pytest.mark.parametrize("target,theta,cap", [(4, 0.5, 0.0), (16, 0.66, 0.0), (8, 0.66, 2.0)])
def test_mac_lists_cover_every_pair_once(target, theta, cap):
    """Bounding-sphere lists: every ordered panel pair exactly once, U symmetric."""
    m = meshgen.bar(length=4e-3, n_w=3, n_h=3, n_l=20, seed=9)
    t = tree.build_mac(m.xyz, m.tri, leaf_target=target, theta=theta, cap=cap)
    count, _ = _coverage(t, m.n_tri)
    assert count.min() == 1 and count.max() == 1
    for i, lst in enumerate(t["U"]):
        for j in lst:
            assert i in t["U"][j]


@pytest.mark.parametrize("theta", [0.5, 0.66])
def test_mac_pairs_obey_the_separation_rule(theta):
    """Radii recomputed by brute force from every panel vertex of each box:
    every V pair satisfies rho_t + rho_s <= theta |c_t - c_s|, and every U pair
    of distinct leaves violates it (near only where it must be)."""
    m = meshgen.coils(outer=1.6e-3, turns=2, step=0.1e-3)
    t = tree.build_mac(m.xyz, m.tri, leaf_target=8, theta=theta, cap=0.0)
    xyz = np.asarray(m.xyz)
    tri = np.asarray(m.tri)
    _, lo, side = tree.root(m.xyz, m.tri)
    sk = t["keys"][t["perm"]]
    nchk = 0
    for lev in range(2, t["L"] + 1):
        h = side / 2.0 ** lev
        bk = t["levels"][lev]
        cell = tree.decode(bk)
        ctr = lo + (cell + 0.5) * h
        bidx = np.searchsorted(bk, sk >> np.uint64(3 * (21 - lev)))
        rad = np.zeros(bk.shape[0])
        for r, p in enumerate(t["perm"]):
            for vtx in tri[p]:
                rad[bidx[r]] = max(rad[bidx[r]], float(np.linalg.norm(xyz[vtx] - ctr[bidx[r]])))
        assert np.allclose(rad, t["radius"][lev], rtol=1e-14, atol=0)
        for b, lst in enumerate(t["V"][lev]):
            for s in lst:
                assert rad[b] + rad[s] <= theta * np.linalg.norm(ctr[b] - ctr[s]) * (1 + 1e-12)
                nchk += 1
        if lev == t["L"]:
            for b, lst in enumerate(t["U"]):
                for s in lst:
                    if s != b:
                        assert rad[b] + rad[s] > theta * np.linalg.norm(ctr[b] - ctr[s]) * (1 - 1e-12)
    assert nchk > 100
