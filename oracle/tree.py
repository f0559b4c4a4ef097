"""Reference octree and interaction lists (oracle, test infrastructure only).

The paper applies the FMM to panel centroids as particles (Sec. II-C) and
defers the tree to refs [22], [23]; the definitions below are the ones the
GPU library documents, written independently here so that its lists can be
compared bit for bit:

* root cube: lo = per-axis minimum of the centroids (c = (v0 + v1 + v2) / 3,
  (((v0 + v1) + v2) + v3) / 4 for a rectangular panel),
  side = largest per-axis extent * (1 + 2^-20);
* cell q = floor((c - lo) / side * 2^21), clipped to [0, 2^21 - 1]; the
  Morton key puts bit b of x, y, z at bits 3b, 3b + 1, 3b + 2;
* panels sorted by (key, index);
* leaf level L = smallest level >= 2 whose mean occupancy of non-empty
  boxes is <= leaf_target (else 20), capped at the deepest level whose box
  side is >= 2 r_max (r_max = largest centroid-to-vertex distance), and at
  least 2;
* with the separation ws (1 or 2), boxes of one level are neighbours when
  their cells differ by at most ws in every direction; U-list of a leaf:
  non-empty neighbouring leaves; V-list of a box (level >= 2): non-empty
  children of the parent's neighbours (parent included) that are not
  neighbours of the box; lists sorted by box index.
"""
import numpy as np


def _vertices(xyz, tri):
    """[N, 4, 3] vertices (the 4th repeats v0 for a triangle) and the quad mask."""
    tri = np.asarray(tri, np.int64)
    if tri.shape[1] == 3:
        tri = np.hstack([tri, tri[:, :1]])
        quad = np.zeros(tri.shape[0], bool)
    else:
        quad = tri[:, 3] >= 0
        tri = np.where(tri >= 0, tri, tri[:, :1])
    return np.asarray(xyz, float)[tri], quad


def centroids(xyz, tri):
    """Vertex mean of each panel: (v0 + v1 + v2) / 3, or (((v0 + v1) + v2) + v3) / 4
    for a rectangle (its centroid, rectangles being parallelograms)."""
    v, quad = _vertices(xyz, tri)
    c3 = (v[:, 0] + v[:, 1] + v[:, 2]) / 3.0
    c4 = (((v[:, 0] + v[:, 1]) + v[:, 2]) + v[:, 3]) / 4.0
    return np.where(quad[:, None], c4, c3)


def morton(q):
    """q: [N, 3] integer cells -> uint64 keys."""
    key = np.zeros(q.shape[0], np.uint64)
    for b in range(21):
        for a in range(3):
            bit = (q[:, a].astype(np.uint64) >> np.uint64(b)) & np.uint64(1)
            key |= bit << np.uint64(3 * b + a)
    return key


def decode(key):
    key = np.asarray(key, np.uint64)
    out = np.zeros((key.shape[0], 3), np.int64)
    for b in range(21):
        for a in range(3):
            out[:, a] |= ((key >> np.uint64(3 * b + a)) & np.uint64(1)).astype(np.int64) << b
    return out


def root(xyz, tri):
    c = centroids(xyz, tri)
    lo = c.min(axis=0)
    ext = np.max(c.max(axis=0) - lo)
    return c, lo, ext * (1.0 + 2.0 ** -20)


def keys(xyz, tri):
    c, lo, side = root(xyz, tri)
    q = np.floor((c - lo) / side * 2097152.0)
    q = np.clip(q, 0, 2097151).astype(np.int64)
    return morton(q)


def build(xyz, tri, leaf_target=32, ws=2):
    k = keys(xyz, tri)
    c, _, side = root(xyz, tri)
    v, _ = _vertices(xyz, tri)
    rmax = np.max(np.sqrt(np.sum((v - c[:, None, :]) ** 2, axis=2)))
    N = k.shape[0]
    perm = np.lexsort((np.arange(N), k))
    sk = k[perm]
    L = 20
    for lev in range(2, 21):
        sh = np.uint64(3 * (21 - lev))
        cnt = np.unique(sk >> sh).shape[0]
        if N / cnt <= leaf_target:
            L = lev
            break
    lsize = 2
    for lev in range(2, 21):
        if side / float(1 << lev) >= 2.0 * rmax:
            lsize = lev
    L = max(2, min(L, lsize))
    levels = []
    for lev in range(L + 1):
        sh = np.uint64(3 * (21 - lev))
        levels.append(np.unique(sk >> sh))
    leaf_keys = levels[L]
    leaf_of = np.searchsorted(leaf_keys, sk >> np.uint64(3 * (21 - L)))

    def lookup(lev, kk):
        arr = levels[lev]
        i = np.searchsorted(arr, kk)
        return i if i < arr.shape[0] and arr[i] == kk else -1

    U = []
    lc = decode(leaf_keys)
    for i in range(leaf_keys.shape[0]):
        lst = []
        for d in np.ndindex(2 * ws + 1, 2 * ws + 1, 2 * ws + 1):
            x = lc[i] + np.array(d) - ws
            if np.any(x < 0) or np.any(x >= (1 << L)):
                continue
            j = lookup(L, morton(x[None])[0])
            if j >= 0:
                lst.append(j)
        U.append(sorted(lst))
    V = {}
    for lev in range(2, L + 1):
        bc = decode(levels[lev])
        Vl = []
        for i in range(levels[lev].shape[0]):
            lst = []
            par = bc[i] >> 1
            for d in np.ndindex(2 * ws + 1, 2 * ws + 1, 2 * ws + 1):
                pn = par + np.array(d) - ws
                if np.any(pn < 0) or np.any(pn >= (1 << (lev - 1))):
                    continue
                if lookup(lev - 1, morton(pn[None])[0]) < 0:
                    continue
                for o in range(8):
                    ch = pn * 2 + np.array([o & 1, (o >> 1) & 1, (o >> 2) & 1])
                    j = lookup(lev, morton(ch[None])[0])
                    if j >= 0 and np.max(np.abs(ch - bc[i])) > ws:
                        lst.append(j)
            Vl.append(sorted(lst))
        V[lev] = Vl
    return {"keys": k, "perm": perm, "L": L, "levels": levels, "leaf_of": leaf_of, "U": U, "V": V}
