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
* build(): with the separation ws (1 or 2), boxes of one level are
  neighbours when their cells differ by at most ws in every direction;
  U-list of a leaf: non-empty neighbouring leaves; V-list of a box (level
  >= 2): non-empty children of the parent's neighbours (parent included)
  that are not neighbours of the box; lists sorted by box index;
* build_mac(): boxes are well separated when the spheres about their
  centres that hold all of their panels' vertices satisfy
  rho_t + rho_s <= theta |c_t - c_s|; near lists are refined level by
  level from the parent's near list (see its docstring).  This rule bounds
  the ratio that governs the convergence of the translated expansions for
  panels of any size, which the cell-distance rule cannot when panels stick
  out of their boxes.
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


def _panel_vertices(xyz, tri):
    """Vertex coordinates [N, 4, 3] and per-panel vertex count (3 or 4)."""
    tri = np.asarray(tri, np.int64)
    if tri.shape[1] == 3:
        tri = np.hstack([tri, -np.ones((tri.shape[0], 1), np.int64)])
    nv = np.where(tri[:, 3] >= 0, 4, 3)
    v = np.asarray(xyz, float)[np.where(tri >= 0, tri, tri[:, :1])]
    return v, nv


def box_geometry(xyz, tri, sk_perm, levels, lo, side, L):
    """Centre and radius of every box of levels 0..L.

    Centre c_b = lo + (cell + 1/2) h_l per axis (h_l = side / 2^l); radius
    rho_b = max over the box's panels and their vertices of |v - c_b| (a flat
    panel lies in the convex hull of its vertices, so its whole surface is
    within rho_b of c_b).  Squared distances are summed x, y, z in that order."""
    xyz = np.asarray(xyz, float)
    v, nv = _panel_vertices(xyz, tri)
    keys_sorted, perm = sk_perm
    vs = v[perm]
    nvs = nv[perm]
    out = {}
    for lev in range(L + 1):
        h = side / float(1 << lev)
        bk = levels[lev]
        cell = decode(bk)
        ctr = np.stack([lo[a] + (cell[:, a] + 0.5) * h for a in range(3)], axis=1)
        bidx = np.searchsorted(bk, keys_sorted >> np.uint64(3 * (21 - lev)))
        r2 = np.zeros(bk.shape[0])
        for j in range(4):
            dx = vs[:, j, 0] - ctr[bidx, 0]
            dy = vs[:, j, 1] - ctr[bidx, 1]
            dz = vs[:, j, 2] - ctr[bidx, 2]
            d2 = dx * dx + dy * dy + dz * dz
            d2 = np.where(nvs > j, d2, 0.0)
            np.maximum.at(r2, bidx, d2)
        out[lev] = (ctr, np.sqrt(r2), bidx)
    return out


def build_mac(xyz, tri, leaf_target=32, theta=0.5, cap=2.0):
    """Uniform-depth octree with interaction lists from a bounding-sphere
    admissibility test (the FMM of Sec. II-C defers to refs [22], [23]; this
    separation rule is the multipole acceptance criterion used with
    expansions about box centres):

    * root cube, keys, panel order and leaf level L as in build(); the depth
      cap side / 2^L >= cap * r_max applies when cap > 0;
    * box centres and radii as in box_geometry();
    * two boxes t, s of one level are well separated when
      rho_t + rho_s <= theta * |c_t - c_s|, with |c_t - c_s| the square root
      of the squared centre distance summed x, y, z;
    * at level 1 every pair is near; at level l >= 2 the candidates of box t
      are the children of the near boxes of t's parent: the well-separated
      ones form t's V-list, the others its near list; the near lists of the
      leaf level are the U-lists;
    * lists sorted by box index.  V offsets (target - source cell) are not
      bounded by a fixed window.
    Returns the dict of build() plus 'centre', 'radius' per level."""
    k = keys(xyz, tri)
    c, lo, side = root(xyz, tri)
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
    if cap > 0:
        lsize = 2
        for lev in range(2, 21):
            if side / float(1 << lev) >= cap * rmax:
                lsize = lev
        L = min(L, lsize)
    L = max(2, L)
    levels = [np.unique(sk >> np.uint64(3 * (21 - lev))) for lev in range(L + 1)]
    geo = box_geometry(xyz, tri, (sk, perm), levels, lo, side, L)
    leaf_of = geo[L][2]
    near = [list(range(levels[1].shape[0])) for _ in range(levels[1].shape[0])]
    V = {}
    for lev in range(2, L + 1):
        ctr, rad, _ = geo[lev]
        bk = levels[lev]
        par = np.searchsorted(levels[lev - 1], bk >> np.uint64(3))
        first = np.searchsorted(bk >> np.uint64(3), levels[lev - 1], side="left")
        last = np.searchsorted(bk >> np.uint64(3), levels[lev - 1], side="right")
        Vl, nl = [], []
        for t in range(bk.shape[0]):
            vl, nn = [], []
            for sp in near[par[t]]:
                for s in range(first[sp], last[sp]):
                    dx = ctr[t, 0] - ctr[s, 0]
                    dy = ctr[t, 1] - ctr[s, 1]
                    dz = ctr[t, 2] - ctr[s, 2]
                    dist = np.sqrt(dx * dx + dy * dy + dz * dz)
                    if s != t and rad[t] + rad[s] <= theta * dist:
                        vl.append(s)
                    else:
                        nn.append(s)
            Vl.append(sorted(vl))
            nl.append(sorted(nn))
        V[lev] = Vl
        near = nl
    return {"keys": k, "perm": perm, "L": L, "levels": levels, "leaf_of": leaf_of, "U": near, "V": V,
            "centre": {lev: geo[lev][0] for lev in geo}, "radius": {lev: geo[lev][1] for lev in geo}}
