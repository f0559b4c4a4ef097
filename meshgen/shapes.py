"""Seeded generators for closed, consistently oriented panel meshes.

Every surface is a closed 2-manifold (each edge in exactly two panels) with
outward-facing panels.  By default the panels are triangles (`tri` is
[n, 3]); with rect=True every lattice quad that is a parallelogram is kept as
one rectangular panel and only the others are split, which gives the hybrid
triangle/rectangle meshes of Sec. II-A (`tri` is then [n, 4], triangles padded
with -1).  Terminal patches are sets of panels tagged with a terminal id; a
port joins a source terminal to a sink terminal.  All lengths are metres,
conductivities S/m, frequencies Hz.

Shapes follow the workloads of the paper's Sec. III (a straight conductor,
two planar square coils); the sizes are the synthetic stand-ins stated in the
design notes, since the paper's own meshes are not published.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class Mesh:
    xyz: np.ndarray          # float64 [n_vert, 3], metres
    tri: np.ndarray          # int32 [n, 3] triangles or [n, 4] panels (rectangles; triangles
                             # padded with -1), outward (counter-clockwise seen from outside)
    cond: np.ndarray         # int32 [n_tri], conductor id
    term: np.ndarray         # int32 [n_tri], terminal id or -1
    ports: list              # list of (source_terminal, sink_terminal)
    sigma: np.ndarray        # float64 [n_cond], S/m
    thickness: np.ndarray    # float64 [n_cond], ESI thickness (metres)
    freqs: np.ndarray        # float64 [n_freq], Hz
    name: str = ""

    @property
    def n_tri(self):
        return int(self.tri.shape[0])

    def port_panels(self, p):
        """(source panel ids, sink panel ids) of port p, int32."""
        s, k = self.ports[p]
        return (np.flatnonzero(self.term == s).astype(np.int32),
                np.flatnonzero(self.term == k).astype(np.int32))

    def translated(self, d):
        m = dataclasses.replace(self)
        m.xyz = self.xyz + np.asarray(d, float)
        return m


class _Builder:
    """Vertex de-duplication by integer key, panel list with tags."""

    def __init__(self, rect=False):
        self.key2id = {}
        self.pts = []
        self.tris = []
        self.tags = []
        self.rect = rect

    def panels(self):
        """[n, 3] triangles, or [n, 4] with -1 padding when rectangles are kept."""
        if not self.rect:
            return np.array(self.tris, np.int32)
        return np.array([t if len(t) == 4 else tuple(t) + (-1,) for t in self.tris], np.int32)

    def _parallelogram(self, a, b, c, d):
        pa, pb, pc, pd = (self.pts[i] for i in (a, b, c, d))
        scale = max(np.linalg.norm(pc - pa), np.linalg.norm(pd - pb))
        return np.linalg.norm(pa + pc - pb - pd) <= 1e-9 * scale

    def vid(self, key, pos):
        i = self.key2id.get(key)
        if i is None:
            i = len(self.pts)
            self.key2id[key] = i
            self.pts.append(np.asarray(pos, float))
        return i

    def quad(self, a, b, c, d, tag, flip_diag=False):
        # a,b,c,d counter-clockwise seen from outside
        if self.rect and self._parallelogram(a, b, c, d):
            self.tris.append((a, b, c, d))
            self.tags.append(tag)
            return
        if flip_diag:
            self.tris += [(a, b, d), (b, c, d)]
        else:
            self.tris += [(a, b, c), (a, c, d)]
        self.tags += [tag, tag]


def _box_surface(bld, size, n, jitter, rng, terminal_faces, cond_tag):
    """Closed box [0,sx]x[0,sy]x[0,sz] meshed on an n=(nx,ny,nz) lattice.

    terminal_faces maps a face name ('z0','z1',...) to a terminal id.
    Interior face vertices are jittered in-plane by +-jitter of the local
    spacing; vertices on box edges stay on the edges.
    """
    sx, sy, sz = size
    nx, ny, nz = n
    h = (sx / nx, sy / ny, sz / nz)
    jit = {}

    def pos(i, j, k):
        p = np.array([i * h[0], j * h[1], k * h[2]])
        key = (i, j, k)
        on = [i in (0, nx), j in (0, ny), k in (0, nz)]
        if jitter > 0 and sum(on) == 1:
            if key not in jit:
                d = rng.uniform(-jitter, jitter, 3) * np.array(h)
                d[on.index(True)] = 0.0
                jit[key] = d
            p = p + jit[key]
        return p

    def v(i, j, k):
        return bld.vid((cond_tag, i, j, k), pos(i, j, k))

    faces = {
        # name: (fixed axis, value index, axis u, axis v, outward sign)
        'x0': (0, 0, 2, 1), 'x1': (0, nx, 1, 2),
        'y0': (1, 0, 0, 2), 'y1': (1, ny, 2, 0),
        'z0': (2, 0, 1, 0), 'z1': (2, nz, 0, 1),
    }
    for name, (ax, val, au, av) in faces.items():
        nu = n[au]
        nv = n[av]
        tag = terminal_faces.get(name, -1)
        for a in range(nu):
            for b in range(nv):
                def idx(da, db):
                    ijk = [0, 0, 0]
                    ijk[ax] = val
                    ijk[au] = a + da
                    ijk[av] = b + db
                    return v(*ijk)
                # (u,v) ordered so that u x v points outward
                bld.quad(idx(0, 0), idx(1, 0), idx(1, 1), idx(0, 1), tag,
                         flip_diag=((a + b) % 2 == 1))


def bar(length=10e-3, width=1e-3, height=1e-3, n_w=5, n_h=5, n_l=50,
        jitter=0.05, seed=1, sigma=5.8e7, thickness=None,
        freqs=(1e3, 1e5, 1e7, 1e9), offset=(0.0, 0.0, 0.0), rect=False) -> Mesh:
    """Straight rectangular bar along z with the two end faces as terminals.

    Terminal 0 (z = length) is the source, terminal 1 (z = 0) the sink.
    The ESI thickness defaults to 2*(cross-section area)/(perimeter), which
    makes the surface model's DC resistance equal rho*L/A.  With rect=True
    (and jitter=0) every face is meshed with rectangles.
    """
    rng = np.random.default_rng(seed)
    bld = _Builder(rect)
    _box_surface(bld, (width, height, length), (n_w, n_h, n_l), jitter, rng,
                 {'z1': 0, 'z0': 1}, 0)
    if thickness is None:
        thickness = 2 * width * height / (2 * (width + height))
    xyz = np.array(bld.pts) + np.asarray(offset, float)
    return Mesh(xyz=xyz, tri=bld.panels(),
                cond=np.zeros(len(bld.tris), np.int32),
                term=np.array(bld.tags, np.int32), ports=[(0, 1)],
                sigma=np.array([sigma]), thickness=np.array([thickness]),
                freqs=np.asarray(freqs, float), name="bar")


def _merge(meshes, name):
    xyz = []
    tri = []
    cond = []
    term = []
    ports = []
    sig = []
    thk = []
    nv = 0
    nt = 0
    nc = 0
    width = max(m.tri.shape[1] for m in meshes)
    for m in meshes:
        xyz.append(m.xyz)
        t = np.full((m.tri.shape[0], width), -1, np.int64)
        t[:, :m.tri.shape[1]] = m.tri
        tri.append(np.where(t >= 0, t + nv, -1))
        cond.append(m.cond + nc)
        tt = m.term.copy()
        tt[tt >= 0] += nt
        term.append(tt)
        ports += [(s + nt, k + nt) for s, k in m.ports]
        sig.append(m.sigma)
        thk.append(m.thickness)
        nv += m.xyz.shape[0]
        nt += int(m.term.max()) + 1
        nc += int(m.cond.max()) + 1
    return Mesh(xyz=np.vstack(xyz), tri=np.vstack(tri).astype(np.int32),
                cond=np.concatenate(cond).astype(np.int32),
                term=np.concatenate(term).astype(np.int32), ports=ports,
                sigma=np.concatenate(sig), thickness=np.concatenate(thk),
                freqs=meshes[0].freqs, name=name)


def two_bars(length=2e-3, width=0.05e-3, gap=0.5e-3, n_w=2, n_l=40, seed=7,
             freqs=(1e9,)) -> Mesh:
    """Two parallel thin square bars along z, centre distance `gap`, one port each."""
    a = bar(length, width, width, n_w, n_w, n_l, jitter=0.0, seed=seed, freqs=freqs)
    b = bar(length, width, width, n_w, n_w, n_l, jitter=0.0, seed=seed + 1, freqs=freqs,
            offset=(gap, 0.0, 0.0))
    return _merge([a, b], "two_bars")


def _spiral_centerline(outer, w, s, turns):
    """Corner points of a rectilinear square spiral, outer end first."""
    h = (outer - w) / 2
    p = w + s
    pts = [np.array([-h, -h])]
    dirs = [np.array([1.0, 0]), np.array([0, 1.0]), np.array([-1.0, 0]), np.array([0, -1.0])]
    lengths = [2 * h, 2 * h, 2 * h]
    k = 1
    while len(lengths) < 4 * turns:
        lengths += [2 * h - k * p, 2 * h - k * p]
        k += 1
    lengths = lengths[:4 * turns]
    for i, L in enumerate(lengths):
        pts.append(pts[-1] + dirs[i % 4] * L)
    return pts


def _swept_trace(bld, corners, z0, w, t, n_w, n_t, step, tag_base, cond_tag, term_ids):
    """Closed surface of a rectangular trace swept along a polyline with mitred corners."""
    corners = [np.asarray(c, float) for c in corners]
    segs = len(corners) - 1
    tang = [(corners[i + 1] - corners[i]) / np.linalg.norm(corners[i + 1] - corners[i]) for i in range(segs)]
    left = [np.array([-d[1], d[0]]) for d in tang]
    stations = []   # (centre xy, lateral vector)
    for i in range(segs):
        L = np.linalg.norm(corners[i + 1] - corners[i])
        ns = max(1, int(math.ceil(L / step)))
        for k in range(ns):
            if k == 0:
                if i == 0:
                    lat = left[0]
                else:
                    lat = (left[i - 1] + left[i]) / (1.0 + float(left[i - 1] @ left[i]))
            else:
                lat = left[i]
            stations.append((corners[i] + (corners[i + 1] - corners[i]) * (k / ns), lat))
    stations.append((corners[-1], left[-1]))
    # ring (lateral s, vertical zz) counter-clockwise seen along the tangent
    ring = []
    for a in range(n_w):
        ring.append((-w / 2 + w * a / n_w, -t / 2))
    for a in range(n_t):
        ring.append((w / 2, -t / 2 + t * a / n_t))
    for a in range(n_w):
        ring.append((w / 2 - w * a / n_w, t / 2))
    for a in range(n_t):
        ring.append((-w / 2, t / 2 - t * a / n_t))
    R = len(ring)

    def rp(si, j):
        c, lat = stations[si]
        s_, zz = ring[j]
        return np.array([c[0] + s_ * lat[0], c[1] + s_ * lat[1], z0 + zz])

    ids = [[bld.vid((cond_tag, 'r', si, j), rp(si, j)) for j in range(R)] for si in range(len(stations))]
    for si in range(len(stations) - 1):
        for j in range(R):
            a = ids[si][j]
            b = ids[si][(j + 1) % R]
            c = ids[si + 1][(j + 1) % R]
            d = ids[si + 1][j]
            # ring runs clockwise seen from outside for increasing j with
            # station index increasing: (a, d, c, b) is outward
            bld.quad(a, d, c, b, -1)
    # end caps: grid in (s, zz); boundary nodes are ring nodes
    for end, si in ((0, 0), (1, len(stations) - 1)):
        tag = term_ids[end]
        grid = {}
        for a in range(n_w + 1):
            for b in range(n_t + 1):
                s_ = -w / 2 + w * a / n_w
                zz = -t / 2 + t * b / n_t
                on_ring = None
                for j, (rs, rz) in enumerate(ring):
                    if abs(rs - s_) < 1e-15 and abs(rz - zz) < 1e-15:
                        on_ring = j
                        break
                if on_ring is not None:
                    grid[a, b] = ids[si][on_ring]
                else:
                    c, lat = stations[si]
                    grid[a, b] = bld.vid((cond_tag, 'cap', end, a, b),
                                         np.array([c[0] + s_ * lat[0], c[1] + s_ * lat[1], z0 + zz]))
        for a in range(n_w):
            for b in range(n_t):
                q = (grid[a, b], grid[a + 1, b], grid[a + 1, b + 1], grid[a, b + 1])
                # lateral x vertical = -tangent for a left-handed frame; the start
                # cap faces -tangent, the end cap +tangent
                if end == 0:
                    bld.quad(q[0], q[1], q[2], q[3], tag)
                else:
                    bld.quad(q[0], q[3], q[2], q[1], tag)


def coils(outer=5e-3, w=0.2e-3, t=35e-6, s=0.2e-3, turns=4, gap=0.5e-3, n_w=3, n_t=1,
          step=0.075e-3, sigma=5.8e7, n_freq=32, fmin=100.0, fmax=1e10, rect=False,
          n_coils=2) -> Mesh:
    """Two parallel square planar spiral coils stacked along z (edge gap `gap`).

    Each coil is one conductor with one port: source on the outer end cap,
    sink on the inner end cap (the external port branch closes the loop).
    The ESI thickness of each trace is its physical thickness t.  With
    rect=True the straight runs are meshed with rectangles and the mitred
    corner panels (trapezoids) with triangles; n_coils=1 keeps the lower coil.
    """
    bld = _Builder(rect)
    corners = _spiral_centerline(outer, w, s, turns)
    _swept_trace(bld, corners, 0.0, w, t, n_w, n_t, step, 0, 0, (0, 1))
    n0 = len(bld.tris)
    if n_coils == 2:
        _swept_trace(bld, corners, t + gap, w, t, n_w, n_t, step, 0, 1, (2, 3))
    # the sweep above emits inward-facing panels; reverse them to outward
    tri = bld.panels()
    if tri.shape[1] == 3:
        tri = tri[:, [0, 2, 1]]
    else:
        quad = tri[:, 3] >= 0
        tri = np.where(quad[:, None], tri[:, [0, 3, 2, 1]], tri[:, [0, 2, 1, 3]]).astype(np.int32)
    cond = np.zeros(len(tri), np.int32)
    cond[n0:] = 1
    term = np.array(bld.tags, np.int32)
    ports = [(0, 1), (2, 3)][:n_coils]
    return Mesh(xyz=np.array(bld.pts), tri=tri, cond=cond, term=term,
                ports=ports, sigma=np.array([sigma, sigma][:n_coils]),
                thickness=np.array([t, t][:n_coils]),
                freqs=np.geomspace(fmin, fmax, n_freq), name="coils")


def panel_edges(tri):
    """Directed edges (a, b) of every panel in vertex order, [n_edges, 2]."""
    tri = np.asarray(tri)
    out = []
    for row in tri:
        vs = [int(x) for x in row if x >= 0]
        out += [(vs[k], vs[(k + 1) % len(vs)]) for k in range(len(vs))]
    return np.array(out, np.int64)


def crop_check(m: Mesh):
    """Return (closed, oriented): every edge in exactly two panels, used once each way."""
    e = panel_edges(m.tri)
    und = np.sort(e, axis=1)
    _, cnt = np.unique(und, axis=0, return_counts=True)
    closed = bool(np.all(cnt == 2))
    _, dcnt = np.unique(e, axis=0, return_counts=True)
    oriented = bool(np.all(dcnt == 1))
    return closed, oriented


# ---------------------------------------------------------------- package (BGA-like)
def _hole_centres(rng, size, n, r, gap, margin):
    """n seeded hole centres in [margin, size - margin]^2, pairwise >= 2r + gap apart."""
    out = []
    tries = 0
    while len(out) < n:
        tries += 1
        if tries > 200000:
            raise ValueError("cannot place %d holes of radius %g in %g" % (n, r, size))
        p = rng.uniform(margin, size - margin, 2)
        if all((p[0] - q[0]) ** 2 + (p[1] - q[1]) ** 2 >= (2 * r + gap) ** 2 for q in out):
            out.append(p)
    return np.array(out).reshape(-1, 2)


def _perforated_face(size, holes, r, h, rng, jitter=0.2):
    """Conforming triangulation of the square [0, size]^2 minus circular holes.

    Boundary points: the square's edges at spacing ~h and each circle at
    n_seg = max(8, ceil(2 pi r / h)) points; interior points: a jittered grid
    at spacing h kept 0.6 h away from every boundary.  The Delaunay
    triangulation of all points (scipy.spatial.Delaunay) holds every boundary
    segment as an edge when no interior point is near it; the triangles whose
    centroid lies inside a hole are removed.  Returns points [n, 2], triangles
    [m, 3] (counter-clockwise), the square boundary loop and one point loop per
    hole (counter-clockwise around the hole)."""
    from scipy.spatial import Delaunay
    ne = max(2, int(math.ceil(size / h)))
    t = np.linspace(0.0, size, ne + 1)
    sq = ([(x, 0.0) for x in t[:-1]] + [(size, y) for y in t[:-1]] +
          [(x, size) for x in t[::-1][:-1]] + [(0.0, y) for y in t[::-1][:-1]])
    pts = list(sq)
    n_sq = len(sq)
    nseg = max(8, int(math.ceil(2 * math.pi * r / h)))
    hole_loops = []
    for (cx, cy) in holes:
        i0 = len(pts)
        for k in range(nseg):
            a = 2 * math.pi * k / nseg
            pts.append((cx + r * math.cos(a), cy + r * math.sin(a)))
        hole_loops.append(list(range(i0, i0 + nseg)))
    g = np.arange(h / 2, size, h)
    gx, gy = np.meshgrid(g, g, indexing="ij")
    cand = np.stack([gx.ravel(), gy.ravel()], 1) + rng.uniform(-jitter, jitter, (gx.size, 2)) * h
    keep = np.all((cand > 0.6 * h) & (cand < size - 0.6 * h), axis=1)
    for (cx, cy) in holes:
        keep &= (cand[:, 0] - cx) ** 2 + (cand[:, 1] - cy) ** 2 > (r + 0.6 * h) ** 2
    pts = np.vstack([np.array(pts), cand[keep]])
    tri = Delaunay(pts).simplices.astype(np.int64)
    cen = pts[tri].mean(axis=1)
    inside = np.zeros(tri.shape[0], bool)
    for (cx, cy) in holes:
        inside |= (cen[:, 0] - cx) ** 2 + (cen[:, 1] - cy) ** 2 < r * r
    tri = tri[~inside]
    # counter-clockwise
    a, b, c = pts[tri[:, 0]], pts[tri[:, 1]], pts[tri[:, 2]]
    cw = (b[:, 0] - a[:, 0]) * (c[:, 1] - a[:, 1]) - (b[:, 1] - a[:, 1]) * (c[:, 0] - a[:, 0]) < 0
    tri[cw] = tri[cw][:, [0, 2, 1]]
    # every boundary segment must be an edge of exactly one triangle
    e = np.sort(np.vstack([tri[:, [0, 1]], tri[:, [1, 2]], tri[:, [2, 0]]]), axis=1)
    ek, cnt = np.unique(e, axis=0, return_counts=True)
    edges = {tuple(x): int(n) for x, n in zip(ek, cnt)}
    loops = [list(range(n_sq))] + hole_loops
    for lp in loops:
        for k in range(len(lp)):
            s = tuple(sorted((lp[k], lp[(k + 1) % len(lp)])))
            if edges.get(s) != 1:
                raise ValueError("boundary segment missing from the triangulation; change the seed or h")
    if np.any(cnt > 2):
        raise ValueError("non-manifold triangulation")
    return pts, tri, loops[0], loops[1:]


def _plane(bld, size, t, z0, holes, r, h, rng, cond_tag, origin=(0.0, 0.0)):
    """Closed surface of a perforated plate [0,size]^2 x [z0 - t/2, z0 + t/2]:
    top and bottom faces, the hole walls and the outer rim (one layer each)."""
    pts, tri, sq, hl = _perforated_face(size, holes, r, h, rng)
    ox, oy = origin
    top = [bld.vid((cond_tag, 'pt', i), (ox + p[0], oy + p[1], z0 + t / 2)) for i, p in enumerate(pts)]
    bot = [bld.vid((cond_tag, 'pb', i), (ox + p[0], oy + p[1], z0 - t / 2)) for i, p in enumerate(pts)]
    for a, b, c in tri:
        bld.tris.append((top[a], top[b], top[c]))      # +z outward
        bld.tags.append(-1)
        bld.tris.append((bot[a], bot[c], bot[b]))      # -z outward
        bld.tags.append(-1)
    # outer rim: square loop counter-clockwise seen from +z, outward = away from the square
    for k in range(len(sq)):
        a, b = sq[k], sq[(k + 1) % len(sq)]
        bld.quad(bot[a], bot[b], top[b], top[a], -1)
    # hole walls: loops counter-clockwise around the hole, outward = towards the hole axis
    for lp in hl:
        for k in range(len(lp)):
            a, b = lp[k], lp[(k + 1) % len(lp)]
            bld.quad(bot[b], bot[a], top[a], top[b], -1)


def _icosphere(bld, centre, r, level, cond_tag):
    """Closed sphere: an icosahedron subdivided `level` times, vertices on the sphere."""
    p = (1 + 5 ** 0.5) / 2
    v = [(-1, p, 0), (1, p, 0), (-1, -p, 0), (1, -p, 0), (0, -1, p), (0, 1, p), (0, -1, -p), (0, 1, -p),
         (p, 0, -1), (p, 0, 1), (-p, 0, -1), (-p, 0, 1)]
    v = [np.array(x, float) / np.linalg.norm(x) for x in v]
    f = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9), (5, 11, 4), (11, 10, 2),
         (10, 7, 6), (7, 1, 8), (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9), (4, 9, 5), (2, 4, 11),
         (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    for _ in range(level):
        mid = {}
        nf = []

        def m(a, b):
            k = (min(a, b), max(a, b))
            if k not in mid:
                x = v[a] + v[b]
                v.append(x / np.linalg.norm(x))
                mid[k] = len(v) - 1
            return mid[k]
        for a, b, c in f:
            ab, bc, ca = m(a, b), m(b, c), m(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        f = nf
    ids = [bld.vid((cond_tag, 's', i), np.asarray(centre) + r * x) for i, x in enumerate(v)]
    for a, b, c in f:
        bld.tris.append((ids[a], ids[b], ids[c]))
        bld.tags.append(-1)


def package(size=10e-3, t=35e-6, n_holes=400, r_hole=0.1e-3, hole_gap=0.05e-3, n_balls=8, r_ball=0.15e-3,
            pitch=0.8e-3, ball_gap=0.05e-3, n_traces=16, trace_w=50e-6, trace_lift=0.1e-3, trace_len=(3e-3, 8e-3),
            n_ports=8, h=42e-6, sphere_level=2, sigma=5.8e7, n_freq=16, fmin=1e6, fmax=5e9, seed=3) -> Mesh:
    """BGA-like package: a perforated ground plane, an array of solder balls
    below it and straight signal traces above it (the package workload of
    Sec. III-B, synthetic).

    * plane: size x size, thickness t, n_holes seeded circular holes of radius
      r_hole at least hole_gap apart (rejection sampling), panels ~h;
    * n_balls x n_balls spheres of radius r_ball at `pitch`, centred under the
      plane, ball_gap below it (floating conductors, no port);
    * n_traces straight traces trace_w x t, trace_lift above the plane, along
      x or y, lengths U(trace_len), placed on free lanes; the first n_ports
      carry a port (source: the far end cap, sink: the near end cap).
    ESI thickness: t for the plane and the traces' 2A/P for the traces,
    2 r_ball / 3 for the balls.  Conductor ids: 0 plane, 1.. balls, then traces."""
    rng = np.random.default_rng(seed)
    bld = _Builder(False)
    holes = _hole_centres(rng, size, n_holes, r_hole, hole_gap, r_hole + hole_gap)
    _plane(bld, size, t, 0.0, holes, r_hole, h, rng, 0)
    conds = [0] * len(bld.tris)
    thick = [t]
    # solder balls
    off = (size - (n_balls - 1) * pitch) / 2
    cid = 1
    for i in range(n_balls):
        for j in range(n_balls):
            n0 = len(bld.tris)
            _icosphere(bld, (off + i * pitch, off + j * pitch, -t / 2 - ball_gap - r_ball), r_ball, sphere_level, cid)
            conds += [cid] * (len(bld.tris) - n0)
            thick.append(2 * r_ball / 3)
            cid += 1
    # traces on lanes: alternate x- and y-directed, lanes at a spacing of 4 widths
    ports = []
    tid = 0
    lanes_x = list(np.arange(0.5e-3, size - 0.5e-3, 4 * trace_w * 3))
    lanes_y = list(lanes_x)
    rng.shuffle(lanes_x)
    rng.shuffle(lanes_y)
    z_tr = t / 2 + trace_lift + t / 2
    for k in range(n_traces):
        L = rng.uniform(*trace_len)
        if k % 2 == 0:
            y = lanes_x.pop()
            x0 = rng.uniform(0.2e-3, size - 0.2e-3 - L)
            corners = [(x0, y), (x0 + L, y)]
            z = z_tr
        else:
            x = lanes_y.pop()
            y0 = rng.uniform(0.2e-3, size - 0.2e-3 - L)
            corners = [(x, y0), (x, y0 + L)]
            z = z_tr + 2 * t          # y traces one layer higher: no crossing with the x traces
        n0 = len(bld.tris)
        _swept_trace(bld, corners, z, trace_w, t, 1, 1, h, 0, cid, (2 * tid, 2 * tid + 1))
        conds += [cid] * (len(bld.tris) - n0)
        thick.append(2 * trace_w * t / (2 * (trace_w + t)))
        if k < n_ports:
            ports.append((2 * tid + 1, 2 * tid))
        tid += 1
        cid += 1
    tri = np.array(bld.tris, np.int64)
    tags = np.array(bld.tags, np.int64)
    # the swept traces emit inward-facing panels (see coils): reverse them
    is_trace = np.array(conds) >= 1 + n_balls * n_balls
    tri[is_trace] = tri[is_trace][:, [0, 2, 1]]
    # terminals are numbered per trace (2 per trace); drop those of port-less traces
    term = tags.copy()
    used = sorted({s for s, _ in ports} | {k_ for _, k_ in ports})
    remap = {o: n for n, o in enumerate(used)}
    term = np.array([remap.get(int(x), -1) if x >= 0 else -1 for x in term], np.int32)
    ports = [(remap[s], remap[k_]) for s, k_ in ports]
    return Mesh(xyz=np.array(bld.pts), tri=tri.astype(np.int32), cond=np.array(conds, np.int32), term=term,
                ports=ports, sigma=np.full(cid, sigma), thickness=np.array(thick),
                freqs=np.geomspace(fmin, fmax, n_freq), name="package")


def package_crop(seed=3) -> Mesh:
    """A 2.8 x 2.8 mm window of the package family at the same panel size and
    feature densities (31 holes, 3 x 3 balls, 4 traces with 2 ports; ~21k
    triangles), small enough for the dense oracle."""
    return package(size=2.8e-3, n_holes=31, n_balls=3, n_traces=4, n_ports=2, trace_len=(1.0e-3, 2.2e-3),
                   seed=seed)


def pop(size=15e-3, t=35e-6, plane_gap=0.2e-3, n_holes=1000, r_hole=0.1e-3, hole_gap=0.05e-3, n_balls=12,
        r_ball=0.2e-3, pitch=1.0e-3, stack_gap=0.5e-3, n_traces=64, trace_w=50e-6, trace_lift=0.1e-3,
        trace_len=(4e-3, 10e-3), n_ports=16, h=42e-6, sphere_level=2, sigma=5.8e7, n_freq=64, fmin=1e3,
        fmax=1e10, seed=5) -> Mesh:
    """Package-on-package stack: two substrates, each with two perforated
    ground planes (plane_gap apart; n_holes seeded holes over the four
    planes), an n_balls x n_balls solder-ball array between the substrates,
    and n_traces straight traces, half above each substrate; the first
    n_ports traces carry a port (far end cap source, near end cap sink).
    Conductor ids: the four planes, the balls, then the traces."""
    rng = np.random.default_rng(seed)
    bld = _Builder(False)
    conds, thick = [], []
    cid = 0
    per = n_holes // 4
    # substrate s: planes at z_s and z_s + plane_gap + t; the upper substrate
    # sits above the balls
    sub_h = plane_gap + 2 * t
    z_sub = [0.0, sub_h + stack_gap + 2 * r_ball]
    for zs in z_sub:
        for zp in (zs, zs + plane_gap + t):
            n0 = len(bld.tris)
            holes = _hole_centres(rng, size, per, r_hole, hole_gap, r_hole + hole_gap)
            _plane(bld, size, t, zp, holes, r_hole, h, rng, cid)
            conds += [cid] * (len(bld.tris) - n0)
            thick.append(t)
            cid += 1
    off = (size - (n_balls - 1) * pitch) / 2
    zb = z_sub[0] + plane_gap + t + t / 2 + stack_gap / 2 + r_ball
    for i in range(n_balls):
        for j in range(n_balls):
            n0 = len(bld.tris)
            _icosphere(bld, (off + i * pitch, off + j * pitch, zb), r_ball, sphere_level, cid)
            conds += [cid] * (len(bld.tris) - n0)
            thick.append(2 * r_ball / 3)
            cid += 1
    ports = []
    lanes = list(np.arange(0.5e-3, size - 0.5e-3, 4 * trace_w * 3))
    lane_pool = {(s_, d): list(rng.permutation(lanes)) for s_ in range(2) for d in range(2)}
    first_trace = cid
    for k in range(n_traces):
        s_ = k % 2                      # substrate
        d = (k // 2) % 2                # direction: x or y
        L = rng.uniform(*trace_len)
        top = z_sub[s_] + plane_gap + t + t / 2
        z = top + trace_lift + t / 2 + (2 * t if d else 0.0)
        lane = lane_pool[(s_, d)].pop()
        a0 = rng.uniform(0.2e-3, size - 0.2e-3 - L)
        corners = [(a0, lane), (a0 + L, lane)] if d == 0 else [(lane, a0), (lane, a0 + L)]
        n0 = len(bld.tris)
        _swept_trace(bld, corners, z, trace_w, t, 1, 1, h, 0, cid, (2 * k, 2 * k + 1))
        conds += [cid] * (len(bld.tris) - n0)
        thick.append(2 * trace_w * t / (2 * (trace_w + t)))
        if k < n_ports:
            ports.append((2 * k + 1, 2 * k))
        cid += 1
    tri = np.array(bld.tris, np.int64)
    tags = np.array(bld.tags, np.int64)
    is_trace = np.array(conds) >= first_trace
    tri[is_trace] = tri[is_trace][:, [0, 2, 1]]
    used = sorted({s_ for s_, _ in ports} | {k_ for _, k_ in ports})
    remap = {o: n for n, o in enumerate(used)}
    term = np.array([remap.get(int(x), -1) if x >= 0 else -1 for x in tags], np.int32)
    ports = [(remap[s_], remap[k_]) for s_, k_ in ports]
    return Mesh(xyz=np.array(bld.pts), tri=tri.astype(np.int32), cond=np.array(conds, np.int32), term=term,
                ports=ports, sigma=np.full(cid, sigma), thickness=np.array(thick),
                freqs=np.geomspace(fmin, fmax, n_freq), name="pop")
