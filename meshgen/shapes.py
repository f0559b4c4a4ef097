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
