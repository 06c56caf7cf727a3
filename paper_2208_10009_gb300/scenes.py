"""Seeded synthetic scenes and Tx/Rx layouts.

This module only builds inputs: triangle meshes with per-triangle face ids, optional
per-face permittivities, and transmitter/receiver positions.  It holds none of the SBR
method's arithmetic, so both the CUDA library's tests and the CPU oracle may use it.

A *face* is a planar polygon given as one or more triangles sharing a face id; the face
sequence of a path names faces, not triangles.  Triangles of one face share vertex ids
along their common edges.

The paper's own scene files (an office with 1573 faces and an outdoor street) are not
available, so these generators stand in for them with seeded procedural geometry shaped
like the paper's indoor and urban workloads.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 2208


def f32_exact(a) -> np.ndarray:
    """Round coordinates to float32 (kept as float64) so that a float32 consumer and a
    float64 consumer see exactly the same geometry."""
    return np.asarray(a, np.float64).astype(np.float32).astype(np.float64)


@dataclass
class Scene:
    verts: np.ndarray            # (V, 3) float64
    tris: np.ndarray             # (T, 3) int32
    tri_face: np.ndarray         # (T,) int32
    nf: int
    face_eps: np.ndarray | None = None   # (F,) float64, <= 0 = perfect reflector
    meta: dict = field(default_factory=dict)

    @property
    def nt(self) -> int:
        return int(len(self.tris))


class _Builder:
    def __init__(self):
        self.v, self.t, self.f = [], [], []
        self.nv = 0
        self.nf = 0

    def quad(self, p0, p1, p3, g=1, face=None):
        """Planar parallelogram p0 + u (p1 - p0) + v (p3 - p0), split into a g x g grid
        of quads (2 triangles each) sharing vertices; one face id for all."""
        p0, p1, p3 = (np.asarray(p, np.float64) for p in (p0, p1, p3))
        fid = self.nf if face is None else face
        if face is None:
            self.nf += 1
        u = np.linspace(0.0, 1.0, g + 1)
        grid = p0[None, None, :] + u[:, None, None] * (p1 - p0)[None, None, :] + u[None, :, None] * (p3 - p0)[None, None, :]
        base = self.nv
        self.v.append(grid.reshape(-1, 3))
        self.nv += (g + 1) * (g + 1)
        i, j = np.meshgrid(np.arange(g), np.arange(g), indexing="ij")
        a = base + i * (g + 1) + j
        b = a + (g + 1)
        c = b + 1
        d = a + 1
        tris = np.stack([np.stack([a, b, c], -1), np.stack([a, c, d], -1)], 2).reshape(-1, 3)
        self.t.append(tris)
        self.f.append(np.full(len(tris), fid, np.int32))
        return fid

    def polygon(self, pts, face=None):
        """Convex planar polygon as a triangle fan; one face id."""
        pts = np.asarray(pts, np.float64)
        fid = self.nf if face is None else face
        if face is None:
            self.nf += 1
        base = self.nv
        self.v.append(pts)
        self.nv += len(pts)
        k = len(pts)
        tris = np.stack([np.full(k - 2, base), base + np.arange(1, k - 1), base + np.arange(2, k)], -1)
        self.t.append(tris)
        self.f.append(np.full(len(tris), fid, np.int32))
        return fid

    def finish(self, **meta) -> Scene:
        v = f32_exact(np.concatenate(self.v))
        t = np.concatenate(self.t).astype(np.int32)
        f = np.concatenate(self.f).astype(np.int32)
        return Scene(v, t, f, self.nf, None, dict(meta))


def box_faces(b: _Builder, lo, hi, g=1, bottom=True, inward=False):
    """Axis-aligned box lo..hi as up to 6 rectangles (5 without the bottom)."""
    x0, y0, z0 = lo
    x1, y1, z1 = hi
    b.quad((x0, y0, z0), (x0, y1, z0), (x0, y0, z1), g)  # x = x0
    b.quad((x1, y0, z0), (x1, y0, z1), (x1, y1, z0), g)  # x = x1
    b.quad((x0, y0, z0), (x0, y0, z1), (x1, y0, z0), g)  # y = y0
    b.quad((x0, y1, z0), (x1, y1, z0), (x0, y1, z1), g)  # y = y1
    if bottom:
        b.quad((x0, y0, z0), (x1, y0, z0), (x0, y1, z0), g)  # z = z0
    b.quad((x0, y0, z1), (x0, y1, z1), (x1, y0, z1), g)  # z = z1


# --------------------------------------------------------------------------- small scenes
def single_plane(size=1000.0, z=0.0, eps=None) -> Scene:
    """One square ground plane z = const (one face, two triangles)."""
    b = _Builder()
    s = size
    b.quad((-s, -s, z), (s, -s, z), (-s, s, z))
    sc = b.finish(name="single_plane")
    if eps is not None:
        sc.face_eps = np.array([eps], np.float64)
    return sc


def corridor(width=4.0, length=2000.0, height=2000.0) -> Scene:
    """Two parallel walls y = 0 (face 0) and y = width (face 1), very long and tall."""
    b = _Builder()
    L, H = length, height
    b.quad((-L, 0.0, -H), (L, 0.0, -H), (-L, 0.0, H))
    b.quad((-L, width, -H), (L, width, -H), (-L, width, H))
    return b.finish(name="corridor", width=width)


def shoebox(L=10.0, W=8.0, H=3.0, g=1) -> Scene:
    """Closed rectangular room [0,L]x[0,W]x[0,H]: 6 faces, 12 triangles (g = 1).
    Face ids: 0 x=0, 1 x=L, 2 y=0, 3 y=W, 4 z=0, 5 z=H."""
    b = _Builder()
    box_faces(b, (0.0, 0.0, 0.0), (L, W, H), g)
    return b.finish(name="shoebox", dims=(L, W, H))


def shoebox_config():
    """Shoebox workload: 10 x 8 x 3 m room, Tx (2, 3, 2), Rx (8, 5, 1.5)."""
    sc = shoebox()
    return sc, f32_exact([[2.0, 3.0, 2.0]]), f32_exact([[8.0, 5.0, 1.5]])


# --------------------------------------------------------------------------- urban canyon
def urban_canyon(seed=SEED_BASE + 2, blocks=20, fmin=20.0, fmax=40.0, street=15.0, hmin=10.0, hmax=60.0,
                 ground_g=55):
    """Seeded 20 x 20 grid of axis-aligned box buildings (footprint U(20, 40) m per side,
    centred in 40 m blocks separated by 15 m streets, heights U(10, 60) m) on a ground
    plane tessellated into ground_g x ground_g quads (~10k triangles in total).  Each
    wall and each roof is its own face; the ground is one face.

    Returns (scene, tx (1,3), rx (256,3)): Tx 25 m above the central street
    intersection, Rx 1.5 m above a 16 x 16 grid of street intersections."""
    rng = np.random.default_rng(seed)
    pitch = fmax + street
    b = _Builder()
    ext = blocks * pitch
    b.quad((-50.0, -50.0, 0.0), (ext + 50.0, -50.0, 0.0), (-50.0, ext + 50.0, 0.0), ground_g)
    for i in range(blocks):
        for j in range(blocks):
            sx, sy = rng.uniform(fmin, fmax, 2)
            h = rng.uniform(hmin, hmax)
            cx, cy = i * pitch + fmax / 2, j * pitch + fmax / 2
            box_faces(b, (cx - sx / 2, cy - sy / 2, 0.0), (cx + sx / 2, cy + sy / 2, h), 1, bottom=False)
    sc = b.finish(name="urban_canyon", seed=seed, blocks=blocks)
    street_c = np.arange(blocks - 1) * pitch + fmax + street / 2  # 19 street centre lines
    mid = blocks // 2 - 1
    tx = np.array([[street_c[mid], street_c[mid], 25.0]])
    sel = street_c[1:17]
    X, Y = np.meshgrid(sel, sel, indexing="ij")
    rx = np.stack([X.ravel(), Y.ravel(), np.full(X.size, 1.5)], -1)
    return sc, f32_exact(tx), f32_exact(rx)


# --------------------------------------------------------------------------- office
def _inside_any(p, boxes, margin=0.05):
    for lo, hi in boxes:
        if np.all(p > lo - margin) and np.all(p < hi + margin):
            return True
    return False


def office(seed=SEED_BASE + 3, nbox=400, ntx=16, nrx=1024, shell=(40.0, 30.0, 4.0), g_shell=40, g_box=3):
    """Seeded office: a closed 40 x 30 x 4 m shell (each wall tessellated g_shell x g_shell)
    with `nbox` random axis-aligned furniture/partition boxes standing on the floor
    (5 faces each, tessellated g_box x g_box): ~55k triangles.  Tx and Rx are seeded
    uniformly in free space (points inside boxes rejected)."""
    rng = np.random.default_rng(seed)
    L, W, H = shell
    b = _Builder()
    box_faces(b, (0.0, 0.0, 0.0), (L, W, H), g_shell)
    boxes = []
    for _ in range(nbox):
        kind = rng.uniform()
        if kind < 0.3:  # partition: thin and tall
            sx, sy = (rng.uniform(1.0, 4.0), rng.uniform(0.05, 0.15))
            if rng.uniform() < 0.5:
                sx, sy = sy, sx
            sz = rng.uniform(1.2, 2.2)
        else:  # desk / cabinet
            sx, sy, sz = rng.uniform(0.5, 2.0), rng.uniform(0.5, 1.5), rng.uniform(0.4, 2.0)
        x = rng.uniform(0.2, L - 0.2 - sx)
        y = rng.uniform(0.2, W - 0.2 - sy)
        lo, hi = np.array([x, y, 0.0]), np.array([x + sx, y + sy, sz])
        boxes.append((lo, hi))
        box_faces(b, lo, hi, g_box, bottom=False)
    sc = b.finish(name="office", seed=seed)

    def free_points(k, zlo, zhi):
        out = []
        while len(out) < k:
            p = rng.uniform((0.3, 0.3, zlo), (L - 0.3, W - 0.3, zhi))
            if not _inside_any(p, boxes):
                out.append(p)
        return np.array(out)

    tx = free_points(ntx, 2.3, 3.7)
    rx = free_points(nrx, 0.5, 3.5)
    return sc, f32_exact(tx), f32_exact(rx)


# --------------------------------------------------------------------------- large city
def large_city(seed=SEED_BASE + 5, blocks=60, pitch=55.0, terrain_cells=700, ntx=4, nrx=4096):
    """Seeded large city: `blocks` x `blocks` extruded random convex polygons (6-12 sides,
    circumradius 10-18 m, heights lognormal with median 25 m) on a heightfield terrain of
    terrain_cells^2 cells (2 triangles each, every terrain triangle its own face): ~1M
    triangles.  Walls extend 3 m below the local terrain height."""
    rng = np.random.default_rng(seed)
    ext = blocks * pitch
    n = terrain_cells
    xs = np.linspace(-60.0, ext + 60.0, n + 1)
    X, Y = np.meshgrid(xs, xs, indexing="ij")

    def height(x, y):
        return 2.0 * np.sin(x / 310.0) * np.cos(y / 270.0) + 1.0 * np.sin((x + y) / 130.0)

    Z = height(X, Y)
    V = np.stack([X, Y, Z], -1).reshape(-1, 3)
    i, j = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    a = i * (n + 1) + j
    bb = a + (n + 1)
    tris = np.stack([np.stack([a, bb, bb + 1], -1), np.stack([a, bb + 1, a + 1], -1)], 2).reshape(-1, 3)
    bld = _Builder()
    bld.v.append(V)
    bld.nv = len(V)
    bld.t.append(tris)
    bld.f.append(np.arange(len(tris), dtype=np.int32))
    bld.nf = len(tris)
    for bi in range(blocks):
        for bj in range(blocks):
            k = int(rng.integers(6, 13))
            r = rng.uniform(10.0, 18.0)
            # evenly spaced corners jittered by up to a third of the spacing: convex, no
            # degenerate edges
            ang = (np.arange(k) + rng.uniform(-1 / 3, 1 / 3, k)) * (2 * np.pi / k) + rng.uniform(0, 2 * np.pi)
            cx, cy = bi * pitch + pitch / 2, bj * pitch + pitch / 2
            px, py = cx + r * np.cos(ang), cy + r * np.sin(ang)
            base = float(height(px, py).min()) - 3.0
            top = float(height(cx, cy)) + float(rng.lognormal(np.log(25.0), 0.5))
            for q in range(k):
                p0 = (px[q], py[q], base)
                p1 = (px[(q + 1) % k], py[(q + 1) % k], base)
                p3 = (px[q], py[q], top)
                bld.quad(p0, p1, p3, 1)
            bld.polygon(np.stack([px, py, np.full(k, top)], -1))
    sc = bld.finish(name="large_city", seed=seed)
    street = np.arange(1, blocks) * pitch
    txi = rng.choice(len(street), size=(ntx, 2))
    tx = np.stack([street[txi[:, 0]], street[txi[:, 1]], np.zeros(ntx)], -1)
    tx[:, 2] = height(tx[:, 0], tx[:, 1]) + 30.0
    side = int(np.sqrt(nrx))
    sel = np.linspace(street[0], street[-1], side)
    RX, RY = np.meshgrid(sel, street[np.linspace(0, len(street) - 1, side).astype(int)], indexing="ij")
    rx = np.stack([RX.ravel(), RY.ravel(), height(RX, RY).ravel() + 1.5], -1)
    return sc, f32_exact(tx), f32_exact(rx)


def jitter(rng, pts, amount):
    """Uniform +-amount jitter of every coordinate (float32-exact)."""
    return f32_exact(pts + rng.uniform(-amount, amount, np.shape(pts)))


# --------------------------------------------------------------------------- random clutter
def _rotation(rng) -> np.ndarray:
    """A uniformly random rotation matrix (from a random unit quaternion)."""
    q = rng.normal(size=4)
    w, x, y, z = q / np.linalg.norm(q)
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
                     [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
                     [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])


def random_clutter(seed=SEED_BASE + 9, nbox=20, room=(20.0, 16.0, 6.0), g_room=2, nrx=4):
    """Seeded closed room (each wall g_room x g_room quads) holding `nbox` boxes of random
    size (0.6-2.5 m per side) in arbitrary orientations, each box side its own face, so that
    no face lies on a coordinate plane; boxes may interpenetrate.  Tx and `nrx` Rx at random
    positions at least 0.3 m outside every box.  Returns (scene, tx (1, 3), rx (nrx, 3))."""
    rng = np.random.default_rng(seed)
    L, W, H = room
    b = _Builder()
    box_faces(b, (0.0, 0.0, 0.0), (L, W, H), g_room)
    frames = []
    for _ in range(nbox):
        half = rng.uniform(0.3, 1.25, 3)
        Rm = _rotation(rng)
        r = float(np.linalg.norm(half))
        c = np.array([rng.uniform(r, L - r), rng.uniform(r, W - r), rng.uniform(r, H - r)])
        corner = lambda sx, sy, sz: c + Rm @ (half * np.array([sx, sy, sz]))
        # the six sides as parallelograms p0 + u (p1 - p0) + v (p3 - p0)
        for s in (-1.0, 1.0):
            b.quad(corner(s, -1, -1), corner(s, 1, -1), corner(s, -1, 1))
            b.quad(corner(-1, s, -1), corner(1, s, -1), corner(-1, s, 1))
            b.quad(corner(-1, -1, s), corner(1, -1, s), corner(-1, 1, s))
        frames.append((c, Rm, half))
    sc = b.finish(name="random_clutter", seed=seed, nbox=nbox)

    def free(p):
        return all(np.any(np.abs(Rm.T @ (p - c)) > half + 0.3) for c, Rm, half in frames)

    pts = []
    while len(pts) < 1 + nrx:
        p = rng.uniform([0.5, 0.5, 0.5], [L - 0.5, W - 0.5, H - 0.5])
        if free(p):
            pts.append(p)
    pts = np.array(pts)
    return sc, f32_exact(pts[:1]), f32_exact(pts[1:])
