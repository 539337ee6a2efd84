"""Seeded synthetic inputs: closed triangle meshes and incident-wave sets.

This module holds geometry and random sampling only — none of the boundary
element arithmetic. It is the single input source shared by the CUDA path,
its tests, the benchmark and the CPU oracle, so that both sides see the same
meshes, vertex numbering and incident fields.

Workloads (the paper meshes at h = 2*pi/(10 k_e), Section 4; its ice
aggregate geometry of Section 5 is not available, so seeded hexagonal-prism
aggregates of the same scale stand in for it):

* ``icosphere(level)``: icosahedron refined ``level`` times, vertices projected
  to the sphere; 20*4**level triangles (level 2: 320, level 4: 5120).
* ``prism_aggregate(...)``: M disjoint hexagonal prisms (aspect ratio
  L/(2a) ~ U[0.5, 2], uniform random orientation, centres by rejection inside
  a sphere of diameter D with a separating-axis gap >= gap), each meshed with
  near-uniform triangles (side quads split in two, caps as six fan sectors).
* ``three_cubes(h)``: the three axis-aligned cubes of side 0.4 of Section 4.
* ``fibonacci_directions(n)`` and ``perpendicular_polarisation(d)``.

All triangles are ordered counter-clockwise seen from outside (outward
normal), vertex ids of each scatterer are contiguous, and ``domain[t]`` is the
scatterer id of triangle ``t``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


@dataclass
class SurfaceMesh:
    verts: np.ndarray   # float64 [nv, 3]
    tris: np.ndarray    # int32   [nt, 3], CCW seen from outside
    domain: np.ndarray  # int32   [nt], scatterer id 0..M-1

    @property
    def n_scatterers(self) -> int:
        return int(self.domain.max()) + 1 if len(self.domain) else 0

    def max_edge_length(self) -> float:
        v = self.verts
        t = self.tris
        e = np.concatenate([v[t[:, 1]] - v[t[:, 0]], v[t[:, 2]] - v[t[:, 1]],
                            v[t[:, 0]] - v[t[:, 2]]])
        return float(np.sqrt((e * e).sum(1)).max())


# --------------------------------------------------------------------------
# sphere
# --------------------------------------------------------------------------
def icosphere(level: int, radius: float = 1.0, centre=(0.0, 0.0, 0.0)) -> SurfaceMesh:
    """Icosahedron refined ``level`` times by edge midpoints, projected to the sphere."""
    p = (1.0 + math.sqrt(5.0)) / 2.0
    v = [(-1, p, 0), (1, p, 0), (-1, -p, 0), (1, -p, 0),
         (0, -1, p), (0, 1, p), (0, -1, -p), (0, 1, -p),
         (p, 0, -1), (p, 0, 1), (-p, 0, -1), (-p, 0, 1)]
    f = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11),
         (1, 5, 9), (5, 11, 4), (11, 10, 2), (10, 7, 6), (7, 1, 8),
         (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9),
         (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    verts = [np.array(x, dtype=np.float64) / np.linalg.norm(x) for x in v]
    faces = list(f)
    for _ in range(level):
        cache = {}

        def mid(a, b):
            key = (a, b) if a < b else (b, a)
            if key not in cache:
                m = verts[a] + verts[b]
                verts.append(m / np.linalg.norm(m))
                cache[key] = len(verts) - 1
            return cache[key]

        nf = []
        for (a, b, c) in faces:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = nf
    V = np.array(verts) * radius + np.asarray(centre, dtype=np.float64)
    T = np.array(faces, dtype=np.int32)
    T = _orient_outward(V, T, np.asarray(centre, dtype=np.float64))
    return SurfaceMesh(V, T, np.zeros(len(T), dtype=np.int32))


def _orient_outward(V, T, centre):
    """Flip triangles whose normal points towards ``centre`` (convex bodies only)."""
    a, b, c = V[T[:, 0]], V[T[:, 1]], V[T[:, 2]]
    n = np.cross(b - a, c - a)
    out = ((a + b + c) / 3.0 - centre)
    flip = (n * out).sum(1) < 0
    T = T.copy()
    T[flip] = T[flip][:, [0, 2, 1]]
    return T


# --------------------------------------------------------------------------
# hexagonal prisms
# --------------------------------------------------------------------------
def _merge_points(points, tol=1e-10):
    """Unique points by rounded coordinates; returns (unique array, index map).

    A point whose rounded key is new also looks in the 26 neighbouring keys,
    so that two copies of one point computed by different formulas merge even
    when they straddle a rounding boundary."""
    key_of = {}
    out = []
    idx = np.empty(len(points), dtype=np.int64)
    scale = 1.0 / tol
    near = [(a, b, c) for a in (-1, 0, 1) for b in (-1, 0, 1) for c in (-1, 0, 1) if (a, b, c) != (0, 0, 0)]
    for i, p in enumerate(points):
        key = (round(p[0] * scale), round(p[1] * scale), round(p[2] * scale))
        j = key_of.get(key)
        if j is None:
            for d in near:
                j = key_of.get((key[0] + d[0], key[1] + d[1], key[2] + d[2]))
                if j is not None and max(abs(out[j][q] - p[q]) for q in range(3)) <= tol:
                    break
                j = None
        if j is None:
            j = len(out)
            key_of[key] = j
            out.append(p)
        idx[i] = j
    return np.array(out), idx


def hexagonal_prism(a: float, length: float, n_side: int, n_len: int):
    """Axis-aligned hexagonal prism (axis z, centred at the origin) mesh.

    ``n_side`` segments per hexagon side, ``n_len`` segments along the axis.
    Triangles: 12*n_side**2 (two caps) + 12*n_side*n_len (sides).
    """
    hexv = [np.array([a * math.cos(math.pi / 3 * i), a * math.sin(math.pi / 3 * i)])
            for i in range(6)]
    pts = []
    tris = []

    def add(p):
        pts.append(p)
        return len(pts) - 1

    z0, z1 = -0.5 * length, 0.5 * length
    # caps: six fan sectors, each subdivided into n_side**2 triangles
    for z in (z0, z1):
        for s in range(6):
            A = np.zeros(2)
            B, C = hexv[s], hexv[(s + 1) % 6]
            n = n_side
            grid = {}
            for i in range(n + 1):
                for j in range(i + 1):
                    # point on the sector: A + i/n (B-A) + j/n (C-B)
                    q = A + (i / n) * (B - A) + (j / n) * (C - B)
                    grid[(i, j)] = add(np.array([q[0], q[1], z]))
            for i in range(n):
                for j in range(i + 1):
                    tris.append((grid[(i, j)], grid[(i + 1, j)], grid[(i + 1, j + 1)]))
                    if j < i:
                        tris.append((grid[(i, j)], grid[(i + 1, j + 1)], grid[(i, j + 1)]))
    # sides: n_side x n_len quads per face, each split in two
    for s in range(6):
        B, C = hexv[s], hexv[(s + 1) % 6]
        grid = {}
        for i in range(n_side + 1):
            q = B + (i / n_side) * (C - B)
            for j in range(n_len + 1):
                z = z0 + (j / n_len) * length
                grid[(i, j)] = add(np.array([q[0], q[1], z]))
        for i in range(n_side):
            for j in range(n_len):
                p00, p10 = grid[(i, j)], grid[(i + 1, j)]
                p01, p11 = grid[(i, j + 1)], grid[(i + 1, j + 1)]
                tris.append((p00, p10, p11))
                tris.append((p00, p11, p01))
    P, idx = _merge_points(pts)
    T = idx[np.array(tris)].astype(np.int32)
    T = _orient_outward(P, T, np.zeros(3))
    return P, T


def _random_rotation(rng):
    """Uniform random rotation matrix (unit quaternion, Shoemake 1992)."""
    u1, u2, u3 = rng.random(3)
    q = np.array([math.sqrt(1 - u1) * math.sin(2 * math.pi * u2),
                  math.sqrt(1 - u1) * math.cos(2 * math.pi * u2),
                  math.sqrt(u1) * math.sin(2 * math.pi * u3),
                  math.sqrt(u1) * math.cos(2 * math.pi * u3)])
    x, y, z, w = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
                     [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
                     [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])


def _prism_corners(a, length, R, c):
    ang = np.arange(6) * math.pi / 3
    ring = np.stack([a * np.cos(ang), a * np.sin(ang)], 1)
    pts = np.concatenate([np.column_stack([ring, np.full(6, -0.5 * length)]),
                          np.column_stack([ring, np.full(6, 0.5 * length)])])
    return pts @ R.T + c


def _prism_axes(R):
    """Face normals and edge directions of a rotated hexagonal prism."""
    ang = np.arange(3) * math.pi / 3
    side_normals = np.stack([np.cos(ang + math.pi / 6), np.sin(ang + math.pi / 6),
                             np.zeros(3)], 1)
    edge_dirs = np.stack([np.cos(ang + math.pi / 2 + math.pi / 6),
                          np.sin(ang + math.pi / 2 + math.pi / 6), np.zeros(3)], 1)
    axis = np.array([[0.0, 0.0, 1.0]])
    faces = np.concatenate([side_normals, axis]) @ R.T
    edges = np.concatenate([edge_dirs, axis]) @ R.T
    return faces, edges


def _sat_axes(F1, E1, F2, E2):
    """Separating-axis candidates of two prisms: face normals and edge cross products."""
    c = np.cross(E1[:, None, :], E2[None, :, :]).reshape(-1, 3)
    nc = np.linalg.norm(c, axis=1)
    keep = nc > 1e-9
    return np.concatenate([F1, F2, c[keep] / nc[keep, None]])


def _sat_gap(P1, P2, axes):
    """Largest separation along the candidate axes (<= true distance)."""
    p1, p2 = P1 @ axes.T, P2 @ axes.T
    gaps = np.maximum(p2.min(0) - p1.max(0), p1.min(0) - p2.max(0))
    return float(gaps.max())


def prism_aggregate(n_prisms: int, tris_per_prism: int | list, seed: int,
                    diameter: float = 1.0, gap: float = 0.0, a0: float = 0.12,
                    aspect=(0.5, 2.0)) -> SurfaceMesh:
    """Seeded aggregate of disjoint hexagonal prisms inside a sphere of ``diameter``.

    Circumradius ``a`` starts at ``a0`` and shrinks by 5% after every 10**4
    rejected placements; the length is ``L = 2a * U[aspect]``. Placement requires
    a separating-axis gap >= ``gap`` between every pair of prisms.
    """
    rng = np.random.default_rng(seed)
    if np.isscalar(tris_per_prism):
        tris_per_prism = [int(tris_per_prism)] * n_prisms
    a = a0
    aspects = rng.uniform(aspect[0], aspect[1], n_prisms)
    rots = [_random_rotation(rng) for _ in range(n_prisms)]
    while True:
        placed = []
        rejections = 0
        ok = True
        for m in range(n_prisms):
            L = 2 * a * aspects[m]
            rho = math.sqrt(a * a + 0.25 * L * L)
            if rho >= 0.5 * diameter:
                ok = False
                break
            F, E = _prism_axes(rots[m])
            axes = [_sat_axes(F, E, q[1], q[2]) for q in placed]
            while True:
                c = rng.uniform(-0.5 * diameter, 0.5 * diameter, 3)
                if np.linalg.norm(c) + rho > 0.5 * diameter:
                    rejections += 1
                else:
                    P = _prism_corners(a, L, rots[m], c)
                    if all(_sat_gap(P, q[0], ax) >= gap for q, ax in zip(placed, axes)):
                        placed.append((P, F, E, c, L))
                        break
                    rejections += 1
                if rejections >= 10_000:
                    ok = False
                    break
            if not ok:
                break
        if ok:
            break
        a *= 0.95
    verts, tris, dom = [], [], []
    off = 0
    for m, (P, F, E, c, L) in enumerate(placed):
        T_target = tris_per_prism[m]
        h = math.sqrt(12.0 * a * (a + L) / T_target)
        n_side = max(1, int(round(a / h)))
        n_len = max(1, int(round(L / h)))
        V, T = hexagonal_prism(a, L, n_side, n_len)
        V = V @ rots[m].T + c
        verts.append(V)
        tris.append(T + off)
        dom.append(np.full(len(T), m, dtype=np.int32))
        off += len(V)
    return SurfaceMesh(np.concatenate(verts), np.concatenate(tris).astype(np.int32),
                       np.concatenate(dom))


# --------------------------------------------------------------------------
# three cubes of Section 4
# --------------------------------------------------------------------------
def cube(origin, side: float, n: int):
    """Axis-aligned cube [origin, origin+side]^3 with n x n quads per face."""
    o = np.asarray(origin, dtype=np.float64)
    pts, tris = [], []

    def add(p):
        pts.append(p)
        return len(pts) - 1

    for axis in range(3):
        for hi in (0, 1):
            u, v = [d for d in range(3) if d != axis]
            grid = {}
            for i in range(n + 1):
                for j in range(n + 1):
                    p = o.copy()
                    p[axis] += hi * side
                    p[u] += side * i / n
                    p[v] += side * j / n
                    grid[(i, j)] = add(p)
            for i in range(n):
                for j in range(n):
                    tris.append((grid[(i, j)], grid[(i + 1, j)], grid[(i + 1, j + 1)]))
                    tris.append((grid[(i, j)], grid[(i + 1, j + 1)], grid[(i, j + 1)]))
    P, idx = _merge_points(pts)
    T = idx[np.array(tris)].astype(np.int32)
    T = _orient_outward(P, T, o + 0.5 * side)
    return P, T


def bipyramid(n: int, radius: float = 1.0, height: float = 1.0) -> SurfaceMesh:
    """Double cone over a regular n-gon: two apex vertices of valence n (edge case)."""
    ang = 2 * math.pi * np.arange(n) / n
    V = np.concatenate([np.column_stack([radius * np.cos(ang), radius * np.sin(ang), np.zeros(n)]),
                        [[0.0, 0.0, height], [0.0, 0.0, -height]]])
    T = []
    for i in range(n):
        j = (i + 1) % n
        T.append((i, j, n))
        T.append((j, i, n + 1))
    T = _orient_outward(V, np.array(T, dtype=np.int32), np.zeros(3))
    return SurfaceMesh(V, T, np.zeros(len(T), dtype=np.int32))


def three_cubes(h: float) -> SurfaceMesh:
    """Three cubes of side 0.4 with front-bottom-left corners at x = -1, 0, 1."""
    n = max(1, int(math.ceil(0.4 / h)))
    verts, tris, dom = [], [], []
    off = 0
    for m, x0 in enumerate((-1.0, 0.0, 1.0)):
        V, T = cube((x0, 0.0, 0.0), 0.4, n)
        verts.append(V)
        tris.append(T + off)
        dom.append(np.full(len(T), m, dtype=np.int32))
        off += len(V)
    return SurfaceMesh(np.concatenate(verts), np.concatenate(tris).astype(np.int32),
                       np.concatenate(dom))


# --------------------------------------------------------------------------
# incident waves and far-field directions
# --------------------------------------------------------------------------
def fibonacci_directions(n: int) -> np.ndarray:
    """n near-uniform unit vectors (golden-angle spiral)."""
    i = np.arange(n, dtype=np.float64)
    z = 1.0 - (2.0 * i + 1.0) / n
    phi = i * math.pi * (3.0 - math.sqrt(5.0))
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    return np.column_stack([r * np.cos(phi), r * np.sin(phi), z])


def perpendicular_polarisation(d: np.ndarray) -> np.ndarray:
    """Unit vector normalise(z x d), or x if d is parallel to z."""
    d = np.atleast_2d(d)
    p = np.cross(np.array([0.0, 0.0, 1.0]), d)
    n = np.linalg.norm(p, axis=1)
    p[n < 1e-12] = np.array([1.0, 0.0, 0.0])
    n[n < 1e-12] = 1.0
    return p / n[:, None]


def sphere_cut_directions(n_theta: int = 181) -> np.ndarray:
    """Directions in the planes phi = 0 and phi = pi/2, theta in [0, pi]."""
    th = np.linspace(0.0, math.pi, n_theta)
    d0 = np.column_stack([np.sin(th), np.zeros_like(th), np.cos(th)])
    d1 = np.column_stack([np.zeros_like(th), np.sin(th), np.cos(th)])
    return np.concatenate([d0, d1])


def plane_wave_x_along_z() -> np.ndarray:
    """[direction, polarisation] of E = x e^{ikz}: shape [1, 6]."""
    return np.array([[0.0, 0.0, 1.0, 1.0, 0.0, 0.0]])


def mesh_for(config: str, seed: int = 0) -> SurfaceMesh:
    """Named workloads: 'sphere320', 'sphere5120', 'sphere<nt>' (icosphere levels)."""
    if config.startswith("sphere"):
        nt = int(config[len("sphere"):])
        level = int(round(math.log(nt / 20, 4)))
        return icosphere(level)
    raise KeyError(config)
