"""Seeded surface triangulations of PEC bodies.

Every mesh is a consistently oriented (counter-clockwise about the outward normal)
triangulation returned as ``verts`` (float64, N_V x 3) and ``tris`` (int32, N_C x 3); all are
closed except ``plate`` and ``open_cylinder`` (open surfaces).

* ``geodesic_sphere(n)``: the icosahedron with each face cut into n^2
  triangles (frequency-n geodesic grid), projected onto the sphere.
  20 n^2 cells, 30 n^2 edges, 10 n^2 + 2 vertices.  Level L of the usual
  midpoint refinement is n = 2^L (level 3: 1280 cells, level 5: 20480).
* ``ellipsoid(n, axes)``: the sphere above mapped by diag(axes).
* ``cube(n, side)``: an n x n grid of squares per face, each split into two
  triangles; 12 n^2 cells, 18 n^2 edges.

Jitter ("3 % of edge length"): every free vertex moves by a uniform random
offset of magnitude at most ``jitter * h_mean`` in its tangent plane and is
projected back onto the surface.  On the cube, face-interior vertices move in
their face, vertices on a cube edge move along that edge and corners stay
fixed, so the sharp edges survive.  All randomness comes from
``numpy.random.default_rng(seed)`` (PCG64).
"""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class Mesh:
    verts: np.ndarray  # (N_V, 3) float64
    tris: np.ndarray  # (N_C, 3) int32, CCW about the outward normal
    name: str = ""

    @property
    def nv(self) -> int:
        return int(self.verts.shape[0])

    @property
    def nc(self) -> int:
        return int(self.tris.shape[0])

    @property
    def n_edges(self) -> int:
        return 3 * self.nc // 2


def _icosahedron():
    t = (1.0 + 5.0 ** 0.5) / 2.0
    v = np.array(
        [
            [-1, t, 0], [1, t, 0], [-1, -t, 0], [1, -t, 0],
            [0, -1, t], [0, 1, t], [0, -1, -t], [0, 1, -t],
            [t, 0, -1], [t, 0, 1], [-t, 0, -1], [-t, 0, 1],
        ],
        dtype=np.float64,
    )
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    f = np.array(
        [
            [0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
            [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
            [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
            [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1],
        ],
        dtype=np.int64,
    )
    return v, f


def _orient_outward(verts, tris):
    """Flip any cell whose normal points towards the body's centre."""
    a, b, c = verts[tris[:, 0]], verts[tris[:, 1]], verts[tris[:, 2]]
    nrm = np.cross(b - a, c - a)
    cen = (a + b + c) / 3.0 - verts.mean(axis=0)
    flip = np.einsum("ij,ij->i", nrm, cen) < 0
    tris = tris.copy()
    tris[flip, 1], tris[flip, 2] = tris[flip, 2].copy(), tris[flip, 1].copy()
    return tris


def _geodesic_grid(n: int):
    """Frequency-n subdivision of the icosahedron, vertices on the unit sphere.

    A grid point of face (a, b, c) with integer weights (n-i-j, i, j) gets the
    key of its nonzero (corner, weight) pairs, so points on shared edges and
    corners are generated once.
    """
    if n < 1:
        raise ValueError("geodesic frequency must be >= 1")
    iv, ifc = _icosahedron()
    index: dict = {}
    pts = []
    tris = []

    def vid(face, i, j):
        w = {face[0]: n - i - j, face[1]: i, face[2]: j}
        key = tuple(sorted((c, wt) for c, wt in w.items() if wt > 0))
        got = index.get(key)
        if got is None:
            p = sum(iv[c] * wt for c, wt in key) / n
            got = len(pts)
            index[key] = got
            pts.append(p)
        return got

    for face in ifc:
        g = {}
        for i in range(n + 1):
            for j in range(n + 1 - i):
                g[i, j] = vid(face, i, j)
        for i in range(n):
            for j in range(n - i):
                tris.append((g[i, j], g[i + 1, j], g[i, j + 1]))
                if i + j + 1 < n:
                    tris.append((g[i + 1, j], g[i + 1, j + 1], g[i, j + 1]))
    verts = np.array(pts, dtype=np.float64)
    verts /= np.linalg.norm(verts, axis=1, keepdims=True)
    tris = np.array(tris, dtype=np.int64)
    return verts, _orient_outward(verts, tris)


def _mean_edge_length(verts, tris):
    e = np.concatenate([tris[:, [0, 1]], tris[:, [1, 2]], tris[:, [2, 0]]])
    e = np.unique(np.sort(e, axis=1), axis=0)
    return float(np.linalg.norm(verts[e[:, 0]] - verts[e[:, 1]], axis=1).mean())


def _tangent_offsets(rng, normals, radius):
    """Uniform angle, uniform magnitude in [0, radius] in each tangent plane."""
    nv = normals.shape[0]
    ref = np.where(np.abs(normals[:, [0]]) < 0.9, [[1.0, 0.0, 0.0]], [[0.0, 1.0, 0.0]])
    t1 = np.cross(normals, ref)
    t1 /= np.linalg.norm(t1, axis=1, keepdims=True)
    t2 = np.cross(normals, t1)
    phi = rng.uniform(0.0, 2.0 * np.pi, nv)
    mag = rng.uniform(0.0, radius, nv)
    return (np.cos(phi) * mag)[:, None] * t1 + (np.sin(phi) * mag)[:, None] * t2


def geodesic_sphere(n: int, radius: float = 1.0, jitter: float = 0.03, seed: int = 1) -> Mesh:
    verts, tris = _geodesic_grid(n)
    if jitter > 0:
        rng = np.random.default_rng(seed)
        h = _mean_edge_length(verts, tris)
        verts = verts + _tangent_offsets(rng, verts, jitter * h)
        verts /= np.linalg.norm(verts, axis=1, keepdims=True)
    return Mesh(verts * radius, tris.astype(np.int32), f"sphere_n{n}_r{radius}_j{jitter}_s{seed}")


def ellipsoid(n: int, axes=(1.0, 0.6, 0.4), jitter: float = 0.03, seed: int = 3) -> Mesh:
    s = geodesic_sphere(n, 1.0, jitter, seed)
    verts = s.verts * np.asarray(axes, dtype=np.float64)[None, :]
    return Mesh(verts, s.tris, f"ellipsoid_n{n}_{axes[0]}x{axes[1]}x{axes[2]}_j{jitter}_s{seed}")


def cube(n: int, side: float = 1.0, jitter: float = 0.03, seed: int = 4) -> Mesh:
    """Closed cube centred at the origin, n x n squares per face."""
    if n < 1:
        raise ValueError("cube grid must be >= 1")
    index: dict = {}
    pts = []

    def vid(p):
        key = tuple(int(round(x)) for x in p)  # integer lattice coordinates in [0, n]
        got = index.get(key)
        if got is None:
            got = len(pts)
            index[key] = got
            pts.append(key)
        return got

    tris = []
    for axis in range(3):
        for side_v in (0, n):
            u_ax, v_ax = [a for a in range(3) if a != axis]
            for i in range(n):
                for j in range(n):
                    q = []
                    for di, dj in ((0, 0), (1, 0), (1, 1), (0, 1)):
                        p = [0, 0, 0]
                        p[axis] = side_v
                        p[u_ax] = i + di
                        p[v_ax] = j + dj
                        q.append(vid(p))
                    tris.append((q[0], q[1], q[2]))
                    tris.append((q[0], q[2], q[3]))
    lat = np.array(pts, dtype=np.float64)
    verts = (lat / n - 0.5) * side
    tris = np.array(tris, dtype=np.int64)
    tris = _orient_outward(verts, tris)
    if jitter > 0:
        rng = np.random.default_rng(seed)
        h = side / n
        on_face = (lat == 0) | (lat == n)  # which coordinates sit on a cube face
        nfix = on_face.sum(axis=1)  # 1 face interior, 2 cube edge, 3 corner
        phi = rng.uniform(0.0, 2.0 * np.pi, lat.shape[0])
        mag = rng.uniform(0.0, jitter * h, lat.shape[0])
        off = np.zeros_like(verts)
        for vi in range(lat.shape[0]):
            free = np.flatnonzero(~on_face[vi])
            if nfix[vi] == 1:
                off[vi, free[0]] = np.cos(phi[vi]) * mag[vi]
                off[vi, free[1]] = np.sin(phi[vi]) * mag[vi]
            elif nfix[vi] == 2:
                off[vi, free[0]] = (1.0 if np.cos(phi[vi]) >= 0 else -1.0) * mag[vi]
        verts = verts + off
    return Mesh(verts, tris.astype(np.int32), f"cube_n{n}_side{side}_j{jitter}_s{seed}")


def torus(nu: int, nv: int, R: float = 1.0, r: float = 0.4, jitter: float = 0.0, seed: int = 6) -> Mesh:
    """Genus-1 torus: an nu x nv grid in (u, v), each quad split into two triangles.

    Jitter moves each vertex by at most ``jitter`` times the mean edge length
    in its (u, v) parameter directions.
    """
    if nu < 3 or nv < 3:
        raise ValueError("torus grid must be at least 3 x 3")
    rng = np.random.default_rng(seed)
    u = 2.0 * np.pi * np.arange(nu) / nu
    v = 2.0 * np.pi * np.arange(nv) / nv
    uu, vv = np.meshgrid(u, v, indexing="ij")
    if jitter > 0:
        h = 0.5 * (2.0 * np.pi * R / nu + 2.0 * np.pi * r / nv)
        uu = uu + rng.uniform(-1, 1, uu.shape) * jitter * h / R
        vv = vv + rng.uniform(-1, 1, vv.shape) * jitter * h / r
    verts = np.stack(
        [(R + r * np.cos(vv)) * np.cos(uu), (R + r * np.cos(vv)) * np.sin(uu), r * np.sin(vv)], axis=-1
    ).reshape(-1, 3)
    idx = lambda i, j: (i % nu) * nv + (j % nv)  # noqa: E731
    tris = []
    for i in range(nu):
        for j in range(nv):
            a, b, c, d = idx(i, j), idx(i + 1, j), idx(i + 1, j + 1), idx(i, j + 1)
            tris.append((a, b, c))
            tris.append((a, c, d))
    tris = np.array(tris, dtype=np.int64)
    # the (u, v) grid orders every cell the same way; flip all if the enclosed volume is negative
    p = verts[tris]
    vol = np.einsum("ij,ij->i", p[:, 0], np.cross(p[:, 1], p[:, 2])).sum() / 6.0
    if vol < 0:
        tris = tris[:, [0, 2, 1]]
    return Mesh(verts, tris.astype(np.int32), f"torus_{nu}x{nv}_R{R}_r{r}")


def plate(n: int, side: float = 1.0, bow: float = 0.0, jitter: float = 0.03, seed: int = 7) -> Mesh:
    """Open square plate (one boundary curve, disk topology): an n x n grid of squares in
    [-side/2, side/2]^2, each split into two triangles along alternating diagonals, normal +z.

    ``bow`` lifts the plate into a shallow cap z = bow (1 - (x^2 + y^2) / (side^2 / 2)).
    Jitter moves interior vertices in the (x, y) plane by at most ``jitter`` times the grid step;
    boundary vertices stay on the square.
    """
    if n < 1:
        raise ValueError("plate grid must be at least 1 x 1")
    rng = np.random.default_rng(seed)
    t = (np.arange(n + 1) / n - 0.5) * side
    xx, yy = np.meshgrid(t, t, indexing="ij")
    if jitter > 0:
        inner = np.zeros(xx.shape, bool)
        inner[1:-1, 1:-1] = True
        h = side / n
        xx = xx + np.where(inner, rng.uniform(-1, 1, xx.shape) * jitter * h, 0.0)
        yy = yy + np.where(inner, rng.uniform(-1, 1, yy.shape) * jitter * h, 0.0)
    zz = bow * (1.0 - (xx**2 + yy**2) / (side**2 / 2.0))
    verts = np.stack([xx, yy, zz], axis=-1).reshape(-1, 3)
    idx = lambda i, j: i * (n + 1) + j  # noqa: E731
    tris = []
    for i in range(n):
        for j in range(n):
            a, b, c, d = idx(i, j), idx(i + 1, j), idx(i + 1, j + 1), idx(i, j + 1)
            if (i + j) % 2 == 0:
                tris += [(a, b, c), (a, c, d)]
            else:
                tris += [(a, b, d), (b, c, d)]
    return Mesh(verts, np.array(tris, dtype=np.int32), f"plate_n{n}_side{side}_bow{bow}_j{jitter}_s{seed}")


def open_cylinder(nu: int, nz: int, radius: float = 0.5, height: float = 1.0, jitter: float = 0.03,
                  seed: int = 8) -> Mesh:
    """Open circular cylinder without end caps (two boundary curves, the topology of an annulus:
    one harmonic field): an nu x nz grid in (angle, z), each quad split into two triangles,
    normal pointing outward.  Jitter moves the vertices off the two rims in (angle, z)."""
    if nu < 3 or nz < 1:
        raise ValueError("cylinder grid must be at least 3 x 1")
    rng = np.random.default_rng(seed)
    u = 2.0 * np.pi * np.arange(nu) / nu
    z = (np.arange(nz + 1) / nz - 0.5) * height
    uu, zz = np.meshgrid(u, z, indexing="ij")
    if jitter > 0:
        inner = np.zeros(uu.shape, bool)
        inner[:, 1:-1] = True
        h = 0.5 * (2.0 * np.pi * radius / nu + height / nz)
        uu = uu + np.where(inner, rng.uniform(-1, 1, uu.shape) * jitter * h / radius, 0.0)
        zz = zz + np.where(inner, rng.uniform(-1, 1, zz.shape) * jitter * h, 0.0)
    verts = np.stack([radius * np.cos(uu), radius * np.sin(uu), zz], axis=-1).reshape(-1, 3)
    idx = lambda i, j: (i % nu) * (nz + 1) + j  # noqa: E731
    tris = []
    for i in range(nu):
        for j in range(nz):
            a, b, c, d = idx(i, j), idx(i + 1, j), idx(i + 1, j + 1), idx(i, j + 1)
            tris += [(a, b, c), (a, c, d)]  # (angle, z) is counter-clockwise about the outward normal
    return Mesh(verts, np.array(tris, dtype=np.int32), f"cylinder_{nu}x{nz}_r{radius}_h{height}_j{jitter}_s{seed}")


def mesh_for_config(name: str) -> Mesh:
    """The seeded meshes of the named workloads.

    ``sphere_l3``: unit sphere, frequency 8 (1280 cells, 1920 unknowns), seed 1.
    ``sphere_l5``: unit sphere, frequency 32 (20480 cells, 30720 unknowns), seed 2.
    ``ellipsoid_40k``: ellipsoid 1.0/0.6/0.4, frequency 37 (41070 unknowns), seed 3.
    ``sphere_90k``: unit sphere, frequency 55 (90750 unknowns), seed 5.
    """
    table = {
        "sphere_l1": lambda: geodesic_sphere(2, seed=1),
        "sphere_l2": lambda: geodesic_sphere(4, seed=1),
        "sphere_l3": lambda: geodesic_sphere(8, seed=1),
        "sphere_l4": lambda: geodesic_sphere(16, seed=2),
        "sphere_l5": lambda: geodesic_sphere(32, seed=2),
        "ellipsoid_40k": lambda: ellipsoid(37, seed=3),
        "sphere_90k": lambda: geodesic_sphere(55, seed=5),
    }
    return table[name]()
