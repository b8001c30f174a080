"""Mesh topology for RWG functions and the quasi-Helmholtz transforms.

Sec. 2, Eq. RWGdef: the n-th RWG function lives on the two cells c_n^+ and
c_n^- adjacent to edge n, with free (opposite) vertices r_n^+ and r_n^-.
Sec. 2, Eq. qHofj: Sigma (N x N_C) and Lambda (N x N_V) map star / loop
coefficients to RWG coefficients; Lambda^T Sigma = 0, Lambda 1 = 0, Sigma 1 = 0.

Open surfaces (Sec. 2: "inner vertices, when Gamma is an open surface"): an edge used by one
cell is a boundary edge and carries no RWG function (the current has no normal component across
the boundary); loop functions belong to the interior vertices only, so Lambda is N x N_V with
N_V the number of interior vertices, and Lambda has full column rank (no all-one null vector).
Sigma 1 = 0 still holds: every RWG edge has exactly two cells.  The vertices of a closed
surface are all interior.

Conventions (the paper fixes none of them):
  * c_n^+ is the lower-index cell of the edge.
  * Sigma[n, c_n^+] = +1, Sigma[n, c_n^-] = -1, since div f_n = +1/A on c^+
    and -1/A on c^- (Eq. RWGdef), i.e. div f_n = sum_c Sigma[n, c] p_c.
  * Lambda: list c_n^+ counter-clockwise as (v1, v2, r_n^+); then
    Lambda[n, v1] = +1, Lambda[n, v2] = -1.  With this rule the loop
    function sum_n Lambda[n, v] f_n equals the surface curl n x grad(lambda_v)
    on every cell, so Lambda^T G_ff Lambda is the P1 stiffness matrix.
"""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp


class MeshError(ValueError):
    pass


@dataclass
class Topology:
    nv: int
    nc: int
    ne: int
    edge_verts: np.ndarray  # (N, 2) vertex ids (v1, v2) in c^+ CCW order
    edge_cells: np.ndarray  # (N, 2) cells (c^+, c^-)
    edge_free: np.ndarray  # (N, 2) free vertices (r^+, r^-)
    cell_edges: np.ndarray  # (N_C, 3) edge opposite local vertex i
    cell_sign: np.ndarray  # (N_C, 3) +1 if the cell is c^+ of that edge, -1 if c^-, 0 on the boundary
    genus: int
    loop_verts: np.ndarray  # (N_V,) mesh vertex of each loop function (the interior vertices)
    loop_of: np.ndarray  # (mesh vertices,) loop index of a vertex, -1 on the boundary
    boundaries: int  # number of boundary curves (0: closed)

    @property
    def nvl(self) -> int:
        """Number of loop functions (interior vertices)."""
        return int(self.loop_verts.shape[0])


def build_topology(tris: np.ndarray, nv: int) -> Topology:
    """RWG edges (used by two cells), their cells and free vertices; boundary edges (one cell)
    carry none; checks orientation and that the surface is a 2-manifold with boundary."""
    tris = np.asarray(tris, dtype=np.int64)
    nc = tris.shape[0]
    if tris.ndim != 2 or tris.shape[1] != 3:
        raise MeshError("tris must be (N_C, 3)")
    if nc == 0 or tris.min() < 0 or tris.max() >= nv:
        raise MeshError("vertex index out of range")
    edges = {}
    for c in range(nc):
        for i in range(3):
            a = int(tris[c, (i + 1) % 3])
            b = int(tris[c, (i + 2) % 3])
            if a == b:
                raise MeshError("degenerate cell")
            key = (min(a, b), max(a, b))
            edges.setdefault(key, []).append((c, i, a, b))
    for key, uses in edges.items():
        if len(uses) > 2:
            raise MeshError("edge %s is used by %d cells (a junction: not a 2-manifold)" % (key, len(uses)))
    inner = sorted(k for k, u in edges.items() if len(u) == 2)
    bnd = sorted(k for k, u in edges.items() if len(u) == 1)
    ne = len(inner)
    edge_verts = np.zeros((ne, 2), np.int64)
    edge_cells = np.zeros((ne, 2), np.int64)
    edge_free = np.zeros((ne, 2), np.int64)
    cell_edges = -np.ones((nc, 3), np.int64)
    cell_sign = np.zeros((nc, 3), np.int64)
    for n, key in enumerate(inner):
        uses = edges[key]
        (c0, i0, a0, b0), (c1, i1, a1, b1) = sorted(uses)
        if not (a0 == b1 and b0 == a1):
            raise MeshError("cells %d and %d are not consistently oriented" % (c0, c1))
        edge_cells[n] = (c0, c1)
        edge_verts[n] = (a0, b0)  # c^+ = c0 traverses the edge a0 -> b0
        edge_free[n] = (tris[c0, i0], tris[c1, i1])
        cell_edges[c0, i0] = n
        cell_sign[c0, i0] = 1
        cell_edges[c1, i1] = n
        cell_sign[c1, i1] = -1
    used = np.zeros(nv, bool)
    used[tris.ravel()] = True
    if not used.all():
        raise MeshError("unreferenced vertex")
    # boundary curves: every boundary vertex has exactly two boundary edges (a 2-manifold with
    # boundary); they form closed curves, counted by walking them
    on_bnd = np.zeros(nv, bool)
    adj = {}
    for a, b in bnd:
        on_bnd[a] = on_bnd[b] = True
        adj.setdefault(a, []).append(b)
        adj.setdefault(b, []).append(a)
    if any(len(x) != 2 for x in adj.values()):
        raise MeshError("a boundary vertex with other than two boundary edges (not a 2-manifold)")
    seen, curves = set(), 0
    for v0 in adj:
        if v0 in seen:
            continue
        curves += 1
        stack = [v0]
        while stack:
            v = stack.pop()
            if v in seen:
                continue
            seen.add(v)
            stack.extend(adj[v])
    chi = nv - (ne + len(bnd)) + nc  # = 2 - 2g - (boundary curves)
    if (2 - chi - curves) % 2 != 0 or 2 - chi - curves < 0:
        raise MeshError("Euler characteristic %d with %d boundary curves: not an orientable surface" % (chi, curves))
    loop_verts = np.flatnonzero(~on_bnd)
    loop_of = -np.ones(nv, np.int64)
    loop_of[loop_verts] = np.arange(loop_verts.shape[0])
    return Topology(nv, nc, ne, edge_verts, edge_cells, edge_free, cell_edges, cell_sign, (2 - chi - curves) // 2,
                    loop_verts, loop_of, curves)


def sigma_matrix(top: Topology) -> sp.csr_matrix:
    """Star transform Sigma in R^{N x N_C} (Eq. qHofj)."""
    rows = np.repeat(np.arange(top.ne), 2)
    cols = top.edge_cells.ravel()
    vals = np.tile([1.0, -1.0], top.ne)
    return sp.csr_matrix((vals, (rows, cols)), shape=(top.ne, top.nc))


def lambda_matrix(top: Topology) -> sp.csr_matrix:
    """Loop transform Lambda in R^{N x N_V} (Eq. qHofj) over the loop (interior) vertices, sign
    rule in the module header; an edge end on the boundary has no entry."""
    rows = np.repeat(np.arange(top.ne), 2)
    cols = top.loop_of[top.edge_verts.ravel()]
    vals = np.tile([1.0, -1.0], top.ne)
    keep = cols >= 0
    return sp.csr_matrix((vals[keep], (rows[keep], cols[keep])), shape=(top.ne, top.nvl))
