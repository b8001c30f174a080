"""Mesh topology for RWG functions and the quasi-Helmholtz transforms.

Sec. 2, Eq. RWGdef: the n-th RWG function lives on the two cells c_n^+ and
c_n^- adjacent to edge n, with free (opposite) vertices r_n^+ and r_n^-.
Sec. 2, Eq. qHofj: Sigma (N x N_C) and Lambda (N x N_V) map star / loop
coefficients to RWG coefficients; Lambda^T Sigma = 0, Lambda 1 = 0, Sigma 1 = 0.

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
    cell_sign: np.ndarray  # (N_C, 3) +1 if the cell is c^+ of that edge else -1
    genus: int


def build_topology(tris: np.ndarray, nv: int) -> Topology:
    """Edges, their two cells and free vertices; checks closedness and orientation."""
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
    ne = len(edges)
    edge_verts = np.zeros((ne, 2), np.int64)
    edge_cells = np.zeros((ne, 2), np.int64)
    edge_free = np.zeros((ne, 2), np.int64)
    cell_edges = -np.ones((nc, 3), np.int64)
    cell_sign = np.zeros((nc, 3), np.int64)
    for n, (key, uses) in enumerate(sorted(edges.items())):
        if len(uses) != 2:
            raise MeshError("edge %s is used by %d cells (not a closed 2-manifold)" % (key, len(uses)))
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
    chi = nv - ne + nc
    if chi % 2 != 0 or chi > 2:
        raise MeshError("Euler characteristic %d is not that of a closed orientable surface" % chi)
    used = np.zeros(nv, bool)
    used[tris.ravel()] = True
    if not used.all():
        raise MeshError("unreferenced vertex")
    return Topology(nv, nc, ne, edge_verts, edge_cells, edge_free, cell_edges, cell_sign, (2 - chi) // 2)


def sigma_matrix(top: Topology) -> sp.csr_matrix:
    """Star transform Sigma in R^{N x N_C} (Eq. qHofj)."""
    rows = np.repeat(np.arange(top.ne), 2)
    cols = top.edge_cells.ravel()
    vals = np.tile([1.0, -1.0], top.ne)
    return sp.csr_matrix((vals, (rows, cols)), shape=(top.ne, top.nc))


def lambda_matrix(top: Topology) -> sp.csr_matrix:
    """Loop transform Lambda in R^{N x N_V} (Eq. qHofj), sign rule in the module header."""
    rows = np.repeat(np.arange(top.ne), 2)
    cols = top.edge_verts.ravel()
    vals = np.tile([1.0, -1.0], top.ne)
    return sp.csr_matrix((vals, (rows, cols)), shape=(top.ne, top.nv))
