"""Gram matrices of the primal bases (Sec. 2).

  G_ll = (lambda_m, lambda_n)   P1 mass matrix; on a cell of area A the local
                                 block is A/12 [[2,1,1],[1,2,1],[1,1,2]]
  G_pp = (p_m, p_n) = diag(1/A_n)                (Eq. patchstddef, p = 1/A on c)
  G_ff = (f_m, f_n)             RWG Gram matrix (7-point rule, exact for degree 2)
  Delta = (grad lambda_m, grad lambda_n)   P1 stiffness (Laplace-Beltrami), Eq. PrimalLaplace
  G_l~p = (lambda~_m, p_n)      mixed Gram matrix of the dual piecewise linear functions and the
                                 primal pulses (Sec. 3, the matrix in P_gSigma)
"""

from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .quadrature import W7


def g_ll(D) -> sp.csr_matrix:
    loc = (np.full((3, 3), 1.0) + np.eye(3)) / 12.0
    rows = np.repeat(D.tris, 3, axis=1).ravel()
    cols = np.tile(D.tris, (1, 3)).ravel()
    vals = (D.area[:, None, None] * loc[None]).reshape(D.nc, 9).ravel()
    return sp.csr_matrix((vals, (rows, cols)), shape=(D.nv, D.nv))


def g_pp(D) -> sp.dia_matrix:
    return sp.diags(1.0 / D.area)


def g_ff(D) -> sp.csr_matrix:
    # half-function (r - P_i)/(2A) on its cell; signs are applied by B
    rel = D.qp[:, None, :, :] - D.verts[D.tris][:, :, None, :]  # (N_C, 3, 7, 3)
    loc = np.einsum("q,ciqx,cjqx->cij", W7, rel, rel) * (D.area / (4.0 * D.area**2))[:, None, None]
    nc = D.nc
    rows = (3 * np.arange(nc)[:, None, None] + np.arange(3)[None, :, None]).repeat(3, axis=2)
    cols = (3 * np.arange(nc)[:, None, None] + np.arange(3)[None, None, :]).repeat(3, axis=1)
    K = sp.csr_matrix((loc.ravel(), (rows.ravel(), cols.ravel())), shape=(3 * nc, 3 * nc))
    return (D.B.T @ K @ D.B).tocsr()


def g_ll_loops(D) -> sp.csr_matrix:
    """G_ll over the loop functions: the P1 mass matrix restricted to the interior vertices
    (all vertices of a closed surface)."""
    idx = D.top.loop_verts
    return g_ll(D)[idx][:, idx].tocsr()


def stiffness_loops(D) -> sp.csr_matrix:
    """The P1 stiffness matrix restricted to the interior vertices."""
    idx = D.top.loop_verts
    return stiffness(D)[idx][:, idx].tocsr()


def stiffness(D) -> sp.csr_matrix:
    """(grad l_m, grad l_n): on a cell, grad l_i = n x e_i / (2A) with e_i the edge opposite i."""
    p = D.verts[D.tris]
    e = np.stack([p[:, 2] - p[:, 1], p[:, 0] - p[:, 2], p[:, 1] - p[:, 0]], axis=1)  # (N_C, 3, 3)
    loc = np.einsum("cix,cjx->cij", e, e) / (4.0 * D.area)[:, None, None]
    rows = np.repeat(D.tris, 3, axis=1).ravel()
    cols = np.tile(D.tris, (1, 3)).ravel()
    return sp.csr_matrix((loc.reshape(D.nc, 9).ravel(), (rows, cols)), shape=(D.nv, D.nv))


def g_lambda_tilde_p(D) -> sp.csr_matrix:
    """Mixed Gram matrix (dual piecewise linear lambda~_m, primal pulse p_n), N_C x N_C (Sec. 3).

    From the definition of the dual piecewise linear functions (Sec. 2): lambda~_m belongs to the
    barycentre of cell m, is linear on each of the six barycentric sub-triangles (vertex, edge
    midpoint, barycentre) of a cell, and takes the values 1 at its own barycentre, 1/NoC(v) at a
    vertex v of cell m (NoC = cells around v), 1/2 at the midpoint of an edge of cell m, and 0 at
    every other barycentre, vertex or midpoint.  (lambda~_m, p_n) = (1/A_n) int_{c_n} lambda~_m:
    each sub-triangle has area A_n/6 and a linear function integrates to the area times the mean
    of its three vertex values, so the entry is the sum over the six sub-triangles of their
    vertex values, divided by 18.  Only cells sharing a vertex with m are in its support.
    """
    tris = D.tris
    noc = np.bincount(tris.ravel(), minlength=D.nv)
    v2c = [[] for _ in range(D.nv)]
    for c in range(D.nc):
        for v in tris[c]:
            v2c[v].append(c)
    rows, cols, vals = [], [], []
    for m in range(D.nc):
        vm = set(int(v) for v in tris[m])
        em = {frozenset((int(tris[m][a]), int(tris[m][(a + 1) % 3]))) for a in range(3)}
        support = sorted({c for v in vm for c in v2c[v]})
        for n in support:
            tn = [int(v) for v in tris[n]]
            total = 0.0
            for a in range(3):  # sub-triangles (vertex tn[a], midpoint of edge (tn[a], tn[b]), barycentre)
                for b in range(3):
                    if a == b:
                        continue
                    vv = 1.0 / noc[tn[a]] if tn[a] in vm else 0.0
                    vmid = 0.5 if frozenset((tn[a], tn[b])) in em else 0.0
                    vbc = 1.0 if n == m else 0.0
                    total += vv + vmid + vbc
            rows.append(m)
            cols.append(n)
            vals.append(total / 18.0)
    return sp.csr_matrix((vals, (rows, cols)), shape=(D.nc, D.nc))
