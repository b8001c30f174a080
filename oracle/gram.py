"""Gram matrices of the primal bases (Sec. 2).

  G_ll = (lambda_m, lambda_n)   P1 mass matrix; on a cell of area A the local
                                 block is A/12 [[2,1,1],[1,2,1],[1,1,2]]
  G_pp = (p_m, p_n) = diag(1/A_n)                (Eq. patchstddef, p = 1/A on c)
  G_ff = (f_m, f_n)             RWG Gram matrix (7-point rule, exact for degree 2)
  Delta = (grad lambda_m, grad lambda_n)   P1 stiffness (Laplace-Beltrami), Eq. PrimalLaplace
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


def stiffness(D) -> sp.csr_matrix:
    """(grad l_m, grad l_n): on a cell, grad l_i = n x e_i / (2A) with e_i the edge opposite i."""
    p = D.verts[D.tris]
    e = np.stack([p[:, 2] - p[:, 1], p[:, 0] - p[:, 2], p[:, 1] - p[:, 0]], axis=1)  # (N_C, 3, 3)
    loc = np.einsum("cix,cjx->cij", e, e) / (4.0 * D.area)[:, None, None]
    rows = np.repeat(D.tris, 3, axis=1).ravel()
    cols = np.tile(D.tris, (1, 3)).ravel()
    return sp.csr_matrix((loc.reshape(D.nc, 9).ravel(), (rows, cols)), shape=(D.nv, D.nv))
