"""Galerkin matrices of the EFIE with RWG functions (Sec. 2).

Definitions (Sec. 2, Eq. RWGdef and the matrix definitions after Eq. EFIE):
  f_n = (r - r_n^+)/(2 A^+) on c_n^+,  (r_n^- - r)/(2 A^-) on c_n^-  (no edge-length factor)
  G(r, r') = e^{i k R} / (4 pi R),  R = |r - r'|,  time convention e^{-i w t}
  [T_A]_mn  = (n x f_m, T_A f_n)  = int int f_m(r) . f_n(r') G dS dS'
  [T_Phi]_mn = (n x f_m, T_Phi f_n) = int int div f_m div' f_n G dS dS'
             = (Sigma V Sigma^T)_mn,  V_st = int int p_s p_t G,  p_s = 1/A_s on c_s
  e_n = (n x f_n, n x E^i) = int f_n . E^i dS
  T = i k T_A + T_Phi / (i k),  T j = -e.
The (n x f_m, n x a) testing reduces to f_m . a because f_m is tangential.
The identity T_Phi = Sigma V Sigma^T (Sec. 3, Eq. TPhiandV, here at every k)
holds because div f_n = sum_c Sigma[n, c] p_c.

Quadrature (the paper states none; readings):
  * far pairs (cells sharing no vertex): 7 x 7 product of the 7-point rule;
  * near pairs (same cell, or sharing an edge or a vertex): singularity
    extraction G = 1/(4 pi R) + (e^{ikR} - 1)/(4 pi R); the first part is
    integrated over the source cell in closed form (``potentials``), the
    second with the 7-point rule (its value at R = 0 is i k / (4 pi)); the
    outer integral uses the 7-point rule.  Extraction is not symmetric in the
    two cells, so each near pair is the mean of both orders (test cell outer),
    which keeps T_A and V complex symmetric.

Every cell-pair integral is reduced to the moments, in centroid-local
coordinates rho = r - c_s and rho' = r' - c_t,
  I0 = int int G,  Ir = int int rho G,  Irp = int int rho' G,  Irr = int int rho.rho' G,
and the local RWG half-functions (edge opposite local vertex i, free vertex
P_i, sign sigma = +1 on c^+ and -1 on c^-) give
  sigma_i sigma_j / (4 A_s A_t) [Irr - b_j.Ir - a_i.Irp + (a_i.b_j) I0]
  (the signs enter through the map B from local half-functions to RWG
  functions, T_A = B^T K B),
  a_i = P_i - c_s,  b_j = P_j - c_t,
while V_st = I0 / (A_s A_t).
"""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp

from .potentials import triangle_potentials
from .quadrature import BARY7, W7, cell_geometry, quad_points
from .topology import Topology, build_topology, lambda_matrix, sigma_matrix

FOUR_PI = 4.0 * np.pi


@dataclass
class Discretization:
    verts: np.ndarray
    tris: np.ndarray
    top: Topology
    area: np.ndarray  # (N_C,)
    normal: np.ndarray  # (N_C, 3)
    cent: np.ndarray  # (N_C, 3)
    qp: np.ndarray  # (N_C, 7, 3) quadrature points
    rho: np.ndarray  # (N_C, 7, 3) quadrature points minus the centroid
    a_loc: np.ndarray  # (N_C, 3, 3) free vertex of local basis i minus centroid
    B: sp.csr_matrix  # (3 N_C, N) local half-function -> RWG map (entries sigma)
    Sigma: sp.csr_matrix
    Lambda: sp.csr_matrix
    near: np.ndarray  # (P, 2) ordered near pairs (s, t), s != t or s == t

    @property
    def N(self):
        return self.top.ne

    @property
    def nc(self):
        return self.top.nc

    @property
    def nv(self):
        return self.top.nv


def discretize(verts, tris) -> Discretization:
    verts = np.asarray(verts, dtype=np.float64)
    tris = np.asarray(tris, dtype=np.int64)
    top = build_topology(tris, verts.shape[0])
    area, normal, cent = cell_geometry(verts, tris)
    qp = quad_points(verts, tris)
    rho = qp - cent[:, None, :]
    a_loc = verts[tris] - cent[:, None, :]
    rows = np.arange(3 * top.nc)
    ce = top.cell_edges.ravel()
    on = ce >= 0  # boundary edges of an open surface carry no RWG function
    B = sp.csr_matrix(
        (top.cell_sign.ravel()[on].astype(np.float64), (rows[on], ce[on])),
        shape=(3 * top.nc, top.ne),
    )
    # near pairs: cells sharing at least one vertex (including s == t)
    v2c = [[] for _ in range(top.nv)]
    for c in range(top.nc):
        for v in tris[c]:
            v2c[v].append(c)
    near = set()
    for cells in v2c:
        for s in cells:
            for t in cells:
                near.add((s, t))
    near = np.array(sorted(near), dtype=np.int64)
    return Discretization(
        verts, tris, top, area, normal, cent, qp, rho, a_loc, B, sigma_matrix(top), lambda_matrix(top), near
    )


def _far_moments(D: Discretization, s_idx, t_idx, k):
    """7 x 7 product-rule moments for every (s, t) in s_idx x t_idx.

    Returns I0 (S, T), Ir (S, T, 3), Irp (S, T, 3), Irr (S, T).
    """
    rs = D.rho[s_idx]  # (S, 7, 3)
    rt = D.rho[t_idx]  # (T, 7, 3)
    dst = D.cent[s_idx][:, None, :] - D.cent[t_idx][None, :, :]  # (S, T, 3)
    diff = dst[:, :, None, None, :] + rs[:, None, :, None, :] - rt[None, :, None, :, :]
    R = np.sqrt(np.einsum("stijx,stijx->stij", diff, diff))
    with np.errstate(divide="ignore", invalid="ignore"):  # coincident points only occur in near pairs,
        G = np.exp(1j * k * R) / (FOUR_PI * R)  # whose far-rule values are replaced
    w = np.outer(W7, W7)[None, None] * (D.area[s_idx][:, None] * D.area[t_idx][None, :])[:, :, None, None]
    with np.errstate(invalid="ignore"):
        wG = w * G  # (S, T, 7, 7)
    I0 = wG.sum(axis=(2, 3))
    Ir = np.einsum("stij,six->stx", wG, rs)
    Irp = np.einsum("stij,tjx->stx", wG, rt)
    Irr = np.einsum("stij,six,tjx->st", wG, rs, rt)
    return I0, Ir, Irp, Irr


def _near_moments_one_order(D: Discretization, s, t, k):
    """Moments of the pair (s test/outer, t source/inner) with singularity extraction."""
    s = np.asarray(s)
    t = np.asarray(t)
    P = s.shape[0]
    r = D.qp[s].reshape(-1, 3)  # (P*7, 3) outer points
    tri_t = np.repeat(D.verts[D.tris[t]], 7, axis=0)  # (P*7, 3, 3)
    S, Vv, p = triangle_potentials(r, tri_t)
    ct = np.repeat(D.cent[t], 7, axis=0)
    J0 = S / FOUR_PI
    J1 = (Vv + (p - ct) * S[:, None]) / FOUR_PI
    # smooth remainder (e^{ikR} - 1)/(4 pi R) with the 7-point inner rule
    At = np.repeat(D.area[t], 7)
    src = np.repeat(D.qp[t], 7, axis=0)  # (P*7, 7, 3)
    rhot = np.repeat(D.rho[t], 7, axis=0)
    R = np.linalg.norm(r[:, None, :] - src, axis=2)  # (P*7, 7)
    safe = np.where(R > 0, R, 1.0)
    half = np.sin(0.5 * k * R)
    g = np.where(R > 0, (-2.0 * half * half + 1j * np.sin(k * R)) / (FOUR_PI * safe), 1j * k / FOUR_PI)
    wg = W7[None, :] * At[:, None] * g
    J0 = J0 + wg.sum(axis=1)
    J1 = J1 + np.einsum("mj,mjx->mx", wg, rhot)
    J0 = J0.reshape(P, 7)
    J1 = J1.reshape(P, 7, 3)
    wo = W7[None, :] * D.area[s][:, None]  # (P, 7)
    rs = D.rho[s]
    I0 = (wo * J0).sum(axis=1)
    Ir = np.einsum("pi,pix->px", wo * J0, rs)
    Irp = np.einsum("pi,pix->px", wo, J1)
    Irr = np.einsum("pi,pix,pix->p", wo, rs, J1)
    return I0, Ir, Irp, Irr


def near_moments(D: Discretization, s, t, k):
    """Symmetrised near-pair moments: mean of the (s outer) and (t outer) orders."""
    a0, ar, arp, arr = _near_moments_one_order(D, s, t, k)
    b0, br, brp, brr = _near_moments_one_order(D, t, s, k)
    # in the (t outer) order the roles of rho and rho' are exchanged
    return 0.5 * (a0 + b0), 0.5 * (ar + brp), 0.5 * (arp + br), 0.5 * (arr + brr)


def _local_block(D: Discretization, s_idx, t_idx, I0, Ir, Irp, Irr):
    """Local half-function couplings K[s, i, t, j] without the signs sigma.

    The signs live in the RWG map B, so T_A = B^T K B.
    """
    a = D.a_loc[s_idx]  # (S, 3, 3)
    b = D.a_loc[t_idx]  # (T, 3, 3)
    term = (
        Irr[:, None, :, None]
        - np.einsum("tjx,stx->sjt", b, Ir).transpose(0, 2, 1)[:, None, :, :]
        - np.einsum("six,stx->sit", a, Irp)[:, :, :, None]
        + np.einsum("six,tjx->sitj", a, b) * I0[:, None, :, None]
    )
    scale = 1.0 / (4.0 * D.area[s_idx][:, None, None, None] * D.area[t_idx][None, None, :, None])
    return term * scale


def pair_moments(D: Discretization, s_idx, k):
    """Moments of every pair (s, t), s in s_idx, t over all cells (far rule or near rule)."""
    s_idx = np.asarray(s_idx, dtype=np.int64)
    t_all = np.arange(D.nc)
    I0, Ir, Irp, Irr = _far_moments(D, s_idx, t_all, k)
    pos = {int(s): i for i, s in enumerate(s_idx)}
    sel = np.isin(D.near[:, 0], s_idx)
    ns, nt = D.near[sel, 0], D.near[sel, 1]
    if ns.size:
        n0, nr, nrp, nrr = near_moments(D, ns, nt, k)
        rows = np.array([pos[int(x)] for x in ns])
        I0[rows, nt] = n0
        Ir[rows, nt] = nr
        Irp[rows, nt] = nrp
        Irr[rows, nt] = nrr
    return I0, Ir, Irp, Irr


def assemble(D: Discretization, k: float, chunk: int = 8):
    """Dense T_A (N x N) and V (N_C x N_C), complex128."""
    nc = D.nc
    K = np.zeros((3 * nc, 3 * nc), dtype=np.complex128)
    V = np.zeros((nc, nc), dtype=np.complex128)
    t_all = np.arange(nc)
    for s0 in range(0, nc, chunk):
        s_idx = np.arange(s0, min(s0 + chunk, nc))
        I0, Ir, Irp, Irr = pair_moments(D, s_idx, k)
        V[s_idx] = I0 / (D.area[s_idx][:, None] * D.area[None, :])
        blk = _local_block(D, s_idx, t_all, I0, Ir, Irp, Irr)  # (S, 3, T, 3)
        K[3 * s0 : 3 * s0 + 3 * len(s_idx)] = blk.reshape(3 * len(s_idx), 3 * nc)
    B = D.B.toarray()
    TA = B.T @ K @ B
    return TA, V


def assemble_rows(D: Discretization, k: float, rows_edges, rows_cells):
    """Sampled rows: T_A[m, :] for m in rows_edges and V[s, :] for s in rows_cells."""
    rows_edges = np.asarray(rows_edges, dtype=np.int64)
    rows_cells = np.asarray(rows_cells, dtype=np.int64)
    TA_rows = np.zeros((rows_edges.size, D.N), dtype=np.complex128)
    B = D.B
    for r, m in enumerate(rows_edges):
        for side in range(2):
            s = int(D.top.edge_cells[m, side])
            i = int(np.flatnonzero(D.top.cell_edges[s] == m)[0])
            I0, Ir, Irp, Irr = pair_moments(D, [s], k)
            blk = _local_block(D, np.array([s]), np.arange(D.nc), I0, Ir, Irp, Irr)[0, i]  # (T, 3)
            TA_rows[r] += D.top.cell_sign[s, i] * (blk.reshape(-1) @ B)
    V_rows = np.zeros((rows_cells.size, D.nc), dtype=np.complex128)
    for r, s in enumerate(rows_cells):
        I0, _, _, _ = pair_moments(D, [s], k)
        V_rows[r] = I0[0] / (D.area[s] * D.area)
    return TA_rows, V_rows


def t_phi(D: Discretization, V: np.ndarray) -> np.ndarray:
    """T_Phi = Sigma V Sigma^T (Sec. 3, Eq. TPhiandV)."""
    S = D.Sigma.toarray()
    return S @ V @ S.T


def t_phi_edgewise(D: Discretization, k: float) -> np.ndarray:
    """T_Phi from its own definition int int div f_m div f_n G (a cross-check of Eq. TPhiandV).

    div f_m = sigma / A_s on each of its cells, so the entry is the sum over the
    four cell pairs of sigma_m sigma_n I0(s, t) / (A_s A_t).
    """
    N = D.N
    out = np.zeros((N, N), dtype=np.complex128)
    I0 = np.zeros((D.nc, D.nc), dtype=np.complex128)
    for s in range(D.nc):
        I0[s] = pair_moments(D, [s], k)[0][0]
    for m in range(N):
        for sm, s in zip((1.0, -1.0), D.top.edge_cells[m]):
            for sn in (1.0, -1.0):
                t = D.top.edge_cells[:, 0 if sn > 0 else 1]
                out[m] += sm * sn * I0[s, t] / (D.area[s] * D.area[t])
    return out


def efie_matrix(D: Discretization, TA: np.ndarray, V: np.ndarray, k: float) -> np.ndarray:
    """T = i k T_A + T_Phi / (i k) (Sec. 2)."""
    return 1j * k * TA + t_phi(D, V) / (1j * k)


def excitation(D: Discretization, k: float, khat, pol) -> np.ndarray:
    """e_n = int f_n . E^i dS, E^i = pol e^{i k khat . r}; columns = plane waves (N x nrhs)."""
    khat = np.atleast_2d(np.asarray(khat, dtype=np.float64))
    pol = np.atleast_2d(np.asarray(pol, dtype=np.complex128))
    nrhs = khat.shape[0]
    phase = np.exp(1j * k * np.einsum("cqx,rx->cqr", D.qp, khat))  # (N_C, 7, nrhs)
    # local half-function value (sigma / (2 A_s)) (r - P_i) dotted with pol
    rel = D.qp[:, None, :, :] - D.verts[D.tris][:, :, None, :]  # (N_C, 3 local, 7, 3)
    dots = np.einsum("ciqx,rx->ciqr", rel, pol)
    w = W7[None, None, :, None] * D.area[:, None, None, None]
    loc = (w * dots * phase[:, None, :, :]).sum(axis=2)  # (N_C, 3, nrhs)
    loc /= (2.0 * D.area)[:, None, None]  # the sign sigma is applied by B
    return D.B.T @ loc.reshape(3 * D.nc, nrhs)


def gap_edges(D: Discretization, origin, normal):
    """Edges of a voltage gap cut by the plane (origin, normal): those whose two cells have their
    centroids on opposite sides.  Returns (edge indices, s) with s = +1 where c^+ lies on the
    negative side (the RWG direction c^+ -> c^- runs along the normal), -1 otherwise."""
    o = np.asarray(origin, dtype=np.float64)
    nh = np.asarray(normal, dtype=np.float64)
    nh = nh / np.linalg.norm(nh)
    side = (D.cent - o) @ nh > 0.0
    cp, cm = D.top.edge_cells[:, 0], D.top.edge_cells[:, 1]
    cut = np.flatnonzero(side[cp] != side[cm])
    return cut, np.where(side[cp[cut]], -1.0, 1.0)


def excitation_voltage_gap(D: Discretization, origin, normal, voltage: complex = 1.0) -> np.ndarray:
    """e_n = int f_n . E^i for a delta-gap source E^i = V delta(s) u (Sec. 4, the Fokker model's
    second excitation; the paper gives no formula, reading: the gap is the closed line of mesh
    edges cut by a plane, u the unit in-surface normal of that line pointing to the plane
    normal's side, s the distance across it).  The delta reduces the surface integral to the
    line integral V int_edge f_n . u dl over the gap edges, evaluated here from the RWG function
    on c^+ (Eq. RWGdef, (r - r^+) / (2 A^+)) with a 5-point Gauss rule along the edge."""
    cut, s = gap_edges(D, origin, normal)
    e = np.zeros(D.N, dtype=np.complex128)
    x, w = np.polynomial.legendre.leggauss(5)
    t, w = 0.5 * (x + 1.0), 0.5 * w
    for n, sg in zip(cut, s):
        v1, v2 = D.verts[D.top.edge_verts[n]]
        cp = D.top.edge_cells[n, 0]
        rp = D.verts[D.top.edge_free[n, 0]]
        ev = v2 - v1
        le = np.linalg.norm(ev)
        # in-surface normal of the edge pointing out of c^+ (away from its free vertex)
        nrm = D.normal[cp]
        out = np.cross(ev, nrm)
        out = out / np.linalg.norm(out)
        if out @ (v1 - rp) < 0:
            out = -out
        pts = v1[None, :] + t[:, None] * ev[None, :]
        f = (pts - rp[None, :]) / (2.0 * D.area[cp])
        flux = le * np.sum(w * (f @ out))
        e[n] = voltage * sg * flux
    return e[:, None]
