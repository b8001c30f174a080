"""Hierarchical low-rank form of T_A and V by adaptive cross approximation (Sec. 4).

TEST INFRASTRUCTURE ONLY (see the package docstring): the oracle of the compressed-operator
path.  Sec. 4 compresses the system matrix with an adaptive cross approximation (ACA) at
tolerance 1e-4, states that any fast method admissible in the frequency range serves, and
that at extremely low frequency the vector potential has to be stored and compressed apart
from the scalar potential so that the first is not lost against the second.  The compressed
operator here therefore compresses T_A (RWG functions) and V (cells) separately; T and the
RF-CMP system are formed from them exactly as from the dense pair (Sec. 2, Sec. 4).  The
cost statement of the complexity section (storage O(N log N) in the admissible range) is the
property the compressed form is built for.

Readings (the paper names the method and its tolerance only):
  * cluster tree: recursive bisection of the index set at the median of the item centres
    along the longest side of the cluster's bounding box, down to clusters of at most
    `leaf` items.  An item's support is a box (an RWG function: the vertices of its two
    cells; a cell: its three vertices); a cluster's box is the union of its items' supports.
  * admissibility: a block (row cluster a, column cluster b) is stored in low rank when
    min(diam a, diam b) <= eta * dist(a, b), diam the box diagonal and dist the distance
    between the two boxes (zero when they touch or overlap), and only when dist > 0: boxes
    that touch never form a low-rank block, boxes of zero extent included.  Since the
    supports are inside the boxes, an admissible block couples only cells that share no
    vertex.
  * block tree: a pair that is not admissible is split into the children of whichever
    clusters have children (both when both do); a pair of two leaves that is not admissible
    is a dense block.
  * ACA with partial pivoting (Bebendorf, Numer. Math. 86, 2000): the approximant
    S_r = sum_l u_l v_l^T is grown one cross at a time; the residual row of the current
    pivot row i is r = A[i, :] - sum_l u_l[i] v_l, its largest entry (modulus) gives the
    pivot column j, v = r / r_j, u = A[:, j] - sum_l v_l[j] u_l, and the next pivot row is
    the largest entry of |u| among rows not yet used.  A residual row that is exactly zero
    is skipped for the next unused row.  The iteration stops after the cross whose size
    ||u|| ||v|| is at most eps ||S_r||_F, with ||S_r||_F^2 updated from the new cross and
    its inner products with the earlier ones.
  * recompression: the ACA factors of a block are orthogonalised (QR of both sides) and
    the small core is cut by its SVD at eps relative to its largest singular value.
  * storage: an admissible block whose crosses would take at least its own entries
    (rank (m + n) >= m n) is stored dense.

Parity status: pinned by tests/test_oracle_lowrank.py: exact recovery of a matrix of known
rank, the interpolation property of the crosses, the Frobenius-norm update against a direct
norm, the error and rank against a truncated SVD of the same block, the block tree's exact
cover and admissibility by brute force, O(n log n) storage growth on a kernel matrix, and
the compressed EFIE operators and RF-CMP solve against the dense ones.
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Cluster:
    """A contiguous range [start, stop) of the cluster order and its support box."""

    start: int
    stop: int
    lo: np.ndarray
    hi: np.ndarray
    children: list = field(default_factory=list)

    @property
    def size(self) -> int:
        return self.stop - self.start

    @property
    def diam(self) -> float:
        return float(np.linalg.norm(self.hi - self.lo))


@dataclass
class ClusterTree:
    root: Cluster
    perm: np.ndarray  # cluster order -> original index

    def leaves(self):
        out, stack = [], [self.root]
        while stack:
            c = stack.pop()
            if c.children:
                stack.extend(reversed(c.children))
            else:
                out.append(c)
        return out


def cluster_tree(centres: np.ndarray, sup_lo: np.ndarray, sup_hi: np.ndarray, leaf: int) -> ClusterTree:
    """Recursive bisection of items with centres (n, 3) and support boxes sup_lo/sup_hi (n, 3)."""
    centres = np.asarray(centres, dtype=np.float64)
    n = centres.shape[0]
    perm = np.arange(n)

    def build(start, stop):
        idx = perm[start:stop]
        lo = sup_lo[idx].min(axis=0)
        hi = sup_hi[idx].max(axis=0)
        node = Cluster(start, stop, lo, hi)
        if stop - start > leaf:
            clo = centres[idx].min(axis=0)
            chi = centres[idx].max(axis=0)
            axis = int(np.argmax(chi - clo))
            # stable sort keeps the split reproducible for equal coordinates
            order = np.argsort(centres[idx, axis], kind="stable")
            perm[start:stop] = idx[order]
            mid = start + (stop - start) // 2
            node.children = [build(start, mid), build(mid, stop)]
        return node

    root = build(0, n) if n > 0 else Cluster(0, 0, np.zeros(3), np.zeros(3))
    return ClusterTree(root, perm)


def box_distance(a: Cluster, b: Cluster) -> float:
    """Euclidean distance between two axis-aligned boxes (0 when they touch or overlap)."""
    gap = np.maximum(0.0, np.maximum(a.lo - b.hi, b.lo - a.hi))
    return float(np.linalg.norm(gap))


def admissible(a: Cluster, b: Cluster, eta: float) -> bool:
    d = box_distance(a, b)
    return d > 0.0 and min(a.diam, b.diam) <= eta * d


@dataclass
class Block:
    """One leaf of the block tree: rows [r0, r1) and columns [c0, c1) in cluster order.

    Dense blocks hold D (r1 - r0, c1 - c0); low-rank blocks hold U (r1 - r0, rank) and
    Vt (rank, c1 - c0) with the block = U @ Vt."""

    r0: int
    r1: int
    c0: int
    c1: int
    D: np.ndarray | None = None
    U: np.ndarray | None = None
    Vt: np.ndarray | None = None

    @property
    def low_rank(self) -> bool:
        return self.U is not None

    @property
    def rank(self) -> int:
        return 0 if self.U is None else self.U.shape[1]


def block_tree(rows: ClusterTree, cols: ClusterTree, eta: float):
    """Leaves of the block tree as (row cluster, column cluster, admissible) triples."""
    out = []
    stack = [(rows.root, cols.root)]
    while stack:
        a, b = stack.pop()
        if a.size == 0 or b.size == 0:
            continue
        if admissible(a, b, eta):
            out.append((a, b, True))
        elif not a.children and not b.children:
            out.append((a, b, False))
        else:
            As = a.children or [a]
            Bs = b.children or [b]
            for x in As:
                for y in Bs:
                    stack.append((x, y))
    return out


def aca(row, col, m: int, n: int, eps: float, max_rank: int | None = None, info: dict | None = None):
    """ACA with partial pivoting of an m x n block given by row(i) -> (n,) and col(j) -> (m,).

    Returns (U (m, r), Vt (r, n)) with the block ~= U @ Vt.  info, if given, receives the
    pivot rows and columns of the crosses and the updated ||S_r||_F^2."""
    if max_rank is None:
        max_rank = min(m, n)
    us, vs = [], []
    prow, pcol = [], []
    norm2 = 0.0  # ||S_r||_F^2
    used = np.zeros(m, dtype=bool)
    i = 0
    while len(us) < max_rank:
        used[i] = True
        r = np.array(row(i), dtype=np.complex128)
        for u, v in zip(us, vs):
            r -= u[i] * v
        j = int(np.argmax(np.abs(r)))
        if r[j] == 0:
            # the residual vanishes on this row: move to the next row not yet used
            free = np.flatnonzero(~used)
            if free.size == 0:
                break
            i = int(free[0])
            continue
        v = r / r[j]
        u = np.array(col(j), dtype=np.complex128)
        for uu, vv in zip(us, vs):
            u -= vv[j] * uu
        # ||S + u v^T||^2 = ||S||^2 + 2 Re sum_l (u_l^H u)(v_l^H v) + ||u||^2 ||v||^2
        cross = sum(np.vdot(uu, u) * np.vdot(vv, v) for uu, vv in zip(us, vs))
        uv2 = np.vdot(u, u).real * np.vdot(v, v).real
        norm2 = norm2 + 2.0 * float(np.real(cross)) + uv2
        us.append(u)
        vs.append(v)
        prow.append(i)
        pcol.append(j)
        if np.sqrt(uv2) <= eps * np.sqrt(max(norm2, 0.0)):
            break
        cand = np.abs(u)
        cand[used] = -1.0
        if cand.max() < 0:
            break
        i = int(np.argmax(cand))
    if info is not None:
        info.update(rows=prow, cols=pcol, norm2=norm2)
    if not us:
        return np.zeros((m, 0), np.complex128), np.zeros((0, n), np.complex128)
    return np.stack(us, axis=1), np.stack(vs, axis=0)


def recompress(U: np.ndarray, Vt: np.ndarray, eps: float):
    """Orthogonalise both factors and cut the core's SVD at eps times its largest value."""
    if U.shape[1] == 0:
        return U, Vt
    Qu, Ru = np.linalg.qr(U)
    Qv, Rv = np.linalg.qr(Vt.T)
    W, s, Zt = np.linalg.svd(Ru @ Rv.T)
    keep = int(np.count_nonzero(s > eps * s[0])) if s[0] > 0 else 0
    return (Qu @ W[:, :keep]) * s[:keep], Zt[:keep] @ Qv.T


@dataclass
class HMatrix:
    """A matrix of shape (m, n) as dense and low-rank blocks in cluster order.

    symmetric: rows and columns share one cluster tree and only the blocks on and above the
    block diagonal (r0 <= c0) are stored; a stored block off the diagonal also stands for its
    transpose below it, so the matrix is exactly complex symmetric, as T_A and V are (Sec. 2)."""

    shape: tuple
    row_perm: np.ndarray  # cluster order -> original row
    col_perm: np.ndarray  # cluster order -> original column
    blocks: list
    symmetric: bool = False

    def storage(self) -> int:
        """Stored complex entries."""
        s = 0
        for b in self.blocks:
            s += b.D.size if b.D is not None else b.U.size + b.Vt.size
        return s

    def matvec(self, x: np.ndarray) -> np.ndarray:
        """y = M x for x (n,) or (n, c), both in the original numbering."""
        xp = np.asarray(x)[self.col_perm]
        yp = np.zeros((self.shape[0],) + xp.shape[1:], dtype=np.complex128)
        for b in self.blocks:
            xs = xp[b.c0 : b.c1]
            yp[b.r0 : b.r1] += b.D @ xs if b.D is not None else b.U @ (b.Vt @ xs)
            if self.symmetric and b.r0 != b.c0:
                xr = xp[b.r0 : b.r1]
                yp[b.c0 : b.c1] += b.D.T @ xr if b.D is not None else b.Vt.T @ (b.U.T @ xr)
        y = np.empty_like(yp)
        y[self.row_perm] = yp
        return y

    def to_dense(self) -> np.ndarray:
        M = np.zeros(self.shape, dtype=np.complex128)
        for b in self.blocks:
            blk = b.D if b.D is not None else b.U @ b.Vt
            M[np.ix_(self.row_perm[b.r0 : b.r1], self.col_perm[b.c0 : b.c1])] = blk
            if self.symmetric and b.r0 != b.c0:
                M[np.ix_(self.col_perm[b.c0 : b.c1], self.row_perm[b.r0 : b.r1])] = blk.T
        return M


def compress(entries, rows: ClusterTree, cols: ClusterTree, eta: float, eps: float, recompress_blocks: bool = True,
             symmetric: bool = False):
    """HMatrix of the matrix whose sub-blocks entries(row_idx, col_idx) returns (original numbering).

    Dense blocks are taken whole; admissible blocks by ACA at eps from single rows and columns.
    symmetric (rows is cols, a complex symmetric matrix): the blocks below the diagonal are
    not compressed but taken as the transposes of their mirror images, and the dense blocks
    on the diagonal are made symmetric (the mean with their transposes)."""
    if symmetric and rows is not cols:
        raise ValueError("a symmetric HMatrix needs one cluster tree for rows and columns")
    m = rows.perm.size
    n = cols.perm.size
    blocks = []
    for a, b, adm in block_tree(rows, cols, eta):
        if symmetric and a.start > b.start:
            continue
        ri = rows.perm[a.start : a.stop]
        ci = cols.perm[b.start : b.stop]
        if not adm:
            Dk = np.asarray(entries(ri, ci), np.complex128)
            if symmetric and a is b:
                Dk = 0.5 * (Dk + Dk.T)  # a diagonal block of a symmetric matrix, up to rounding
            blocks.append(Block(a.start, a.stop, b.start, b.stop, D=Dk))
            continue
        U, Vt = aca(lambda i: entries(ri[i : i + 1], ci)[0], lambda j: entries(ri, ci[j : j + 1])[:, 0],
                    ri.size, ci.size, eps)
        if recompress_blocks:
            U, Vt = recompress(U, Vt, eps)
        if U.shape[1] * (ri.size + ci.size) >= ri.size * ci.size:
            # the crosses would take at least the block's own entries: stored dense
            blocks.append(Block(a.start, a.stop, b.start, b.stop, D=np.asarray(entries(ri, ci), np.complex128)))
            continue
        blocks.append(Block(a.start, a.stop, b.start, b.stop, U=U, Vt=Vt))
    return HMatrix((m, n), rows.perm, cols.perm, blocks, symmetric)


# ---------------------------------------------------------------- the EFIE operators


def cell_supports(D):
    """Centres and support boxes of the cells (the domains of the p_s of V)."""
    P = D.verts[D.tris]  # (N_C, 3, 3)
    return D.cent, P.min(axis=1), P.max(axis=1)


def edge_supports(D):
    """Centres (edge midpoints) and support boxes (both cells) of the RWG functions of T_A."""
    _, lo, hi = cell_supports(D)
    ec = D.top.edge_cells  # (N, 2)
    mid = 0.5 * (D.verts[D.top.edge_verts[:, 0]] + D.verts[D.top.edge_verts[:, 1]])
    return mid, np.minimum(lo[ec[:, 0]], lo[ec[:, 1]]), np.maximum(hi[ec[:, 0]], hi[ec[:, 1]])


@dataclass
class CompressedEFIE:
    """T_A and V compressed apart (Sec. 4), with the trees they share rows and columns on."""

    TA: HMatrix
    V: HMatrix
    edge_tree: ClusterTree
    cell_tree: ClusterTree


def compress_efie(D, TA: np.ndarray, V: np.ndarray, eps: float = 1e-4, eta: float = 1.0, leaf: int = 32):
    """Compress the dense T_A and V of one mesh and wavenumber at tolerance eps."""
    et = cluster_tree(*edge_supports(D), leaf)
    ct = cluster_tree(*cell_supports(D), leaf)
    HA = compress(lambda r, c: TA[np.ix_(r, c)], et, et, eta, eps, symmetric=True)
    HV = compress(lambda r, c: V[np.ix_(r, c)], ct, ct, eta, eps, symmetric=True)
    return CompressedEFIE(HA, HV, et, ct)
