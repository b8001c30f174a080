"""Pins of the compressed-operator oracle (Sec. 4: T_A and V compressed apart by ACA at 1e-4).

Held to what the mathematics fixes, not to the oracle itself: a matrix of known rank is
recovered exactly; the approximant interpolates the block on every pivot row and column;
the updated Frobenius norm equals a direct norm; the error is within the tolerance of a
truncated SVD of the same block and the rank near its eps-rank; the block tree covers every
entry exactly once and its low-rank blocks are separated (brute force over the supports);
storage grows like n log n on a kernel matrix; and on the EFIE the separately compressed
T_A and V give the dense operators' current at every wavenumber, while compressing T whole
loses the vector potential at low frequency (the cancellation Sec. 4 warns of).
"""

import numpy as np
import pytest

import synth
from oracle import efie, krylov, lowrank as L, rfcmp


def _fib_sphere(n):
    """n points on the unit sphere by the Fibonacci lattice."""
    i = np.arange(n) + 0.5
    z = 1.0 - 2.0 * i / n
    r = np.sqrt(1.0 - z * z)
    ph = np.pi * (1.0 + 5**0.5) * i
    return np.stack([r * np.cos(ph), r * np.sin(ph), z], axis=1)


def _laplace(P, Q):
    """Entries 1/(4 pi |p - q|) (0 where p = q)."""
    def ent(r, c):
        d = np.linalg.norm(P[r][:, None] - Q[c][None], axis=2)
        g = np.zeros_like(d)
        np.divide(1.0, 4.0 * np.pi * d, out=g, where=d > 0)
        return g.astype(np.complex128)

    return ent


def _separated_block(m=120, n=90, shift=4.0, seed=3):
    rng = np.random.default_rng(seed)
    P = rng.uniform(-0.5, 0.5, (m, 3))
    Q = rng.uniform(-0.5, 0.5, (n, 3)) + np.array([shift, 0.0, 0.0])
    return _laplace(P, Q)(np.arange(m), np.arange(n))


def test_aca_recovers_a_matrix_of_known_rank():
    rng = np.random.default_rng(1)
    m, n, r = 70, 55, 5
    A = (rng.standard_normal((m, r)) + 1j * rng.standard_normal((m, r))) @ (
        rng.standard_normal((r, n)) + 1j * rng.standard_normal((r, n)))
    U, Vt = L.aca(lambda i: A[i], lambda j: A[:, j], m, n, 1e-12)
    assert r <= U.shape[1] <= r + 1  # the last cross may be a rounding-level one that stops it
    assert np.linalg.norm(A - U @ Vt) <= 1e-12 * np.linalg.norm(A)
    U2, Vt2 = L.recompress(U, Vt, 1e-12)
    assert U2.shape[1] == r
    assert np.linalg.norm(A - U2 @ Vt2) <= 1e-12 * np.linalg.norm(A)


def test_aca_crosses_interpolate_and_norm_update_is_exact():
    A = _separated_block()
    info = {}
    U, Vt = L.aca(lambda i: A[i], lambda j: A[:, j], *A.shape, 1e-6, info=info)
    E = A - U @ Vt
    scale = np.abs(A).max()
    # the approximant reproduces the block on every pivot row and pivot column
    assert np.abs(E[info["rows"], :]).max() <= 1e-12 * scale
    assert np.abs(E[:, info["cols"]]).max() <= 1e-12 * scale
    assert len(set(info["rows"])) == len(info["rows"])
    assert np.isclose(info["norm2"], np.linalg.norm(U @ Vt) ** 2, rtol=1e-12)


@pytest.mark.parametrize("eps", [1e-3, 1e-4, 1e-6])
def test_aca_error_and_rank_against_truncated_svd(eps):
    A = _separated_block()
    U, Vt = L.aca(lambda i: A[i], lambda j: A[:, j], *A.shape, eps)
    U, Vt = L.recompress(U, Vt, eps)
    err = np.linalg.norm(A - U @ Vt) / np.linalg.norm(A)
    s = np.linalg.svd(A, compute_uv=False)
    tail = np.sqrt(np.cumsum((s**2)[::-1]))[::-1] / np.linalg.norm(A)  # tail[r] = ||A - A_r|| / ||A||
    eps_rank = int(np.argmax(np.append(tail, 0.0) <= eps))
    assert err <= 10 * eps
    assert U.shape[1] <= eps_rank + 3
    # no rank-r approximant beats the truncated SVD (Eckart-Young); the cross one is close to it
    r = U.shape[1]
    assert err >= (tail[r] if r < s.size else 0.0) * (1 - 1e-9)


def test_cluster_tree_partitions_and_bounds_its_items():
    P = _fib_sphere(500)
    h = 0.05
    T = L.cluster_tree(P, P - h, P + h, leaf=24)
    assert np.array_equal(np.sort(T.perm), np.arange(500))
    stack = [T.root]
    while stack:
        c = stack.pop()
        idx = T.perm[c.start : c.stop]
        assert np.all(P[idx] - h >= c.lo - 1e-15) and np.all(P[idx] + h <= c.hi + 1e-15)
        if c.children:
            a, b = c.children
            assert a.start == c.start and a.stop == b.start and b.stop == c.stop
            assert abs(a.size - b.size) <= 1
            stack.extend(c.children)
        else:
            assert 0 < c.size <= 24


@pytest.mark.parametrize("eta", [0.5, 1.0, 2.0])
def test_block_tree_covers_every_entry_once_and_separates_low_rank_blocks(eta):
    P = _fib_sphere(800)
    h = 0.05
    lo, hi = P - h, P + h
    T = L.cluster_tree(P, lo, hi, leaf=16)
    count = np.zeros((800, 800), dtype=np.int64)
    n_lr = 0
    for a, b, adm in L.block_tree(T, T, eta):
        ri, ci = T.perm[a.start : a.stop], T.perm[b.start : b.stop]
        count[np.ix_(ri, ci)] += 1
        if adm:
            n_lr += 1
            # brute force: every pair of supports is at least the box distance apart, and the
            # admissibility inequality holds for the boxes the supports span
            gap = np.maximum(0.0, np.maximum(lo[ri][:, None] - hi[ci][None], lo[ci][None] - hi[ri][:, None]))
            dmin = np.linalg.norm(gap, axis=2).min()
            bl, bh = lo[ri].min(0), hi[ri].max(0)
            cl, ch = lo[ci].min(0), hi[ci].max(0)
            dbox = np.linalg.norm(np.maximum(0.0, np.maximum(bl - ch, cl - bh)))
            assert dmin >= dbox - 1e-12 and dbox > 0
            assert min(np.linalg.norm(bh - bl), np.linalg.norm(ch - cl)) <= eta * dbox
        else:
            assert not a.children and not b.children
    assert np.all(count == 1)
    assert n_lr > 0


def test_symmetric_storage_is_exactly_symmetric_and_matches_the_full_form():
    P = _fib_sphere(600)
    h = 0.04
    T = L.cluster_tree(P, P - h, P + h, leaf=32)
    ent = _laplace(P, P)
    full = L.compress(ent, T, T, 1.0, 1e-6)
    sym = L.compress(ent, T, T, 1.0, 1e-6, symmetric=True)
    M = ent(np.arange(600), np.arange(600))
    Ds = sym.to_dense()
    assert np.array_equal(Ds, Ds.T)
    assert sym.storage() < 0.6 * full.storage()
    x = np.random.default_rng(2).standard_normal((600, 3)) + 0j
    assert np.linalg.norm(sym.matvec(x) - Ds @ x) <= 1e-13 * np.linalg.norm(Ds @ x)
    for H in (full, sym):
        assert np.linalg.norm(H.matvec(x) - M @ x) <= 1e-5 * np.linalg.norm(M @ x)


@pytest.mark.slow
def test_storage_grows_like_n_log_n():
    """The complexity statement of the paper's cost section: O(N log N) storage with a fast method."""
    out = {}
    for n in (2000, 8000):
        P = _fib_sphere(n)
        h = np.sqrt(4 * np.pi / n)
        T = L.cluster_tree(P, P - h / 2, P + h / 2, leaf=32)
        H = L.compress(_laplace(P, P), T, T, 1.0, 1e-4, symmetric=True)
        out[n] = H.storage()
    assert out[8000] / 8000**2 < 0.5 * out[2000] / 2000**2  # far from dense growth
    per = {n: out[n] / (n * np.log2(n)) for n in out}
    assert per[8000] < 1.5 * per[2000]


# ---------------------------------------------------------------- the EFIE operators (Sec. 4)

EPS = 1e-4  # the paper's ACA tolerance


def _sphere(memo):
    def make():
        m = synth.geodesic_sphere(8)  # 1920 RWG functions, 1280 cells
        D = efie.discretize(m.verts, m.tris)
        return D, rfcmp.factors(D)

    return memo(("lowrank_sphere8",), make)


def _ops(memo, k):
    D, _ = _sphere(memo)
    return memo(("lowrank_sphere8_ops", k), lambda: efie.assemble(D, k))


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.slow
def test_separate_compression_keeps_the_vector_potential_at_low_frequency(memo):
    """Compressing T whole at 1e-4 loses i k T_A against Sigma V Sigma^T / (i k) at ka = 1e-3;
    compressing T_A and V apart keeps the LU current within a few eps."""
    D, _ = _sphere(memo)
    k = 1e-3
    TA, V = _ops(memo, k)
    C = L.compress_efie(D, TA, V, eps=EPS)
    assert C.TA.storage() < 0.5 * TA.size and C.V.storage() < 0.5 * V.size
    x = np.random.default_rng(4).standard_normal(D.N) + 0j
    assert _rel(C.TA.matvec(x), TA @ x) <= EPS
    xs = np.random.default_rng(5).standard_normal(D.nc) + 0j
    assert _rel(C.V.matvec(xs), V @ xs) <= EPS
    kh, pol = synth.plane_wave_z()
    e = efie.excitation(D, k, kh, pol)
    T = efie.efie_matrix(D, TA, V, k)
    j = krylov.lu_solve(T, -e)
    j_sep = krylov.lu_solve(efie.efie_matrix(D, C.TA.to_dense(), C.V.to_dense(), k), -e)
    assert _rel(j_sep, j) <= 5 * EPS
    whole = L.compress(lambda r, c: T[np.ix_(r, c)], C.edge_tree, C.edge_tree, 1.0, EPS, symmetric=True)
    j_whole = krylov.lu_solve(whole.to_dense(), -e)
    assert _rel(j_whole, j) > 0.1


@pytest.mark.slow
@pytest.mark.parametrize("k", [1.0, 1e-5])
def test_rfcmp_on_compressed_operators_matches_the_dense_solve(memo, k):
    """The RF-CMP system built from the compressed pair is Hermitian positive definite as the
    dense one (the compressed T_A, V are exactly complex symmetric) and gives its current."""
    D, F = _sphere(memo)
    TA, V = _ops(memo, k)
    C = L.compress_efie(D, TA, V, eps=EPS)
    TAc, Vc = C.TA.to_dense(), C.V.to_dense()
    assert np.array_equal(TAc, TAc.T) and np.array_equal(Vc, Vc.T)
    kh, pol = synth.plane_wave_z()
    e = efie.excitation(D, k, kh, pol)
    sc = rfcmp.power_scaling(F, TA, V, k)
    j, it, _ = rfcmp.solve(F, TA, V, k, sc, e, 1e-10)
    jc, itc, _ = rfcmp.solve(F, TAc, Vc, k, sc, e, 1e-10)
    assert _rel(jc, j) <= 5 * EPS
    assert abs(itc - it) <= 2
