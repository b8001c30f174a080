"""Pins of the oracle's theory variant of the outer preconditioner (Sec. 3, Eq. Pgs).

P_gS = Sigma (Sigma^T Sigma)^+ G_l~p^{-1} Sigma^T with the mixed Gram matrix G_l~p of the dual
piecewise linear functions and the primal pulses.  The oracle integrates the dual functions over
the barycentric sub-triangles (their definition, Sec. 2); these tests hold it to the closed-form
case formula the paper prints for G_l~p (Sec. 3), to the partition of unity of the dual functions
(every column sums to 1) and to symmetry and diagonal dominance, and hold the P_gS system to the
paper's statements: Hermitian positive definite, bounded as k -> 0, and the same current as the
plain EFIE (j = -T^{-1} e).
"""

import numpy as np
import pytest

import synth
from oracle import efie, gram, krylov, rfcmp, topology


MESHES = {
    "sphere": lambda: synth.geodesic_sphere(3, seed=7),  # valences 5 and 6
    "cube": lambda: synth.cube(3),  # valences 3 to 6
    "torus": lambda: synth.torus(8, 6, jitter=0.03),  # genus 1
    "ellipsoid": lambda: synth.ellipsoid(3),
}


def _disc(memo, name):
    def make():
        m = MESHES[name]()
        return efie.discretize(m.verts, m.tris)

    return memo(("gs_disc", name), make)


def _paper_formula(D):
    """G_l~p from the case formula of Sec. 3: entries 2/18 (9/2 + sum_i 1/NoC(v_i)) on the
    diagonal, 2/18 (1/2 + 1/NoC(e+) + 1/NoC(e-)) for cells sharing the edge (e+, e-),
    2/18 (1/NoC(v)) for cells sharing only the vertex v, 0 otherwise."""
    tris = [set(int(v) for v in t) for t in D.tris]
    noc = np.bincount(D.tris.ravel(), minlength=D.nv)
    G = np.zeros((D.nc, D.nc))
    for m in range(D.nc):
        for n in range(D.nc):
            common = tris[m] & tris[n]
            if m == n:
                G[m, n] = 2 / 18 * (9 / 2 + sum(1 / noc[v] for v in tris[m]))
            elif len(common) == 2:
                a, b = sorted(common)
                G[m, n] = 2 / 18 * (1 / 2 + 1 / noc[a] + 1 / noc[b])
            elif len(common) == 1:
                (v,) = common
                G[m, n] = 2 / 18 * (1 / noc[v])
    return G


@pytest.mark.parametrize("name", ["sphere", "cube", "torus", "ellipsoid"])
def test_gtp_matches_the_printed_formula_and_sums_to_one(memo, name):
    D = _disc(memo, name)
    G = gram.g_lambda_tilde_p(D).toarray()
    assert np.abs(G - _paper_formula(D)).max() <= 1e-15
    # partition of unity of the dual piecewise linear functions: sum_m lambda~_m = 1
    assert np.abs(G.sum(axis=0) - 1.0).max() <= 1e-14
    assert np.abs(G - G.T).max() <= 1e-15
    off = np.abs(G).sum(axis=1) - np.diag(G)
    assert (np.diag(G) > off).all()  # strictly diagonally dominant, hence positive definite
    assert np.linalg.eigvalsh(G)[0] > 0


def test_pgs_is_an_oblique_map_onto_the_star_space(memo):
    D = _disc(memo, "sphere")
    F = memo(("gs_fac", "sphere"), lambda: rfcmp.factors(D))
    # range in range(Sigma), loops annihilated (Sigma^T Lambda = 0), P_S P_gS = P_gS
    assert np.abs(F.P_gS @ F.Lambda).max() <= 1e-12
    assert np.abs(F.P_S @ F.P_gS - F.P_gS).max() <= 1e-12
    # but not the orthogonal projector itself: neither idempotent nor Hermitian
    assert np.abs(F.P_gS @ F.P_gS - F.P_gS).max() > 1e-3
    assert np.abs(F.P_gS - F.P_gS.T).max() > 1e-3


@pytest.mark.parametrize("k", [1.0, 1e-2, 1e-5])
def test_gsigma_system_hpd_and_bounded(memo, k):
    D = _disc(memo, "sphere")
    F = memo(("gs_fac", "sphere"), lambda: rfcmp.factors(D))
    TA, V = memo(("gs_op", k), lambda: efie.assemble(D, k))
    T = efie.efie_matrix(D, TA, V, k)
    sc = rfcmp.kscale(k)  # the scaling of Sec. 3: alpha = sqrt k, beta = 1/sqrt k, gamma = k
    A, _, _ = rfcmp.dense_system(F, T, sc, "gsigma")
    ev = np.linalg.eigvalsh(0.5 * (A + A.conj().T))
    assert ev[0] > 0
    assert ev[-1] / ev[0] < 20  # bounded independently of k (Sec. 3)


def test_gsigma_structured_equals_dense_and_solution_equals_lu(memo):
    D = _disc(memo, "sphere")
    F = memo(("gs_fac", "sphere"), lambda: rfcmp.factors(D))
    k = 1.0
    TA, V = memo(("gs_op", k), lambda: efie.assemble(D, k))
    T = efie.efie_matrix(D, TA, V, k)
    sc = rfcmp.kscale(k)
    A, Bmap, Po = rfcmp.dense_system(F, T, sc, "gsigma")
    rng = np.random.default_rng(3)
    x = rng.standard_normal(D.N) + 1j * rng.standard_normal(D.N)
    ref = A @ x
    assert np.linalg.norm(rfcmp.apply_A_gsigma(F, TA, V, k, sc, x) - ref) <= 1e-12 * np.linalg.norm(ref)
    e = efie.excitation(D, k, [[0.0, 0.0, 1.0]], [[1.0, 0.0, 0.0]])[:, 0]
    b = Bmap @ e
    assert np.linalg.norm(rfcmp.apply_rhs_gsigma(F, TA, V, k, sc, e) - b) <= 1e-12 * np.linalg.norm(b)
    j, _, _ = rfcmp.solve(F, TA, V, k, sc, e, 1e-12, outer="gsigma")
    jl = krylov.lu_solve(T, -e)
    assert np.linalg.norm(j - jl) <= 1e-10 * np.linalg.norm(jl)
    js, _, _ = rfcmp.solve(F, TA, V, k, sc, e, 1e-12)  # the numerical variant reaches the same current
    assert np.linalg.norm(js - jl) <= 1e-10 * np.linalg.norm(jl)


def test_torus_gsigma_solution(memo):
    # multiply connected: P_LH carries the quasi-harmonic part, P_gS maps onto stars only
    D = _disc(memo, "torus")
    assert D.top.genus == 1
    F = memo(("gs_fac", "torus"), lambda: rfcmp.factors(D))
    k = 2.0
    TA, V = efie.assemble(D, k)
    T = efie.efie_matrix(D, TA, V, k)
    e = efie.excitation(D, k, [[0.0, 0.0, 1.0]], [[1.0, 0.0, 0.0]])[:, 0]
    j, _, _ = rfcmp.solve(F, TA, V, k, rfcmp.kscale(k), e, 1e-12, outer="gsigma")
    jl = krylov.lu_solve(T, -e)
    assert np.linalg.norm(j - jl) <= 1e-9 * np.linalg.norm(jl)
