"""Pins of the oracle on open surfaces (Sec. 2: loop functions of the inner vertices only).

An edge used by one cell is a boundary edge and carries no RWG function; the loop functions
belong to the interior vertices.  Held to what the definitions fix: the dimension count
N = N_V + N_C - 1 + H with H = 2g + b - 1 harmonic fields (b boundary curves), Lambda of full
column rank, Sigma 1 = 0 and Lambda^T Sigma = 0, Lambda^T G_ff Lambda = the P1 stiffness matrix
of the interior vertices (Eq. PrimalLaplace); and the RF-CMP system: Hermitian positive
definite, its structured application equal to the dense one, its current equal to the LU
solution of T j = -e, and its condition number bounded as k -> 0 while cond(T) grows.
"""

import numpy as np
import pytest

import synth
from oracle import efie, gram, krylov, rfcmp

MESHES = {
    "plate": lambda: synth.plate(5),  # disk: H = 0
    "cap": lambda: synth.plate(5, bow=0.15, seed=9),  # curved disk
    "cylinder": lambda: synth.open_cylinder(8, 3),  # annulus: H = 1
}


def _disc(memo, name):
    return memo(("open_disc", name), lambda: efie.discretize(MESHES[name]().verts, MESHES[name]().tris))


@pytest.mark.parametrize("name,harmonic", [("plate", 0), ("cap", 0), ("cylinder", 1)])
def test_dimension_count_and_transforms(memo, name, harmonic):
    D = _disc(memo, name)
    t = D.top
    assert t.boundaries == (2 if name == "cylinder" else 1) and t.genus == 0
    assert t.nvl < t.nv  # the boundary vertices carry no loop function
    S, L = D.Sigma.toarray(), D.Lambda.toarray()
    assert np.abs(S @ np.ones(t.nc)).max() == 0.0  # every RWG edge has two cells
    assert np.linalg.matrix_rank(L) == t.nvl  # full column rank: no all-one null vector
    assert np.abs(L.T @ S).max() == 0.0
    rank = np.linalg.matrix_rank(np.hstack([L, S]))
    assert t.ne - rank == harmonic  # harmonic fields: 2g + b - 1
    assert t.ne == t.nvl + t.nc - 1 + harmonic
    # loop-loop Gram = P1 stiffness of the interior vertices (Eq. PrimalLaplace)
    K = L.T @ gram.g_ff(D).toarray() @ L
    assert np.abs(K - gram.stiffness_loops(D).toarray()).max() <= 1e-12 * np.abs(K).max()


def test_closed_surfaces_keep_every_vertex(memo):
    m = synth.geodesic_sphere(2, seed=1)
    D = efie.discretize(m.verts, m.tris)
    assert D.top.boundaries == 0 and D.top.nvl == D.top.nv
    assert np.array_equal(D.top.loop_verts, np.arange(D.top.nv))


@pytest.mark.parametrize("name,k", [("plate", 1.0), ("plate", 1e-3), ("cap", 2.0), ("cylinder", 1.5)])
def test_open_surface_rfcmp_solution_equals_lu(memo, name, k):
    D = _disc(memo, name)
    F = memo(("open_fac", name), lambda: rfcmp.factors(D))
    TA, V = memo(("open_op", name, k), lambda: efie.assemble(D, k))
    T = efie.efie_matrix(D, TA, V, k)
    sc = rfcmp.kscale(k)
    A, Bmap, Po = rfcmp.dense_system(F, T, sc)
    ev = np.linalg.eigvalsh(0.5 * (A + A.conj().T))
    assert ev[0] > 0  # Hermitian positive definite
    # Hermitian by construction; the rounding of the dense composition grows like 1/k^2 (the
    # same on closed surfaces: 3.5e-7 of the largest entry on a sphere at k = 1e-3)
    assert np.abs(A - A.conj().T).max() <= 1e-11 / k**2 * np.abs(A).max()
    if k >= 0.1:  # at low k the dense composition cancels; the structured form is the stable one
        rng = np.random.default_rng(4)
        x = rng.standard_normal(D.N) + 1j * rng.standard_normal(D.N)
        ref = A @ x
        assert np.linalg.norm(rfcmp.apply_A(F, TA, V, k, sc, x) - ref) <= 1e-11 * np.linalg.norm(ref)
    e = efie.excitation(D, k, [[0.0, 0.0, 1.0]], [[1.0, 0.0, 0.0]])[:, 0]
    j, _, _ = rfcmp.solve(F, TA, V, k, sc, e, 1e-12)
    jl = krylov.lu_solve(T, -e)
    # the LU solution of T carries cond(T) eps, about 1e-8 relative at k = 1e-3
    assert np.linalg.norm(j - jl) <= (1e-9 if k >= 0.1 else 1e-7) * np.linalg.norm(jl)


def test_open_surface_conditioning_is_frequency_stable(memo):
    D = _disc(memo, "plate")
    F = memo(("open_fac", "plate"), lambda: rfcmp.factors(D))
    conds, tconds = [], []
    for k in (1.0, 1e-2, 1e-4):
        TA, V = memo(("open_op", "plate", k), lambda: efie.assemble(D, k))
        T = efie.efie_matrix(D, TA, V, k)
        A, _, _ = rfcmp.dense_system(F, T, rfcmp.kscale(k))
        conds.append(np.linalg.cond(A))
        tconds.append(np.linalg.cond(T))
    assert max(conds) / min(conds) < 1.5  # bounded down to the static limit
    assert tconds[2] / tconds[0] > 1e6  # the plain EFIE: cond grows like 1/k^2
