"""The theory variant of the outer preconditioner on the GPU (Sec. 3, Eq. Pgs).

P_o = P_LH / alpha + i P_gS / beta with P_gS = Sigma (Sigma^T Sigma)^+ G_l~p^{-1} Sigma^T.  The
library builds G_l~p from the case formula of Sec. 3 and its dense inverse by Newton-Schulz
refinement from a Jacobi start; the oracle integrates the dual functions and inverts densely.
Held to the oracle: the factor (1e-11), P_gS, P_o and P_o^H (1e-11), the application of A (1e-9
against the oracle's composition over the library's own stored matrices), and the current of a
solve (1e-6 against the oracle's LU solution, and against the numerical variant's current).
"""

import numpy as np
import pytest

import synth
from oracle import efie, krylov, rfcmp

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1803_08333_gb300 as rf  # noqa: E402

MESHES = {
    "l2": lambda: synth.geodesic_sphere(4, seed=1),  # 320 cells, N = 480
    "torus": lambda: synth.torus(6, 10, jitter=0.02),  # genus 1
    "cube": lambda: synth.cube(4),  # valences 3 to 6
}


@pytest.fixture(scope="module")
def ctx():
    from paper_1803_08333_gb300 import build

    build.build()
    yield rf.Context(0)


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _case(memo, name, k):
    m = MESHES[name]()
    D = memo(("gsg_disc", name), lambda: efie.discretize(m.verts, m.tris))
    F = memo(("gsg_fac", name), lambda: rfcmp.factors(D))
    TA, V = memo(("gsg_op", name, k), lambda: efie.assemble(D, k))
    return m, D, F, TA, V


@pytest.mark.parametrize("name", ["l2", "torus", "cube"])
def test_gtp_inverse_factor(ctx, memo, name):
    m, D, F, _, _ = _case(memo, name, 1.0)
    op = rf.Operator(ctx, m.verts, m.tris, 1.0, scaling="k", outer="gsigma")
    assert _rel(op.export("GTP_INV").cpu().numpy(), F.Gtp_inv) <= 1e-11


@pytest.mark.parametrize("name,k", [("l2", 1.0), ("l2", 1e-3), ("torus", 1.5), ("cube", 0.5)])
def test_gsigma_application_and_preconditioners(ctx, memo, name, k):
    m, D, F, TA, V = _case(memo, name, k)
    sc = rfcmp.kscale(k)
    op = rf.Operator(ctx, m.verts, m.tris, k, scaling="k", outer="gsigma")
    gTA = op.export("T_A").cpu().numpy().astype(np.complex128)
    gV = op.export("V").cpu().numpy().astype(np.complex128)
    rng = np.random.default_rng(5)
    x = rng.standard_normal((6, op.N)) + 1j * rng.standard_normal((6, op.N))
    wide = op.apply("A", torch.from_numpy(x)).cpu().numpy()  # 6 columns: exact-digit products
    x = x[:2]
    got = op.apply("A", torch.from_numpy(x)).cpu().numpy()
    for c in range(2):
        assert _rel(wide[c], got[c]) <= 1e-11
        assert _rel(got[c], rfcmp.apply_A_gsigma(F, gTA, gV, k, sc, x[c])) <= 1e-9
        assert _rel(got[c], rfcmp.apply_A_gsigma(F, TA, V, k, sc, x[c])) <= 1e-5
    Po, _ = rfcmp.preconditioners(F, sc, "gsigma")
    for which, M in (("P_GSIGMA", F.P_gS), ("P_O", Po), ("P_O_ADJ", Po.conj().T)):
        y = op.precondition(which, torch.from_numpy(x)).cpu().numpy()
        assert _rel(y.T, M @ x.T) <= 1e-11, which


@pytest.mark.parametrize("name,k", [("l2", 1.0), ("torus", 2.0), ("cube", 0.7)])
def test_gsigma_solution_matches_lu(ctx, memo, name, k):
    m, D, F, TA, V = _case(memo, name, k)
    kh, pol = synth.random_plane_waves(3, seed=8)
    J = krylov.lu_solve(efie.efie_matrix(D, TA, V, k), -efie.excitation(D, k, kh, pol)).T
    op = rf.Operator(ctx, m.verts, m.tris, k, scaling="k", outer="gsigma")
    e = op.rhs_planewave(kh, pol)
    for precision in ("mixed", "ff"):
        j, rep = op.solve(e, tol=1e-10, precision=precision)
        assert all(r.converged for r in rep)
        jh = j.cpu().numpy()
        for c in range(3):
            assert _rel(jh[c], J[c]) <= 1e-6, (precision, c, _rel(jh[c], J[c]))


@pytest.mark.parametrize("k", [1e-2, 1e-5])
def test_gsigma_low_frequency_current_equals_the_numerical_variant(ctx, memo, k):
    m, D, F, TA, V = _case(memo, "l2", k)
    e_args = synth.plane_wave_z()
    opg = rf.Operator(ctx, m.verts, m.tris, k, scaling="k", outer="gsigma")
    ops = rf.Operator(ctx, m.verts, m.tris, k, scaling="k")
    jg, rg = opg.solve(opg.rhs_planewave(*e_args), tol=1e-10)
    js, rs = ops.solve(ops.rhs_planewave(*e_args), tol=1e-10)
    assert rg[0].converged and rs[0].converged
    # both at residual 1e-10 of well-conditioned systems (the same current, -T^{-1} e)
    assert _rel(jg.cpu().numpy(), js.cpu().numpy()) <= 1e-7
    # and the oracle's FP64 RF-CMP solve with P_gS
    jo, _, _ = rfcmp.solve(F, TA, V, k, rfcmp.kscale(k), efie.excitation(D, k, *e_args)[:, 0], 1e-12,
                           outer="gsigma")
    assert _rel(jg.cpu().numpy()[0], jo) <= 1e-6
