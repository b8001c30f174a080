"""Open surfaces on the GPU (Sec. 2: loop functions of the inner vertices only).

RWG functions on the edges shared by two cells, loop functions on the interior vertices, G_ll the
P1 mass matrix restricted to them.  Held to the oracle: T_A and V (1e-5, real and imaginary parts
separately), the factors (1e-11), P_o (1e-11), the application of A against the oracle's
composition over the library's own stored matrices (1e-9), the currents against the oracle's LU
solution (1e-6, mixed and float-float, down to ka = 1e-3), and the RCS (1e-3 dB).  Meshes: a
plate (disk), a curved cap, an open cylinder (two boundary curves, one harmonic field).
"""

import numpy as np
import pytest

import synth
from oracle import efie, farfield, krylov, rfcmp

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1803_08333_gb300 as rf  # noqa: E402

MESHES = {
    "plate": lambda: synth.plate(12),  # 288 cells, 408 unknowns, 121 loop functions
    "cap": lambda: synth.plate(10, bow=0.15, seed=9),
    "cylinder": lambda: synth.open_cylinder(16, 8),  # 256 cells, 368 unknowns
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
    D = memo(("open_gdisc", name), lambda: efie.discretize(m.verts, m.tris))
    F = memo(("open_gfac", name), lambda: rfcmp.factors(D))
    TA, V = memo(("open_gop", name, k), lambda: efie.assemble(D, k))
    return m, D, F, TA, V


@pytest.mark.parametrize("name,k", [("plate", 1.0), ("plate", 1e-3), ("cap", 2.0), ("cylinder", 1.5)])
def test_open_surface_operator_and_factors(ctx, memo, name, k):
    m, D, F, TA, V = _case(memo, name, k)
    op = rf.Operator(ctx, m.verts, m.tris, k, scaling="k")
    info = op.info()
    assert (info.n_edges, info.n_cells, info.n_vertices) == (D.N, D.nc, D.top.nvl)
    assert info.boundaries == D.top.boundaries and info.genus == 0
    ev, ec = op.edges()
    assert np.array_equal(ev, D.top.edge_verts) and np.array_equal(ec, D.top.edge_cells)
    gTA = op.export("T_A").cpu().numpy().astype(np.complex128)
    gV = op.export("V").cpu().numpy().astype(np.complex128)
    for got, ref in ((gTA, TA), (gV, V)):
        assert _rel(got.real, ref.real) <= 1e-5 and _rel(got.imag, ref.imag) <= 1e-5
    assert _rel(op.export("LPLUS").cpu().numpy(), F.Lplus) <= 1e-11
    assert _rel(op.export("GLL_INV").cpu().numpy(), F.Gll_inv) <= 1e-11
    sc = rfcmp.kscale(k)
    rng = np.random.default_rng(6)
    x = rng.standard_normal((2, op.N)) + 1j * rng.standard_normal((2, op.N))
    got = op.apply("A", torch.from_numpy(x)).cpu().numpy()
    for c in range(2):
        assert _rel(got[c], rfcmp.apply_A(F, gTA, gV, k, sc, x[c])) <= 1e-9
    Po, _ = rfcmp.preconditioners(F, sc)
    y = op.precondition("P_O", torch.from_numpy(x)).cpu().numpy()
    assert _rel(y.T, Po @ x.T) <= 1e-11


@pytest.mark.parametrize("name,k", [("plate", 1.0), ("plate", 1e-3), ("cap", 2.0), ("cylinder", 1.5)])
def test_open_surface_currents_match_lu(ctx, memo, name, k):
    m, D, F, TA, V = _case(memo, name, k)
    kh, pol = synth.random_plane_waves(3, seed=14)
    J = krylov.lu_solve(efie.efie_matrix(D, TA, V, k), -efie.excitation(D, k, kh, pol)).T
    op = rf.Operator(ctx, m.verts, m.tris, k)
    e = op.rhs_planewave(kh, pol)
    assert _rel(e.cpu().numpy().T, efie.excitation(D, k, kh, pol)) <= 1e-12
    for precision in ("mixed", "ff"):
        j, rep = op.solve(e, tol=1e-10, precision=precision)
        assert all(r.converged for r in rep), rep
        jh = j.cpu().numpy()
        # LU of T at k = 1e-3 carries cond(T) eps, about 1e-8
        for c in range(3):
            assert _rel(jh[c], J[c]) <= 1e-6, (precision, c, _rel(jh[c], J[c]))
    if k >= 1.0:
        th = np.linspace(0, np.pi, 91)
        dirs = farfield.cut_directions(th, 0.4)
        ref = farfield.bistatic_rcs(D, J[0], k, dirs)
        got = op.farfield(j[:1], dirs)[0]
        keep = ref > ref.max() * 1e-4
        assert np.abs(got[keep] - 10 * np.log10(ref[keep])).max() <= 1e-3


def test_open_surface_refusals(ctx):
    m = MESHES["plate"]()
    with pytest.raises(rf.RfcmpError):  # the theory variant needs a closed surface
        rf.Operator(ctx, m.verts, m.tris, 1.0, outer="gsigma")
    s = synth.plate(1)  # two cells: every vertex on the boundary, no loop function
    with pytest.raises(rf.RfcmpError):
        rf.Operator(ctx, s.verts, s.tris, 1.0)


def test_large_plate_factor_build_and_solve(ctx):
    """The 100 x 100 plate (20000 cells, 29800 unknowns): the Newton-Schulz refinement of
    (Sigma^T Sigma)^+ floors near a 1e-12 residual on this open surface and must be kept there
    (not fall back or fail), and the solve converges at ka = 1 and 1e-4."""
    m = synth.plate(100, seed=7)
    for k in (1.0, 1e-4):
        op = rf.Operator(ctx, m.verts, m.tris, k)
        assert op.N == 29800 and op.info().boundaries == 1
        j, rep = op.solve(op.rhs_planewave(*synth.plane_wave_z()), tol=1e-6)
        assert rep[0].converged and rep[0].residual <= 1e-6, rep
        op.close()
