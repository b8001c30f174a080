"""Batched excitations: 512 plane waves in one multi-column solve.

Seeded uniform directions on S^2 with random polarisations on a PEC ellipsoid (semi-axes
1.0 / 0.6 / 0.4), ka = 2.  The inner iterations of a 512-column solve run on the split-BF16
tensor-core GEMM and the refinement residuals on the exact-digit GEMM, so these tests hold that
path to the solution tolerance of 1e-6:
  * 1920 unknowns: four sampled columns against the oracle's dense LU solution;
  * 7680 unknowns: four sampled columns against the same columns solved one at a time in the
    float-float single-column form (itself held to the oracle in test_gpu_parity.py).
"""

import numpy as np
import pytest

import synth
from oracle import efie, krylov

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1803_08333_gb300 as rf  # noqa: E402

KA = 2.0
SAMPLE = [0, 137, 290, 511]


@pytest.fixture(scope="module")
def ctx():
    from paper_1803_08333_gb300 import build

    build.build()
    yield rf.Context(0)


def _rel_cols(a, b):
    return np.linalg.norm(a - b, axis=1) / np.linalg.norm(b, axis=1)


def test_512_columns_match_oracle_lu(ctx):
    m = synth.ellipsoid(8, seed=3)  # 1280 cells, N = 1920
    kh, pol = synth.random_plane_waves(512, seed=33)
    op = rf.Operator(ctx, m.verts, m.tris, KA)
    e = op.rhs_planewave(kh, pol)
    j, rep = op.solve(e, tol=1e-9)
    assert all(r.converged and r.residual <= 1e-9 for r in rep)
    D = efie.discretize(m.verts, m.tris)
    TA, V = efie.assemble(D, KA)
    E = efie.excitation(D, KA, kh[SAMPLE], pol[SAMPLE])
    J = krylov.lu_solve(efie.efie_matrix(D, TA, V, KA), -E).T
    err = _rel_cols(j.cpu().numpy()[SAMPLE], J)
    assert err.max() <= 1e-6, err


def test_512_columns_match_single_column_solves(ctx):
    m = synth.ellipsoid(16, seed=3)  # 5120 cells, N = 7680
    kh, pol = synth.random_plane_waves(512, seed=33)
    op = rf.Operator(ctx, m.verts, m.tris, KA)
    e = op.rhs_planewave(kh, pol)
    j, rep = op.solve(e, tol=1e-9)
    assert all(r.converged and r.residual <= 1e-9 for r in rep)
    js = []
    for c in SAMPLE:
        jc, rc = op.solve(e[c : c + 1], tol=1e-10, precision="ff")
        assert rc[0].converged
        js.append(jc.cpu().numpy()[0])
    err = _rel_cols(j.cpu().numpy()[SAMPLE], np.array(js))
    assert err.max() <= 1e-6, err
