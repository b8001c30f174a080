"""Serving on the GPU: each result is the oracle's current, and the same alone and in the mix.

Requests for one operator share a running batch session: later ones join it between refinement
sweeps, so a served current comes out of a solve whose membership changed while it ran.  Each
is held to the oracle's LU solution of T j = -e (Sec. 2) and to a standalone solve.
"""

import numpy as np
import pytest

import synth
from oracle import efie, krylov

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1803_08333_gb300 import serve  # noqa: E402
import paper_1803_08333_gb300 as rf  # noqa: E402


def test_results_alone_equal_results_in_the_mix(memo):
    from paper_1803_08333_gb300 import build

    build.build()
    meshes = [synth.geodesic_sphere(4, seed=1), synth.cube(4), synth.ellipsoid(3)]
    names = ["l2", "cube4", "ell3"]
    rng = np.random.default_rng(12)
    jobs = []
    for i in range(12):
        m = meshes[i % 3]
        k = [0.5, 1e-3, 1.7][i % 3]
        nr = int(rng.integers(1, 24))
        kh, pol = synth.random_plane_waves(nr, seed=100 + i)
        jobs.append((m, k, kh, pol))
    be = serve.GpuBackend(0)
    srv = serve.Server(be, hbm_budget=0, workers=2)
    futs = [srv.submit(m.verts, m.tris, k, kh, pol, tol=1e-10) for (m, k, kh, pol) in jobs]
    res = [f.result(timeout=600) for f in futs]
    st = srv.stats()
    srv.close()
    assert st["requests"] == 12 and st["mean_batch_columns"] >= 1
    assert st["mean_batch_columns"] > np.mean([len(j[2]) for j in jobs])  # requests shared solves
    ctx = rf.Context(0)
    for i, ((m, k, kh, pol), r) in enumerate(zip(jobs, res)):
        D = memo(("srv_disc", names[i % 3]), lambda: efie.discretize(m.verts, m.tris))
        TA, V = memo(("srv_op", names[i % 3], k), lambda: efie.assemble(D, k))
        J = krylov.lu_solve(efie.efie_matrix(D, TA, V, k), -efie.excitation(D, k, kh, pol)).T
        for c in range(len(kh)):
            assert np.linalg.norm(r.j[c] - J[c]) <= 1e-6 * np.linalg.norm(J[c]), (i, c)
        op = rf.Operator(ctx, m.verts, m.tris, k)
        j, rep = op.solve(op.rhs_planewave(kh, pol), tol=1e-10)
        alone = j.cpu().numpy()
        assert all(x <= 1e-10 for x in r.residuals)
        err = np.linalg.norm(r.j - alone) / np.linalg.norm(alone)
        # both solve the same system to relative residual 1e-10; merged columns take the
        # multi-column (tensor-core) products and their own rounding, so they agree to about
        # cond * 1e-10, with cond below 1e3 for these meshes
        assert err <= 1e-7, err
        op.close()


def test_trim_releases_wide_buffers_and_rebuilds_them():
    ctx = rf.Context(0)
    m = synth.geodesic_sphere(5, seed=2)
    op = rf.Operator(ctx, m.verts, m.tris, 0.9)
    kh, pol = synth.random_plane_waves(12, seed=5)
    e = op.rhs_planewave(kh, pol)
    j1, r1 = op.solve(e, tol=1e-9)  # 12 columns: planes and digits get built
    wide = ctx.bytes_in_use()
    op.trim()
    assert ctx.bytes_in_use() < wide
    j2, r2 = op.solve(e, tol=1e-9)
    assert ctx.bytes_in_use() == wide
    assert all(r.converged for r in r1 + r2)
    assert (torch.linalg.norm(j2 - j1) / torch.linalg.norm(j1)).item() <= 1e-8
    op.close()
    ctx.close()
