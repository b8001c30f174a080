"""The device-resident solve loop (Sec. 4: CG on the RF-CMP system with accurate refinement).

The loop runs either as one CUDA graph per op (refinement sweeps and CG iterations as nested
WHILE conditional nodes whose conditions the solve's kernels set on the device) or eagerly, the
same kernels launched one by one.  The loop's own reductions are fixed-order, but the GEMVs add
FP64 partials of different CTAs with atomics, whose order follows the timing: the two drivers
agree to the accuracy of the solve, iteration for iteration, and both must meet the oracle.
"""

import numpy as np
import pytest

import synth
from oracle import efie, krylov

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1803_08333_gb300 as rf  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    from paper_1803_08333_gb300 import build

    build.build()
    yield rf.Context(0)
    rf.set_solve_graphs(True)


def _solve_both(op, e, **kw):
    prev = rf.set_solve_graphs(True)
    try:
        jg, rg = op.solve(e, **kw)  # also builds what wide products need on first use
        l0 = rf.launch_count()
        jg2, rg2 = op.solve(e, **kw)  # replays the captured graph
        lg = rf.launch_count() - l0
        rf.set_solve_graphs(False)
        l0 = rf.launch_count()
        je, re_ = op.solve(e, **kw)
        le = rf.launch_count() - l0
    finally:
        rf.set_solve_graphs(prev)
    return (jg, rg, lg), (jg2, rg2), (je, re_, le)


def _same_reports_iters(a, b):
    return [(r.iterations, r.refinements) for r in a] == [(r.iterations, r.refinements) for r in b]


@pytest.mark.parametrize("nr,precision", [(1, "mixed"), (2, "mixed"), (6, "mixed"), (1, "ff"), (5, "ff")])
def test_graph_and_eager_loops_agree(ctx, nr, precision):
    m = synth.geodesic_sphere(4, seed=1)  # N = 480
    op = rf.Operator(ctx, m.verts, m.tris, 0.8)
    kh, pol = synth.random_plane_waves(nr, seed=21)
    e = op.rhs_planewave(kh, pol)
    (jg, rg, lg), (jg2, rg2), (je, re_, le) = _solve_both(op, e, tol=1e-8, precision=precision)
    for rep in (rg, rg2, re_):
        assert all(r.converged and r.residual <= 1e-8 for r in rep), rep
    for j in (jg2, je):
        assert float(torch.linalg.norm(j - jg) / torch.linalg.norm(jg)) <= 1e-7
    for rep in (rg2, re_):
        assert all(abs(a.iterations - b.iterations) <= 1 and a.refinements == b.refinements for a, b in zip(rg, rep))
    if _same_reports_iters(rg2, re_):
        assert lg == le  # the same kernels, whichever driver launched them


def test_graph_loop_matches_oracle_ff_and_mixed(ctx, memo):
    m = synth.geodesic_sphere(4, seed=1)
    k = 1.3
    D = memo(("kry_disc",), lambda: efie.discretize(m.verts, m.tris))
    TA, V = memo(("kry_op", k), lambda: efie.assemble(D, k))
    kh, pol = synth.random_plane_waves(3, seed=5)
    E = efie.excitation(D, k, kh, pol)
    J = krylov.lu_solve(efie.efie_matrix(D, TA, V, k), -E)
    op = rf.Operator(ctx, m.verts, m.tris, k)
    e = op.rhs_planewave(kh, pol)
    for precision in ("mixed", "ff"):
        j, rep = op.solve(e, tol=1e-10, precision=precision)
        jh = j.cpu().numpy().T
        err = np.linalg.norm(jh - J, axis=0) / np.linalg.norm(J, axis=0)
        assert err.max() <= 1e-6, (precision, err)
        assert all(r.converged and r.residual <= 1e-10 for r in rep)


def test_iteration_cap_and_refinement_cap(ctx):
    m = synth.geodesic_sphere(3, seed=2)
    op = rf.Operator(ctx, m.verts, m.tris, 1.0)
    e = op.rhs_planewave(*synth.plane_wave_z())
    for graphs in (True, False):
        prev = rf.set_solve_graphs(graphs)
        try:
            _, rep = op.solve(e, tol=1e-12, max_iter=3)
            assert rep[0].iterations == 3 and not rep[0].converged
            _, rep = op.solve(e, tol=1e-12, max_refine=0)
            assert rep[0].iterations == 0 and rep[0].refinements == 0
            _, rep = op.solve(e, tol=1e-12, max_refine=1, inner_tol=0.5)
            assert rep[0].refinements == 1
        finally:
            rf.set_solve_graphs(prev)


def test_profiling_inside_graphs(ctx):
    m = synth.geodesic_sphere(12, seed=3)  # N = 4320
    op = rf.Operator(ctx, m.verts, m.tris, 0.5)
    e = op.rhs_planewave(*synth.plane_wave_z())
    op.solve(e, tol=1e-6)  # warm: workspace and graph
    avg = {}
    for graphs in (True, False):
        prev = rf.set_solve_graphs(graphs)
        rf.profile_enable(True)
        try:
            _, rep = op.solve(e, tol=1e-6)
            prof = rf.profile_read()
        finally:
            rf.profile_enable(False)
            rf.set_solve_graphs(prev)
        fam = prof["gemv_c64_f32"]
        assert fam["launches"] >= 4 * rep[0].iterations
        avg[graphs] = fam["total_ms"] / fam["launches"]
    # device timestamps (graph) and CUDA events (eager) time the same launches
    assert 0.6 < avg[True] / avg[False] < 1.4, avg
