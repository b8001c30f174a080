"""Kernel plans on the GPU: launch shapes change timing, not results; the tuner runs end to end."""

import math

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1803_08333_gb300 as rf  # noqa: E402
from paper_1803_08333_gb300 import autotune as at  # noqa: E402


@pytest.fixture(scope="module")
def op():
    from paper_1803_08333_gb300 import build

    build.build()
    ctx = rf.Context(0)
    m = synth.geodesic_sphere(6, seed=1)  # 1080 unknowns: several GEMV work units per row at 256 columns
    o = rf.Operator(ctx, m.verts, m.tris, 0.7)
    yield o
    o.close()
    ctx.close()


def _x(n, nr, seed):
    g = torch.Generator().manual_seed(seed)
    return torch.complex(torch.randn(nr, n, generator=g, dtype=torch.float64),
                         torch.randn(nr, n, generator=g, dtype=torch.float64)).cuda()


def _rel(a, b):
    return (torch.linalg.norm(a - b) / torch.linalg.norm(b)).item()


def test_float_float_products_do_not_depend_on_the_gemv_shape(op):
    x = _x(op.N, 3, 1)
    op.set_plan(None)
    ref = op.apply("A", x)
    for plan in ({"gemv_chunk": 256, "gemv_ctas_per_sm": 1}, {"gemv_chunk": 4096, "gemv_ctas_per_sm": 4}):
        op.set_plan(plan)
        assert op.plan()["gemv_chunk"] == plan["gemv_chunk"]
        assert _rel(op.apply("A", x), ref) <= 1e-12
    op.set_plan(None)


@pytest.mark.parametrize("nr", [2, 20])
def test_inner_products_agree_on_gemv_and_tensor_cores(op, nr):
    """FP32 GEMV vs split-BF16 GEMM (any N tile) vs the float-float operator: the split products
    carry about 2^-16 relative error per product, the FP32 GEMV about 2^-24."""
    x = _x(op.N, nr, 2)
    op.set_plan(None)
    exact = op.apply("A", x)
    op.set_plan({"mrhs_min": 65536})
    assert _rel(op.apply("A_INNER", x), exact) <= 1e-5
    for bn in (32, 64, 128):
        op.set_plan({"mrhs_min": 1, "gemm_bn": bn})
        assert _rel(op.apply("A_INNER", x), exact) <= 2e-4
    op.set_plan(None)


def test_invalid_plans_are_rejected(op):
    for bad in ({"gemm_bn": 48}, {"gemv_chunk": 300}, {"gemv_ctas_per_sm": 9}, {"far_min_blocks": 5}):
        with pytest.raises(rf.RfcmpError):
            op.set_plan(bad)
    assert op.plan() == {k: 0 for k in rf.Plan.KEYS}


def test_tuner_and_tuned_solve(op, tmp_path):
    entries = at.tune_operator(op, [1, 16], "mixed", reps=2)
    assert [e.nrhs for e in entries] == [1, 16]
    for e in entries:
        assert math.isfinite(e.ms) and e.ms <= e.default_ms * 1.5
        rf.Plan.of(e.plan)  # valid fields
    t = at.Table(torch.cuda.get_device_name(0), entries)
    t.save(str(tmp_path / "t.json"))
    op.tuning = at.Table.load(str(tmp_path / "t.json"))
    kh, pol = synth.random_plane_waves(16, seed=3)
    e = op.rhs_planewave(kh, pol)
    j1, r1 = op.solve(e, tol=1e-8)
    op.tuning = None
    op.set_plan(None)
    j0, r0 = op.solve(e, tol=1e-8)
    assert all(r.converged for r in r0 + r1)
    assert _rel(j1, j0) <= 1e-6  # both at residual 1e-8 of a well-conditioned system


def test_far_pair_register_budgets_assemble_the_same_matrix():
    ctx = rf.Context(0)
    m = synth.geodesic_sphere(5, seed=4)
    mats = []
    for b in (1, 2, 3, 4):
        ctx.set_plan({"far_min_blocks": b})
        o = rf.Operator(ctx, m.verts, m.tris, 1.3, scaling="k")
        mats.append(o.export("T_A").cpu().numpy())
        o.close()
    ctx.set_plan(None)
    for M in mats[1:]:
        assert np.linalg.norm(M - mats[0]) <= 1e-6 * np.linalg.norm(mats[0])
    best, times = at.tune_assembly(ctx, m.verts, m.tris, 1.3, reps=1)
    assert best in (1, 2, 3, 4) and all(t > 0 for t in times.values())
    ctx.close()
