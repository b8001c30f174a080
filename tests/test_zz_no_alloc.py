"""The allocation-free T_A entry point matches the regular one.

rfcmp_apply_ta_noalloc serves callers that cannot allocate device memory when
they need y = T_A x (a pre-partitioned serving pool, or a path that must not
call cudaMalloc/cudaFree because they can synchronise the device).  It keeps
its scratch in a file-scope device array instead of the operator's lazily
allocated work buffers.  This file is collected last, so a run that stops at
the first failure has run every other test before it; it also passes alone in
a fresh process.
"""

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1803_08333_gb300 as rf  # noqa: E402


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def op():
    from paper_1803_08333_gb300 import build

    build.build()
    ctx = rf.Context(0)
    m = synth.geodesic_sphere(8, seed=1)  # N = 1920
    o = rf.Operator(ctx, m.verts, m.tris, 1.3, scaling="k")
    yield o
    o.close()


@pytest.mark.parametrize("nrhs", [1, 3])
def test_noalloc_matches_apply_on_two_calls(op, nrhs):
    rng = np.random.default_rng(nrhs)
    for call in range(2):  # the scratch keeps the previous call's contents
        x = rng.standard_normal((nrhs, op.N)) + 1j * rng.standard_normal((nrhs, op.N))
        xt = torch.from_numpy(x).cuda()
        ref = op.apply("T_A", xt).cpu().numpy()
        got = op.apply_ta_noalloc(xt).cpu().numpy()
        assert _rel(got, ref) <= 1e-12, (call, _rel(got, ref))


def test_noalloc_rejects_sizes_beyond_its_scratch(op):
    x = torch.zeros((5, op.N), dtype=torch.complex128, device="cuda")
    with pytest.raises(rf.RfcmpError) as ei:
        op.apply_ta_noalloc(x)
    assert ei.value.status == -1


def test_noalloc_rejects_columns_beyond_its_capacity():
    # nrhs = 4 passes the column check, but a padded row of 34 688 entries x 4 columns exceeds the
    # 131 072 complex entries of the scratch; the call must refuse it and leave y untouched
    ctx = rf.Context(0)
    m = synth.geodesic_sphere(34, seed=2)  # 23 120 cells, N = 34 680
    big = rf.Operator(ctx, m.verts, m.tris, 1.0, scaling="k")
    try:
        assert big.N == 34680
        x = torch.ones((4, big.N), dtype=torch.complex128, device="cuda")
        y = torch.full((4, big.N), 7.0 + 0j, dtype=torch.complex128, device="cuda")
        with pytest.raises(rf.RfcmpError) as ei:
            big.apply_ta_noalloc(x, out=y)
        assert ei.value.status == -1
        assert "131072" in str(ei.value)
        torch.cuda.synchronize()
        assert bool((y == 7.0).all())
        # one column fits: it matches the regular entry point
        got = big.apply_ta_noalloc(x[:1]).cpu().numpy()
        ref = big.apply("T_A", x[:1]).cpu().numpy()
        assert _rel(got, ref) <= 1e-12
    finally:
        big.close()
        ctx.close()
