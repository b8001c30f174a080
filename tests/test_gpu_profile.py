"""Profiling counters under long runs and concurrent use.

With profiling on, every instrumented launch is bracketed by a pair of CUDA events that the
library resolves in batches.  These tests run more launches of one kernel family than a batch
holds, and two threads that profile the same family at once, and then check that the next
ordinary call still succeeds and still matches the oracle: a profiling fault must never
surface as the failure of an unrelated launch.
"""

import threading

import numpy as np
import pytest

import synth
from oracle import efie

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1803_08333_gb300 as rf  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    from paper_1803_08333_gb300 import build

    build.build()
    yield rf.Context(0)


def _x(n, nr, seed):
    rng = np.random.default_rng(seed)
    return torch.from_numpy(rng.standard_normal((nr, n)) + 1j * rng.standard_normal((nr, n))).cuda()


def _ta_check(op, m, k):
    D = efie.discretize(m.verts, m.tris)
    TA, _ = efie.assemble(D, k)
    TA64 = op.export("T_A").cpu().numpy().astype(np.complex128)
    assert np.linalg.norm(TA64 - TA) / np.linalg.norm(TA) < 1e-5
    x = _x(op.N, 1, 5)
    y = op.apply("T_A", x).cpu().numpy()[0]
    ref = TA64 @ x.cpu().numpy()[0]
    assert np.linalg.norm(y - ref) / np.linalg.norm(ref) < 1e-12


def test_more_profiled_launches_than_one_batch(ctx):
    m = synth.geodesic_sphere(1, seed=9)  # 20 cells, N = 30
    op = rf.Operator(ctx, m.verts, m.tris, 1.0, scaling="k")
    x = _x(op.N, 1, 1)
    rf.profile_enable(True)
    try:
        for _ in range(5200):
            op.apply("T_A", x)
        prof = rf.profile_read()
    finally:
        rf.profile_enable(False)
    fam = max(prof.values(), key=lambda v: v["launches"])
    assert fam["launches"] >= 5200, prof
    assert fam["total_ms"] > 0.0
    # the next launches (and a whole solve) must not inherit an error from the counters
    _ta_check(op, m, 1.0)
    e = op.rhs_planewave(*synth.plane_wave_z())
    _, rep = op.solve(e, tol=1e-8)
    assert rep[0].converged


def test_two_threads_profile_one_family(ctx):
    m = synth.geodesic_sphere(2, seed=3)  # 80 cells, N = 120
    ops = [rf.Operator(ctx, m.verts, m.tris, 1.0, scaling="k") for _ in range(2)]
    errors = []

    def work(op, seed):
        try:
            s = torch.cuda.Stream()
            with torch.cuda.stream(s):
                x = _x(op.N, 1, seed)
                for _ in range(3000):
                    op.apply("T_A", x)
            s.synchronize()
        except Exception as exc:  # pragma: no cover - reported below
            errors.append(exc)

    rf.profile_enable(True)
    try:
        th = [threading.Thread(target=work, args=(op, i)) for i, op in enumerate(ops)]
        for t in th:
            t.start()
        for t in th:
            t.join()
        prof = rf.profile_read()
    finally:
        rf.profile_enable(False)
    assert not errors, errors
    assert sum(v["launches"] for v in prof.values()) >= 6000
    for op in ops:
        _ta_check(op, m, 1.0)
