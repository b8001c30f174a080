"""Host-side logic of the continuous-batching server (fake backend, no GPU)."""

import time

import numpy as np
import pytest

import synth
from paper_1803_08333_gb300 import serve


def _mesh(n, seed=1):
    m = synth.geodesic_sphere(n, seed=seed)
    return m.verts, m.tris


def test_all_requests_complete_with_their_columns():
    be = serve.FakeBackend()
    srv = serve.Server(be, hbm_budget=0, workers=2)
    v, t = _mesh(2)
    futs = [srv.submit(v, t, 1.0 + 0.1 * (i % 3), np.tile([[0, 0, 1.0]], (i % 4 + 1, 1)),
                       np.tile([[1.0, 0, 0]], (i % 4 + 1, 1))) for i in range(20)]
    for i, f in enumerate(futs):
        r = f.result(timeout=10)
        assert r.j.shape == (i % 4 + 1, 3 * t.shape[0] // 2)
    srv.close()
    st = srv.stats()
    assert st["requests"] == 20 and st["columns"] == sum(i % 4 + 1 for i in range(20))
    assert st["p50_ms"] is not None and st["p99_ms"] >= st["p50_ms"]


def test_requests_join_a_running_solve_between_sweeps():
    be = serve.FakeBackend(solve_seconds=0.05)
    be.steps_per_column = 3
    srv = serve.Server(be, hbm_budget=0, workers=1, max_batch_columns=64)
    v, t = _mesh(2)
    kh, pol = synth.plane_wave_z()
    first = srv.submit(v, t, 1.0, kh, pol)
    time.sleep(0.02)  # the first solve is in its first sweep; these join it at the next sweep
    rest = [srv.submit(v, t, 1.0, kh, pol) for _ in range(5)]
    r0 = first.result(timeout=10)
    rr = [f.result(timeout=10) for f in rest]
    srv.close()
    assert len(be.sessions) == 1  # one running solve took all six requests
    assert srv.stats()["joined_running_solve"] == 5
    assert r0.batch_columns == 6 and {r.batch_columns for r in rr} == {6}
    assert r0.latency_s < min(r.latency_s + 0.02 for r in rr) + 0.06  # the first left before the others
    assert len(be.created) == 1  # the operator stayed resident


def test_merged_mode_solves_waiting_requests_together():
    be = serve.FakeBackend(solve_seconds=0.05)
    srv = serve.Server(be, hbm_budget=0, workers=1, max_batch_columns=64, continuous=False)
    v, t = _mesh(2)
    kh, pol = synth.plane_wave_z()
    first = srv.submit(v, t, 1.0, kh, pol)
    time.sleep(0.02)  # the first solve is running; these queue behind it and merge
    rest = [srv.submit(v, t, 1.0, kh, pol) for _ in range(5)]
    assert first.result(timeout=10).batch_columns == 1
    assert {f.result(timeout=10).batch_columns for f in rest} == {5}
    st = srv.stats()
    srv.close()
    assert st["solves"] == 2 and st["joined_running_solve"] == 0
    assert not getattr(be, "sessions", [])


def test_a_full_session_leaves_the_rest_waiting():
    be = serve.FakeBackend(solve_seconds=0.02)
    srv = serve.Server(be, hbm_budget=0, workers=1, max_batch_columns=4)
    v, t = _mesh(2)
    kh, pol = synth.random_plane_waves(3, seed=1)
    futs = [srv.submit(v, t, 1.0, kh, pol) for _ in range(4)]  # 12 columns through 4 slots
    res = [f.result(timeout=10) for f in futs]
    srv.close()
    assert all(r.j.shape[0] == 3 for r in res)
    assert max(srv.stats()["mean_batch_columns"] for _ in [0]) <= 4


def test_admission_respects_the_budget_and_evicts_lru():
    be = serve.FakeBackend()
    one = serve.op_footprint(42, 80, 1, with_factors=False)
    budget = int(2.5 * serve.op_footprint(42, 80, 1, with_factors=True))
    srv = serve.Server(be, hbm_budget=budget, workers=2)
    v, t = _mesh(2)
    kh, pol = synth.plane_wave_z()
    futs = [srv.submit(v, t, 0.5 + i, kh, pol) for i in range(8)]  # 8 distinct wavenumbers
    for f in futs:
        f.result(timeout=10)
    srv.close()
    assert be.max_in_use <= budget
    assert len(be.destroyed) >= 8 - budget // one


def test_a_failing_batch_fails_only_its_requests():
    class Flaky(serve.FakeBackend):
        def admit(self, sess, khat, pol, stream):
            if sess["op"]["scene"][1] == 2.0:
                raise RuntimeError("boom")
            return super().admit(sess, khat, pol, stream)

    srv = serve.Server(Flaky(), hbm_budget=0, workers=2)
    v, t = _mesh(2)
    kh, pol = synth.plane_wave_z()
    good = srv.submit(v, t, 1.0, kh, pol)
    bad = srv.submit(v, t, 2.0, kh, pol)
    assert good.result(timeout=10).j.shape[0] == 1
    with pytest.raises(RuntimeError):
        bad.result(timeout=10)
    srv.close()


def test_poisson_workload_is_seeded():
    a = serve.poisson_workload(50, 20.0, seed=4)
    b = serve.poisson_workload(50, 20.0, seed=4)
    assert a == b
    t = np.array([x[0] for x in a])
    assert np.all(np.diff(t) > 0)
    assert all(1 <= x[2] <= 64 for x in a)
    assert len({x[1] for x in a}) <= 48
    assert len({x[1][:2] for x in a}) <= 12  # scenes share meshes


def test_warm_makes_operators_resident_within_budget():
    be = serve.FakeBackend()
    one = serve.op_footprint(*_mesh(3)[0].shape[:1], _mesh(3)[1].shape[0], 1, with_factors=True)
    srv = serve.Server(be, hbm_budget=int(2.5 * one), workers=1)
    v, t = _mesh(3)
    assert srv.warm(v, t, 1.0) and srv.warm(v, t, 2.0) and srv.warm(v, t, 1.0)
    assert be.created == [(serve.mesh_key(v, t), 1.0), (serve.mesh_key(v, t), 2.0)]
    kh, pol = synth.plane_wave_z()
    srv.submit(v, t, 2.0, kh, pol).result(timeout=10)
    assert len(be.created) == 2  # the warm operator served the request
    srv.close()
    assert be.in_use == 0


def test_footprint_counts_what_a_wider_solve_builds():
    nv, nc = 1922, 3840
    cold = serve.op_footprint(nv, nc, 1, with_factors=True)
    assert serve.op_footprint(nv, nc, 64, with_factors=True) > cold
    # a resident operator that already solved 64 columns adds nothing for 32 more
    assert serve.op_footprint(nv, nc, 32, with_factors=True, widest=64) == 0
    # one that only solved single columns still has to build the planes and digits
    grow = serve.op_footprint(nv, nc, 16, with_factors=True, widest=1)
    assert grow >= 32 * (3 * nc // 2) ** 2


def test_eviction_falls_back_to_dropping_the_factor_cache():
    be = serve.FakeBackend()
    v, t = _mesh(3)
    one = serve.op_footprint(v.shape[0], t.shape[0], 1, with_factors=False)
    srv = serve.Server(be, hbm_budget=int(0.5 * one), workers=1)
    assert not srv.warm(v, t, 1.0)  # cannot fit even after dropping the cache
    assert getattr(be, "cache_clears", 0) == 1
    srv.close()


def test_idle_operators_are_trimmed_before_they_are_evicted():
    be = serve.FakeBackend()
    v, t = _mesh(3)
    nv, nc = v.shape[0], t.shape[0]
    base = serve.op_footprint(nv, nc, 1, with_factors=False)
    wide = serve.op_footprint(nv, nc, 32, with_factors=True, widest=1)
    # room for two resident operators and one wide solve's planes, not two
    srv = serve.Server(be, hbm_budget=2 * base + int(1.5 * wide), workers=1)
    kh, pol = synth.random_plane_waves(32, seed=2)
    srv.submit(v, t, 1.0, kh, pol).result(timeout=10)
    srv.submit(v, t, 2.0, kh, pol).result(timeout=10)
    srv.close()
    assert getattr(be, "trims", 0) >= 1  # the first operator gave its planes back ...
    assert be.destroyed == [(serve.mesh_key(v, t), 1.0), (serve.mesh_key(v, t), 2.0)]  # ... and stayed until close
    assert be.in_use == 0


def test_a_request_wider_than_a_session_gets_its_own():
    be = serve.FakeBackend(solve_seconds=0.01)
    srv = serve.Server(be, hbm_budget=0, workers=1, max_batch_columns=4)
    v, t = _mesh(2)
    kh, pol = synth.random_plane_waves(6, seed=3)
    r = srv.submit(v, t, 1.0, kh, pol).result(timeout=10)
    srv.close()
    assert r.j.shape == (6, 3 * t.shape[0] // 2)
    assert be.sessions[0]["cap"] == 6  # opened as wide as the request


def test_reservations_are_released_after_sessions_and_failures():
    class Flaky(serve.FakeBackend):
        def step(self, sess, stream):
            if sess["op"]["scene"][1] == 3.0:
                raise RuntimeError("boom")
            return super().step(sess, stream)

    be = Flaky(solve_seconds=0.005)
    srv = serve.Server(be, hbm_budget=10**12, workers=2, max_batch_columns=8)
    v, t = _mesh(2)
    kh, pol = synth.random_plane_waves(3, seed=5)
    futs = [srv.submit(v, t, 1.0 + (i % 3), kh, pol) for i in range(12)]
    ok = [f for i, f in enumerate(futs) if 1.0 + (i % 3) != 3.0]
    bad = [f for i, f in enumerate(futs) if 1.0 + (i % 3) == 3.0]
    for f in ok:
        assert f.result(timeout=10).j.shape[0] == 3
    for f in bad:
        with pytest.raises(RuntimeError):
            f.result(timeout=10)
    srv.close()
    assert srv._reserved == 0 and not srv._busy
    st = srv.stats()
    assert st["requests"] == len(ok) and st["solves"] >= 3
