"""Batch sessions (rfcmp_batch_*): columns that join and leave a running RF-CMP solve.

Each column's arithmetic is that of a standalone solve: the same kernels, its own CG scalars
and stopping test.  Columns admitted while others are mid-solve, and columns admitted into
slots freed by finished ones, must reach the same current as the standalone multi-column solve
(to the solve tolerance times the conditioning) and as the oracle's LU solution of the plain
EFIE system T j = -e (Sec. 2, the current RF-CMP computes; Sec. 3).
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
    c = rf.Context(0)
    yield c
    c.close()


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _lu(memo, m, key, k, kh, pol):
    D = memo(("bs_disc", key), lambda: efie.discretize(m.verts, m.tris))
    TA, V = memo(("bs_op", key, k), lambda: efie.assemble(D, k))
    return krylov.lu_solve(efie.efie_matrix(D, TA, V, k), -efie.excitation(D, k, kh, pol)).T


@pytest.mark.parametrize("k,precision", [(1.0, "mixed"), (1e-3, "mixed"), (1.5, "ff")])
def test_columns_joining_mid_solve_match_lu_and_the_standalone_solve(ctx, memo, k, precision):
    m = synth.geodesic_sphere(4, seed=1)  # 320 cells, N = 480
    kh, pol = synth.random_plane_waves(7, seed=21)
    J = _lu(memo, m, "l2", k, kh, pol)
    op = rf.Operator(ctx, m.verts, m.tris, k)
    e = op.rhs_planewave(kh, pol)
    ja, ra = op.solve(e, tol=1e-10, precision=precision)
    alone = ja.cpu().numpy()
    assert all(r.converged for r in ra)

    sess = op.batch(5, tol=1e-10, precision=precision)
    got, reps = {}, {}
    slot_col = {}
    for c, s in zip(range(3), sess.admit(e[0:3])):  # three columns start
        slot_col[s] = c
    assert sess.counts() == (3, 0, 2)
    nxt = 3
    steps = 0
    while slot_col or nxt < 7:
        fin = sess.step()
        steps += 1
        if fin:
            j, rep = sess.take(fin)
            for s, jr, r in zip(fin, j.cpu().numpy(), rep):
                c = slot_col.pop(s)
                got[c], reps[c] = jr, r
        # after the first sweep, and whenever slots free up, the next columns join
        free = sess.counts()[2]
        if free and nxt < 7:
            n = min(free, 7 - nxt, 2)
            for c, s in zip(range(nxt, nxt + n), sess.admit(e[nxt : nxt + n])):
                slot_col[s] = c
            nxt += n
        assert steps < 64
    assert sess.counts() == (0, 0, 5)
    sess.close()
    for c in range(7):
        assert reps[c].converged and reps[c].residual <= 1e-10, (c, reps[c])
        # the same system to relative residual 1e-10 on both sides; their products round
        # differently (sweep membership changes the multi-column product path), cond < 1e3 here
        assert _rel(got[c], alone[c]) <= 1e-7, (c, _rel(got[c], alone[c]))
        assert _rel(got[c], J[c]) <= 1e-6, (c, _rel(got[c], J[c]))
    op.close()


def test_session_errors_and_reuse(ctx):
    m = synth.geodesic_sphere(3, seed=2)
    op = rf.Operator(ctx, m.verts, m.tris, 0.8)
    kh, pol = synth.random_plane_waves(3, seed=4)
    e = op.rhs_planewave(kh, pol)
    sess = op.batch(2, tol=1e-8)
    slots = sess.admit(e[0:2])
    assert sorted(slots) == [0, 1]
    with pytest.raises(rf.RfcmpError):
        sess.admit(e[2:3])  # no free slot
    with pytest.raises(rf.RfcmpError):
        sess.take(slots[0])  # still running
    with pytest.raises(rf.RfcmpError):
        op.batch(0)
    done = []
    for _ in range(32):
        done += sess.step()
        if len(done) == 2:
            break
    assert sorted(done) == [0, 1]
    assert sess.step() == []  # nothing running: a no-op
    with pytest.raises(rf.RfcmpError):
        sess.take([done[0], done[0]])  # listed twice
    j0, (r0,) = sess.take(done[0])
    assert r0.converged and r0.residual <= 1e-8
    # the freed slot takes a new column; its report starts from scratch
    (s,) = sess.admit(e[2:3])
    assert s == done[0]
    for _ in range(32):
        if sess.step():
            break
    j21, r21 = sess.take([s, done[1]])  # two columns, finished in different sweeps, in one take
    assert all(r.converged for r in r21)
    j2, j1 = j21[0:1], j21[1:2]
    sess.close()
    ref, rr = op.solve(e, tol=1e-8)  # the operator is usable after the session
    for c, j in ((0, j0), (1, j1), (2, j2)):
        assert (torch.linalg.norm(j[0] - ref[c]) / torch.linalg.norm(ref[c])).item() <= 1e-5
    op.close()
