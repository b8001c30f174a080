"""The paper's remaining experiments on synthetic meshes (Sec. 4), on the GPU.

  * voltage-gap (delta-gap) excitation, the second excitation of the Fokker experiment: the
    library's e against the oracle's line integral of the RWG functions across the gap, and the
    current of the RF-CMP solve against the oracle's LU solution (ka = 1) and its FP64 RF-CMP
    solve (ka = 1e-3);
  * dense-discretization stability (Fig. SphereH): at fixed ka the iteration count of the
    preconditioned CG stays flat from 120 to 30720 unknowns, with the current against the oracle
    up to 1920 unknowns;
  * a multiply connected structure (the toroidal structure of Sec. 4) at 10368 unknowns: flat
    iterations from ka = 1 to 1e-5, the residual of sampled rows of T j = -e checked with rows
    the oracle assembles, and the same current from both outer preconditioners.
"""

import numpy as np
import pytest

import synth
from oracle import efie, krylov, rfcmp

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1803_08333_gb300 as rf  # noqa: E402

GAP = ([0.0, 0.0, 0.05], [0.1, 0.2, 1.0])


@pytest.fixture(scope="module")
def ctx():
    from paper_1803_08333_gb300 import build

    build.build()
    yield rf.Context(0)


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_voltage_gap_excitation_matches_oracle(ctx):
    m = synth.geodesic_sphere(8, seed=1)
    D = efie.discretize(m.verts, m.tris)
    op = rf.Operator(ctx, m.verts, m.tris, 1.0, scaling="k")
    e = op.rhs_voltage_gap(*GAP, voltage=2.0 - 0.5j).cpu().numpy()[0]
    ref = efie.excitation_voltage_gap(D, *GAP, voltage=2.0 - 0.5j)[:, 0]
    assert np.abs(e - ref).max() <= 1e-13 * np.abs(ref).max()


@pytest.mark.parametrize("ka", [1.0, 1e-3])
def test_voltage_gap_solution(ctx, memo, ka):
    m = synth.geodesic_sphere(8, seed=1)
    D = memo(("gap_disc",), lambda: efie.discretize(m.verts, m.tris))
    TA, V = efie.assemble(D, ka)
    e_ref = efie.excitation_voltage_gap(D, *GAP)[:, 0]
    if ka >= 0.1:
        ref = krylov.lu_solve(efie.efie_matrix(D, TA, V, ka), -e_ref)
    else:  # LU of T loses digits at low frequency; the oracle's FP64 RF-CMP solve does not
        F = memo(("gap_fac",), lambda: rfcmp.factors(D))
        ref, _, _ = rfcmp.solve(F, TA, V, ka, rfcmp.kscale(ka), e_ref, 1e-12)
    op = rf.Operator(ctx, m.verts, m.tris, ka)
    j, rep = op.solve(op.rhs_voltage_gap(*GAP), tol=1e-10)
    assert rep[0].converged
    assert _rel(j.cpu().numpy()[0], ref) <= 1e-6


def test_h_sweep_iterations_flat(ctx, memo):
    ka = 0.1
    kh, pol = synth.plane_wave_z()
    iters = {}
    for n in (2, 4, 8, 16, 32):
        m = synth.geodesic_sphere(n, seed=2)
        op = rf.Operator(ctx, m.verts, m.tris, ka)
        j, rep = op.solve(op.rhs_planewave(kh, pol), tol=1e-6)
        assert rep[0].converged
        iters[op.N] = rep[0].iterations
        if n <= 8:
            D = efie.discretize(m.verts, m.tris)
            TA, V = efie.assemble(D, ka)
            J = krylov.lu_solve(efie.efie_matrix(D, TA, V, ka), -efie.excitation(D, ka, kh, pol)[:, 0])
            j10, _ = op.solve(op.rhs_planewave(kh, pol), tol=1e-10)
            assert _rel(j10.cpu().numpy()[0], J) <= 1e-6
        op.close()
        ctx.clear_cache()
    # bounded in h: 120 to 30720 unknowns within a few iterations of each other
    assert max(iters.values()) - min(iters.values()) <= 4, iters
    assert max(iters.values()) <= 16, iters


@pytest.fixture(scope="module")
def big_torus():
    return synth.torus(96, 36, jitter=0.03, seed=6)  # 6912 cells, 10368 unknowns, genus 1


def test_torus_10k_iterations_flat_in_k(ctx, big_torus):
    m = big_torus
    kh, pol = synth.plane_wave_z()
    iters = []
    for ka in (1.0, 1e-2, 1e-5):
        op = rf.Operator(ctx, m.verts, m.tris, ka)
        assert op.info().genus == 1 and op.N == 10368
        j, rep = op.solve(op.rhs_planewave(kh, pol), tol=1e-6)
        assert rep[0].converged
        iters.append(rep[0].iterations)
        op.close()
    assert max(iters) <= 2 * min(iters) + 4, iters


def test_torus_10k_sampled_residual_and_outer_variants(ctx, big_torus):
    m = big_torus
    ka = 1.0
    kh, pol = synth.plane_wave_z()
    op = rf.Operator(ctx, m.verts, m.tris, ka)
    j, rep = op.solve(op.rhs_planewave(kh, pol), tol=1e-10)
    assert rep[0].converged
    jh = j.cpu().numpy()[0]
    # rows of T j + e from rows the oracle assembles: T = i k T_A + Sigma V Sigma^T / (i k)
    D = efie.discretize(m.verts, m.tris)
    rows = np.array([0, 1777, 5000, 10367])
    cells = np.unique(D.top.edge_cells[rows].ravel())
    TA_rows, V_rows = efie.assemble_rows(D, ka, rows, cells)
    Vr = {int(c): V_rows[i] for i, c in enumerate(cells)}
    S = D.Sigma
    e = efie.excitation(D, ka, kh, pol)[:, 0]
    sj = S.T @ jh
    for i, mrow in enumerate(rows):
        cp, cm = D.top.edge_cells[mrow]
        tphi = (Vr[int(cp)] - Vr[int(cm)]) @ sj
        res = 1j * ka * (TA_rows[i] @ jh) + tphi / (1j * ka) + e[mrow]
        # complex64 operator storage: rows agree with the oracle to ~1e-6 of their scale
        scale = abs(1j * ka * (np.abs(TA_rows[i]) @ np.abs(jh))) + abs((np.abs(Vr[int(cp)]) + np.abs(Vr[int(cm)])) @ np.abs(sj)) / ka
        assert abs(res) <= 1e-5 * scale, (mrow, abs(res), scale)
    # the theory variant reaches the same current
    opg = rf.Operator(ctx, m.verts, m.tris, ka, scaling="k", outer="gsigma")
    jg, rg = opg.solve(opg.rhs_planewave(kh, pol), tol=1e-10)
    assert rg[0].converged
    assert _rel(jg.cpu().numpy()[0], jh) <= 1e-7
