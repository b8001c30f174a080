"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed
forms (Mie series, sphere capacitance, Rayleigh limit, quadrature exactness),
exact identities of the quasi-Helmholtz algebra (Sec. 2, Sec. 3.2), brute
force (polar integration of the singular potentials) and the spectral
statements of the paper (HPD system, bounded condition number, CG bound).
"""

import math

import numpy as np
import pytest

import synth
from oracle import efie, farfield, gram, krylov, mie, potentials, quadrature, rfcmp, topology


def _disc(memo, n, seed=1):
    return memo(("disc", n, seed), lambda: efie.discretize(*_mesh(n, seed)))


def _mesh(n, seed):
    m = synth.geodesic_sphere(n, seed=seed)
    return m.verts, m.tris


def _op(memo, n, k, seed=1):
    D = _disc(memo, n, seed)
    return memo(("op", n, k, seed), lambda: efie.assemble(D, k))


# ---------------------------------------------------------------- quadrature
@pytest.mark.parametrize("deg", range(6))
def test_seven_point_rule_exact_to_degree_five(deg):
    # int_T l1^a l2^b l3^c dS = 2 A a! b! c! / (a+b+c+2)!  (A = 1/2 on the unit triangle)
    for a in range(deg + 1):
        for b in range(deg + 1 - a):
            c = deg - a - b
            exact = 2 * 0.5 * math.factorial(a) * math.factorial(b) * math.factorial(c) / math.factorial(deg + 2)
            q = 0.5 * np.sum(quadrature.W7 * quadrature.BARY7[:, 0] ** a * quadrature.BARY7[:, 1] ** b * quadrature.BARY7[:, 2] ** c)
            assert abs(q - exact) < 1e-15


def test_seven_point_rule_not_exact_at_degree_six():
    q = 0.5 * np.sum(quadrature.W7 * quadrature.BARY7[:, 0] ** 6)
    exact = 2 * 0.5 * math.factorial(6) / math.factorial(8)
    assert abs(q - exact) > 1e-6


# ---------------------------------------------------------------- potentials
def _polar_brute(r, T, n=300):
    """int_T 1/R and int_T (r'-p)/R by polar integration about the projection p."""
    cr = np.cross(T[1] - T[0], T[2] - T[0])
    nh = cr / np.linalg.norm(cr)
    d = (r - T[0]) @ nh
    p = r - d * nh
    x, w = np.polynomial.legendre.leggauss(n)
    s = 0.5 * (x + 1)
    ws = 0.5 * w
    S = 0.0
    V = np.zeros(3)
    for i in range(3):
        a = T[i] - p
        b = T[(i + 1) % 3] - p
        jac = np.cross(a, b) @ nh
        for si, wsi in zip(s, ws):
            e = (1 - si) * a + si * b
            q = s[:, None] * e[None, :]
            R = np.sqrt((q**2).sum(1) + d * d)
            f = ws * s / R
            S += jac * wsi * f.sum()
            V += jac * wsi * (f[:, None] * q).sum(0)
    return S, V


@pytest.mark.parametrize(
    "r",
    [
        [0.3, 0.3, 0.0],  # interior, in plane (singular)
        [0.3, 0.3, 0.05],  # near, off plane
        [1.5, -0.4, 0.2],  # far
        [0.5, 0.05, 0.0],  # in plane, near an edge
        [1.0, 0.1, 0.0],  # at a vertex
        [0.6, 0.5, -0.01],  # near the far edge, below
        [-0.5, 0.4, 0.0],  # in plane, outside
    ],
)
def test_analytic_potentials_match_polar_quadrature(r):
    T = np.array([[0.0, 0, 0], [1.0, 0.1, 0], [0.2, 0.9, 0.0]])
    r = np.array(r)
    S, Vv, _ = potentials.triangle_potentials(r[None], T[None])
    Sb, Vb = _polar_brute(r, T)
    assert abs(S[0] - Sb) < 1e-12 * max(1, abs(Sb))
    assert np.abs(Vv[0] - Vb).max() < 1e-12


def test_potential_far_field_limit():
    # far away, int 1/R -> A / |r - c|
    T = np.array([[0.0, 0, 0], [1.0, 0.1, 0], [0.2, 0.9, 0.0]])
    r = np.array([300.0, 200.0, 500.0])
    S, _, _ = potentials.triangle_potentials(r[None], T[None])
    A = 0.5 * np.linalg.norm(np.cross(T[1] - T[0], T[2] - T[0]))
    assert abs(S[0] - A / np.linalg.norm(r - T.mean(0))) < 1e-5 * S[0]  # next term is O((size/distance)^2)


# ---------------------------------------------------------------- topology
@pytest.mark.parametrize("mesh", ["sphere", "cube", "torus", "ellipsoid"])
def test_quasi_helmholtz_identities(mesh):
    m = {
        "sphere": lambda: synth.geodesic_sphere(3, seed=7),
        "cube": lambda: synth.cube(3),
        "torus": lambda: synth.torus(10, 6, jitter=0.03),
        "ellipsoid": lambda: synth.ellipsoid(3),
    }[mesh]()
    top = topology.build_topology(m.tris, m.nv)
    S = topology.sigma_matrix(top).toarray()
    L = topology.lambda_matrix(top).toarray()
    assert np.array_equal(S.T @ L, np.zeros((top.nc, top.nv)))  # Sec. 2: Lambda^T Sigma = 0
    assert np.array_equal(L @ np.ones(top.nv), np.zeros(top.ne))  # Lambda 1 = 0
    assert np.array_equal(S @ np.ones(top.nc), np.zeros(top.ne))  # Sigma 1 = 0
    g = 1 if mesh == "torus" else 0
    assert top.genus == g
    PS = S @ np.linalg.pinv(S.T @ S, rcond=1e-10, hermitian=True) @ S.T
    PL = L @ np.linalg.pinv(L.T @ L, rcond=1e-10, hermitian=True) @ L.T
    assert abs(np.trace(PS) - (top.nc - 1)) < 1e-8
    assert abs(np.trace(PL) - (top.nv - 1)) < 1e-8
    # quasi-harmonic subspace: rank of I - P_Lambda - P_Sigma is 2g
    assert abs(np.trace(np.eye(top.ne) - PS - PL) - 2 * g) < 1e-8


def test_topology_open_surfaces_and_invalid_meshes():
    m = synth.geodesic_sphere(2)
    # one cell removed: an open surface (a disk) with one boundary curve of three edges, whose
    # vertices carry no loop function
    t = topology.build_topology(m.tris[:-1], m.nv)
    assert t.boundaries == 1 and t.genus == 0 and t.ne == 30 * 4 - 3 and t.nvl == m.nv - 3
    bad = m.tris.copy()
    bad[0] = bad[0, [0, 2, 1]]
    with pytest.raises(topology.MeshError):  # inconsistent orientation
        topology.build_topology(bad, m.nv)
    junction = np.vstack([m.tris, m.tris[:1, [0, 2, 1]]])  # an edge shared by three cells
    with pytest.raises(topology.MeshError):
        topology.build_topology(junction, m.nv)
    # two holes meeting at one vertex: a boundary vertex with four boundary edges
    v = int(m.tris[0, 0])
    around = [c for c in range(m.nc) if v in m.tris[c]]
    pinched = np.delete(m.tris, [around[0], around[2]], axis=0)
    with pytest.raises(topology.MeshError):
        topology.build_topology(pinched, m.nv)


# ---------------------------------------------------------------- projectors
def test_projectors_and_pseudo_inverse(memo):
    D = _disc(memo, 2)
    F = memo(("fac", 2), lambda: rfcmp.factors(D))
    assert rfcmp.pseudo_inverse_check(F) < 1e-12  # Sec. 3.2 identity vs SVD pinv
    I = np.eye(D.N)
    assert np.abs(F.P_S @ F.P_S - F.P_S).max() < 1e-12
    assert np.abs(F.P_S + F.P_LH - I).max() == 0
    assert np.abs(F.P_S @ F.Sigma - F.Sigma).max() < 1e-12
    assert np.abs(F.P_S @ F.Lambda).max() < 1e-12
    assert abs(np.trace(F.P_S) - (D.nc - 1)) < 1e-9


# ---------------------------------------------------------------- Gram matrices
def test_gram_matrices(memo):
    D = _disc(memo, 2)
    Gll = gram.g_ll(D)
    assert abs(Gll.sum() - D.area.sum()) < 1e-13 * D.area.sum()  # 1^T G_ll 1 = |Gamma|
    Gff = gram.g_ff(D).toarray()
    Lam = D.Lambda.toarray()
    Delta = gram.stiffness(D).toarray()
    # Lambda^T G_ff Lambda = Delta (Eq. PrimalLaplace); pins RWG scaling and Lambda signs
    assert np.abs(Lam.T @ Gff @ Lam - Delta).max() < 1e-12 * np.abs(Delta).max()
    assert np.abs(Delta @ np.ones(D.nv)).max() < 1e-12
    Gpp = gram.g_pp(D).toarray()
    assert np.allclose(np.diag(Gpp), 1.0 / D.area)


# ---------------------------------------------------------------- operators
def test_operator_symmetry_and_tphi_identity(memo):
    D = _disc(memo, 2)
    k = 1.3
    TA, V = _op(memo, 2, k)
    assert np.abs(TA - TA.T).max() <= 1e-14 * np.abs(TA).max()
    assert np.abs(V - V.T).max() <= 1e-14 * np.abs(V).max()
    TP = efie.t_phi(D, V)
    TPe = efie.t_phi_edgewise(D, k)  # from int int div f div f G directly
    assert np.abs(TP - TPe).max() <= 1e-13 * np.abs(TP).max()
    # divergence-free loop currents are annihilated by T_Phi
    assert np.abs(TP @ D.Lambda.toarray()).max() <= 1e-13 * np.abs(TP).max()


def test_sphere_capacitance_converges_h2(memo):
    # static single layer with p = 1/A: 1^T V0^{-1} 1 = total charge at unit potential = 4 pi (a = 1)
    errs = []
    for n in (2, 4):
        _, V = _op(memo, n, 1e-9)
        q = np.linalg.solve(V.real, np.ones(V.shape[0]))
        errs.append(abs(q.sum() - 4 * np.pi) / (4 * np.pi))
    assert errs[1] < 0.015
    assert 2.5 < errs[0] / errs[1] < 6.0  # second order in h


def test_excitation_static_closed_form(memo):
    # at k = 0, e_n = pol . int f_n = pol . ((c+ - r+)/2 - (c- - r-)/2)
    D = _disc(memo, 2)
    pol = np.array([0.3, -0.2, 0.9])
    e = efie.excitation(D, 0.0, [[0, 0, 1.0]], [pol])[:, 0]
    c = D.cent
    top = D.top
    ref = ((c[top.edge_cells[:, 0]] - D.verts[top.edge_free[:, 0]]) / 2 - (c[top.edge_cells[:, 1]] - D.verts[top.edge_free[:, 1]]) / 2) @ pol
    assert np.abs(e - ref).max() < 1e-14


# ---------------------------------------------------------------- Mie series
def test_mie_rayleigh_limit():
    x = 1e-3
    th = np.linspace(0, np.pi, 13)
    sE, sH = mie.pec_sphere_rcs(x, 1.0, th)
    k = x
    refE = 4 * np.pi / k**2 * x**6 * (0.5 - np.cos(th)) ** 2
    refH = 4 * np.pi / k**2 * x**6 * (1 - 0.5 * np.cos(th)) ** 2
    # the E-plane pattern has a null at cos t = 1/2, so compare against the peak
    assert np.abs(sE - refE).max() < 1e-5 * refE.max()
    assert np.abs(sH - refH).max() < 1e-5 * refH.max()


def test_mie_optical_backscatter():
    # large ka: monostatic RCS of a sphere tends to pi a^2
    vals = [mie.pec_sphere_rcs(ka, 1.0, np.array([np.pi]))[0][0] / np.pi for ka in (60.0, 80.0, 100.0)]
    assert all(abs(v - 1) < 0.05 for v in vals)


def _rcs_error_db(D, j, k):
    th = np.linspace(0, np.pi, 37)
    worst = 0.0
    for phi, idx in ((0.0, 0), (np.pi / 2, 1)):
        s = farfield.bistatic_rcs(D, j, k, farfield.cut_directions(th, phi))
        sm = mie.pec_sphere_rcs(k, 1.0, th)[idx]
        keep = sm > sm.max() * 1e-4  # within 40 dB of the peak (nulls excluded)
        worst = max(worst, np.abs(10 * np.log10(s[keep] / sm[keep])).max())
    return worst


@pytest.mark.slow
def test_efie_rcs_matches_mie_and_converges(memo):
    kh, pol = synth.plane_wave_z()
    errs = []
    for n in (4, 8):
        D = _disc(memo, n)
        TA, V = _op(memo, n, 1.0)
        T = efie.efie_matrix(D, TA, V, 1.0)
        e = efie.excitation(D, 1.0, kh, pol)[:, 0]
        j = krylov.lu_solve(T, -e)
        errs.append(_rcs_error_db(D, j, 1.0))
    assert errs[1] < 0.15  # level 3, ka = 1
    assert errs[1] < 0.5 * errs[0]


# ---------------------------------------------------------------- RF-CMP
@pytest.mark.parametrize("k", [1.0, 1e-2, 1e-5])
def test_rfcmp_system_hpd_and_bounded(memo, k):
    D = _disc(memo, 2)
    F = memo(("fac", 2), lambda: rfcmp.factors(D))
    TA, V = _op(memo, 2, k)
    T = efie.efie_matrix(D, TA, V, k)
    sc = rfcmp.power_scaling(F, TA, V, k, exact=True)
    A, _, _ = rfcmp.dense_system(F, T, sc)
    H = 0.5 * (A + A.conj().T)
    ev = np.linalg.eigvalsh(H)
    assert ev[0] > 0
    assert ev[-1] / ev[0] < 20  # bounded as k -> 0 (Sec. 4, Fig. SphereF)
    sv = np.linalg.svd(T, compute_uv=False)
    if k == 1e-2:
        # plain EFIE: cond grows like k^-2 (Sec. 2)
        assert sv[0] / sv[-1] > 1e5
    if k == 1.0:
        assert np.linalg.norm(A - A.conj().T) / np.linalg.norm(A) < 1e-12


def test_rfcmp_structured_equals_dense_at_ka1(memo):
    D = _disc(memo, 2)
    F = memo(("fac", 2), lambda: rfcmp.factors(D))
    k = 1.0
    TA, V = _op(memo, 2, k)
    T = efie.efie_matrix(D, TA, V, k)
    sc = rfcmp.Scaling(0.7, 0.6, 0.12)
    A, Bm, _ = rfcmp.dense_system(F, T, sc)
    x = rfcmp.splitmix_start(D.N, 11) + 1j * rfcmp.splitmix_start(D.N, 12)
    assert np.linalg.norm(rfcmp.apply_A(F, TA, V, k, sc, x) - A @ x) < 1e-12 * np.linalg.norm(A @ x)
    e = efie.excitation(D, k, *synth.plane_wave_z())[:, 0]
    assert np.linalg.norm(rfcmp.apply_rhs(F, TA, V, k, sc, e) - Bm @ e) < 1e-12 * np.linalg.norm(Bm @ e)


def test_rfcmp_solution_equals_lu_and_scaling_independent(memo):
    D = _disc(memo, 2)
    F = memo(("fac", 2), lambda: rfcmp.factors(D))
    k = 1.0
    TA, V = _op(memo, 2, k)
    T = efie.efie_matrix(D, TA, V, k)
    e = efie.excitation(D, k, *synth.plane_wave_z())[:, 0]
    jl = krylov.lu_solve(T, -e)
    sc = rfcmp.power_scaling(F, TA, V, k)
    j1, it1, _ = rfcmp.solve(F, TA, V, k, sc, e, 1e-13)
    j2, it2, _ = rfcmp.solve(F, TA, V, k, rfcmp.kscale(k), e, 1e-13)
    assert np.linalg.norm(j1 - jl) < 1e-10 * np.linalg.norm(jl)
    assert np.linalg.norm(j2 - jl) < 1e-10 * np.linalg.norm(jl)
    # CG iteration bound (Eq. Niter)
    A, _, _ = rfcmp.dense_system(F, T, sc)
    ev = np.linalg.eigvalsh(0.5 * (A + A.conj().T))
    assert it1 <= math.ceil(0.5 * math.sqrt(ev[-1] / ev[0]) * math.log(2 / 1e-13))


def test_power_iteration_close_to_exact_norms(memo):
    D = _disc(memo, 2)
    F = memo(("fac", 2), lambda: rfcmp.factors(D))
    TA, V = _op(memo, 2, 1.0)
    p = rfcmp.power_scaling(F, TA, V, 1.0, steps=60, rtol=0.0)
    x = rfcmp.power_scaling(F, TA, V, 1.0, exact=True)
    for a, b in ((p.alpha, x.alpha), (p.beta, x.beta), (p.gamma, x.gamma)):
        assert abs(a - b) < 0.02 * b
        assert a <= b * (1 + 1e-12)  # Rayleigh quotients approach the top eigenvalue from below


def test_kscale_reduces_to_theory_scaling():
    sc = rfcmp.kscale(0.04)
    assert sc.alpha == pytest.approx(0.2) and sc.beta == pytest.approx(5.0) and sc.gamma == pytest.approx(0.04)


def test_low_frequency_rcs_matches_rayleigh_mie(memo):
    # RF-CMP stays accurate where the plain EFIE loses its loop part (Sec. 4, Fig. Sphere_RCS)
    D = _disc(memo, 4)
    F = memo(("fac", 4), lambda: rfcmp.factors(D))
    k = 1e-4
    TA, V = _op(memo, 4, k)
    e = efie.excitation(D, k, *synth.plane_wave_z())[:, 0]
    sc = rfcmp.power_scaling(F, TA, V, k)
    j, it, _ = rfcmp.solve(F, TA, V, k, sc, e, 1e-12)
    assert it < 60
    assert _rcs_error_db(D, j, k) < 0.5


def test_splitmix_reference_values():
    # splitmix64 from state 0 gives 0xE220A8397B1DCDAF first (published test value)
    u = rfcmp.splitmix_start(1, 0)[0] + 0.5
    assert u == (0xE220A8397B1DCDAF >> 11) / float(1 << 53)


# ---------------------------------------------------------------- Krylov
def test_cg_and_cgs_on_small_systems():
    rng = np.random.default_rng(5)
    M = rng.standard_normal((40, 40)) + 1j * rng.standard_normal((40, 40))
    H = M @ M.conj().T + 40 * np.eye(40)
    b = rng.standard_normal(40) + 1j * rng.standard_normal(40)
    x, it, res = krylov.cg(lambda v: H @ v, b, 1e-12)
    assert np.linalg.norm(x - np.linalg.solve(H, b)) < 1e-10 * np.linalg.norm(x)
    G = M + 15 * np.eye(40)
    y, it2, res2 = krylov.cgs(lambda v: G @ v, b, 1e-12)
    assert np.linalg.norm(y - np.linalg.solve(G, b)) < 1e-9 * np.linalg.norm(y)


# ---------------------------------------------------------------- voltage gap
def test_voltage_gap_flux_and_loop():
    # the flux of an (unnormalised) RWG function through its own edge is 1, so a delta gap of
    # voltage V gives e_n = +-V on the gap edges; the gap edges close into a loop around the cut
    m = synth.geodesic_sphere(4, seed=5)
    D = efie.discretize(m.verts, m.tris)
    origin, normal = [0.0, 0.0, 0.1], [0.2, 0.1, 1.0]
    e = efie.excitation_voltage_gap(D, origin, normal, 2.5)[:, 0]
    cut, s = efie.gap_edges(D, origin, normal)
    assert cut.size > 0
    assert np.abs(np.abs(e[cut]) - 2.5).max() <= 1e-13
    assert np.abs(np.delete(e, cut)).max() == 0.0
    assert np.array_equal(np.sign(e[cut].real), s)
    # a closed line: every vertex touched by the gap edges meets two of them
    vs, counts = np.unique(D.top.edge_verts[cut].ravel(), return_counts=True)
    assert (counts % 2 == 0).all()
    # the impressed field is a gradient jump across the line: e is Sigma times the indicator of one side
    side = ((D.cent - origin) @ (np.array(normal) / np.linalg.norm(normal)) > 0).astype(float)
    assert np.abs(e.real - 2.5 * (D.Sigma @ (1.0 - side))).max() <= 1e-13


@pytest.mark.slow
def test_dense_discretization_stability():
    # Sec. 4 (Fig. SphereH): the RF-CMP condition number stays bounded as h -> 0 at fixed k,
    # while the plain EFIE's grows like h^-2 (here N = 120 -> 480, h halves)
    cond_A, cond_T = [], []
    for n in (2, 4):
        m = synth.geodesic_sphere(n, seed=1)
        D = efie.discretize(m.verts, m.tris)
        F = rfcmp.factors(D)
        k = 0.5
        TA, V = efie.assemble(D, k)
        T = efie.efie_matrix(D, TA, V, k)
        cond_A.append(rfcmp.condition_number(F, T, rfcmp.power_scaling(F, TA, V, k, exact=True)))
        sv = np.linalg.svd(T, compute_uv=False)
        cond_T.append(sv[0] / sv[-1])
    assert max(cond_A) < 10 and cond_A[1] / cond_A[0] < 1.1
    assert 3.5 < cond_T[1] / cond_T[0] < 5.0
