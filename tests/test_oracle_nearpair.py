"""Pins of the oracle's near-pair integrals and sampled rows against independent quadrature.

The oracle integrates cell pairs that share a vertex by singularity extraction: closed-form
integrals of 1/R and (r' - p)/R over the source cell, the bounded remainder
(e^{ikR} - 1)/(4 pi R) = (-2 sin^2(kR/2) + i sin kR)/(4 pi R) by the 7-point rule (value
i k/(4 pi) at R = 0), a 7-point outer rule, and the mean of both orders.  The reference here
integrates the FULL kernel e^{ikR}/(4 pi R) over the source cell with no extraction: polar
coordinates about the foot of the observation point on the source plane, one sub-triangle per
edge, Gauss-Legendre in the edge parameter and, in the radial direction, the substitution
rho = |d| sinh(s) (d = height above the plane), which turns rho drho / R into |d| sinh(s) ds
and leaves an analytic integrand.  Outer rule and the mean of both orders are the oracle's
stated definition of a near-pair entry and are taken over; everything inside the source-cell
integral is independent.

What the comparison can resolve:
  * k = 0: both sides are exact up to the reference's quadrature (1e-11 at 120 x 120 points).
  * Im G = sin(kR)/(4 pi R) is an even power series in R, so the oracle's 7-point remainder rule
    integrates it up to a (kh)^6/5040 term: imaginary parts agree to ~1e-9 (k = 1) and ~1e-6
    (k = 3) on a mesh with h ~ 0.14.  They carry the i k/(4 pi) value at R = 0 (15 % of the
    self-pair Im I0 comes from the seven coincident points) and the sin kR form.
  * Re G - 1/(4 pi R) = -2 sin^2(kR/2)/(4 pi R) ~ -k^2 R/(8 pi) has a kink at R = 0 that the
    7-point rule integrates to within 3-8 % on a self pair (the error falls about 8x per
    subdivision of the source cell: quadrature, not formula), 0.3 % on an edge pair and 0.1 %
    on a vertex pair; the real remainder is held to 12 %, 1 % and 0.3 %, which a dropped
    factor (100 %) or sign (200 %) in -2 sin^2(kR/2) exceeds by far.
"""

import numpy as np
import pytest

import synth
from oracle import efie
from oracle.quadrature import W7

FOUR_PI = 4.0 * np.pi


# ---------------------------------------------------------------- independent source-cell integral
def _inner_reference(r, T, ct, k, n=120):
    """int_T G(r, r') dS' and int_T (r' - ct) G(r, r') dS', G = e^{ikR}/(4 pi R), by polar quadrature."""
    cr = np.cross(T[1] - T[0], T[2] - T[0])
    nh = cr / np.linalg.norm(cr)
    d = (r - T[0]) @ nh
    p = r - d * nh
    x, w = np.polynomial.legendre.leggauss(n)
    g, wg = 0.5 * (x + 1.0), 0.5 * w
    J0 = 0j
    J1 = np.zeros(3, complex)
    size = np.linalg.norm(T[1] - T[0])
    for i in range(3):
        a = T[i] - p
        b = T[(i + 1) % 3] - p
        jac = np.cross(a, b) @ nh  # twice the signed area of (p, P_i, P_i+1)
        e = (1.0 - g)[:, None] * a[None] + g[:, None] * b[None]  # edge points relative to p
        L = np.linalg.norm(e, axis=1)
        if abs(d) > 1e-12 * size:
            smax = np.arcsinh(L / abs(d))
            s = g[None, :] * smax[:, None]
            u = abs(d) * np.sinh(s) / L[:, None]  # radial fraction along p -> edge point
            wt = wg[None, :] * smax[:, None] * abs(d) * np.sinh(s) / L[:, None] ** 2  # u du / R
            R = abs(d) * np.cosh(s)
        else:
            u = np.broadcast_to(g[None, :], (n, n))
            wt = np.broadcast_to(wg[None, :] / L[:, None], (n, n))
            R = u * L[:, None]
        rp = p[None, None, :] + u[:, :, None] * e[:, None, :]
        ww = jac * wg[:, None] * wt * np.exp(1j * k * R) / FOUR_PI
        J0 += ww.sum()
        J1 += np.einsum("ab,abx->x", ww, rp - ct)
    return J0, J1


def _reference_one_order(D, s, t, k, n):
    T = D.verts[D.tris[t]]
    I0 = 0j
    Ir = np.zeros(3, complex)
    Irp = np.zeros(3, complex)
    Irr = 0j
    for q in range(7):
        r = D.qp[s, q]
        J0, J1 = _inner_reference(r, T, D.cent[t], k, n)
        w = W7[q] * D.area[s]
        rho = r - D.cent[s]
        I0 += w * J0
        Ir += w * rho * J0
        Irp += w * J1
        Irr += w * (rho @ J1)
    return I0, Ir, Irp, Irr


def _reference_moments(D, s, t, k, n=120):
    a = _reference_one_order(D, s, t, k, n)
    b = _reference_one_order(D, t, s, k, n)
    # with t outer, rho and rho' exchange roles
    return 0.5 * (a[0] + b[0]), 0.5 * (a[1] + b[2]), 0.5 * (a[2] + b[1]), 0.5 * (a[3] + b[3])


def _oracle_moments(D, s, t, k):
    I0, Ir, Irp, Irr = efie.near_moments(D, np.array([s]), np.array([t]), k)
    return I0[0], Ir[0], Irp[0], Irr[0]


@pytest.fixture(scope="module")
def l3():
    m = synth.geodesic_sphere(8, seed=1)  # h ~ 0.14
    D = efie.discretize(m.verts, m.tris)
    s = 5
    cand = D.near[D.near[:, 0] == s, 1]
    shared = [len(set(D.tris[s]) & set(D.tris[t])) for t in cand]
    pairs = {kind: (s, int(cand[shared.index(nv)])) for kind, nv in (("self", 3), ("edge", 2), ("vertex", 1))}
    return D, pairs


def _rel(a, b):
    a, b = np.ravel(a), np.ravel(b)
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("kind", ["self", "edge", "vertex"])
def test_near_moments_static_match_polar_reference(l3, kind):
    D, pairs = l3
    s, t = pairs[kind]
    o = _oracle_moments(D, s, t, 0.0)
    r = _reference_moments(D, s, t, 0.0)
    for name, oi, ri in zip(("I0", "Ir", "Irp", "Irr"), o, r):
        assert np.abs(np.imag(oi)).max() == 0.0
        assert _rel(np.real(oi), np.real(ri)) < 1e-9, (kind, name, _rel(np.real(oi), np.real(ri)))


@pytest.mark.parametrize("k,tol", [(1.0, 5e-8), (3.0, 3e-6)])
@pytest.mark.parametrize("kind", ["self", "edge", "vertex"])
def test_near_moments_imaginary_part_match_reference(l3, kind, k, tol):
    D, pairs = l3
    s, t = pairs[kind]
    o = _oracle_moments(D, s, t, k)
    r = _reference_moments(D, s, t, k)
    for name, oi, ri in zip(("I0", "Ir", "Irp", "Irr"), o, r):
        e = _rel(np.imag(oi), np.imag(ri))
        assert e < tol, (kind, k, name, e)


REAL_REMAINDER_TOL = {"self": 0.12, "edge": 1e-2, "vertex": 3e-3}


@pytest.mark.parametrize("k", [1.0, 3.0])
@pytest.mark.parametrize("kind", ["self", "edge", "vertex"])
def test_near_moments_real_remainder_match_reference(l3, kind, k):
    # Re of the bounded remainder: moments at k minus the static moments, on both sides
    D, pairs = l3
    s, t = pairs[kind]
    o, o0 = _oracle_moments(D, s, t, k), _oracle_moments(D, s, t, 0.0)
    r, r0 = _reference_moments(D, s, t, k), _reference_moments(D, s, t, 0.0)
    for name, a, a0, b, b0 in zip(("I0", "Ir", "Irp", "Irr"), o, o0, r, r0):
        e = _rel(np.real(a) - np.real(a0), np.real(b) - np.real(b0))
        assert e < REAL_REMAINDER_TOL[kind], (kind, k, name, e)


def test_self_pair_value_at_coincident_points_is_visible(l3):
    # the seven coincident points of a self pair carry i k/(4 pi) x sum_q (w_q A)^2 of Im I0:
    # dropping that value would move Im I0 by far more than the tolerance above
    D, pairs = l3
    s, _ = pairs["self"]
    k = 1.0
    share = k / FOUR_PI * np.sum((W7 * D.area[s]) ** 2)
    im = np.imag(_reference_moments(D, s, s, k)[0])
    assert share / im > 0.1


# ---------------------------------------------------------------- T_A rows straight from the RWG functions
def _rwg_on_cell(D, m, c):
    """(sigma, free vertex) of RWG function m on cell c: f_m = sigma (r - P)/(2 A_c)."""
    cp, cm = D.top.edge_cells[m]
    ev = set(D.top.edge_verts[m].tolist())
    free = [v for v in D.tris[c] if v not in ev]
    assert len(free) == 1
    return (1.0 if c == cp else -1.0), D.verts[free[0]]


def _direct_cell_pair(D, m, n, s, t, k, near, cache):
    """int_s int_t f_m(r) . f_n(r') G dS dS' from the definition of the RWG functions."""
    sm, Pm = _rwg_on_cell(D, m, s)
    sn, Pn = _rwg_on_cell(D, n, t)
    fm = sm * (D.qp[s] - Pm) / (2.0 * D.area[s])  # (7, 3)
    fn = sn * (D.qp[t] - Pn) / (2.0 * D.area[t])
    if not near:
        R = np.linalg.norm(D.qp[s][:, None, :] - D.qp[t][None, :, :], axis=2)
        w = np.outer(W7 * D.area[s], W7 * D.area[t])
        return np.sum(w * np.exp(1j * k * R) / (FOUR_PI * R) * (fm @ fn.T))
    # near: 7-point outer rule, independent inner integral, mean of both orders
    tot = 0j
    for (a, fa, b, sb, Pb) in ((s, fm, t, sn, Pn), (t, fn, s, sm, Pm)):
        Tb = D.verts[D.tris[b]]
        for q in range(7):
            key = (a, q, b, k)
            if key not in cache:
                cache[key] = _inner_reference(D.qp[a, q], Tb, D.cent[b], k, n=96)
            J0, J1 = cache[key]
            inner = sb / (2.0 * D.area[b]) * (J1 + (D.cent[b] - Pb) * J0)  # int_b f(r') G
            tot += 0.5 * W7[q] * D.area[a] * (fa[q] @ inner)
    return tot


def test_ta_rows_from_rwg_definition():
    m_ = synth.geodesic_sphere(3, seed=4)  # 180 cells, N = 270
    D = efie.discretize(m_.verts, m_.tris)
    c0 = 7
    rows = [int(e) for e in D.top.cell_edges[c0]]
    near = {(int(a), int(b)) for a, b in D.near}
    cache = {}
    for k in (1e-8, 1.0):
        TA_rows, _ = efie.assemble_rows(D, k, rows, [])
        for r, m in enumerate(rows):
            direct = np.zeros(D.N, complex)
            for n in range(D.N):
                for s in D.top.edge_cells[m]:
                    for t in D.top.edge_cells[n]:
                        direct[n] += _direct_cell_pair(D, m, n, int(s), int(t), k, (int(s), int(t)) in near, cache)
            got = TA_rows[r]
            # far entries: the same 7 x 7 rule, only the algebra differs
            far = np.array([all((int(s), int(t)) not in near for s in D.top.edge_cells[m] for t in D.top.edge_cells[n])
                            for n in range(D.N)])
            assert np.abs(got[far] - direct[far]).max() <= 1e-12 * np.abs(direct).max()
            if k < 1e-6:  # static: exact up to the reference quadrature
                assert _rel(got.real, direct.real) < 1e-9
            else:
                assert _rel(got.imag, direct.imag) < 1e-8
                assert _rel(got.real, direct.real) < 1e-3


# ---------------------------------------------------------------- sampled rows = full assembly
@pytest.mark.parametrize("ka", [1.0, 1e-5])
def test_assemble_rows_matches_assemble(ka):
    m = synth.geodesic_sphere(4, seed=1)  # 320 cells, N = 480
    D = efie.discretize(m.verts, m.tris)
    TA, V = efie.assemble(D, ka)
    rng = np.random.default_rng(11)
    re = rng.choice(D.N, 9, replace=False)
    rc = rng.choice(D.nc, 7, replace=False)
    TA_rows, V_rows = efie.assemble_rows(D, ka, re, rc)
    for got, full in ((TA_rows, TA[re]), (V_rows, V[rc])):
        assert np.abs(got - full).max() <= 1e-13 * np.abs(full).max()
    # the columns of the same indices (both matrices are complex symmetric)
    assert np.abs(TA_rows - TA[:, re].T).max() <= 1e-13 * np.abs(TA).max()
    assert np.abs(V_rows - V[:, rc].T).max() <= 1e-13 * np.abs(V).max()
