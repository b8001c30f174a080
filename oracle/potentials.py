"""Closed-form integrals of 1/R and (r' - p)/R over a flat triangle.

The paper leaves the singular integration to the reader.  The reading taken
(singularity extraction on near pairs) needs, for an observation point r and a
source triangle T with unit normal n, height d = n.(r - P_0) and projection
p = r - d n:

  S(r)   = int_T 1 / |r - r'| dS'
  Vv(r)  = int_T (r' - p) / |r - r'| dS'

Both follow from Stokes' theorem on the plane of T as sums over its three
edges (the classical closed forms of Wilton et al., 1984, and Graglia, 1993).
For edge i running from P_a to P_b (counter-clockwise about n):
  l = unit edge vector, u = l x n (outward in-plane edge normal),
  l+ = (P_b - p).l, l- = (P_a - p).l, P0 = (P_a - p).u (signed),
  R0^2 = P0^2 + d^2, R+- = sqrt(l+-^2 + R0^2),
  F = ln((R+ + l+)/(R- + l-)),
  S  = sum_i [ P0 F - |d| (atan(P0 l+/(R0^2 + |d| R+)) - atan(P0 l-/(R0^2 + |d| R-))) ]
  Vv = 1/2 sum_i u [ R0^2 F + l+ R+ - l- R- ].
R +- l is evaluated as R0^2 / (R -+ l) when l < 0 to avoid cancellation; F is
taken as 0 when R0 vanishes (the point lies on the edge line, where every
term carrying F is multiplied by P0 or R0^2).
"""

from __future__ import annotations

import numpy as np


def _rpl(R, l, R02):
    """R + l computed without cancellation (R >= |l|)."""
    safe = np.where(R - l > 0, R - l, 1.0)
    return np.where(l > 0, R + l, R02 / safe)


def triangle_potentials(r: np.ndarray, tri: np.ndarray):
    """S and Vv for observation points r (M, 3) and triangles tri (M, 3, 3).

    Returns S (M,), Vv (M, 3) and the projection p (M, 3).
    """
    r = np.asarray(r, dtype=np.float64)
    P = np.asarray(tri, dtype=np.float64)
    cr = np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0])
    n = cr / np.linalg.norm(cr, axis=1, keepdims=True)
    d = np.einsum("mj,mj->m", r - P[:, 0], n)
    p = r - d[:, None] * n
    ad = np.abs(d)
    S = np.zeros(r.shape[0])
    Vv = np.zeros_like(r)
    for i in range(3):
        Pa = P[:, i]
        Pb = P[:, (i + 1) % 3]
        ev = Pb - Pa
        le = np.linalg.norm(ev, axis=1, keepdims=True)
        lh = ev / le
        u = np.cross(lh, n)
        lp = np.einsum("mj,mj->m", Pb - p, lh)
        lm = np.einsum("mj,mj->m", Pa - p, lh)
        P0 = np.einsum("mj,mj->m", Pa - p, u)
        R02 = P0 * P0 + d * d
        Rp = np.sqrt(lp * lp + R02)
        Rm = np.sqrt(lm * lm + R02)
        scale = le[:, 0]
        tiny = R02 <= (1e-30 * scale * scale)
        num = _rpl(Rp, lp, R02)
        den = _rpl(Rm, lm, R02)
        F = np.where(tiny, 0.0, np.log(np.where(tiny, 1.0, num / np.where(tiny, 1.0, den))))
        denp = R02 + ad * Rp
        denm = R02 + ad * Rm
        at = np.where(
            ad > 0,
            np.arctan2(P0 * lp, np.where(denp > 0, denp, 1.0)) - np.arctan2(P0 * lm, np.where(denm > 0, denm, 1.0)),
            0.0,
        )
        S += P0 * F - ad * at
        Vv += 0.5 * u * (R02 * F + lp * Rp - lm * Rm)[:, None]
    return S, Vv, p
