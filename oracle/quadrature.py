"""Triangle quadrature and per-cell geometry.

The paper states no quadrature.  The workloads name a 7-point triangle rule;
the reading taken is Radon's degree-5 rule (centroid plus two orbits of three
points), exact for polynomials of total degree <= 5.  In barycentric
coordinates (l1, l2, l3), weights summing to 1 (multiplied by the area):
  (1/3, 1/3, 1/3)                     9/40
  (a, a, 1-2a) and permutations       (155 - sqrt15)/1200,  a = (6 - sqrt15)/21
  (b, b, 1-2b) and permutations       (155 + sqrt15)/1200,  b = (6 + sqrt15)/21
"""

from __future__ import annotations

import numpy as np

_S15 = np.sqrt(15.0)
_A = (6.0 - _S15) / 21.0
_B = (6.0 + _S15) / 21.0
_WA = (155.0 - _S15) / 1200.0
_WB = (155.0 + _S15) / 1200.0

BARY7 = np.array(
    [
        [1.0 / 3.0, 1.0 / 3.0, 1.0 / 3.0],
        [_A, _A, 1.0 - 2.0 * _A],
        [_A, 1.0 - 2.0 * _A, _A],
        [1.0 - 2.0 * _A, _A, _A],
        [_B, _B, 1.0 - 2.0 * _B],
        [_B, 1.0 - 2.0 * _B, _B],
        [1.0 - 2.0 * _B, _B, _B],
    ]
)
W7 = np.array([9.0 / 40.0, _WA, _WA, _WA, _WB, _WB, _WB])


def cell_geometry(verts: np.ndarray, tris: np.ndarray):
    """Area, unit normal (from the CCW order) and centroid of every cell."""
    p = verts[tris]  # (N_C, 3 vertices, 3)
    cr = np.cross(p[:, 1] - p[:, 0], p[:, 2] - p[:, 0])
    twice = np.linalg.norm(cr, axis=1)
    return 0.5 * twice, cr / twice[:, None], p.mean(axis=1)


def quad_points(verts: np.ndarray, tris: np.ndarray, bary: np.ndarray = BARY7) -> np.ndarray:
    """Quadrature points r = sum_i l_i p_i of every cell: (N_C, Q, 3)."""
    p = verts[tris]
    return np.einsum("qi,cij->cqj", bary, p)
