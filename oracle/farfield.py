"""Scattered far field and bistatic radar cross section of a surface current.

With e^{-i w t} and j normalised by the wave impedance (Sec. 2), the far field
of the scattered wave is E^s ~ i k e^{ikr}/(4 pi r) (N - rhat (rhat . N)) with
the radiation vector N(rhat) = int j(r') e^{-i k rhat . r'} dS', so for a
unit-amplitude incident wave sigma = (k^2 / 4 pi) |N - rhat (rhat . N)|^2.
The surface integral uses the 7-point rule on every cell.
"""

from __future__ import annotations

import numpy as np

from .quadrature import W7


def radiation_vector(D, j: np.ndarray, k: float, dirs: np.ndarray) -> np.ndarray:
    """N(rhat) for RWG coefficients j (N,) and directions dirs (M, 3): (M, 3) complex."""
    jl = D.B @ j  # local half-function coefficients, sign included: (3 N_C,)
    jl = jl.reshape(D.nc, 3)
    rel = D.qp[:, None, :, :] - D.verts[D.tris][:, :, None, :]  # (N_C, 3, 7, 3)
    # current density at each quadrature point: sum_i jl_i (r - P_i) / (2 A)
    J = np.einsum("ci,ciqx->cqx", jl, rel) / (2.0 * D.area)[:, None, None]
    w = W7[None, :] * D.area[:, None]  # (N_C, 7)
    phase = np.exp(-1j * k * np.einsum("cqx,mx->mcq", D.qp, dirs))
    return np.einsum("mcq,cq,cqx->mx", phase, w, J)


def bistatic_rcs(D, j: np.ndarray, k: float, dirs: np.ndarray) -> np.ndarray:
    """sigma (m^2) in the directions dirs (M, 3)."""
    Nv = radiation_vector(D, j, k, dirs)
    perp = Nv - dirs * np.einsum("mx,mx->m", dirs, Nv)[:, None]
    return (k * k / (4.0 * np.pi)) * np.einsum("mx,mx->m", perp, perp.conj()).real


def cut_directions(theta: np.ndarray, phi: float) -> np.ndarray:
    """Unit vectors (sin t cos p, sin t sin p, cos t) on a constant-phi cut."""
    return np.stack(
        [np.sin(theta) * np.cos(phi), np.sin(theta) * np.sin(phi), np.cos(theta)], axis=1
    )
