"""Seeded plane-wave excitations E^i(r) = p e^{i k khat . r} (e^{-i w t})."""

from __future__ import annotations

import numpy as np


def plane_wave_z():
    """x-polarised plane wave travelling along +z: (khat, pol), each (1, 3)."""
    return np.array([[0.0, 0.0, 1.0]]), np.array([[1.0, 0.0, 0.0]])


def random_plane_waves(nrhs: int, seed: int = 33):
    """Directions: normalised Gaussian triples; polarisation cos(psi) theta + sin(psi) phi.

    psi ~ U[0, 2 pi).  theta/phi are the spherical unit vectors of the direction,
    so the polarisation is orthogonal to khat.
    """
    rng = np.random.default_rng(seed)
    d = rng.standard_normal((nrhs, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    th = np.arccos(np.clip(d[:, 2], -1.0, 1.0))
    ph = np.arctan2(d[:, 1], d[:, 0])
    e_th = np.stack([np.cos(th) * np.cos(ph), np.cos(th) * np.sin(ph), -np.sin(th)], axis=1)
    e_ph = np.stack([-np.sin(ph), np.cos(ph), np.zeros_like(ph)], axis=1)
    psi = rng.uniform(0.0, 2.0 * np.pi, nrhs)
    pol = np.cos(psi)[:, None] * e_th + np.sin(psi)[:, None] * e_ph
    return d, pol
