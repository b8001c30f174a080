"""Stored expected values (tests/golden, written by make_golden.py from the oracle alone)."""

import os

import numpy as np

from oracle import mie

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "mie_pec_sphere.txt")


def _load():
    rows = np.loadtxt(GOLDEN)
    return rows[:, 0], rows[:, 1], rows[:, 2], rows[:, 3]


def test_mie_table_reproduces():
    """The oracle's Mie series still gives the stored table."""
    ka, th, s_e, s_h = _load()
    for k in np.unique(ka):
        sel = ka == k
        e, h = mie.pec_sphere_rcs(k, 1.0, np.radians(th[sel]))
        np.testing.assert_allclose(e / np.pi, s_e[sel], rtol=1e-10, atol=0)
        np.testing.assert_allclose(h / np.pi, s_h[sel], rtol=1e-10, atol=0)


def test_mie_table_rayleigh_rows():
    """The ka = 0.01 rows follow the dipole (Rayleigh) limit of a small PEC sphere, electric dipole
    4 pi a^3 E and magnetic dipole -2 pi a^3 H: sigma_E / (pi a^2) = 4 (ka)^4 (cos t - 1/2)^2,
    sigma_H / (pi a^2) = 4 (ka)^4 (1 - cos t / 2)^2, up to O((ka)^2) corrections."""
    ka, th, s_e, s_h = _load()
    sel = ka == 0.01
    c = np.cos(np.radians(th[sel]))
    ref_e = 4 * 0.01**4 * (c - 0.5) ** 2
    ref_h = 4 * 0.01**4 * (1 - 0.5 * c) ** 2
    keep = np.abs(c - 0.5) > 0.1  # the E-plane zero at 60 degrees
    np.testing.assert_allclose(s_e[sel][keep], ref_e[keep], rtol=1e-3)
    np.testing.assert_allclose(s_h[sel], ref_h, rtol=1e-3)
    # backscatter 9 (ka)^4 in both planes
    back = th[sel] == 180
    np.testing.assert_allclose(s_e[sel][back], 9 * 0.01**4, rtol=1e-3)
