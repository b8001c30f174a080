"""Writes the stored expected values under tests/golden from the oracle alone.

mie_pec_sphere.txt: normalised bistatic cross sections sigma / (pi a^2) of a perfectly conducting
sphere of radius a = 1 m (Mie series, oracle.mie: the reference solution the RCS of the EFIE
solves is compared with) at ka = 0.01, 0.5, 1, 2, 3 and theta = 0, 30, ..., 180 degrees, on the
E-plane (phi = 0) and H-plane (phi = 90 deg) cuts.  The file pins the oracle against silent
drift; tests/test_golden.py also holds its ka = 0.01 rows to the Rayleigh (dipole) limit.

    python tests/golden/make_golden.py
"""

import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import mie  # noqa: E402

KA = (0.01, 0.5, 1.0, 2.0, 3.0)
THETA_DEG = tuple(range(0, 181, 30))


def table():
    th = np.radians(np.asarray(THETA_DEG, dtype=np.float64))
    rows = []
    for ka in KA:
        s_e, s_h = mie.pec_sphere_rcs(ka, 1.0, th)
        for t, e, h in zip(THETA_DEG, s_e / np.pi, s_h / np.pi):
            rows.append((ka, t, e, h))
    return rows


def main():
    path = os.path.join(HERE, "mie_pec_sphere.txt")
    with open(path, "w") as f:
        f.write("# sigma/(pi a^2) of a PEC sphere, Mie series (oracle.mie), written by make_golden.py\n")
        f.write("# ka theta_deg sigma_E_norm sigma_H_norm\n")
        for ka, t, e, h in table():
            f.write("%.17g %d %.17g %.17g\n" % (ka, t, e, h))
    print("wrote", path)


if __name__ == "__main__":
    main()
