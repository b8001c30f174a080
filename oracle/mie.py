"""Mie series of a perfectly conducting sphere (textbook closed form).

Incident x-polarised plane wave along +z, e^{-i w t}, sphere radius a, size
parameter x = k a.  With the Riccati-Bessel functions psi_n(x) = x j_n(x) and
xi_n(x) = x h_n^(1)(x), the coefficients of a perfect conductor are
  a_n = psi_n'(x) / xi_n'(x),   b_n = psi_n(x) / xi_n(x),
the amplitudes
  S1 = sum (2n+1)/(n(n+1)) (a_n pi_n + b_n tau_n),
  S2 = sum (2n+1)/(n(n+1)) (a_n tau_n + b_n pi_n),
with pi_n = P_n^1(cos t)/sin t and tau_n = d P_n^1(cos t)/dt from their
three-term recurrences, and the bistatic cross sections
  sigma_E(t) = 4 pi |S2|^2 / k^2   (phi = 0 cut, the plane of E),
  sigma_H(t) = 4 pi |S1|^2 / k^2   (phi = 90 deg cut).
The spherical Bessel functions are scipy's (a library routine as a step).
"""

from __future__ import annotations

import numpy as np
from scipy.special import spherical_jn, spherical_yn


def _angular(nmax: int, mu: np.ndarray):
    pi = np.zeros((nmax + 1, mu.size))
    tau = np.zeros((nmax + 1, mu.size))
    pi[1] = 1.0
    tau[1] = mu
    for n in range(2, nmax + 1):
        pi[n] = ((2 * n - 1) * mu * pi[n - 1] - n * pi[n - 2]) / (n - 1)
        tau[n] = n * mu * pi[n] - (n + 1) * pi[n - 1]
    return pi, tau


def pec_sphere_amplitudes(ka: float, theta: np.ndarray, nmax: int | None = None):
    x = float(ka)
    if nmax is None:
        nmax = int(np.ceil(x + 4.05 * x ** (1.0 / 3.0) + 10))
    n = np.arange(1, nmax + 1)
    jn = spherical_jn(n, x)
    yn = spherical_yn(n, x)
    jnp = spherical_jn(n, x, derivative=True)
    ynp = spherical_yn(n, x, derivative=True)
    psi = x * jn
    dpsi = jn + x * jnp
    xi = x * (jn + 1j * yn)
    dxi = (jn + 1j * yn) + x * (jnp + 1j * ynp)
    an = dpsi / dxi
    bn = psi / xi
    pi, tau = _angular(nmax, np.cos(theta))
    c = ((2 * n + 1) / (n * (n + 1)))[:, None]
    S1 = (c * (an[:, None] * pi[1:] + bn[:, None] * tau[1:])).sum(axis=0)
    S2 = (c * (an[:, None] * tau[1:] + bn[:, None] * pi[1:])).sum(axis=0)
    return S1, S2


def pec_sphere_rcs(k: float, a: float, theta: np.ndarray):
    """(sigma_E, sigma_H) in m^2 on the phi = 0 and phi = 90 deg cuts."""
    S1, S2 = pec_sphere_amplitudes(k * a, np.asarray(theta, dtype=np.float64))
    return 4.0 * np.pi * np.abs(S2) ** 2 / k**2, 4.0 * np.pi * np.abs(S1) ** 2 / k**2
