"""The refinement-free Calderon multiplicative preconditioner (Sec. 3, Sec. 4).

System (Sec. 3, Eq. NewFormulation):
  P_o^H T^H P_m T P_o i = -P_o^H T^H P_m e,   j = P_o i.
Numerical variant used by the paper (Sec. 4, first display):
  P_o   = P_LH / alpha + i P_S / beta
  P_mL  = Lambda G_ll^{-1} Lambda^T / alpha^2 + P_LH / gamma
  P_mS  = Sigma (Sigma^T Sigma)^+ G_pp^{-1} (Sigma^T Sigma)^+ Sigma^T / beta^2
  P_m   = P_mL + P_mS
with the quasi-Helmholtz projectors (Sec. 2)
  P_S = Sigma (Sigma^T Sigma)^+ Sigma^T,  P_LH = I - P_S,
and the pseudo-inverse from the identity of Sec. 3.2
  (Sigma^T Sigma + 1 1^T / N_C)^{-1} = (Sigma^T Sigma)^+ + 1 1^T / N_C.

alpha, beta, gamma (Sec. 4, second display).  Reading: the norms are taken of
the frequency-scaled pieces i k T_A and T_Phi / (i k) of T, and M_S is P_mS
without its 1/beta^2 (the printed beta formula would otherwise contain beta):
  alpha^4 = k^2      || P_LH T_A^H Lambda G_ll^{-1} Lambda^T T_A P_LH ||_2
  beta^4  = k^{-2}   || P_S T_Phi^H M_S T_Phi P_S ||_2
  gamma   = k^2/alpha^2 || P_LH T_A^H P_LH T_A P_LH ||_2
so each principal diagonal block of the system has unit norm.  Under the
closed-form choice alpha = sqrt k, beta = 1/sqrt k, gamma = k (Sec. 4, third
display) the variant reduces to the theory scaling of Sec. 3.  The norms are
estimated by power iteration (Sec. 4) from a start vector given by the caller
(``splitmix_start``), Rayleigh quotient estimate; at most 30 steps, stopping once
the estimate changes by at most 1e-3 (relative) between steps (the paper states
neither; the solution does not depend on these choices).

Theory variant of the outer preconditioner (Sec. 3, Eq. NewFormulation and Eq. Pgs):
  P_o = P_LH / alpha + i P_gS / beta,  P_gS = Sigma (Sigma^T Sigma)^+ G_l~p^{-1} Sigma^T,
with G_l~p the mixed Gram matrix of the dual piecewise linear functions and the primal pulses
(``gram.g_lambda_tilde_p``); P_m is unchanged.  With alpha = sqrt k, beta = 1/sqrt k,
gamma = k this is the formulation of Sec. 3 exactly.  P_gS is not a projector (nor Hermitian);
the solution j = P_o i is the same, -T^{-1} e.  ``outer="gsigma"`` selects it below.

Low-frequency-stable application (reading of Eq. LastProofBigUmformung with
the separate storage of T_A and V, Sec. 4): the products that vanish exactly,
Sigma^T P_LH = 0, Lambda^T Sigma = 0, P_LH Sigma = 0 and
(Sigma^T Sigma)^+ (Sigma^T Sigma) = I - 1 1^T / N_C, are applied
symbolically, so T_Phi only ever meets star-range vectors.  ``apply_A`` is
that form; ``dense_system`` forms the same matrix naively for small problems.
"""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.linalg as sla

from . import gram


def splitmix_start(n: int, seed: int) -> np.ndarray:
    """Deterministic start vector: u_i = splitmix64(seed * 2^32 + i) / 2^64 - 1/2.

    splitmix64 (Steele, Lea, Flood 2014): z += 0x9E3779B97F4A7C15;
    z = (z ^ z>>30) * 0xBF58476D1CE4E5B9; z = (z ^ z>>27) * 0x94D049BB133111EB;
    z ^ z>>31.  The top 53 bits give u in [0, 1).
    """
    M = (1 << 64) - 1
    out = np.empty(n)
    for i in range(n):
        z = (seed * (1 << 32) + i + 0x9E3779B97F4A7C15) & M
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M
        z = z ^ (z >> 31)
        out[i] = (z >> 11) * (1.0 / (1 << 53)) - 0.5
    return out


@dataclass
class Factors:
    """Topology and metric factors, independent of k."""

    Sigma: np.ndarray  # dense (N, N_C)
    Lambda: np.ndarray  # dense (N, N_V)
    Lplus: np.ndarray  # (Sigma^T Sigma)^+
    Gll_inv: np.ndarray  # G_ll^{-1}
    Gpp_inv: np.ndarray  # diag(A)
    P_S: np.ndarray
    P_LH: np.ndarray
    Gtp_inv: np.ndarray  # G_l~p^{-1} (dual piecewise linear x primal pulse, Sec. 3)
    P_gS: np.ndarray  # Sigma (Sigma^T Sigma)^+ G_l~p^{-1} Sigma^T (Eq. Pgs)


def factors(D) -> Factors:
    S = D.Sigma.toarray()
    L = D.Lambda.toarray()
    nc = D.nc
    J = np.full((nc, nc), 1.0 / nc)
    Lplus = np.linalg.inv(S.T @ S + J) - J  # Sec. 3.2 identity
    Gll_inv = np.linalg.inv(gram.g_ll_loops(D).toarray())
    Gpp_inv = np.diag(D.area)
    P_S = S @ Lplus @ S.T
    if D.top.boundaries == 0:
        Gtp_inv = np.linalg.inv(gram.g_lambda_tilde_p(D).toarray())
        P_gS = S @ Lplus @ Gtp_inv @ S.T
    else:  # the dual functions of Sec. 2 are defined on closed surfaces only
        Gtp_inv = P_gS = None
    return Factors(S, L, Lplus, Gll_inv, Gpp_inv, P_S, np.eye(D.N) - P_S, Gtp_inv, P_gS)


@dataclass
class Scaling:
    alpha: float
    beta: float
    gamma: float


def kscale(k: float) -> Scaling:
    """alpha = sqrt k, beta = 1/sqrt k, gamma = k (Sec. 4, third display)."""
    return Scaling(np.sqrt(k), 1.0 / np.sqrt(k), k)


def power_norm(apply, x0: np.ndarray, steps: int, rtol: float = 0.0) -> float:
    """Largest eigenvalue of an HPSD operator: normalised power steps, Rayleigh quotient.

    Stops after `steps` steps, or earlier (after at least 2) once the Rayleigh quotient
    changes by at most rtol relative to its value.
    """
    x = x0.astype(np.complex128)
    x = x / np.linalg.norm(x)
    lam = 0.0
    for it in range(steps):
        y = apply(x)
        prev, lam = lam, np.vdot(x, y).real
        x = y / np.linalg.norm(y)
        if rtol > 0 and it >= 1 and abs(lam - prev) <= rtol * abs(lam):
            break
    return lam


def block_operators(F: Factors, TA: np.ndarray, V: np.ndarray):
    """The three HPSD operators whose norms define alpha, beta, gamma (unscaled by k)."""
    S = F.Sigma
    MS = S @ F.Lplus @ F.Gpp_inv @ F.Lplus @ S.T
    TPhi = S @ V @ S.T
    LGL = F.Lambda @ F.Gll_inv @ F.Lambda.T
    X = F.P_LH @ TA.conj().T @ LGL @ TA @ F.P_LH
    Y = F.P_S @ TPhi.conj().T @ MS @ TPhi @ F.P_S
    Z = F.P_LH @ TA.conj().T @ F.P_LH @ TA @ F.P_LH
    return X, Y, Z


def power_scaling(F: Factors, TA, V, k: float, steps: int = 30, exact: bool = False, rtol: float = 1e-3) -> Scaling:
    """alpha, beta, gamma by power iteration (Sec. 4), or by exact norms (for pins)."""
    X, Y, Z = block_operators(F, TA, V)
    N = TA.shape[0]
    if exact:
        nx, ny, nz = (np.linalg.eigvalsh(0.5 * (M + M.conj().T))[-1] for M in (X, Y, Z))
    else:
        nx = power_norm(lambda v: X @ v, splitmix_start(N, 1), steps, rtol)
        ny = power_norm(lambda v: Y @ v, splitmix_start(N, 2), steps, rtol)
        nz = power_norm(lambda v: Z @ v, splitmix_start(N, 3), steps, rtol)
    alpha = (k * k * nx) ** 0.25
    beta = (ny / (k * k)) ** 0.25
    gamma = k * k / (alpha * alpha) * nz
    return Scaling(alpha, beta, gamma)


def preconditioners(F: Factors, sc: Scaling, outer: str = "sigma"):
    """Dense P_o and P_m of the numerical variant (Sec. 4); outer="gsigma": P_gS in P_o (Sec. 3)."""
    S = F.Sigma
    Po = F.P_LH / sc.alpha + 1j * (F.P_gS if outer == "gsigma" else F.P_S) / sc.beta
    PmL = F.Lambda @ F.Gll_inv @ F.Lambda.T / sc.alpha**2 + F.P_LH / sc.gamma
    PmS = S @ F.Lplus @ F.Gpp_inv @ F.Lplus @ S.T / sc.beta**2
    return Po, PmL + PmS


def dense_system(F: Factors, T: np.ndarray, sc: Scaling, outer: str = "sigma"):
    """A = P_o^H T^H P_m T P_o and the map b = -P_o^H T^H P_m e (Sec. 3, Eq. NewFormulation)."""
    Po, Pm = preconditioners(F, sc, outer)
    left = Po.conj().T @ T.conj().T @ Pm
    return left @ T @ Po, -left, Po


def apply_A_gsigma(F: Factors, TA, V, k: float, sc: Scaling, x: np.ndarray) -> np.ndarray:
    """A x with P_o = P_LH / alpha + i P_gS / beta, in the low-frequency-stable order.

    With z = L^+ Sigma^T x (x_L = x - Sigma z) and z' = L^+ G^{-1} Sigma^T x (G = G_l~p):
      T P_o x = u + Sigma w,  u = T_A (i k x_L / alpha - k Sigma z' / beta),
                               w = V Pi G^{-1} Sigma^T x / (k beta),  Pi = I - 1 1^T / N_C
    (Sigma^T x_L = 0 and Sigma^T Sigma L^+ = Pi); y = P_m T P_o x as in ``apply_A``; and
      A x = -(i k / alpha) P_LH u' - (k / beta) Sigma G^{-1} L^+ Sigma^T u'
            + Sigma G^{-1} Pi conj(V) L q / (k beta),  u' = conj(T_A) y,  L = Sigma^T Sigma,
    from P_gS^H = Sigma G^{-1} L^+ Sigma^T and Sigma^T y = L q.
    """
    S, Lp, Gi = F.Sigma, F.Lplus, F.Gtp_inv
    a, b, g = sc.alpha, sc.beta, sc.gamma
    s = S.T @ x
    x_L = x - S @ (Lp @ s)
    t = Gi @ s
    u = TA @ (1j * k * x_L / a - k * (S @ (Lp @ t)) / b)
    w = V @ (t - t.mean()) / (k * b)
    zu = Lp @ (S.T @ u)
    uL = u - S @ zu
    q = Lp @ (F.Gpp_inv @ (zu + w - w.mean())) / b**2
    y = F.Lambda @ (F.Gll_inv @ (F.Lambda.T @ u)) / a**2 + uL / g + S @ q
    up = TA.conj() @ y
    zp = Lp @ (S.T @ up)
    vp = V.conj() @ (S.T @ (S @ q)) / (k * b)
    return -(1j * k / a) * (up - S @ zp) + S @ (Gi @ (-(k / b) * zp + vp - vp.mean()))


def apply_rhs_gsigma(F: Factors, TA, V, k: float, sc: Scaling, e: np.ndarray) -> np.ndarray:
    """b = -P_o^H T^H P_m e with P_gS in P_o; P_m e and T^H as in ``apply_rhs``."""
    S, Lp, Gi = F.Sigma, F.Lplus, F.Gtp_inv
    a, b, g = sc.alpha, sc.beta, sc.gamma
    ze = Lp @ (S.T @ e)
    eL = e - S @ ze
    q = Lp @ (F.Gpp_inv @ ze) / b**2
    y = F.Lambda @ (F.Gll_inv @ (F.Lambda.T @ e)) / a**2 + eL / g + S @ q
    up = TA.conj() @ y
    tv = S @ (V.conj() @ (S.T @ (S @ q)))
    th = -1j * k * up + (1j / k) * tv
    zt = Lp @ (S.T @ th)
    return -((th - S @ zt) / a - 1j * (S @ (Gi @ zt)) / b)


def apply_A(F: Factors, TA, V, k: float, sc: Scaling, x: np.ndarray) -> np.ndarray:
    """A x in the low-frequency-stable order (module header).

    With x_S = P_S x, x_L = x - x_S:
      T P_o x = u + Sigma w,  u = T_A (i k x_L / alpha - k x_S / beta),  w = V Sigma^T x / (k beta)
      y = P_m T P_o x = Lambda G_ll^{-1} Lambda^T u / alpha^2 + P_LH u / gamma + Sigma q,
          q = L^+ G_pp^{-1} (L^+ Sigma^T u + w - mean(w)) / beta^2
      A x = -(i k / alpha) P_LH u' - (k / beta) P_S u' + Sigma conj(V) L q / (k beta),
          u' = conj(T_A) y,  L = Sigma^T Sigma.
    """
    S, Lp = F.Sigma, F.Lplus
    a, b, g = sc.alpha, sc.beta, sc.gamma
    x_S = S @ (Lp @ (S.T @ x))
    x_L = x - x_S
    u = TA @ (1j * k * x_L / a - k * x_S / b)
    w = V @ (S.T @ x) / (k * b)
    zu = Lp @ (S.T @ u)
    uL = u - S @ zu
    q = Lp @ (F.Gpp_inv @ (zu + w - w.mean())) / b**2
    y = F.Lambda @ (F.Gll_inv @ (F.Lambda.T @ u)) / a**2 + uL / g + S @ q
    up = TA.conj() @ y
    zp = Lp @ (S.T @ up)
    up_S = S @ zp
    up_L = up - up_S
    Lq = S.T @ (S @ q)
    return -(1j * k / a) * up_L - (k / b) * up_S + S @ (V.conj() @ Lq) / (k * b)


def apply_rhs(F: Factors, TA, V, k: float, sc: Scaling, e: np.ndarray) -> np.ndarray:
    """b = -P_o^H T^H P_m e in the same order (e has no analytically zero parts)."""
    S, Lp = F.Sigma, F.Lplus
    a, b, g = sc.alpha, sc.beta, sc.gamma
    ze = Lp @ (S.T @ e)
    eL = e - S @ ze
    q = Lp @ (F.Gpp_inv @ ze) / b**2
    y = F.Lambda @ (F.Gll_inv @ (F.Lambda.T @ e)) / a**2 + eL / g + S @ q
    # T^H y = -i k conj(T_A) y + (i/k) Sigma conj(V) Sigma^T y
    up = TA.conj() @ y
    Sty = S.T @ (S @ q)  # Sigma^T y: the loop and P_LH parts of y vanish under Sigma^T
    tv = S @ (V.conj() @ Sty)
    th = -1j * k * up + (1j / k) * tv
    zt = Lp @ (S.T @ th)
    th_S = S @ zt
    th_L = th - th_S
    return -(th_L / a - 1j * th_S / b)


def solve(F: Factors, TA, V, k: float, sc: Scaling, e: np.ndarray, tol: float, maxiter: int = 5000,
          outer: str = "sigma"):
    """RF-CMP solve with CG (Sec. 4): returns j = P_o i, iterations, CG residual."""
    from .krylov import cg

    gs = outer == "gsigma"
    bvec = (apply_rhs_gsigma if gs else apply_rhs)(F, TA, V, k, sc, e)
    Aop = apply_A_gsigma if gs else apply_A
    i, it, res = cg(lambda v: Aop(F, TA, V, k, sc, v), bvec, tol, maxiter)
    s = F.Sigma.T @ i
    x_L = i - F.Sigma @ (F.Lplus @ s)
    x_S = F.Sigma @ (F.Lplus @ (F.Gtp_inv @ s if gs else s))
    j = x_L / sc.alpha + 1j * x_S / sc.beta
    return j, it, res


def condition_number(F: Factors, T, sc: Scaling, outer: str = "sigma") -> float:
    A, _, _ = dense_system(F, T, sc, outer)
    ev = np.linalg.eigvalsh(0.5 * (A + A.conj().T))
    return ev[-1] / ev[0]


def pseudo_inverse_check(F: Factors) -> float:
    """|| L^+ - pinv(L) || / || pinv(L) || with L = Sigma^T Sigma (SVD-based pinv)."""
    L = F.Sigma.T @ F.Sigma
    P = sla.pinvh(L)
    return np.linalg.norm(F.Lplus - P) / np.linalg.norm(P)
