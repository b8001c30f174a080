"""Krylov solvers and the dense direct solve.

CG is the solver for the Hermitian positive definite RF-CMP system and CGS
the one for the non-Hermitian comparators (Sec. 4, Fokker experiment).  Both
are the textbook recurrences, start from x0 = 0 and stop when the recursively
updated residual satisfies ||r|| / ||b|| <= tol (the solver's own residual;
the paper does not say which residual its tolerance refers to).
"""

from __future__ import annotations

import numpy as np


def cg(apply, b: np.ndarray, tol: float, maxiter: int = 10000):
    """Conjugate gradients for an HPD operator.  Returns (x, iterations, rel. residual)."""
    x = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    rr = np.vdot(r, r).real
    bn = np.sqrt(np.vdot(b, b).real)
    if bn == 0:
        return x, 0, 0.0
    it = 0
    while np.sqrt(rr) / bn > tol and it < maxiter:
        Ap = apply(p)
        alpha = rr / np.vdot(p, Ap).real
        x = x + alpha * p
        r = r - alpha * Ap
        rr_new = np.vdot(r, r).real
        p = r + (rr_new / rr) * p
        rr = rr_new
        it += 1
    return x, it, np.sqrt(rr) / bn


def cgs(apply, b: np.ndarray, tol: float, maxiter: int = 10000):
    """Conjugate gradients squared (Sonneveld) with the shadow residual r0~ = b."""
    x = np.zeros_like(b)
    r = b.copy()
    rt = b.copy()
    bn = np.linalg.norm(b)
    if bn == 0:
        return x, 0, 0.0
    rho_old = 1.0
    p = np.zeros_like(b)
    q = np.zeros_like(b)
    it = 0
    while np.linalg.norm(r) / bn > tol and it < maxiter:
        rho = np.vdot(rt, r)
        if rho == 0:
            break
        if it == 0:
            u = r.copy()
            p = u.copy()
        else:
            beta = rho / rho_old
            u = r + beta * q
            p = u + beta * (q + beta * p)
        v = apply(p)
        alpha = rho / np.vdot(rt, v)
        q = u - alpha * v
        uq = u + q
        x = x + alpha * uq
        r = r - alpha * apply(uq)
        rho_old = rho
        it += 1
    return x, it, np.linalg.norm(r) / bn


def lu_solve(T: np.ndarray, rhs: np.ndarray) -> np.ndarray:
    """Dense LU with partial pivoting (LAPACK gesv through numpy)."""
    return np.linalg.solve(T, rhs)
