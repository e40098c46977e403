"""Electrode-charge solves in FP64, plain dense linear algebra (test infrastructure only).

A library primitive (LU, inverse) serves as a step; nothing is blocked or reordered
beyond what the cited equation states.
"""
from __future__ import annotations

import numpy as np


def solve_bordered(e, b, q_sol: float = 0.0):
    """Charges under the electroneutrality constraint, straight from its definition:
    E q = b - mu_c 1 (Eq. 29) together with 1^T q + Q^sol = 0 (the constraint behind
    Eq. 34), i.e. the bordered system [[E, 1], [1^T, 0]] [q; mu_c] = [b; -Q^sol].
    Returns (q, mu_c)."""
    e = np.asarray(e, dtype=np.float64)
    n = e.shape[0]
    a = np.zeros((n + 1, n + 1))
    a[:n, :n] = e
    a[:n, n] = 1.0
    a[n, :n] = 1.0
    rhs = np.concatenate([np.asarray(b, dtype=np.float64), [-q_sol]])
    sol = np.linalg.solve(a, rhs)
    return sol[:n], sol[n]


def neutralizing_vector(e):
    """d' = E^-1 1 (Eq. S9), C^ele = 1^T d' (Eq. 32) and d = d' / C^ele (Eq. S8).
    Returns (d, d_prime, c_ele)."""
    e = np.asarray(e, dtype=np.float64)
    dp = np.linalg.solve(e, np.ones(e.shape[0]))
    c = float(dp.sum())
    return dp / c, dp, c


def two_step(e, b, q_sol: float = 0.0):
    """The paper's two-step method (Eq. 35): q^b = E^-1 b, then
    q = q^b - (Q^b + Q^sol) d with Q^b = 1^T q^b and d from Eq. S8-S9."""
    qb = np.linalg.solve(np.asarray(e, dtype=np.float64), np.asarray(b, dtype=np.float64))
    d, _, _ = neutralizing_vector(e)
    return qb - (qb.sum() + q_sol) * d


def neutralize(qb, d, q_sol: float = 0.0):
    """Second step of Eq. 35 applied to a given first-step solution q^b."""
    qb = np.asarray(qb, dtype=np.float64)
    return qb - (qb.sum() + q_sol) * np.asarray(d, dtype=np.float64)


def s_matrix(e):
    """Scalfi's S = E^-1 (I - 1 d^T) (Eq. 33); q = S b when Q^sol = 0."""
    einv = np.linalg.inv(np.asarray(e, dtype=np.float64))
    n = einv.shape[0]
    ones = np.ones(n)
    d = einv @ ones / (ones @ einv @ ones)
    return einv @ (np.eye(n) - np.outer(ones, d))


def pcg(e, b, precond=None, x0=None, tol: float = 1e-6, maxit: int = 10_000,
        flexible: bool = True):
    """Preconditioned conjugate gradient on E x = b (Sec. III B 2: P E q = P b).

    ``precond`` is a dense matrix P (z = P r), or None for plain CG.  Stops when
    ||b - E x||_2 / ||b||_2 <= tol on the recursively updated residual.  With
    ``flexible`` the Polak-Ribiere form beta = r_{k+1}^T (z_{k+1} - z_k) / (r_k^T z_k)
    is used, which stays valid for the non-symmetric PCG-DC preconditioner.
    Returns (x, iterations, relative residual)."""
    e = np.asarray(e, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    r = b - e @ x
    bn = np.linalg.norm(b)
    if bn == 0.0:
        return x, 0, 0.0
    apply = (lambda v: v.copy()) if precond is None else (lambda v: precond @ v)
    z = apply(r)
    p = z.copy()
    rz = r @ z
    rel = np.linalg.norm(r) / bn
    it = 0
    while rel > tol and it < maxit:
        q = e @ p
        alpha = rz / (p @ q)
        x += alpha * p
        r_new = r - alpha * q
        it += 1
        rel = np.linalg.norm(r_new) / bn
        if rel <= tol:
            r = r_new
            break
        z_new = apply(r_new)
        if flexible:
            beta = (r_new @ (z_new - z)) / rz
        else:
            beta = (r_new @ z_new) / rz
        rz = r_new @ z_new
        p = z_new + beta * p
        r, z = r_new, z_new
    return x, it, rel


def jacobi(e):
    """Plain diagonal preconditioner P = diag(E)^-1 (the baseline of the charge solve)."""
    return np.diag(1.0 / np.diag(np.asarray(e, dtype=np.float64)))
