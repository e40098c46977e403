"""Galvanostatic charge-discharge (GCD) constraint in FP64 (test infrastructure only).

Each of M electrodes holds a given total charge Q_a^0 while its atoms stay at one common
potential shift Delta mu_a (Supplementary Note, "Galvanostatic charge-discharge (GCD)
simulation", Eq. S14-S21, and "Iterative approach for GCD-CPM", Eq. S22-S24).  Atoms are
assigned to electrodes by integer labels 0 .. M-1.  Plain dense linear algebra: a library
solve or inverse serves as a step, nothing else is reordered.
"""
from __future__ import annotations

import numpy as np


def indicators(labels, m: int):
    """B [N, M]: column h is b^h of Eq. S22, one on the atoms of electrode h."""
    labels = np.asarray(labels)
    return (labels[:, None] == np.arange(m)[None, :]).astype(np.float64)


def solve_bordered_gcd(e, b, labels, q0):
    """The definition: the stationary point of Eq. S14.  Its derivative in q_i gives
    E q = b + Delta u with Delta u_i = Delta mu of atom i's electrode (Eq. S15), and the
    multipliers enforce B^T q = Q^0; together the bordered system
    [[E, -B], [B^T, 0]] [q; Delta mu] = [b; Q^0].  Returns (q, Delta mu [M])."""
    e = np.asarray(e, dtype=np.float64)
    q0 = np.asarray(q0, dtype=np.float64)
    n, m = e.shape[0], len(q0)
    bm = indicators(labels, m)
    a = np.zeros((n + m, n + m))
    a[:n, :n] = e
    a[:n, n:] = -bm
    a[n:, :n] = bm.T
    sol = np.linalg.solve(a, np.concatenate([np.asarray(b, dtype=np.float64), q0]))
    return sol[:n], sol[n:]


def capacitance_coefficients(e, labels, m: int):
    """A = (a^1 .. a^M) with a^h = E^-1 b^h (Eq. S23) and the capacitance coefficients
    C_ab = sum over atoms of electrode a of a^b (Eq. S24).  Returns (A [N, M], C [M, M])."""
    bm = indicators(labels, m)
    amat = np.linalg.solve(np.asarray(e, dtype=np.float64), bm)
    return amat, bm.T @ amat


def gcd_two_step(e, b, labels, q0):
    """The paper's two-step GCD charges: q^b = E^-1 b, Delta Q_a = Q_a^0 - (charge of
    q^b on electrode a), Delta u_E = C_E^-1 Delta Q_E (Eq. S20), q = q^b + A Delta u_E
    (Eq. S16-S17 with the columns of Eq. S23).  Returns (q, Delta mu [M])."""
    q0 = np.asarray(q0, dtype=np.float64)
    m = len(q0)
    qb = np.linalg.solve(np.asarray(e, dtype=np.float64), np.asarray(b, dtype=np.float64))
    amat, cmat = capacitance_coefficients(e, labels, m)
    dq = q0 - indicators(labels, m).T @ qb
    dmu = np.linalg.solve(cmat, dq)
    return qb + amat @ dmu, dmu


def joint_capacitance(cmat):
    """C(Q, -Q) of two electrodes carrying opposite charges (Eq. S21):
    (C_aa C_bb - C_ab^2) / (C_aa + 2 C_ab + C_bb) = |C_E| / C^ele."""
    cmat = np.asarray(cmat, dtype=np.float64)
    return (cmat[0, 0] * cmat[1, 1] - cmat[0, 1] * cmat[1, 0]) / cmat.sum()
