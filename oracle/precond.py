"""The PCG-DC preconditioner, built atom by atom, and the sparsified-inverse
preconditioners PCG-Normal and PCG-Full it is compared with (test infrastructure only).

Sec. III B 2, steps 1)-3) and Eq. 36-37.  Readings where the text leaves room:
* neighbours of tau are the atoms j with r_tau_j <= r_cut (inclusive), tau included;
  the minimum-image distance is used (r_cut must be below half of every box edge);
* the off-diagonal entry is (erfc(g r) - erfc(g r_cut)) / r for r < r_cut, read
  literally from Eq. 36, which makes it continuous (zero) at r_cut;
* P is used as built (column tau of M_tau^-1); it is not symmetric.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erfc


def _min_image(d, box):
    L = np.asarray(box, dtype=np.float64)
    return d - L * np.round(d / L)


def neighbours(xyz, box, rcut: float):
    """For every atom, the sorted indices j (itself included) with |r_tau - r_j| <= rcut."""
    xyz = np.asarray(xyz, dtype=np.float64)
    if 2.0 * rcut >= min(float(v) for v in box):
        raise ValueError("r_cut must be below half of every box edge")
    out = []
    for t in range(xyz.shape[0]):
        d = _min_image(xyz - xyz[t], box)
        r = np.sqrt(np.einsum("ij,ij->i", d, d))
        out.append(np.nonzero(r <= rcut)[0])
    return out


def local_matrix(idx, xyz, alpha, box, g_dc: float, rcut: float):
    """M_tau of Eq. 36 over the neighbourhood ``idx``."""
    pts = np.asarray(xyz, dtype=np.float64)[idx]
    n = len(idx)
    m = np.zeros((n, n))
    for a in range(n):
        d = _min_image(pts - pts[a], box)
        r = np.sqrt(np.einsum("ij,ij->i", d, d))
        for c in range(n):
            if a == c:
                m[a, c] = math.sqrt(2.0 / math.pi) * float(alpha[idx[a]])
            elif r[c] < rcut:
                m[a, c] = (erfc(g_dc * r[c]) - erfc(g_dc * rcut)) / r[c]
    return m


def dc_preconditioner(xyz, alpha, box, g_dc: float, rcut: float):
    """Dense P: column tau holds column tau of M_tau^-1 on tau's neighbours, zeros
    elsewhere (Sec. III B 2 steps 1-3).  Returns (P, neighbour lists)."""
    xyz = np.asarray(xyz, dtype=np.float64)
    n = xyz.shape[0]
    nb = neighbours(xyz, box, rcut)
    p = np.zeros((n, n))
    for t in range(n):
        idx = nb[t]
        m = local_matrix(idx, xyz, alpha, box, g_dc, rcut)
        minv = np.linalg.inv(m)
        pos = int(np.nonzero(idx == t)[0][0])
        p[idx, t] = minv[:, pos]
    return p, nb


def p_gap(p, sum_einv: float, nb):
    """Eq. 37: p_gap = (sum_ij e^-1_ij - sum_ij p_ij) / n_zero, n_zero = number of
    entries of P outside the neighbour pattern."""
    n = p.shape[0]
    nnz = sum(len(x) for x in nb)
    n_zero = n * n - nnz
    return (sum_einv - float(p.sum())) / n_zero


def fill_gap(p, nb, gap: float):
    """P with every entry outside the neighbour pattern replaced by p_gap (Eq. 37)."""
    out = np.full_like(p, gap)
    for t, idx in enumerate(nb):
        out[idx, t] = p[idx, t]
    return out


def sparsified_inverse(e, xyz, box, rcut: float, strict: bool = True):
    """PCG-Normal / PCG-Full (Sec. III B 2, Fig. 2a-c, Fig. 6a): P keeps the entries of
    E^-1 for the pairs within rcut and is zero elsewhere.  PCG-Normal: r_ij < r_cut
    (strict, as printed).  PCG-Full: every pair of the neighbour list, read as the
    real-space cutoff (pass it with strict=False).  r_ij is the minimum-image distance, so
    a pair counts once whatever its images.  Returns (P, pattern lists)."""
    xyz = np.asarray(xyz, dtype=np.float64)
    einv = np.linalg.inv(np.asarray(e, dtype=np.float64))
    d = _min_image(xyz[:, None, :] - xyz[None, :, :], box)
    r = np.sqrt(np.einsum("ijk,ijk->ij", d, d))
    mask = r < rcut if strict else r <= rcut
    return np.where(mask, einv, 0.0), [np.nonzero(mask[:, t])[0] for t in range(len(xyz))]
