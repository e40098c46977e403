"""Forces on the electrolyte ions from the electrode's Gaussian charges, in FP64 (test
infrastructure only).

The energy of the electrode-ion coupling is U = sum_i sum_I q_i q_I e_iI(alpha_i), with
e_iI the point-Gaussian entry of Eq. 25 (the same Ewald form as Eq. 22: real space,
reciprocal space, the constant -pi/(V g^2) and, with the slab correction, Eq. 39).  The
force on ion I is -dU/dr_I.  Its real-space part is the derivative of the pair potential
erf(alpha r)/r of Eq. S25 with the Ewald screening erf(g r)/r taken out.  Eq. S25 prints
the Gaussian-Gaussian force with alpha_ij in the first term and alpha_i in the second;
the derivative of erf(alpha_ij r)/r has alpha_ij in both, which for a point ion
(alpha_iI = alpha_i, Sec. II A) is the same thing.  Units: charges in e, lengths in A,
forces in e^2/A^2 (times k_e for eV/A).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erfc

from .ewald import _image_ranges, kvectors


def _radial_derivative(g: float, alpha, r):
    """d/dr of erfc(g r)/r - erfc(alpha r)/r (alpha may be inf: a point charge)."""
    two_pi = 2.0 / math.sqrt(math.pi)
    point = np.isinf(alpha)
    a = np.where(point, 0.0, alpha)
    gauss = np.where(point, 0.0, two_pi * a * np.exp(-(a * r) ** 2))
    erfc_a = np.where(point, 0.0, erfc(a * r))
    return (-two_pi * g * np.exp(-(g * r) ** 2) + gauss) / r - (erfc(g * r) - erfc_a) / (r * r)


def forces_on_ions(xyz, alpha, q, ion_xyz, ion_q, box, g: float, rc: float,
                   eps: float = 1e-8, slab: bool = True):
    """F_I = -q_I sum_i q_i d e_iI / d r_I for every ion I; shape [N_ion, 3]."""
    xyz = np.asarray(xyz, dtype=np.float64)
    alpha = np.asarray(alpha, dtype=np.float64)
    q = np.asarray(q, dtype=np.float64)
    ion_xyz = np.asarray(ion_xyz, dtype=np.float64)
    ion_q = np.asarray(ion_q, dtype=np.float64)
    L = np.asarray(box, dtype=np.float64)
    vol = float(np.prod(L))
    grad = np.zeros_like(ion_xyz)  # d/dr_I of sum_i q_i e_iI
    # real space: d = r_i - r_I + R_n, r = |d|, so dr/dr_I = -d / r
    nr = _image_ranges(box, rc)
    shifts = np.array([(i, j, k) for i in range(-nr[0], nr[0] + 1)
                       for j in range(-nr[1], nr[1] + 1)
                       for k in range(-nr[2], nr[2] + 1)], dtype=np.float64) * L
    d0 = xyz[:, None, :] - ion_xyz[None, :, :]  # [N, N_ion, 3]
    a_iI = np.broadcast_to(alpha[:, None], d0.shape[:2])
    for s in shifts:
        d = d0 + s
        r = np.sqrt(np.einsum("abk,abk->ab", d, d))
        mask = r < rc
        if not np.any(mask):
            continue
        fr = np.zeros_like(r)
        fr[mask] = _radial_derivative(g, a_iI[mask], r[mask])
        grad -= np.einsum("a,ab,abk->bk", q, fr / np.where(mask, r, 1.0), d)
    # reciprocal space: d/dr_I cos(K . (r_i - r_I)) = sin(K . (r_i - r_I)) K
    _, kvec, w = kvectors(box, g, eps)
    phase = xyz @ kvec.T  # [N, M]
    ion_phase = ion_xyz @ kvec.T  # [N_ion, M]
    c, s_ = q @ np.cos(phase), q @ np.sin(phase)  # [M]
    # sum_i q_i sin(K.r_i - K.r_I) = S_K cos(K.r_I) - C_K sin(K.r_I)
    sin_sum = s_[None, :] * np.cos(ion_phase) - c[None, :] * np.sin(ion_phase)
    grad += (sin_sum * w[None, :]) @ kvec
    # slab correction (Eq. 39): d/dz_I of -(2 pi/V)(z_i - z_I)^2 is (4 pi/V)(z_i - z_I)
    if slab:
        grad[:, 2] += (4.0 * math.pi / vol) * (q @ xyz[:, 2] - q.sum() * ion_xyz[:, 2])
    return -ion_q[:, None] * grad
