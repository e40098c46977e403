"""Gaussian Ewald sums in FP64, written out term by term (test infrastructure only).

Conventions.  Gaussian units as in Sec. II A (the 1/(4 pi eps0) factor is dropped), so
E is in 1/A and a potential per unit charge is in e/A; ``KE`` converts e/A to volts.
The Ewald splitting parameter is ``g`` (the paper's eta in Eq. 12-23); the electrode
charge inverse width is ``alpha[i]`` (the paper's alpha_i, Eq. 4).  ``alpha = inf``
marks a point charge.
"""
from __future__ import annotations

import math
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
from scipy.special import erfc

# CODATA e / (4 pi eps0 * 1 Angstrom) in volts: converts e/A to V.
KE = 14.399645478

SQRT_PI = math.sqrt(math.pi)


def kvectors(box, g: float, eps: float = 1e-8):
    """Half-space reciprocal lattice vectors and their weights (Eq. 13, Eq. 20).

    K = 2 pi (h/Lx, k/Ly, l/Lz) != 0 with |K| <= Kc, Kc = 2 g sqrt(ln(1/eps)), so the
    dropped Gaussian factor exp(-K^2/4g^2) is below eps.  Only one of each +-K pair is
    kept (h > 0, or h = 0 and k > 0, or h = k = 0 and l > 0), so the weight is doubled:
    W_K = 2 * (4 pi / V) * exp(-K^2 / 4 g^2) / K^2.

    Returns (hkl int64 [M,3], K float64 [M,3], W float64 [M]).
    """
    lx, ly, lz = (float(v) for v in box)
    vol = lx * ly * lz
    kc = 2.0 * g * math.sqrt(math.log(1.0 / eps))
    hmax = int(math.floor(kc * lx / (2.0 * math.pi)))
    kmax = int(math.floor(kc * ly / (2.0 * math.pi)))
    lmax = int(math.floor(kc * lz / (2.0 * math.pi)))
    h, k, l = np.meshgrid(np.arange(0, hmax + 1), np.arange(-kmax, kmax + 1),
                          np.arange(-lmax, lmax + 1), indexing="ij")
    h, k, l = h.ravel(), k.ravel(), l.ravel()
    half = (h > 0) | ((h == 0) & (k > 0)) | ((h == 0) & (k == 0) & (l > 0))
    h, k, l = h[half], k[half], l[half]
    kvec = np.stack([2.0 * math.pi * h / lx, 2.0 * math.pi * k / ly, 2.0 * math.pi * l / lz],
                    axis=1)
    k2 = np.einsum("ij,ij->i", kvec, kvec)
    keep = k2 <= kc * kc
    kvec, k2 = kvec[keep], k2[keep]
    hkl = np.stack([h[keep], k[keep], l[keep]], axis=1).astype(np.int64)
    w = 2.0 * (4.0 * math.pi / vol) * np.exp(-k2 / (4.0 * g * g)) / k2
    return hkl, kvec, w


def mix_alpha(a, b):
    """Gaussian cross-width law alpha_ij^-2 = alpha_i^-2 + alpha_j^-2 (Sec. II A, after
    Eq. 5).  A point charge (inf) leaves the other width (alpha_ij = alpha_i); two point
    charges give inf."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    inv2 = np.where(np.isinf(a), 0.0, 1.0 / np.where(np.isinf(a), 1.0, a) ** 2) + \
        np.where(np.isinf(b), 0.0, 1.0 / np.where(np.isinf(b), 1.0, b) ** 2)
    with np.errstate(divide="ignore"):
        return np.where(inv2 == 0.0, np.inf, 1.0 / np.sqrt(inv2))


def _erfc_over_r(x, r):
    """erfc(x)/r with erfc(inf) = 0."""
    return np.where(np.isinf(x), 0.0, erfc(np.where(np.isinf(x), 0.0, x))) / r


def _image_ranges(box, rc):
    return [int(math.ceil(rc / float(l))) + 1 for l in box]


def real_space_pairs(ra, rb, alpha_ab, box, g: float, rc: float, same_set: bool):
    """Real-space part of Eq. 22 / Eq. 20 for every (a, b) pair:
    sum over images n with |r_ab + R_n| < rc of erfc(g r)/r - erfc(alpha_ab r)/r.
    With same_set, the n = 0 image of a = b (r = 0) is excluded (the diagonal case of
    Eq. 22 is added by ``interaction_matrix``)."""
    ra = np.asarray(ra, dtype=np.float64)
    rb = np.asarray(rb, dtype=np.float64)
    L = np.asarray(box, dtype=np.float64)
    na, nb = ra.shape[0], rb.shape[0]
    out = np.zeros((na, nb))
    nr = _image_ranges(box, rc)
    shifts = np.array([(i, j, k) for i in range(-nr[0], nr[0] + 1)
                       for j in range(-nr[1], nr[1] + 1)
                       for k in range(-nr[2], nr[2] + 1)], dtype=np.float64) * L
    alpha_ab = np.broadcast_to(np.asarray(alpha_ab, dtype=np.float64), (na, nb))
    rows = max(1, 2_000_000 // max(1, nb))

    def block(a0):
        d = ra[a0:a0 + rows, None, :] - rb[None, :, :]  # [c, nb, 3]
        aab = alpha_ab[a0:a0 + rows]
        for s in shifts:
            dd = d + s
            r = np.sqrt(np.einsum("abk,abk->ab", dd, dd))
            mask = r < rc
            if same_set and not np.any(s):
                ia = np.arange(a0, min(na, a0 + rows))
                mask[ia - a0, ia] = False
            if not np.any(mask):
                continue
            rm = r[mask]
            out[a0:a0 + rows][mask] += _erfc_over_r(g * rm, rm) - _erfc_over_r(aab[mask] * rm, rm)

    # row blocks are independent; numpy releases the GIL, so they run on all host cores
    with ThreadPoolExecutor(max_workers=os.cpu_count() or 1) as pool:
        list(pool.map(block, range(0, na, rows)))
    return out


def kspace_pairs(ra, rb, box, g: float, eps: float = 1e-8):
    """Reciprocal part of Eq. 22-23 in the difference form, pair by pair:
    sum_K W_K cos(K . (r_a - r_b)) over the half-space table of ``kvectors``."""
    _, kvec, w = kvectors(box, g, eps)
    ra = np.asarray(ra, dtype=np.float64)
    rb = np.asarray(rb, dtype=np.float64)
    na, nb, m = ra.shape[0], rb.shape[0], kvec.shape[0]
    out = np.empty((na, nb))
    # tiles of (a rows) x (b columns) x M phases of about 4e6 elements each, so the
    # memory stays bounded however large the sets are
    cb = max(1, min(nb, 4_000_000 // max(1, m)))
    ca = max(1, 4_000_000 // max(1, cb * m))

    def tile(t):
        a0, b0 = t
        d = ra[a0:a0 + ca, None, :] - rb[None, b0:b0 + cb, :]  # [ca, cb, 3]
        out[a0:a0 + ca, b0:b0 + cb] = np.cos(d @ kvec.T) @ w    # phases [ca, cb, M]

    # numpy releases the GIL inside cos/matmul, so tiles run on all host cores.
    tiles = [(a0, b0) for a0 in range(0, na, ca) for b0 in range(0, nb, cb)]
    with ThreadPoolExecutor(max_workers=os.cpu_count() or 1) as pool:
        list(pool.map(tile, tiles))
    return out


def kspace_matrix_factored(xyz, box, g: float, eps: float = 1e-8, chunk: int = 2048):
    """Reciprocal part of Eq. 22-23 for every pair through the angle-addition identity
    cos(K.(r_i - r_j)) = cos(K.r_i) cos(K.r_j) + sin(K.r_i) sin(K.r_j):
    sum_K W_K cos(K.r_ij) = (C W C^T + S W S^T)_ij with C_iK = cos(K.r_i), S_iK = sin(K.r_i).
    The sum over K is a library matrix product (FP64 BLAS), taken over chunks of the
    k-vector table so memory stays bounded.  Equal to ``kspace_pairs`` up to rounding; it
    serves electrodes where the pairwise difference form is too slow."""
    _, kvec, w = kvectors(box, g, eps)
    xyz = np.asarray(xyz, dtype=np.float64)
    n = xyz.shape[0]
    out = np.zeros((n, n))
    for k0 in range(0, kvec.shape[0], chunk):
        ph = xyz @ kvec[k0:k0 + chunk].T                  # K . r_i, [n, c]
        sw = np.sqrt(w[k0:k0 + chunk])
        c = np.cos(ph) * sw
        out += c @ c.T
        c = np.sin(ph) * sw
        out += c @ c.T
    return out


def kspace_potential_factored(xyz, ion_xyz, ion_q, box, g: float, eps: float = 1e-8,
                              chunk: int = 2048):
    """sum_I q_I sum_K W_K cos(K.(r_i - r_I)) for every electrode atom i, through the same
    identity: sum_K W_K [cos(K.r_i) Re S(K) + sin(K.r_i) Im S(K)] with the structure factor
    S(K) = sum_I q_I exp(i K.r_I).  Equal to ``kspace_pairs(...) @ ion_q`` up to rounding."""
    _, kvec, w = kvectors(box, g, eps)
    xyz = np.asarray(xyz, dtype=np.float64)
    ion_xyz = np.asarray(ion_xyz, dtype=np.float64)
    ion_q = np.asarray(ion_q, dtype=np.float64)
    out = np.zeros(xyz.shape[0])
    for k0 in range(0, kvec.shape[0], chunk):
        kc = kvec[k0:k0 + chunk]
        phi = ion_xyz @ kc.T                               # K . r_I, [n_ion, c]
        re, im = np.cos(phi).T @ ion_q, np.sin(phi).T @ ion_q
        ph = xyz @ kc.T
        out += np.cos(ph) @ (w[k0:k0 + chunk] * re) + np.sin(ph) @ (w[k0:k0 + chunk] * im)
    return out


def interaction_matrix(xyz, alpha, box, g: float, rc: float, eps: float = 1e-8,
                       slab: bool = True, kspace: str = "difference"):
    """The Gaussian Ewald interaction matrix E of Eq. 22, entry by entry.

    e_ij = [real space, Eq. 22 first case, summed over images within rc]
         + [reciprocal space, Eq. 23: (4 pi/V) sum_{K != 0} exp(-K^2/4g^2)/K^2 cos(K.r_ij)]
         - pi / (V g^2)
         + (i == j) * (-2 g / sqrt(pi) + 2 alpha_ii / sqrt(pi)),  alpha_ii = alpha_i/sqrt(2)
         + [slab] -(2 pi / V) [(z_i - z_j)^2 + Lz^2 / 6]   (Yeh-Ballenger, Eq. 39)

    The reciprocal prefactor is 4 pi / V as in Eq. 16 (Eq. 23 prints a second 4 pi that
    phi-hat already carries).  The diagonal Gaussian self-energy is Eq. 6,
    sqrt(2/pi) alpha_i; a point charge (alpha = inf) has none (end of Sec. II C).
    ``kspace`` = "factored" sums the reciprocal part by ``kspace_matrix_factored`` (the
    FP64 BLAS form for large electrodes) instead of the pairwise difference form."""
    xyz = np.asarray(xyz, dtype=np.float64)
    alpha = np.asarray(alpha, dtype=np.float64)
    n = xyz.shape[0]
    lx, ly, lz = (float(v) for v in box)
    vol = lx * ly * lz
    a_ij = mix_alpha(alpha[:, None], alpha[None, :])
    e = real_space_pairs(xyz, xyz, a_ij, box, g, rc, same_set=True)
    if kspace == "factored":
        e += kspace_matrix_factored(xyz, box, g, eps)
    else:
        e += kspace_pairs(xyz, xyz, box, g, eps)
    e -= math.pi / (vol * g * g)
    self_e = np.where(np.isinf(alpha), 0.0, math.sqrt(2.0 / math.pi) * np.where(np.isinf(alpha), 0.0, alpha))
    e[np.arange(n), np.arange(n)] += -2.0 * g / SQRT_PI + self_e
    if slab:
        z = xyz[:, 2]
        e += -(2.0 * math.pi / vol) * ((z[:, None] - z[None, :]) ** 2 + lz * lz / 6.0)
    return e


def electrolyte_potential(xyz, alpha, ion_xyz, ion_q, box, g: float, rc: float,
                          eps: float = 1e-8, slab: bool = True, kspace: str = "difference"):
    """b^sol_i = sum_I q_I e_iI(alpha_i) (Eq. 25) for point-charge ions.

    e_iI uses the point-Gaussian coefficient alpha_iI = alpha_i (Sec. II A, after Eq. 5)
    in the same Ewald form as Eq. 22 (off-diagonal case), plus -pi/(V g^2) and, with
    ``slab``, the Eq. 39 correction.  ``kspace`` = "factored" sums the reciprocal part
    through the ions' structure factors (``kspace_potential_factored``).  Returns b^sol
    in e/A, shape [N]."""
    xyz = np.asarray(xyz, dtype=np.float64)
    alpha = np.asarray(alpha, dtype=np.float64)
    ion_xyz = np.asarray(ion_xyz, dtype=np.float64)
    ion_q = np.asarray(ion_q, dtype=np.float64)
    lx, ly, lz = (float(v) for v in box)
    vol = lx * ly * lz
    a_iI = np.broadcast_to(alpha[:, None], (xyz.shape[0], ion_xyz.shape[0]))
    e = real_space_pairs(xyz, ion_xyz, a_iI, box, g, rc, same_set=False)
    if kspace != "factored":
        e += kspace_pairs(xyz, ion_xyz, box, g, eps)
    e -= math.pi / (vol * g * g)
    if slab:
        z, zi = xyz[:, 2], ion_xyz[:, 2]
        e += -(2.0 * math.pi / vol) * ((z[:, None] - zi[None, :]) ** 2 + lz * lz / 6.0)
    out = e @ ion_q
    if kspace == "factored":
        out += kspace_potential_factored(xyz, ion_xyz, ion_q, box, g, eps)
    return out


def rhs_volts(chi, bsol):
    """b_i = chi_i - b^sol_i (Eq. 25) with chi in V and b^sol in e/A; returns V."""
    return np.asarray(chi, dtype=np.float64) - KE * np.asarray(bsol, dtype=np.float64)


# ----------------------------------------------------------------------------------------
# Neutral-equivalent form (the form the GPU library stores).
#
# Eq. 39 expands to -(2 pi/V)(z_i^2 + z_j^2) + (4 pi/V) z_i z_j - (2 pi/V) Lz^2/6, and the
# Ewald constant -pi/(V g^2) is the same for every entry.  Write E = E_n + u 1^T + 1 u^T
# + k0 1 1^T with u_i = -(2 pi/V) z_i^2 and k0 = -pi/(V g^2) - (2 pi/V) Lz^2/6.  For charges
# with 1^T q = -Q^sol (Eq. 34):  E q = E_n q - Q^sol u + (u^T q - k0 Q^sol) 1.  The 1-term
# is absorbed by the multiplier mu_c of Eq. 29-30, and the -Q^sol u term is cancelled by
# the matching Q^sol z_i^2 term of b^sol.  So the neutral q of (E, b) equals the neutral q
# of (E_n, b_n) with the forms below; E_n is positive definite (Gram matrix of the
# reciprocal sum plus a dipole term), E itself is indefinite along 1 for slabs.
# ----------------------------------------------------------------------------------------

def neutral_form_matrix(e, xyz, box, g: float, slab: bool = True):
    """E_n = E + pi/(V g^2) + (2 pi/V)(z_i^2 + z_j^2 + Lz^2/6)."""
    lx, ly, lz = (float(v) for v in box)
    vol = lx * ly * lz
    out = np.array(e, dtype=np.float64) + math.pi / (vol * g * g)
    if slab:
        z = np.asarray(xyz, dtype=np.float64)[:, 2]
        out += (2.0 * math.pi / vol) * (z[:, None] ** 2 + z[None, :] ** 2 + lz * lz / 6.0)
    return out


def neutral_form_bsol(bsol, xyz, ion_xyz, ion_q, box, g: float, slab: bool = True):
    """b^sol_n = b^sol + pi Q/(V g^2) + (2 pi/V)(sum_I q_I z_I^2 + Q z_i^2 + Q Lz^2/6),
    Q = sum_I q_I (the electrode-ion counterpart of ``neutral_form_matrix``)."""
    lx, ly, lz = (float(v) for v in box)
    vol = lx * ly * lz
    ion_q = np.asarray(ion_q, dtype=np.float64)
    qs = float(ion_q.sum())
    out = np.array(bsol, dtype=np.float64) + math.pi * qs / (vol * g * g)
    if slab:
        z = np.asarray(xyz, dtype=np.float64)[:, 2]
        zi = np.asarray(ion_xyz, dtype=np.float64)[:, 2]
        out += (2.0 * math.pi / vol) * (float(ion_q @ (zi * zi)) + qs * z * z + qs * lz * lz / 6.0)
    return out
