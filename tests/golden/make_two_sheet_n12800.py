"""Writes two_sheet_n12800.npz: the FP64 oracle's answers for the 12,800-atom two-sheet
cell (two graphene sheets of 40 x 40 rectangular cells, 98.4 x 170.4 x 90 A, g = 0.3,
r_c = 12 A, k-space to 1e-8) with one frame of 2,000 ions (1,000 of each sign, 2.5 A
apart, seed 20211106 + 2000), computed by oracle/ alone:

* b_neutral: the extrinsic potential b = chi - k_e b^sol (Eq. 25) in the neutral-equivalent
  form the library returns (volts);
* q: the neutral charges of the bordered electroneutral system (Eq. 29 with Eq. 34);
* d: the neutralising vector d = E_n^-1 1 / (1^T E_n^-1 1) (Eq. S8-S9);
* the ion positions and charges the answers belong to.

The pairwise difference form of the reciprocal sum is too slow at this size, so E and
b^sol take the factored FP64 BLAS form (oracle.ewald.kspace_matrix_factored /
kspace_potential_factored, pinned to the difference form on small cells).  About ten
minutes on eight host cores:

    python tests/golden/make_two_sheet_n12800.py
"""
import hashlib
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import ewald as ew  # noqa: E402
from oracle import solve as sv  # noqa: E402
from paper_2111_06704_gb300 import workloads as wl  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "two_sheet_n12800.npz")


def electrode_digest(xyz, alpha):
    return hashlib.sha256(np.ascontiguousarray(xyz).tobytes() +
                          np.ascontiguousarray(alpha).tobytes()).hexdigest()


def main():
    g, rc, eps = wl.G_EWALD, wl.RCUT_REAL, wl.KSPACE_EPS
    el = wl.two_sheet_electrode(40, 40)
    rng = np.random.default_rng(wl.seed_for(2, 0))
    ions, q_ion = wl.random_ions(rng, 1000, 1000, el.box, min_sep=2.5)
    t0 = time.time()
    e = ew.interaction_matrix(el.xyz, el.alpha, el.box, g, rc, eps, True, kspace="factored")
    print(f"E: {time.time() - t0:.0f} s", flush=True)
    bsol = ew.electrolyte_potential(el.xyz, el.alpha, ions, q_ion, el.box, g, rc, eps, True,
                                    kspace="factored")
    print(f"b^sol: {time.time() - t0:.0f} s", flush=True)
    q_sol = float(q_ion.sum())
    q, _ = sv.solve_bordered(e, ew.rhs_volts(el.chi, bsol) / ew.KE, q_sol)
    print(f"q: {time.time() - t0:.0f} s", flush=True)
    en = ew.neutral_form_matrix(e, el.xyz, el.box, g, True)
    del e
    d, _, c_ele = sv.neutralizing_vector(en)
    b_n = ew.rhs_volts(el.chi, ew.neutral_form_bsol(bsol, el.xyz, ions, q_ion, el.box, g, True))
    np.savez(OUT, ion_xyz=ions, ion_q=q_ion, b_neutral=b_n, q=q, d=d,
             c_ele_neutral=np.float64(c_ele), q_sol=np.float64(q_sol),
             params=np.array([g, rc, eps]),
             electrode_sha256=np.array(electrode_digest(el.xyz, el.alpha)))
    print(f"wrote {OUT} in {time.time() - t0:.0f} s", flush=True)


if __name__ == "__main__":
    main()
