"""Many-column solves with the inner float matvec and residual replacement (matvec_mode 0,
the default for two or more right-hand sides of a float-stored E) against the
error-free matvec throughout (matvec_mode 1) and against the oracle.

The inner matvec sums in float, so between replacements the recursive residual drifts
from the true one; convergence is declared on the replaced (true) residual only, so the
reported relative residual is that of b - E x with the stored E, recomputed here on the
host in FP64, and the charges reach the oracle's as the error-free solve's do.
"""
import numpy as np
import pytest

from oracle import ewald as ew
from paper_2111_06704_gb300 import cpm
from paper_2111_06704_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def true_relres(e_n, b_volts, q):
    b = b_volts / ew.KE
    return np.linalg.norm(b - q @ e_n.T, axis=1) / np.linalg.norm(b, axis=1)


@pytest.mark.parametrize("frames", [2, 17])  # one group, and a ragged second group of 16
def test_fast_and_exact_matvec_solves_agree(small_cell_oracle, frames):
    oc = small_cell_oracle
    el, base = oc.work.electrode, oc.work.electrolyte
    rng = np.random.default_rng(wl.seed_for(3, 21))
    xyz = wl.perturb_frames(rng, base.xyz[0], frames, 0.5, el.box)
    q_ion = np.broadcast_to(base.q[0], (frames, base.n_ion)).copy()
    out = {}
    for mode in (0, 1):
        ctx = cpm.Context(el.box, matvec_mode=mode)
        ctx.cpm_build_E(el.xyz, el.alpha)
        b, qsol = ctx.cpm_potential(xyz, q_ion, el.chi)
        for tol in (1e-6, 1e-10):
            q, it, rel = ctx.cpm_solve(b, tol=tol, maxit=2000)
            e_n = ctx.cpm_get_E(cpm.CPM_E_STORED)
            tr = true_relres(e_n, b, q)
            assert np.all(rel <= tol) and np.all(tr <= 1.01 * tol), (mode, tol)
            assert np.allclose(rel, tr, rtol=1e-3, atol=0)  # the reported one is the true one
            out[(mode, tol)] = (q, it)
        ctx.close()
    q0, it0 = out[(0, 1e-10)]
    q1, it1 = out[(1, 1e-10)]
    assert np.linalg.norm(q0 - q1) <= 1e-8 * np.linalg.norm(q1)
    assert np.all(it0 <= it1 + 8)


def test_fast_matvec_many_columns_against_the_oracle():
    # 3,200 atoms (several 64-row blocks, E rows of 25 stages), 16 frames: every frame's
    # neutral charges against the oracle's bordered solve (factored FP64 k-space form)
    el = wl.two_sheet_electrode(20, 20)
    rng = np.random.default_rng(wl.seed_for(3, 22))
    base, q_ion = wl.random_ions(rng, 250, 250, el.box, min_sep=None)
    xyz = wl.perturb_frames(rng, base, 16, 0.5, el.box)
    qi = np.broadcast_to(q_ion, (16, q_ion.shape[0])).copy()
    ctx = cpm.Context(el.box)
    ctx.cpm_build_E(el.xyz, el.alpha)
    b, qsol = ctx.cpm_potential(xyz, qi, el.chi)
    q, it, rel = ctx.cpm_solve(b, tol=1e-10, maxit=3000)
    q = ctx.cpm_neutralize(q, qsol)
    ctx.close()
    e = ew.interaction_matrix(el.xyz, el.alpha, el.box, wl.G_EWALD, wl.RCUT_REAL,
                              wl.KSPACE_EPS, True, kspace="factored")
    from oracle import solve as sv
    for f in (0, 7, 15):
        bsol = ew.electrolyte_potential(el.xyz, el.alpha, xyz[f], qi[f], el.box, wl.G_EWALD,
                                        wl.RCUT_REAL, wl.KSPACE_EPS, True, kspace="factored")
        q_ref, _ = sv.solve_bordered(e, ew.rhs_volts(el.chi, bsol) / ew.KE, float(qi[f].sum()))
        assert np.linalg.norm(q[f] - q_ref) < 1e-6 * np.linalg.norm(q_ref), f
