"""The 12,800-atom workload in the launch configuration bench.py times (BF16X6 build,
PCG-DC, tol 1e-6), checked where the oracle can follow at this size: sampled rows of E
and sampled entries of b against the direct FP64 sums, and properties that hold at any
size (E symmetric, the solver's residual against the stored E recomputed in FP64 on the
host, sum q = -Q^sol, sum d = 1).

Tolerances as in the small-cell parity tests: E and b entries to 1e-6 of the largest
entry; the residual to the solve tolerance.
"""
import hashlib
import os

import numpy as np
import pytest

from oracle import ewald as ew
from paper_2111_06704_gb300 import cpm
from paper_2111_06704_gb300 import workloads as wl

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

ROWS = [0, 4321, 12799]  # first atom, a middle one, the last one (upper sheet)

# the oracle's answers for this cell and frame, written by
# tests/golden/make_two_sheet_n12800.py (oracle/ alone: FP64 sums, bordered solve)
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                      "two_sheet_n12800.npz")


@pytest.fixture(scope="module")
def full():
    work = wl.precision_cell()
    el, io = work.electrode, work.electrolyte
    ctx = cpm.Context(el.box)  # defaults: BF16X6, PCG-DC
    ctx.cpm_build_E(el.xyz, el.alpha)
    b, qsol = ctx.cpm_potential(io.xyz, io.q, el.chi)
    qb, it, rel = ctx.cpm_solve(b, tol=1e-6, maxit=2000)
    q = ctx.cpm_neutralize(qb.copy(), qsol)
    e_n = ctx.cpm_get_E(cpm.CPM_E_STORED)
    yield work, ctx, e_n, b, qsol, qb, q, it, rel
    ctx.close()


def test_sampled_rows_of_E(full):
    work, ctx, e_n, *_ = full
    el = work.electrode
    g, rc, eps = wl.G_EWALD, wl.RCUT_REAL, wl.KSPACE_EPS
    rows = el.xyz[ROWS]
    a_ij = ew.mix_alpha(el.alpha[ROWS, None], el.alpha[None, :])
    ref = ew.kspace_pairs(rows, el.xyz, el.box, g, eps)
    # real space of the row atoms against every atom; their own r = 0 terms are the
    # diagonal case (Eq. 22), added with the self energy below
    for k, i in enumerate(ROWS):
        others = np.delete(np.arange(el.n), i)
        ref[k, others] += ew.real_space_pairs(el.xyz[i:i + 1], el.xyz[others],
                                              a_ij[k:k + 1, others], el.box, g, rc, False)[0]
        ref[k, i] += ew.real_space_pairs(el.xyz[i:i + 1], el.xyz[i:i + 1], a_ij[k, i],
                                         el.box, g, rc, True)[0, 0]
        ref[k, i] += -2 * g / np.sqrt(np.pi) + np.sqrt(2 / np.pi) * el.alpha[i]
    # neutral-equivalent form: the Ewald constant and the rank-2 part of Eq. 39 dropped,
    # the dipole part (4 pi / V) z_i z_j kept
    vol = float(np.prod(el.box))
    z = el.xyz[:, 2]
    ref += (4 * np.pi / vol) * z[ROWS, None] * z[None, :]
    assert np.abs(e_n[ROWS] - ref).max() < 1e-6 * np.abs(ref).max()
    # symmetry of the whole stored matrix
    assert np.array_equal(e_n, e_n.T)


def test_sampled_entries_of_b(full):
    work, ctx, e_n, b, qsol, *_ = full
    el, io = work.electrode, work.electrolyte
    rows = ROWS
    bsol = ew.electrolyte_potential(el.xyz[rows], el.alpha[rows], io.xyz[0], io.q[0], el.box,
                                    wl.G_EWALD, wl.RCUT_REAL, wl.KSPACE_EPS)
    bsol_n = ew.neutral_form_bsol(bsol, el.xyz[rows], io.xyz[0], io.q[0], el.box, wl.G_EWALD)
    ref = ew.rhs_volts(el.chi[rows], bsol_n)
    assert np.abs(b[0, rows] - ref).max() < 1e-6 * np.abs(b).max()
    assert qsol[0] == pytest.approx(io.q[0].sum())


def test_solution_properties(full):
    work, ctx, e_n, b, qsol, qb, q, it, rel = full
    assert rel[0] <= 1e-6 and it[0] < 200
    # the residual of the first step against the stored matrix, recomputed in FP64
    r = b[0] / ew.KE - e_n @ qb[0]
    assert np.linalg.norm(r) / np.linalg.norm(b[0] / ew.KE) <= 1.01e-6
    assert abs(q.sum() + qsol.sum()) < 1e-12 * np.abs(q).sum()
    d = ctx.cpm_get_d()
    assert d.sum() == pytest.approx(1.0, abs=1e-12)


def test_charges_against_the_oracle(full):
    # the whole q vector of the 12,800-atom cell against the oracle's bordered solve, in
    # the default BF16X6 build: converged (tol 1e-10) within the 1e-6 parity bar, and in
    # the bench's configuration (tol 1e-6) within what that residual allows
    gold = np.load(GOLDEN)
    work, ctx, *_ = full
    el = work.electrode
    digest = hashlib.sha256(np.ascontiguousarray(el.xyz).tobytes() +
                            np.ascontiguousarray(el.alpha).tobytes()).hexdigest()
    assert str(gold["electrode_sha256"]) == digest
    b, qsol = ctx.cpm_potential(gold["ion_xyz"][None], gold["ion_q"][None], el.chi)
    assert np.abs(b[0] - gold["b_neutral"]).max() < 1e-6 * np.abs(gold["b_neutral"]).max()
    assert qsol[0] == pytest.approx(float(gold["q_sol"]), abs=1e-12)
    qb, _, rel = ctx.cpm_solve(b, tol=1e-6, maxit=2000)
    q6 = ctx.cpm_neutralize(qb, qsol)[0]
    err6 = np.linalg.norm(q6 - gold["q"]) / np.linalg.norm(gold["q"])
    qb, _, rel = ctx.cpm_solve(b, tol=1e-10, maxit=4000)
    assert rel[0] <= 1e-10
    q = ctx.cpm_neutralize(qb, qsol)[0]
    err = np.linalg.norm(q - gold["q"]) / np.linalg.norm(gold["q"])
    d = ctx.cpm_get_d()
    err_d = np.linalg.norm(d - gold["d"]) / np.linalg.norm(gold["d"])
    print(f"q error: {err:.3e} converged, {err6:.3e} at tol 1e-6; d error {err_d:.3e}")
    assert err < 1e-6
    assert err_d < 1e-6
    assert err6 < 1e-5
