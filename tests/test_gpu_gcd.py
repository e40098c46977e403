"""Fixed charge per electrode (GCD, Eq. S14-S24) through the C ABI against the FP64
oracle (oracle/gcd.py).  The library works with the neutral-equivalent E_n; the charges,
the differences of the electrodes' shifts and Eq. S21's joint capacitance do not depend
on that form, so those are compared.
"""
import math

import numpy as np
import pytest

from oracle import ewald as ew
from oracle import gcd
from paper_2111_06704_gb300 import cpm
from paper_2111_06704_gb300 import workloads as wl
from tests import _cases, _golden

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

PREC = {"fp64": cpm.CPM_PREC_FP64, "bf16x6": cpm.CPM_PREC_BF16X6}
Q_TOL = {"fp64": 1e-9, "bf16x6": 1e-6}
SOLVE_TOL = {"fp64": 1e-12, "bf16x6": 1e-10}  # float-stored E: the solves' floor


def _three_electrodes(el):
    """The lower sheet, and the upper sheet split in x."""
    upper = el.xyz[:, 2] > 15.0
    return (upper.astype(int) + (upper & (el.xyz[:, 0] > el.box[0] / 2))).astype(np.int32)


@pytest.mark.parametrize("prec", ["fp64", "bf16x6"])
def test_gcd_charges_match_the_oracle(prec):
    work = _cases.tiny_two_sheet(q_sol=2)
    el, io = work.electrode, work.electrolyte
    oc = _cases.oracle_case(work)
    labels = _three_electrodes(el)
    q0 = np.array([[-0.7, 0.3, -1.6]])  # sums to -Q^sol
    ctx = cpm.Context(el.box, precision=PREC[prec], rcut_dc=3.0)
    ctx.cpm_build_E(el.xyz, el.alpha)
    _, iters, rel = ctx.cpm_gcd_setup(labels, tol=SOLVE_TOL[prec])
    assert np.all(rel <= SOLVE_TOL[prec]) and np.all(iters > 0)
    b, qsol = ctx.cpm_potential(io.xyz, io.q, el.chi)
    q, _, _ = ctx.cpm_solve(b, tol=SOLVE_TOL[prec])
    q, dmu = ctx.cpm_gcd_charges(q, q0, qsol)
    b_paper = ew.rhs_volts(el.chi, oc.bsol_paper[0]) / ew.KE
    q_ref, dmu_ref = gcd.gcd_two_step(oc.e_paper, b_paper, labels, q0[0])
    assert np.linalg.norm(q[0] - q_ref) / np.linalg.norm(q_ref) < Q_TOL[prec]
    for a in range(3):
        assert q[0, labels == a].sum() == pytest.approx(q0[0, a], abs=1e-10)
    # shifts in volts, up to one constant
    shift = (dmu[0] - dmu[0, 0]) - (dmu_ref - dmu_ref[0]) * ew.KE
    assert np.abs(shift).max() < 1e-6 * np.abs(dmu_ref * ew.KE).max()
    ctx.close()


def test_one_electrode_is_the_neutralisation():
    # m = 1 with Q^0 = -Q^sol is Eq. 35's second step
    work = _cases.tiny_two_sheet(q_sol=2)
    el, io = work.electrode, work.electrolyte
    ctx = cpm.Context(el.box, precision=cpm.CPM_PREC_FP64, rcut_dc=3.0)
    ctx.cpm_build_E(el.xyz, el.alpha)
    ctx.cpm_gcd_setup(np.zeros(el.n, np.int32), tol=1e-12)
    b, qsol = ctx.cpm_potential(io.xyz, io.q, el.chi)
    qb, _, _ = ctx.cpm_solve(b, tol=1e-12)
    q1 = ctx.cpm_neutralize(qb.copy(), qsol)
    q2, _ = ctx.cpm_gcd_charges(qb.copy(), -qsol[:, None], qsol)
    # the build solves E d' = 1 to 1e-10, so d carries ~kappa x 1e-10 relative error
    assert np.abs(q1 - q2).max() < 1e-7 * np.abs(q1).max()
    ctx.close()


@pytest.mark.parametrize("prec", ["fp64", "bf16x6"])
def test_joint_capacitance_of_a_two_sheet_capacitor(prec):
    # Eq. S21 for two ideal graphene sheets 30 A apart: the parallel-plate capacitor with
    # each sheet's lattice part (Table 1's U^GRA and the neighbours' screening), in e/V
    from scipy.special import erfc
    bond, d, alpha = 1.42, 30.0, wl.ALPHA
    u = float(next(r for r in _golden.rows("table1_2d_lattices.txt")
                   if r[0] == "GRA" and r[1] == "1.420")[3])
    a, b = wl.ideal_graphene_cell(bond)
    lo = wl.graphene_sheet(4, 3, 0.0, a, b)
    hi = wl.graphene_sheet(4, 3, d, a, b)
    xyz = np.vstack([lo, hi])
    ctx = cpm.Context((4 * a, 3 * b, 90.0), precision=PREC[prec], rcut_dc=3.0)
    ctx.cpm_build_E(xyz, np.full(len(xyz), alpha))
    c, _, _ = ctx.cpm_gcd_setup(np.r_[np.zeros(len(lo)), np.ones(len(hi))].astype(np.int32),
                                tol=SOLVE_TOL[prec])
    cell = wl.graphene_sheet(1, 1, 0.0, a, b)[:, :2]
    sites = np.array([(ix * a + x, iy * b + y) for ix in range(-12, 13)
                      for iy in range(-12, 13) for x, y in cell])
    r = np.hypot(*(sites - cell[0]).T)
    r = r[(r > 1e-9) & (r < 30.0)]
    w = math.sqrt(2 / math.pi) * alpha - u - np.sum(erfc(ew.mix_alpha(alpha, alpha) * r) / r)
    ref = len(lo) / (4 * math.pi * d / (a * b / 4) + 2 * w) / ew.KE
    # the Ewald settings alone leave ~6e-9 (the oracle at the same settings)
    assert gcd.joint_capacitance(c) == pytest.approx(ref, rel=1e-8 if prec == "fp64" else 2e-6)
    ctx.close()


def test_gcd_rejects_what_it_cannot_serve():
    work = _cases.tiny_two_sheet()
    el = work.electrode
    ctx = cpm.Context(el.box, rcut_dc=3.0)
    ctx.cpm_build_E(el.xyz, el.alpha)
    labels = _three_electrodes(el)

    def status(fn, *args):
        with pytest.raises(cpm.CpmError) as ei:
            fn(*args)
        return ei.value.status

    qb = np.zeros((1, el.n))
    assert status(ctx.cpm_gcd_charges, qb, np.zeros((1, 3))) == cpm.CPM_EINVAL  # no setup
    assert status(ctx.cpm_gcd_setup, labels, 2) == cpm.CPM_EINVAL  # label 2 with m = 2
    assert status(ctx.cpm_gcd_setup, labels, 4) == cpm.CPM_EINVAL  # electrode 3 empty
    ctx.cpm_gcd_setup(labels)
    assert status(ctx.cpm_gcd_charges, qb, np.array([[0.1, 0.0, 0.0]])) == cpm.CPM_EINVAL
    ctx.cpm_build_E(el.xyz, el.alpha)  # a rebuild drops the setup
    assert status(ctx.cpm_gcd_charges, qb, np.zeros((1, 3))) == cpm.CPM_EINVAL
    ctx.close()
