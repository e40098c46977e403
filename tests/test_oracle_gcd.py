"""Pins of the GCD oracle (fixed charge per electrode, Eq. S14-S24) to things other than
itself: the electroneutral two-step method it generalises (Eq. 35), its own definition as
a bordered system (Eq. S14-S15), the constant-potential charges it must give back when
handed their electrode totals, and the closed-form capacitance of a two-sheet graphene
capacitor (Eq. S21 against parallel plates plus Table 1's lattice potential)."""
import math

import numpy as np
import pytest

from oracle import ewald as ew
from oracle import gcd
from oracle import solve as sv
from paper_2111_06704_gb300 import workloads as wl
from tests import _cases, _golden


def _two_sheet_case(q_sol):
    work = _cases.tiny_two_sheet(q_sol=q_sol)
    el, io = work.electrode, work.electrolyte
    e = ew.interaction_matrix(el.xyz, el.alpha, el.box, 0.3, 12.0, 1e-8, True)
    bsol = ew.electrolyte_potential(el.xyz, el.alpha, io.xyz[0], io.q[0], el.box, 0.3, 12.0)
    labels = (el.xyz[:, 2] > 15.0).astype(int)  # electrode 0: the sheet at z = 0
    return el, io, e, bsol, labels


@pytest.mark.parametrize("q_sol", [0, 2])
def test_one_electrode_is_the_two_step_method(q_sol):
    # M = 1 with Q^0 = -Q^sol: a^1 = E^-1 1 = d', C_E = C^ele, so Eq. S16-S20 become
    # Eq. 35's q^b - (Q^b + Q^sol) d
    el, io, e, bsol, _ = _two_sheet_case(q_sol)
    b = ew.rhs_volts(el.chi, bsol) / ew.KE
    qs = float(io.q[0].sum())
    q, dmu = gcd.gcd_two_step(e, b, np.zeros(el.n, int), [-qs])
    ref = sv.two_step(e, b, qs)
    assert np.abs(q - ref).max() < 1e-10 * np.abs(ref).max()
    _, mu = sv.solve_bordered(e, b, qs)
    assert dmu[0] == pytest.approx(-mu, rel=1e-9)  # the same multiplier, opposite sign


@pytest.mark.parametrize("m", [2, 3])
def test_two_step_equals_the_bordered_definition(m):
    el, io, e, bsol, labels = _two_sheet_case(2)
    if m == 3:  # split the upper sheet in x as well
        labels = labels + ((labels == 1) & (el.xyz[:, 0] > el.box[0] / 2)).astype(int)
    b = ew.rhs_volts(el.chi, bsol) / ew.KE
    q0 = np.array([-0.7, 0.3, -0.1][:m])
    q, dmu = gcd.gcd_two_step(e, b, labels, q0)
    qd, dmud = gcd.solve_bordered_gcd(e, b, labels, q0)
    scale = np.abs(qd).max()
    assert np.abs(q - qd).max() < 1e-10 * scale
    assert np.allclose(dmu, dmud, rtol=1e-9, atol=0)
    # the constraints hold and every electrode is one equipotential (Eq. S15)
    for a in range(m):
        on = labels == a
        assert q[on].sum() == pytest.approx(q0[a], abs=1e-12)
        assert np.allclose((e @ q - b)[on], dmu[a], rtol=0, atol=1e-10 * np.abs(b).max())
    # C_E is symmetric, with positive self and negative mutual coefficients (Eq. S21)
    _, c = gcd.capacitance_coefficients(e, labels, m)
    assert np.allclose(c, c.T, rtol=1e-10)
    assert np.all(np.diag(c) > 0) and np.all(c[~np.eye(m, dtype=bool)] < 0)


@pytest.mark.parametrize("neutral_form", [False, True])
def test_gcd_gives_back_the_constant_potential_charges(neutral_form):
    # Handed the electrode totals of the constant-potential solution, GCD returns those
    # charges; chi, constant on each electrode, is absorbed into the shifts (Eq. S14), so
    # without it the shifts differ by the potential difference.  The neutral-equivalent
    # E_n gives the same charges (its remainder only moves every shift by one constant).
    el, io, e, bsol, labels = _two_sheet_case(2)
    qs = float(io.q[0].sum())
    b = ew.rhs_volts(el.chi, bsol) / ew.KE
    q_cpm = sv.two_step(e, b, qs)
    q0 = np.array([q_cpm[labels == 0].sum(), q_cpm[labels == 1].sum()])
    if neutral_form:
        e = ew.neutral_form_matrix(e, el.xyz, el.box, 0.3)
        bsol = ew.neutral_form_bsol(bsol, el.xyz, io.xyz[0], io.q[0], el.box, 0.3)
    q, dmu = gcd.gcd_two_step(e, -bsol, labels, q0)
    assert np.abs(q - q_cpm).max() < 1e-10 * np.abs(q_cpm).max()
    assert dmu[1] - dmu[0] == pytest.approx(1.0 / ew.KE, rel=1e-9)  # chi: -0.5 / +0.5 V


def test_capacitor_joint_capacitance_closed_form():
    # Two ideal graphene sheets 30 A apart as electrodes a and b, no ions: Eq. S21's
    # C(Q, -Q) = |C_E| / C^ele against the parallel-plate capacitor with each sheet's
    # lattice part, N_s / (4 pi d / A_atom + 2 W), W = sqrt(2/pi) alpha - U^GRA - S
    # (the charge per unit potential difference of the closed-form capacitor pin)
    from scipy.special import erfc
    bond, d, alpha = 1.42, 30.0, 1.979
    u = float(next(r for r in _golden.rows("table1_2d_lattices.txt")
                   if r[0] == "GRA" and r[1] == "1.420")[3])
    a, b = wl.ideal_graphene_cell(bond)
    lo = wl.graphene_sheet(4, 3, 0.0, a, b)
    hi = wl.graphene_sheet(4, 3, d, a, b)
    xyz = np.vstack([lo, hi])
    e = ew.interaction_matrix(xyz, np.full(len(xyz), alpha), (4 * a, 3 * b, 90.0), 0.3,
                              18.0, 1e-14, True)
    labels = np.r_[np.zeros(len(lo), int), np.ones(len(hi), int)]
    _, c = gcd.capacitance_coefficients(e, labels, 2)
    cell = wl.graphene_sheet(1, 1, 0.0, a, b)[:, :2]
    sites = np.array([(ix * a + x, iy * b + y) for ix in range(-12, 13)
                      for iy in range(-12, 13) for x, y in cell])
    r = np.hypot(*(sites - cell[0]).T)
    r = r[(r > 1e-9) & (r < 30.0)]
    w = math.sqrt(2 / math.pi) * alpha - u - np.sum(erfc(ew.mix_alpha(alpha, alpha) * r) / r)
    ref = len(lo) / (4 * math.pi * d / (a * b / 4) + 2 * w)
    assert gcd.joint_capacitance(c) == pytest.approx(ref, rel=1e-11)
    assert gcd.joint_capacitance(c) == pytest.approx(np.linalg.det(c) / c.sum(), rel=1e-12)
    # the charges for +-Q: one sheet at Q / C(Q, -Q) above the other
    q, dmu = gcd.gcd_two_step(e, np.zeros(len(xyz)), labels, [-1.0, 1.0])
    assert dmu[1] - dmu[0] == pytest.approx(1.0 / gcd.joint_capacitance(c), rel=1e-10)
