"""Pins of the electrode-ion force oracle (Eq. S25 inside the Ewald sum of Eq. 22 / 25):
central finite differences of the oracle's own coupling energy q^T b^sol, which shares
no derivative code with it, for Gaussian and point electrode charges, with and without
the slab correction, ion by ion and for a common shift of all ions."""
import numpy as np
import pytest

from oracle import ewald as ew
from oracle import forces as fo
from oracle import solve as sv
from tests import _cases


def _energy(el, alpha, q, ion_xyz, ion_q, slab):
    bsol = ew.electrolyte_potential(el.xyz, alpha, ion_xyz, ion_q, el.box, 0.3, 18.0, 1e-14,
                                    slab)
    return float(q @ bsol)


@pytest.mark.parametrize("slab", [True, False])
@pytest.mark.parametrize("point", [False, True])
@pytest.mark.parametrize("close", [False, True])
def test_forces_are_minus_the_energy_gradient(slab, point, close):
    work = _cases.tiny_two_sheet(q_sol=2)
    el, io = work.electrode, work.electrolyte
    alpha = np.full(el.n, np.inf) if point else el.alpha
    rng = np.random.default_rng(4)
    q = rng.normal(0.0, 0.01, el.n)
    ion_xyz, ion_q = io.xyz[0].copy(), io.q[0]
    if close:
        # ion 0 at 0.6 A from an electrode atom, where the Gaussian's own terms of
        # Eq. S25 (erf(alpha r) / r and its exponential) are of order one
        ion_xyz[0] = el.xyz[5] + np.array([0.3, -0.2, 0.49])
    f = fo.forces_on_ions(el.xyz, alpha, q, ion_xyz, ion_q, el.box, 0.3, 18.0, 1e-14, slab)
    h = 1e-4  # larger steps: truncation ~h^2; smaller: rounding of the energy sums
    for ion in (0, 3, 7):
        for k in range(3):
            xp, xm = ion_xyz.copy(), ion_xyz.copy()
            xp[ion, k] += h
            xm[ion, k] -= h
            fd = -(_energy(el, alpha, q, xp, ion_q, slab) -
                   _energy(el, alpha, q, xm, ion_q, slab)) / (2 * h)
            assert f[ion, k] == pytest.approx(fd, rel=1e-6, abs=1e-9 * np.abs(f).max())


def test_total_force_under_a_common_shift():
    # with the constant-potential charges of the oracle's solve: the summed force on the
    # ions is minus the derivative of U when every ion moves by the same vector
    work = _cases.tiny_two_sheet(q_sol=0)
    el, io = work.electrode, work.electrolyte
    oc = _cases.oracle_case(work)
    q = oc.q[0]
    f = fo.forces_on_ions(el.xyz, el.alpha, q, io.xyz[0], io.q[0], el.box, 0.3, 18.0, 1e-14,
                          False)
    h = 1e-4  # larger steps: truncation ~h^2; smaller: rounding of the energy sums
    for k in range(3):
        xp, xm = io.xyz[0].copy(), io.xyz[0].copy()
        xp[:, k] += h
        xm[:, k] -= h
        fd = -(_energy(el, el.alpha, q, xp, io.q[0], False) -
               _energy(el, el.alpha, q, xm, io.q[0], False)) / (2 * h)
        assert f[:, k].sum() == pytest.approx(fd, rel=1e-6, abs=1e-9)
