"""Pins of the sparsified-inverse preconditioners (PCG-Normal, PCG-Full; Sec. III B 2)
to their limits and to the behaviour Fig. 6a reports: a wider cutoff never costs
iterations, P = E^-1 converges at once, a P reduced to the diagonal of E^-1 (a cutoff
below the nearest-neighbour distance) gains nothing over plain CG, and the p_gap shift of
Eq. 37 helps a little."""
import numpy as np
import pytest

from oracle import ewald as ew
from oracle import precond as pc
from oracle import solve as sv
from tests import _cases


@pytest.fixture(scope="module")
def cell():
    oc = _cases.small_cell_oracle()
    return oc, oc.b_neutral_volts[0] / ew.KE


def _iters(e, b, p):
    _, it, rel = sv.pcg(e, b, p, tol=1e-6, maxit=500)
    assert rel <= 1e-6
    return it


def test_limits(cell):
    oc, b = cell
    el = oc.work.electrode
    e = oc.e_neutral
    whole, _ = pc.sparsified_inverse(e, el.xyz, el.box, 1e3)
    assert np.allclose(whole, np.linalg.inv(e), rtol=0, atol=0)
    assert _iters(e, b, whole) == 1  # P = E^-1
    diag, pattern = pc.sparsified_inverse(e, el.xyz, el.box, 1.0)  # nearest neighbour 1.42
    assert all(len(x) == 1 for x in pattern)
    assert np.allclose(diag, np.diag(np.diag(np.linalg.inv(e))), rtol=0, atol=0)
    # symmetric up to the rounding of the inverse, with a symmetric pattern (unlike
    # PCG-DC's P)
    assert np.abs(whole - whole.T).max() < 1e-12 * np.abs(whole).max()
    p8, nb8 = pc.sparsified_inverse(e, el.xyz, el.box, 8.0)
    mask = p8 != 0.0
    assert np.array_equal(mask, mask.T) and sum(len(x) for x in nb8) == mask.sum()


def test_fig6a_order(cell):
    oc, b = cell
    el = oc.work.electrode
    e = oc.e_neutral
    sum_inv = float(np.linalg.inv(e).sum())
    counts, gapped = [], []
    for rcut, strict in [(12.0, False), (8.0, True), (4.0, True), (2.0, True), (1.0, True)]:
        p, nb = pc.sparsified_inverse(e, el.xyz, el.box, rcut, strict)
        counts.append(_iters(e, b, p))
        gapped.append(_iters(e, b, pc.fill_gap(p, nb, pc.p_gap(p, sum_inv, nb))))
    # PCG-Full, then PCG-Normal at 8, 4, 2 and 1 A: never fewer iterations for less of E^-1
    assert counts == sorted(counts) and counts[0] < counts[-1]
    # the diagonal of E^-1 alone is no better than plain CG
    assert counts[-1] >= _iters(e, b, None)
    # the shift helps a little and never hurts
    assert all(g <= c for g, c in zip(gapped, counts)) and sum(gapped) < sum(counts)
