"""PCG-Normal and PCG-Full (Sec. III B 2, Fig. 6a) on the GPU against the oracle's
sparsified inverse (oracle/precond.py) on the 512-atom cell: the pattern entry by entry,
P within what the float storage of E allows, iteration counts to 1e-6 within one of the
oracle's PCG with its own P, the charges within the parity bar, and Fig. 6a's order
(more of E^-1 never costs iterations).

E is stored in float, so its inverse differs from the FP64 oracle's by up to
kappa(E_n) x 6e-8 relative (kappa = 171 here): P is compared to 1e-4 of its largest entry.
"""
import numpy as np
import pytest

from oracle import ewald as ew
from oracle import precond as pc
from oracle import solve as sv
from paper_2111_06704_gb300 import cpm

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

CASES = [("full", cpm.CPM_PRECOND_FULL, 12.0, False), ("normal8", cpm.CPM_PRECOND_NORMAL, 8.0, True),
         ("normal4", cpm.CPM_PRECOND_NORMAL, 4.0, True), ("normal2", cpm.CPM_PRECOND_NORMAL, 2.0, True)]


@pytest.mark.parametrize("name,pre,rcut,strict", CASES)
def test_sparsified_inverse_against_the_oracle(small_cell_oracle, name, pre, rcut, strict):
    oc = small_cell_oracle
    el = oc.work.electrode
    kw = {"rcut_real": 12.0} if pre == cpm.CPM_PRECOND_FULL else {"rcut_dc": rcut}
    ctx = cpm.Context(el.box, precond=pre, **kw)
    ctx.cpm_build_E(el.xyz, el.alpha)
    off, idx, val = ctx.cpm_get_precond()
    p_ref, pattern = pc.sparsified_inverse(oc.e_neutral, el.xyz, el.box, rcut, strict)
    assert np.array_equal(np.diff(off), [len(x) for x in pattern])
    scale = np.abs(p_ref).max()
    for j in range(el.n):
        cols = idx[off[j]:off[j + 1]]
        assert np.array_equal(cols, pattern[j])  # symmetric pattern: row j = column j
        assert np.abs(val[off[j]:off[j + 1]] - p_ref[j, cols]).max() <= 1e-4 * scale
    b = oc.b_neutral_volts
    q, it, rel = ctx.cpm_solve(b, tol=1e-6)
    _, it_ref, _ = sv.pcg(oc.e_neutral, b[0] / ew.KE, p_ref, tol=1e-6, maxit=500)
    assert abs(int(it[0]) - it_ref) <= 1, (name, int(it[0]), it_ref)
    q, _, rel = ctx.cpm_solve(b, tol=1e-10, maxit=2000)
    assert rel[0] <= 1e-10
    assert np.linalg.norm(q[0] - oc.qb_neutral[0]) < 1e-6 * np.linalg.norm(oc.qb_neutral[0])
    ctx.close()


def test_fig6a_order_on_the_gpu(small_cell_oracle):
    oc = small_cell_oracle
    el = oc.work.electrode
    counts = []
    for name, pre, rcut, strict in CASES:
        kw = {"rcut_real": 12.0} if pre == cpm.CPM_PRECOND_FULL else {"rcut_dc": rcut}
        ctx = cpm.Context(el.box, precond=pre, **kw)
        ctx.cpm_build_E(el.xyz, el.alpha)
        _, it, _ = ctx.cpm_solve(oc.b_neutral_volts, tol=1e-6)
        counts.append(int(it[0]))
        ctx.close()
    assert counts == sorted(counts) and counts[0] < counts[-1]
