"""The matrix path (Eq. 33 with Eq. 35) through the C ABI: q = S b - Q^sol d against the
FP64 oracle's neutral charges and against the iterative path on the same context."""
import numpy as np
import pytest

from paper_2111_06704_gb300 import cpm
from tests import _cases

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

PREC = {"fp64": cpm.CPM_PREC_FP64, "bf16x6": cpm.CPM_PREC_BF16X6}
Q_TOL = {"fp64": 1e-9, "bf16x6": 1e-6}
SOLVE_TOL = {"fp64": 1e-12, "bf16x6": 1e-10}  # float-stored E: the solves' floor


@pytest.mark.parametrize("prec", ["fp64", "bf16x6"])
@pytest.mark.parametrize("q_sol", [0, 3])
def test_matrix_path_matches_the_oracle_and_the_solve(prec, q_sol):
    work = _cases.tiny_two_sheet(q_sol=q_sol, n_ion=9 if q_sol else 8)
    el, io = work.electrode, work.electrolyte
    oc = _cases.oracle_case(work)
    ctx = cpm.Context(el.box, precision=PREC[prec], rcut_dc=3.0)
    ctx.cpm_build_E(el.xyz, el.alpha)
    assert ctx.cpm_smatrix_build(tol=SOLVE_TOL[prec]) > 0
    b, qsol = ctx.cpm_potential(io.xyz, io.q, el.chi)
    q = ctx.cpm_smatrix_charges(b, qsol)
    assert np.linalg.norm(q - oc.q) / np.linalg.norm(oc.q) < Q_TOL[prec]
    # neutral to the accuracy of the columns E^-1 e_j (cpm_neutralize makes it exact)
    assert q[0].sum() == pytest.approx(-q_sol, abs=1e-6 * np.abs(q[0]).sum())
    q_it, _, _, _, _ = cpm.charges(ctx, io.xyz, io.q, el.chi, tol=SOLVE_TOL[prec])
    assert np.abs(q - q_it).max() < 1e-7 * np.abs(q_it).max()
    ctx.close()


def test_matrix_path_many_frames_and_rejections():
    work = _cases.tiny_two_sheet()
    el = work.electrode
    ctx = cpm.Context(el.box, precision=cpm.CPM_PREC_FP64, rcut_dc=3.0)
    ctx.cpm_build_E(el.xyz, el.alpha)
    with pytest.raises(cpm.CpmError) as ei:
        ctx.cpm_smatrix_charges(np.zeros((1, el.n)))
    assert ei.value.status == cpm.CPM_EINVAL  # before cpm_smatrix_build
    ctx.cpm_smatrix_build()
    rng = np.random.default_rng(3)
    b = rng.standard_normal((7, el.n))  # seven frames (not a multiple of four) at once
    q = ctx.cpm_smatrix_charges(b)
    for f in range(7):
        assert np.array_equal(q[f], ctx.cpm_smatrix_charges(b[f:f + 1])[0])
    ctx.cpm_build_E(el.xyz, el.alpha)  # a rebuild drops S
    with pytest.raises(cpm.CpmError) as ei:
        ctx.cpm_smatrix_charges(b)
    assert ei.value.status == cpm.CPM_EINVAL
    ctx.close()
