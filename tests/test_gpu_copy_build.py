"""cpm_build_E_copy through the C ABI: a context built from another context's E (the
plain FP64 PCG baseline on electrodes whose FP64 k-space build is out of reach).

The copy holds the source's stored E_n widened exactly to FP64, its d and diagonal (and
its PCG-DC preconditioner when asked), so its solves are the solves of the same matrix in
FP64 arithmetic: they reach the oracle's charges like the source's, and the source's own
solve to the same tolerance.
"""
import numpy as np
import pytest

from paper_2111_06704_gb300 import cpm

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def src(small_cell_oracle):
    el = small_cell_oracle.work.electrode
    ctx = cpm.Context(el.box)  # BF16X6, PCG-DC
    ctx.cpm_build_E(el.xyz, el.alpha)
    yield ctx
    ctx.close()


def test_fp64_jacobi_copy_solves_the_same_matrix(src, small_cell_oracle):
    oc = small_cell_oracle
    el, io = oc.work.electrode, oc.work.electrolyte
    dst = cpm.Context(el.box, precision=cpm.CPM_PREC_FP64, precond=cpm.CPM_PRECOND_JACOBI)
    dst.cpm_build_E_copy(src)
    assert np.array_equal(dst.cpm_get_E(cpm.CPM_E_STORED), src.cpm_get_E(cpm.CPM_E_STORED))
    assert np.array_equal(dst.cpm_get_d(), src.cpm_get_d())
    assert dst.cpm_get_info()["c_ele"] == src.cpm_get_info()["c_ele"]
    b, qsol = src.cpm_potential(io.xyz, io.q, el.chi)
    q, it, rel = dst.cpm_solve(b, tol=1e-12, maxit=5000)
    assert rel[0] <= 1e-12
    q = dst.cpm_neutralize(q, qsol)
    assert rel_l2(q, oc.q) < 1e-6
    q_src, _, _ = src.cpm_solve(b, tol=1e-12, maxit=5000)
    q_src = src.cpm_neutralize(q_src, qsol)
    assert rel_l2(q, q_src) < 1e-9
    # no k-space tables on the copy: the potential is the source's job
    with pytest.raises(cpm.CpmError) as ei:
        dst.cpm_potential(io.xyz, io.q, el.chi)
    assert ei.value.status == cpm.CPM_EINVAL
    dst.close()


def test_copy_with_pcg_dc_and_argument_checks(src, small_cell_oracle):
    oc = small_cell_oracle
    el, io = oc.work.electrode, oc.work.electrolyte
    dst = cpm.Context(el.box, precision=cpm.CPM_PREC_FP64)  # PCG-DC, copied from src
    dst.cpm_build_E_copy(src)
    off, idx, val = dst.cpm_get_precond()
    off0, idx0, val0 = src.cpm_get_precond()
    assert np.array_equal(off, off0) and np.array_equal(idx, idx0) and np.array_equal(val, val0)
    b, qsol = src.cpm_potential(io.xyz, io.q, el.chi)
    q, it, rel = dst.cpm_solve(b, tol=1e-10, maxit=2000)
    _, it_src, _ = src.cpm_solve(b, tol=1e-10, maxit=2000)
    assert abs(int(it[0]) - int(it_src[0])) <= 1
    assert rel_l2(dst.cpm_neutralize(q, qsol), oc.q) < 1e-6
    dst.close()
    # another box, or a PCG-DC setting the source does not have, is refused
    other = cpm.Context((el.box[0] + 1.0, el.box[1], el.box[2]), precision=cpm.CPM_PREC_FP64)
    with pytest.raises(cpm.CpmError) as ei:
        other.cpm_build_E_copy(src)
    assert ei.value.status == cpm.CPM_EINVAL
    other.close()
    other = cpm.Context(el.box, precision=cpm.CPM_PREC_FP64, rcut_dc=6.0)
    with pytest.raises(cpm.CpmError) as ei:
        other.cpm_build_E_copy(src)
    assert ei.value.status == cpm.CPM_EINVAL
    other.close()
