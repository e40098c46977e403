"""The cluster-resident PCG (solver_path 2: one thread-block cluster per right-hand side,
the whole solve in one launch) against the kernel path (solver_path 1) and the oracle,
through the C ABI, and the online autotuner that picks between them (solver_path 0).

Both paths run the same iteration on the same stored matrix (error-free float-pair
matvec, FP64 vectors and reductions); only the order of the FP64 partial sums differs, so
the charges agree to the solve tolerance and the iteration counts to within one.
"""
import numpy as np
import pytest

from paper_2111_06704_gb300 import cpm
from paper_2111_06704_gb300 import workloads as wl
from tests import _cases

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


def solve_both(work, b, tol, q0=None, **params):
    el = work.electrode
    out = {}
    for path in (1, 2):
        ctx = cpm.Context(el.box, solver_path=path, **params)
        ctx.cpm_build_E(el.xyz, el.alpha)
        q = None if q0 is None else q0.copy()
        q, it, rel = ctx.cpm_solve(b, q, use_guess=q0 is not None, tol=tol, maxit=3000)
        assert ctx.cpm_get_info()["solve_path"] == path
        out[path] = (q, it, rel)
        ctx.close()
    return out


@pytest.mark.parametrize("pre", [cpm.CPM_PRECOND_DC, cpm.CPM_PRECOND_JACOBI,
                                 cpm.CPM_PRECOND_NONE])
def test_cluster_path_equals_kernel_path(small_cell_oracle, pre):
    oc = small_cell_oracle
    b = oc.b_neutral_volts
    out = solve_both(oc.work, b, 1e-10, precond=pre)
    (q1, it1, r1), (q2, it2, r2) = out[1], out[2]
    assert r2[0] <= 1e-10
    assert rel_l2(q2, q1) < 1e-8
    assert abs(int(it1[0]) - int(it2[0])) <= 1
    assert rel_l2(q2[0], oc.qb_neutral[0]) < 1e-6


def test_cluster_path_many_frames_with_a_guess(small_cell_oracle):
    oc = small_cell_oracle
    el, base = oc.work.electrode, oc.work.electrolyte
    rng = np.random.default_rng(wl.seed_for(3, 31))
    xyz = wl.perturb_frames(rng, base.xyz[0], 9, 0.5, el.box)
    q_ion = np.broadcast_to(base.q[0], (9, base.n_ion)).copy()
    ctx = cpm.Context(el.box)
    ctx.cpm_build_E(el.xyz, el.alpha)
    b, _ = ctx.cpm_potential(xyz, q_ion, el.chi)
    ctx.close()
    q0 = np.tile(oc.qb_neutral[0], (9, 1))  # the unperturbed frame's charges as guess
    out = solve_both(oc.work, b, 1e-9, q0=q0)
    (q1, it1, _), (q2, it2, r2) = out[1], out[2]
    assert np.all(r2 <= 1e-9)
    for f in range(9):
        assert rel_l2(q2[f], q1[f]) < 1e-7
    # the kernel path's inner iterations sum in float (the streamed matvec and the
    # many-column PCG-DC apply) between exact residual replacements, the cluster path's
    # are error-free throughout: near a 1e-9 tolerance a replacement that reopens a column
    # costs it an iteration or two
    assert np.all(np.abs(it1.astype(int) - it2.astype(int)) <= 2)


@pytest.mark.parametrize("cells", [(3, 2), (11, 9)])  # 48 and 792 atoms: ragged row slices
def test_cluster_path_odd_sizes(cells):
    el = wl.two_sheet_electrode(*cells)
    rng = np.random.default_rng(5)
    ions, q = wl.random_ions(rng, 20, 20, el.box, min_sep=1.0)
    work = wl.Workload("odd", el, wl.Electrolyte(ions[None], q[None]))
    ctx = cpm.Context(el.box, rcut_dc=3.0 if el.n < 100 else 8.0)
    ctx.cpm_build_E(el.xyz, el.alpha)
    b, _ = ctx.cpm_potential(ions[None], q[None], el.chi)
    ctx.close()
    out = solve_both(work, b, 1e-10, rcut_dc=3.0 if el.n < 100 else 8.0)
    assert rel_l2(out[2][0], out[1][0]) < 1e-8 and out[2][2][0] <= 1e-10


def test_cluster_path_failures_come_back_as_status():
    work = _cases.tiny_two_sheet()
    el, io = work.electrode, work.electrolyte
    ctx = cpm.Context(el.box, rcut_dc=3.0, solver_path=2, precond=cpm.CPM_PRECOND_NONE)
    ctx.cpm_build_E(el.xyz, el.alpha)
    b, _ = ctx.cpm_potential(io.xyz, io.q, el.chi)
    q, it, rel = ctx.cpm_solve(b, tol=1e-14, maxit=2, allow_noconv=True)
    assert it[0] == 2 and rel[0] > 1e-14
    bad = b.copy()
    bad[0, 3] = np.nan
    with pytest.raises(cpm.CpmError) as ei:
        ctx.cpm_solve(bad, tol=1e-8)
    assert ei.value.status == cpm.CPM_EBREAKDOWN
    q, it, rel = ctx.cpm_solve(b, tol=1e-8)  # the context still solves
    assert rel[0] <= 1e-8
    ctx.close()


def test_autotuner_settles_on_one_path(small_cell_oracle):
    oc = small_cell_oracle
    el = oc.work.electrode
    ctx = cpm.Context(el.box)  # solver_path 0
    ctx.cpm_build_E(el.xyz, el.alpha)
    b = oc.b_neutral_volts
    paths = []
    for _ in range(4):
        q, it, rel = ctx.cpm_solve(b, tol=1e-9)
        paths.append(ctx.cpm_get_info()["solve_path"])
        assert rel_l2(q[0], oc.qb_neutral[0]) < 1e-6
    # the build's own one-column solve (E d' = 1) tried the cluster path; the first solve
    # here tries the kernel path; from then on the faster of the two is kept
    assert paths[0] == 1 and paths[1] == paths[2] == paths[3]
    ctx.cpm_build_E(el.xyz, el.alpha)  # a rebuild starts the tuning again
    ctx.cpm_solve(b, tol=1e-9)
    assert ctx.cpm_get_info()["solve_path"] == 1
    ctx.close()
