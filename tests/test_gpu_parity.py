"""CUDA path against the FP64 oracle, element by element, through the C ABI.

Tolerances.  FP64 mode: the same sums in double precision in a different order, so
E and b agree to ~1e-12 of their largest entry and the converged charges to the solve
tolerance.  FP32 mode: E is rounded to float (6e-8 relative); its reciprocal part is
accumulated from the heaviest weights down, the heaviest exactly in double and the rest
in short float chunks summed in double; phases are exact fixed point before one float
rounding.  Entry errors then sit near the float rounding of E (~1e-8 absolute), so the
element checks use 1e-6 of the largest entry and the charges 1e-6 relative (L2) after a
solve to 1e-9.
"""
import numpy as np
import pytest

from oracle import ewald as ew
from oracle import precond as pc
from paper_2111_06704_gb300 import cpm
from paper_2111_06704_gb300 import workloads as wl
from tests import _cases

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

PREC = {"fp64": cpm.CPM_PREC_FP64, "fp32": cpm.CPM_PREC_FP32, "bf16x6": cpm.CPM_PREC_BF16X6}
E_TOL = {"fp64": 1e-12, "fp32": 1e-6, "bf16x6": 1e-6}
B_TOL = {"fp64": 1e-11, "fp32": 1e-6, "bf16x6": 1e-6}
Q_TOL = {"fp64": 1e-9, "fp32": 1e-6, "bf16x6": 1e-6}


def make_ctx(work, prec="fp32", **kw):
    el = work.electrode
    ctx = cpm.Context(el.box, precision=PREC[prec], **kw)
    ctx.cpm_build_E(el.xyz, el.alpha)
    return ctx


def rel_max(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / np.abs(b).max()


def rel_l2(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b)


# ------------------------------------------------------------------ small cell (N=512)

@pytest.fixture(scope="module")
def oc():
    return _cases.small_cell_oracle()


@pytest.fixture(scope="module", params=["fp64", "fp32", "bf16x6"])
def built(request, oc):
    ctx = make_ctx(oc.work, request.param)
    yield request.param, ctx
    ctx.close()


def test_interaction_matrix_matches_oracle(built, oc):
    prec, ctx = built
    e_n = ctx.cpm_get_E(cpm.CPM_E_STORED)
    assert rel_max(e_n, oc.e_neutral) < E_TOL[prec]
    e_p = ctx.cpm_get_E(cpm.CPM_E_PAPER)
    assert rel_max(e_p, oc.e_paper) < E_TOL[prec]
    assert np.array_equal(e_n, e_n.T)  # mirrored: exactly symmetric


def test_apply_E_is_the_stored_matrix_times_p(built, oc):
    # the solver's matvec applies the stored matrix exactly up to FP64 summation: the
    # float path keeps every product and partial-sum rounding error
    prec, ctx = built
    rng = np.random.default_rng(2)
    p = rng.standard_normal((3, oc.work.electrode.n))
    q = ctx.cpm_apply_E(p)
    e_n = ctx.cpm_get_E(cpm.CPM_E_STORED)
    ref = p @ e_n.T
    assert np.abs(q - ref).max() <= 1e-12 * np.abs(ref).max()
    assert np.abs(q - p @ oc.e_neutral.T).max() <= E_TOL[prec] * 50 * np.abs(ref).max()


def test_potential_matches_oracle(built, oc):
    prec, ctx = built
    io, el = oc.work.electrolyte, oc.work.electrode
    b, qsol = ctx.cpm_potential(io.xyz, io.q, el.chi)
    assert rel_max(b, oc.b_neutral_volts) < B_TOL[prec]
    assert np.allclose(qsol, oc.q_sol)


def test_charges_match_oracle(built, oc):
    prec, ctx = built
    io, el = oc.work.electrolyte, oc.work.electrode
    q, iters, rel, b, qsol = cpm.charges(ctx, io.xyz, io.q, el.chi, tol=1e-12 if prec == "fp64" else 1e-10)
    assert np.all(rel <= (1e-12 if prec == "fp64" else 1e-9))
    print(f"512 atoms, {prec} build: q error {rel_l2(q, oc.q):.2e}, "
          f"b error {rel_max(b, oc.b_neutral_volts):.2e} of max|b|")
    assert rel_l2(q, oc.q) < Q_TOL[prec]
    assert abs(q.sum() + oc.q_sol.sum()) < 1e-12 * np.abs(q).sum()  # Eq. 34


def test_first_step_and_neutralizing_vector(built, oc):
    prec, ctx = built
    d = ctx.cpm_get_d()
    assert d.sum() == pytest.approx(1.0, abs=1e-12)
    assert rel_l2(d, oc.d_neutral) < Q_TOL[prec]
    info = ctx.cpm_get_info()
    assert info["c_ele"] == pytest.approx(oc.c_ele_neutral, rel=Q_TOL[prec])
    q, _, _ = ctx.cpm_solve(oc.b_neutral_volts, tol=1e-12 if prec == "fp64" else 1e-10)
    assert rel_l2(q, oc.qb_neutral) < Q_TOL[prec]


@pytest.mark.parametrize("pre", [cpm.CPM_PRECOND_NONE, cpm.CPM_PRECOND_JACOBI,
                                 cpm.CPM_PRECOND_DC])
def test_every_preconditioner_reaches_the_oracle(oc, pre):
    ctx = make_ctx(oc.work, "fp32", precond=pre)
    io, el = oc.work.electrolyte, oc.work.electrode
    q, iters, rel, _, _ = cpm.charges(ctx, io.xyz, io.q, el.chi, tol=1e-9)
    assert rel_l2(q, oc.q) < 1e-6
    ctx.close()


def test_dc_preconditioner_needs_fewer_iterations(oc):
    io, el = oc.work.electrolyte, oc.work.electrode
    its = {}
    for pre in (cpm.CPM_PRECOND_JACOBI, cpm.CPM_PRECOND_DC):
        ctx = make_ctx(oc.work, "fp32", precond=pre)
        _, it, _, _, _ = cpm.charges(ctx, io.xyz, io.q, el.chi, tol=1e-6)
        its[pre] = int(it[0])
        ctx.close()
    assert its[cpm.CPM_PRECOND_DC] < its[cpm.CPM_PRECOND_JACOBI]


def test_dc_preconditioner_matches_oracle(oc):
    # P of Eq. 36 entry by entry (pattern exact, values to FP64 rounding of the local
    # eliminations) and p_gap of Eq. 37 from the library's own 1^T E_n^-1 1
    el = oc.work.electrode
    ctx = make_ctx(oc.work, "fp32")
    off, idx, val = ctx.cpm_get_precond()
    p_ref, nb = pc.dc_preconditioner(el.xyz, el.alpha, el.box, wl.G_DC, wl.RCUT_DC)
    assert off[-1] == sum(len(x) for x in nb)
    for j in range(el.n):
        cols = idx[off[j]:off[j + 1]]
        assert np.array_equal(cols, nb[j])  # the pattern is symmetric: j's row = j's list
        np.testing.assert_allclose(val[off[j]:off[j + 1]], p_ref[j, cols], rtol=0,
                                   atol=1e-11 * np.abs(p_ref).max())
    info = ctx.cpm_get_info()
    if info["p_gap"] != 0.0:
        gap = pc.p_gap(p_ref, info["c_ele"], nb)
        n_zero = el.n ** 2 - off[-1]
        assert abs(info["p_gap"] - gap) <= 1e-10 * (abs(info["c_ele"]) + np.abs(p_ref).sum()) / n_zero
    ctx.close()


def test_device_pointers_give_the_same_answer(oc):
    # one solver path for both calls (the autotuner may otherwise time another path on the
    # second call), so the sums are the same bit for bit
    ctx = make_ctx(oc.work, "fp32", solver_path=1)
    io, el = oc.work.electrolyte, oc.work.electrode
    q_host, _, _, b_host, _ = cpm.charges(ctx, io.xyz, io.q, el.chi, tol=1e-9)
    dev = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    b = torch.empty((1, el.n), dtype=torch.float64, device="cuda")
    qs = torch.empty(1, dtype=torch.float64, device="cuda")
    ctx.cpm_potential(dev(io.xyz), dev(io.q), dev(el.chi), b, qs)
    q = torch.zeros((1, el.n), dtype=torch.float64, device="cuda")
    ctx.cpm_solve(b, q, tol=1e-9)
    ctx.cpm_neutralize(q, qs)
    assert np.array_equal(b.cpu().numpy(), b_host)
    assert np.array_equal(q.cpu().numpy(), q_host)
    ctx.close()


def test_previous_step_guess(oc):
    # Eq. 26: starting from the converged charges leaves nothing to do
    ctx = make_ctx(oc.work, "fp32")
    io, el = oc.work.electrolyte, oc.work.electrode
    b, qsol = ctx.cpm_potential(io.xyz, io.q, el.chi)
    q, it0, _ = ctx.cpm_solve(b, tol=1e-8)
    q2, it1, _ = ctx.cpm_solve(b, q.copy(), use_guess=True, tol=1e-8)
    # the fresh residual b - E q may sit just above the recursive one: a step or two
    assert it1[0] <= 2 and 3 * it1[0] < it0[0]
    assert rel_l2(q2, q) < 1e-8
    ctx.close()


# ------------------------------------------------- ragged / edge cases (fast oracle)

@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16x6"])
@pytest.mark.parametrize("q_sol", [0, 3])
def test_tiny_cell_with_images_and_net_charge(prec, q_sol):
    # 48 atoms (not a tile multiple), box edges below 2 rc (many images), and a
    # monopolar electrolyte (Q^sol != 0, Eq. 34).
    work = _cases.tiny_two_sheet(q_sol=q_sol, n_ion=9 if q_sol else 8)
    oc = _cases.oracle_case(work)
    ctx = make_ctx(work, prec, rcut_dc=3.0)
    assert rel_max(ctx.cpm_get_E(cpm.CPM_E_PAPER), oc.e_paper) < E_TOL[prec]
    io, el = work.electrolyte, work.electrode
    q, _, _, b, qsol = cpm.charges(ctx, io.xyz, io.q, el.chi, tol=1e-12 if prec == "fp64" else 1e-10)
    assert rel_max(b, oc.b_neutral_volts) < B_TOL[prec]
    assert qsol[0] == q_sol
    assert rel_l2(q, oc.q) < Q_TOL[prec]
    ctx.close()


@pytest.fixture(scope="module")
def wide_cell():
    # box edges 29.5 x 29.8 A, above 2 r_cut = 24 A: one image per direction, so the real
    # space takes the far electrode-ion pairs (erfc(g r) / r <= 1e-4 1/A) in float in the
    # FP32 and BF16X6 builds, and in FP64 in the FP64 build
    el = wl.two_sheet_electrode(12, 7)
    rng = np.random.default_rng(wl.seed_for(1, 7))
    frames = [wl.random_ions(rng, 200, 200, el.box, min_sep=2.5) for _ in range(3)]
    io = wl.Electrolyte(np.stack([f[0] for f in frames]), np.stack([f[1] for f in frames]))
    g, rc, eps = wl.G_EWALD, wl.RCUT_REAL, wl.KSPACE_EPS
    ref = []
    for f in range(io.frames):
        bsol = ew.electrolyte_potential(el.xyz, el.alpha, io.xyz[f], io.q[f], el.box, g, rc, eps)
        bsn = ew.neutral_form_bsol(bsol, el.xyz, io.xyz[f], io.q[f], el.box, g)
        ref.append(ew.rhs_volts(el.chi, bsn))
    return el, io, np.array(ref)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16x6"])
def test_potential_with_float_far_pairs(prec, wide_cell):
    el, io, ref = wide_cell
    ctx = cpm.Context(el.box, precision=PREC[prec], rcut_dc=3.0)
    ctx.cpm_build_E(el.xyz, el.alpha)
    b, qsol = ctx.cpm_potential(io.xyz, io.q, el.chi)
    err = rel_max(b, ref)
    print(f"{prec}: b max error {err:.2e} of the largest entry")
    assert err < B_TOL[prec]
    assert np.all(qsol == 0)
    ctx.close()


@pytest.mark.parametrize("prec", ["fp64", "bf16x6"])
def test_one_atom_electrode(prec):
    # The degenerate electrode: one atom, so d = 1 (Eq. S8) and Eq. 35 gives it the whole
    # compensating charge, q = -Q^sol, whatever b is; E is its self-interaction alone.
    work = _cases.tiny_two_sheet(q_sol=3, n_ion=9)
    el, io = work.electrode, work.electrolyte
    one = wl.Workload("one atom", wl.Electrode(el.xyz[:1], el.alpha[:1], el.chi[:1], el.box),
                      io)
    oc = _cases.oracle_case(one)
    ctx = make_ctx(one, prec, rcut_dc=3.0)
    assert rel_max(ctx.cpm_get_E(cpm.CPM_E_PAPER), oc.e_paper) < E_TOL[prec]
    assert np.allclose(ctx.cpm_get_d(), 1.0, rtol=0, atol=1e-12)
    q, _, _, b, qsol = cpm.charges(ctx, io.xyz, io.q, el.chi[:1], tol=1e-10)
    assert rel_max(b, oc.b_neutral_volts) < B_TOL[prec]
    assert qsol[0] == 3 and q.shape == (1, 1)
    assert q[0, 0] == pytest.approx(-3.0, abs=1e-12) and oc.q[0, 0] == pytest.approx(-3.0)
    ctx.close()


def test_no_ions_and_many_frames():
    work = _cases.tiny_two_sheet()
    el = work.electrode
    oc = _cases.oracle_case(wl.Workload("empty", el, wl.Electrolyte(np.zeros((1, 0, 3)),
                                                                     np.zeros((1, 0)))))
    ctx = make_ctx(work, "fp64", rcut_dc=3.0)
    b, qsol = ctx.cpm_potential(np.zeros((1, 0, 3)), np.zeros((1, 0)), el.chi)
    assert rel_max(b, oc.b_neutral_volts) < 1e-12 and qsol[0] == 0
    # five frames at once equal five single-frame calls
    rng = np.random.default_rng(5)
    frames = [wl.random_ions(rng, 4, 4, el.box, min_sep=1.0) for _ in range(5)]
    xyz = np.stack([f[0] for f in frames])
    qq = np.stack([f[1] for f in frames])
    bb, _ = ctx.cpm_potential(xyz, qq, el.chi)
    for f in range(5):
        b1, _ = ctx.cpm_potential(xyz[f:f + 1], qq[f:f + 1], el.chi)
        assert np.array_equal(bb[f], b1[0])
    ctx.close()


def test_errors_are_reported_not_raised_in_c():
    work = _cases.tiny_two_sheet()
    el = work.electrode
    ctx = cpm.Context(el.box, rcut_dc=3.0)
    with pytest.raises(cpm.CpmError) as ei:
        ctx.cpm_solve(np.zeros((1, el.n)))
    assert ei.value.status == cpm.CPM_ENOTBUILT
    ctx.cpm_build_E(el.xyz, el.alpha)
    with pytest.raises(cpm.CpmError) as ei:
        ctx.cpm_solve(np.ones((1, el.n)), tol=-1.0)
    assert ei.value.status == cpm.CPM_EINVAL
    ctx.close()
    bad = cpm.Context(el.box, rcut_dc=20.0)  # above half the box edge
    with pytest.raises(cpm.CpmError) as ei:
        bad.cpm_build_E(el.xyz, el.alpha)
    assert ei.value.status == cpm.CPM_EINVAL
    bad.close()


def test_maxit_reports_no_convergence(oc):
    ctx = make_ctx(oc.work, "fp32", precond=cpm.CPM_PRECOND_NONE)
    b = oc.b_neutral_volts
    q, it, rel = ctx.cpm_solve(b, tol=1e-12, maxit=3, allow_noconv=True)
    assert it[0] == 3 and rel[0] > 1e-12
    with pytest.raises(cpm.CpmError) as ei:
        ctx.cpm_solve(b, tol=1e-12, maxit=3)
    assert ei.value.status == cpm.CPM_ENOCONV
    ctx.close()
