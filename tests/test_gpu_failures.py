"""Failure paths made on the host, through the C ABI: each bad input or failing resource
comes back as its status code with the context still usable afterwards.

* non-finite coordinates, or a Gaussian width that is neither positive nor INFINITY,
  are refused by cpm_build_E (CPM_EINVAL) before any kernel uses them;
* an allocator callback that returns NULL gives CPM_ENOMEM;
* a right-hand side or a guess holding NaN or Inf stops the solve with CPM_EBREAKDOWN
  (the PCG's scalars turn non-finite; Eq. 25's b must be finite);
* an unconverged solve returns CPM_ENOCONV with its residual set.
"""
import numpy as np
import pytest

from paper_2111_06704_gb300 import cpm
from tests import _cases

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


@pytest.fixture(scope="module")
def tiny():
    return _cases.tiny_two_sheet()


@pytest.mark.parametrize("what", ["nan_xyz", "inf_xyz", "zero_alpha", "nan_alpha"])
def test_build_refuses_bad_geometry(tiny, what):
    el = tiny.electrode
    xyz, alpha = el.xyz.copy(), el.alpha.copy()
    if what == "nan_xyz":
        xyz[5, 1] = np.nan
    elif what == "inf_xyz":
        xyz[7, 2] = np.inf
    elif what == "zero_alpha":
        alpha[3] = 0.0
    else:
        alpha[0] = np.nan
    ctx = cpm.Context(el.box, rcut_dc=3.0)
    with pytest.raises(cpm.CpmError) as ei:
        ctx.cpm_build_E(xyz, alpha)
    assert ei.value.status == cpm.CPM_EINVAL
    # the context builds the good geometry afterwards
    ctx.cpm_build_E(el.xyz, el.alpha)
    assert np.isfinite(ctx.cpm_get_E(cpm.CPM_E_STORED)).all()
    ctx.close()


def test_allocator_returning_null_gives_enomem(tiny):
    el = tiny.electrode
    calls = []

    def alloc(nbytes):
        calls.append(nbytes)
        return None

    ctx = cpm.Context(el.box, allocator=(alloc, lambda ptr: None), rcut_dc=3.0)
    with pytest.raises(cpm.CpmError) as ei:
        ctx.cpm_build_E(el.xyz, el.alpha)
    assert ei.value.status == cpm.CPM_ENOMEM and calls
    ctx.close()


@pytest.mark.parametrize("bad", [np.nan, np.inf])
@pytest.mark.parametrize("where", ["b", "guess"])
def test_non_finite_right_hand_side_or_guess_breaks_down(tiny, bad, where):
    el, io = tiny.electrode, tiny.electrolyte
    ctx = cpm.Context(el.box, rcut_dc=3.0)
    ctx.cpm_build_E(el.xyz, el.alpha)
    b, _ = ctx.cpm_potential(io.xyz, io.q, el.chi)
    q0 = np.zeros_like(b)
    if where == "b":
        b[0, 4] = bad
    else:
        q0[0, 4] = bad
    with pytest.raises(cpm.CpmError) as ei:
        ctx.cpm_solve(b, q0, use_guess=where == "guess", tol=1e-8)
    assert ei.value.status == cpm.CPM_EBREAKDOWN
    # the context still solves a good right-hand side
    b, _ = ctx.cpm_potential(io.xyz, io.q, el.chi)
    q, it, rel = ctx.cpm_solve(b, tol=1e-8)
    assert rel[0] <= 1e-8 and np.isfinite(q).all()
    ctx.close()


def test_maxit_gives_enoconv_with_the_residual(tiny):
    el, io = tiny.electrode, tiny.electrolyte
    ctx = cpm.Context(el.box, rcut_dc=3.0, precond=cpm.CPM_PRECOND_NONE)
    ctx.cpm_build_E(el.xyz, el.alpha)
    b, _ = ctx.cpm_potential(io.xyz, io.q, el.chi)
    q, it, rel = ctx.cpm_solve(b, tol=1e-14, maxit=2, allow_noconv=True)
    assert it[0] == 2 and rel[0] > 1e-14 and np.isfinite(q).all()
    with pytest.raises(cpm.CpmError) as ei:
        ctx.cpm_solve(b, tol=1e-14, maxit=2)
    assert ei.value.status == cpm.CPM_ENOCONV
    ctx.close()
