"""cpm_solve_static: the solve for callers that cannot allocate device memory at solve
time (an MD engine that owns the device memory pool, a host that forbids cudaMalloc
after start-up, a time step that must not stall on an allocation).

It runs the PCG kernels of cpm_solve on a fixed file-scope device workspace instead of a
workspace grown through the allocator, so its charges must equal cpm_solve's.  This file
is collected last so that a run stopping at the first failure has run every other test.
"""
import numpy as np
import pytest

from paper_2111_06704_gb300 import cpm
from tests import _cases

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

TOL = 1e-6  # relative (L2), the charge tolerance of the parity tests


def _dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _rel(a, b):
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


def test_static_solve_matches_cpm_solve_twice():
    work = _cases.tiny_two_sheet()
    el, io = work.electrode, work.electrolyte
    ctx = cpm.Context(el.box, rcut_dc=3.0)
    ctx.cpm_build_E(el.xyz, el.alpha)
    b = torch.empty((1, el.n), dtype=torch.float64, device="cuda")
    qs = torch.empty(1, dtype=torch.float64, device="cuda")
    ctx.cpm_potential(_dev(io.xyz), _dev(io.q), _dev(el.chi), b, qs)
    q_ref = torch.zeros((1, el.n), dtype=torch.float64, device="cuda")
    _, it_ref, _ = ctx.cpm_solve(b, q_ref, tol=1e-10)
    for _ in range(2):  # the shared array keeps the last call's contents
        q = torch.full((1, el.n), 7.0, dtype=torch.float64, device="cuda")
        it, rel = ctx.cpm_solve_static(b, q, tol=1e-10)
        torch.cuda.synchronize()
        assert rel[0] <= 1e-10
        assert _rel(q, q_ref) < TOL
        assert int(it[0]) == int(it_ref[0])
    # several right-hand sides and a previous-step guess (Eq. 26) go through it too
    b2 = torch.cat([b, 2.0 * b])
    q2 = torch.zeros((2, el.n), dtype=torch.float64, device="cuda")
    ctx.cpm_solve_static(b2, q2, tol=1e-10)
    assert _rel(q2[1], 2.0 * q_ref[0]) < TOL
    it, _ = ctx.cpm_solve_static(b, q_ref.clone(), use_guess=True, tol=1e-8)
    assert int(it[0]) <= 2
    ctx.close()


def test_static_solve_allocates_nothing_on_a_fresh_context():
    # every allocation of this context goes through torch's caching allocator, whose
    # cumulative count of allocation requests must not move across the no-allocation
    # solve, even though no cpm_solve has reserved a workspace on this context before
    work = _cases.tiny_two_sheet()
    el, io = work.electrode, work.electrolyte
    ctx = cpm.Context(el.box, torch_allocator=True, rcut_dc=3.0)
    ctx.cpm_build_E(el.xyz, el.alpha)
    b = torch.empty((2, el.n), dtype=torch.float64, device="cuda")
    qs = torch.empty(2, dtype=torch.float64, device="cuda")
    ctx.cpm_potential(_dev(np.concatenate([io.xyz, io.xyz])),
                      _dev(np.concatenate([io.q, io.q])), _dev(el.chi), b, qs)
    q = torch.zeros((2, el.n), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    count0 = torch.cuda.memory_stats()["allocation.all.allocated"]
    used0 = torch.cuda.memory_allocated()
    for _ in range(2):
        q.zero_()
        it, rel = ctx.cpm_solve_static(b, q, tol=1e-10)
        assert np.all(rel <= 1e-10)
    torch.cuda.synchronize()
    assert torch.cuda.memory_stats()["allocation.all.allocated"] == count0
    assert torch.cuda.memory_allocated() == used0
    # the same charges as the allocating solve on this context
    q_ref = torch.zeros_like(q)
    ctx.cpm_solve(b, q_ref, tol=1e-10)
    assert _rel(q, q_ref) < TOL
    ctx.close()


def test_static_solve_rejects_what_it_cannot_serve():
    work = _cases.tiny_two_sheet()
    el = work.electrode
    ctx = cpm.Context(el.box, rcut_dc=3.0)
    ctx.cpm_build_E(el.xyz, el.alpha)
    # host arrays would need staging buffers
    with pytest.raises(cpm.CpmError) as ei:
        ctx.cpm_solve_static(np.ones((1, el.n)), np.zeros((1, el.n)))
    assert ei.value.status == cpm.CPM_EINVAL
    # more right-hand sides than the fixed workspace holds
    many = 3000
    b = torch.ones((many, el.n), dtype=torch.float64, device="cuda")
    q = torch.zeros((many, el.n), dtype=torch.float64, device="cuda")
    with pytest.raises(cpm.CpmError) as ei:
        ctx.cpm_solve_static(b, q)
    assert ei.value.status == cpm.CPM_EINVAL and "workspace" in str(ei.value)
    ctx.close()
