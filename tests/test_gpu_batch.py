"""Ragged batches: several electrodes of different sizes solved by one PCG over all of
them (cpm_batch_*), against the same systems solved one context at a time, which the
parity tests pin to the oracle.

Every system runs the same iteration as its own solve: the matvec arithmetic is the same
and only the partition of the FP64 dot products differs, so charges agree to the
solve tolerance and iteration counts to within one.
"""
import numpy as np
import pytest

from paper_2111_06704_gb300 import cpm
from paper_2111_06704_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


@pytest.fixture(scope="module")
def systems():
    works = wl.ragged_systems(count=5, n_lo=450, n_hi=1500, seed=7)
    ctxs, bs, qss = [], [], []
    for w in works:
        el, io = w.electrode, w.electrolyte
        c = cpm.Context(el.box, precision=cpm.CPM_PREC_FP32)
        c.cpm_build_E(el.xyz, el.alpha)
        b, qs = c.cpm_potential(io.xyz, io.q, el.chi)
        ctxs.append(c)
        bs.append(b[0])
        qss.append(qs[0])
    yield works, ctxs, bs, np.array(qss)
    for c in ctxs:
        c.close()


def test_sizes_are_ragged(systems):
    works = systems[0]
    sizes = [w.electrode.n for w in works]
    assert len(set(sizes)) == len(sizes) and min(sizes) >= 400


def test_batch_solve_matches_single_solves(systems):
    works, ctxs, bs, qss = systems
    single, its = [], []
    for c, b in zip(ctxs, bs):
        q, it, rel = c.cpm_solve(b[None], tol=1e-10)
        single.append(q[0])
        its.append(int(it[0]))
    batch = cpm.Batch(ctxs)
    q, it, rel = batch.solve(np.concatenate(bs), tol=1e-10)
    assert np.all(rel <= 1e-10)
    parts = np.split(q, np.cumsum(batch.sizes)[:-1])
    for k, (qb, qs_) in enumerate(zip(parts, single)):
        assert np.linalg.norm(qb - qs_) <= 1e-8 * np.linalg.norm(qs_), k
        assert abs(int(it[k]) - its[k]) <= 1
    # Eq. 35 per system with its own d
    qn = batch.neutralize(q.copy(), qss)
    for k, (c, qb) in enumerate(zip(ctxs, np.split(qn, np.cumsum(batch.sizes)[:-1]))):
        ref = c.cpm_neutralize(parts[k][None].copy(), qss[k:k + 1])[0]
        assert np.abs(qb - ref).max() <= 1e-12 * np.abs(ref).max()
        assert abs(qb.sum() + qss[k]) < 1e-12 * np.abs(qb).sum()
    batch.close()


def test_batch_with_device_vectors_and_a_converged_guess(systems):
    works, ctxs, bs, _ = systems
    batch = cpm.Batch(ctxs[::-1])  # another order, another largest-first layout
    b = torch.tensor(np.concatenate(bs[::-1]), device="cuda")
    q = torch.zeros_like(b)
    _, it, rel = batch.solve(b, q, tol=1e-10)
    q_host = q.cpu().numpy()
    # restarting from the converged charges needs (almost) no iteration
    _, it2, rel2 = batch.solve(b, q.clone(), use_guess=True, tol=1e-9)
    assert np.all(it2 <= 1) and np.all(rel2 <= 1e-9)
    # a single-system batch is the plain solve
    one = cpm.Batch(ctxs[:1])
    q1, it1, _ = one.solve(bs[0], tol=1e-10)
    qs_, its_, _ = ctxs[0].cpm_solve(bs[0][None], tol=1e-10)
    assert np.linalg.norm(q1 - qs_[0]) <= 1e-8 * np.linalg.norm(qs_[0])
    assert np.isfinite(q_host).all()
    one.close()
    batch.close()


def test_batch_rejects_mixed_configurations(systems):
    works, ctxs, _, _ = systems
    el = works[0].electrode
    f64 = cpm.Context(el.box, precision=cpm.CPM_PREC_FP64)
    f64.cpm_build_E(el.xyz, el.alpha)
    with pytest.raises(cpm.CpmError):
        cpm.Batch([ctxs[0], f64])
    unbuilt = cpm.Context(el.box)
    with pytest.raises(cpm.CpmError):
        cpm.Batch([ctxs[0], unbuilt])
    f64.close()
    unbuilt.close()
