"""Batched and ragged solves through the C ABI against the FP64 oracle, frame by frame
and system by system (Eq. 25 with the two-step method of Eq. 35 and the bordered
definition of Eq. 29 and Eq. 34).

* Eight frames of the 512-atom cell in one cpm_potential, one cpm_solve over eight
  right-hand sides and one cpm_neutralize; frame 5 carries a net electrolyte charge
  (Q^sol = +6 e), so its second step moves charge between the electrode and the ions.
* Three independent electrodes of 450 to 1,000 atoms as one ragged batch
  (cpm_batch_solve / cpm_batch_neutralize), each with its own E, P and d.

Every q is compared with the oracle's bordered solve to 1e-6 relative (L2), after a
solve to 1e-10: the parity bar of the single-frame tests.
"""
import numpy as np
import pytest

from oracle import ewald as ew
from oracle import solve as sv
from paper_2111_06704_gb300 import cpm
from paper_2111_06704_gb300 import workloads as wl
from tests import _cases

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

Q_TOL = 1e-6


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


def oracle_charges(el, e_paper, ion_xyz, ion_q, kspace="difference"):
    bsol = ew.electrolyte_potential(el.xyz, el.alpha, ion_xyz, ion_q, el.box, wl.G_EWALD,
                                    wl.RCUT_REAL, wl.KSPACE_EPS, True, kspace=kspace)
    q_sol = float(np.sum(ion_q))
    q, _ = sv.solve_bordered(e_paper, ew.rhs_volts(el.chi, bsol) / ew.KE, q_sol)
    return q, q_sol


def test_eight_frames_in_one_solve_match_the_oracle(small_cell_oracle):
    oc = small_cell_oracle
    el, base = oc.work.electrode, oc.work.electrolyte
    rng = np.random.default_rng(wl.seed_for(3, 7))
    xyz = wl.perturb_frames(rng, base.xyz[0], 8, 0.5, el.box)
    q_ion = np.broadcast_to(base.q[0], (8, base.n_ion)).copy()
    anions = np.flatnonzero(q_ion[5] < 0)[:3]
    q_ion[5, anions] = 1.0  # frame 5: Q^sol = +6
    ctx = cpm.Context(el.box)
    ctx.cpm_build_E(el.xyz, el.alpha)
    b, qsol = ctx.cpm_potential(xyz, q_ion, el.chi)
    q, it, rel = ctx.cpm_solve(b, tol=1e-10, maxit=2000)
    assert np.all(rel <= 1e-10)
    q = ctx.cpm_neutralize(q, qsol)
    ctx.close()
    errs = []
    for f in range(8):
        q_ref, q_sol = oracle_charges(el, oc.e_paper, xyz[f], q_ion[f])
        assert qsol[f] == pytest.approx(q_sol, abs=1e-12)
        errs.append(rel_l2(q[f], q_ref))
        assert errs[-1] < Q_TOL, f
        assert abs(q[f].sum() + q_sol) <= 1e-12 * np.abs(q[f]).sum()  # Eq. 34
    assert qsol[5] == pytest.approx(6.0)
    print(f"8-frame batch: q error (L2, relative) up to {max(errs):.2e}")


def test_ragged_batch_matches_the_oracle_system_by_system():
    works = wl.ragged_systems(count=3, n_lo=450, n_hi=1000, seed=3)  # 896, 480, 728 atoms
    sizes = [w.electrode.n for w in works]
    assert len(set(sizes)) == 3 and min(sizes) >= 450 and max(sizes) <= 1000
    ctxs, bs, qss, refs = [], [], [], []
    for w in works:
        el, io = w.electrode, w.electrolyte
        c = cpm.Context(el.box)
        c.cpm_build_E(el.xyz, el.alpha)
        b, qs = c.cpm_potential(io.xyz, io.q, el.chi)
        ctxs.append(c)
        bs.append(b[0])
        qss.append(qs[0])
        # the factored FP64 k-space form (pinned to the pairwise form on CPU) keeps the
        # oracle at seconds per system
        e = ew.interaction_matrix(el.xyz, el.alpha, el.box, wl.G_EWALD, wl.RCUT_REAL,
                                  wl.KSPACE_EPS, True, kspace="factored")
        refs.append(oracle_charges(el, e, io.xyz[0], io.q[0], kspace="factored")[0])
    batch = cpm.Batch(ctxs)
    q, it, rel = batch.solve(np.concatenate(bs), tol=1e-10, maxit=2000)
    assert np.all(rel <= 1e-10)
    q = batch.neutralize(q, np.array(qss))
    batch.close()
    for k, part in enumerate(np.split(q, np.cumsum(sizes)[:-1])):
        print(f"ragged system of {sizes[k]} atoms: q error {rel_l2(part, refs[k]):.2e}")
        assert rel_l2(part, refs[k]) < Q_TOL, k
        assert abs(part.sum() + qss[k]) <= 1e-12 * np.abs(part).sum()
    for c in ctxs:
        c.close()
