"""Shared test cases: seeded workloads and the oracle's answers for them."""
from __future__ import annotations

import dataclasses
import functools

import numpy as np

from oracle import ewald as ew
from oracle import precond as pc
from oracle import solve as sv
from paper_2111_06704_gb300 import workloads as wl


@dataclasses.dataclass
class OracleCase:
    work: wl.Workload
    g: float
    rc: float
    eps: float
    e_paper: np.ndarray       # Eq. 22 + Eq. 39, 1/A
    e_neutral: np.ndarray     # neutral-equivalent form
    bsol_paper: np.ndarray    # [F, N] e/A
    b_neutral_volts: np.ndarray  # [F, N] V
    q: np.ndarray             # [F, N] neutral charges (e), bordered solve
    qb_neutral: np.ndarray    # [F, N] E_n^-1 b_n
    d_neutral: np.ndarray     # [N]
    c_ele_neutral: float
    q_sol: np.ndarray         # [F]


def oracle_case(work: wl.Workload, g=wl.G_EWALD, rc=wl.RCUT_REAL, eps=wl.KSPACE_EPS,
                slab=True) -> OracleCase:
    el, io = work.electrode, work.electrolyte
    e = ew.interaction_matrix(el.xyz, el.alpha, el.box, g, rc, eps, slab)
    en = ew.neutral_form_matrix(e, el.xyz, el.box, g, slab)
    d, _, c = sv.neutralizing_vector(en)
    bs, bn, qs, qq, qb = [], [], [], [], []
    for f in range(io.frames):
        bsol = ew.electrolyte_potential(el.xyz, el.alpha, io.xyz[f], io.q[f], el.box, g, rc,
                                        eps, slab)
        q_sol = float(io.q[f].sum())
        b = ew.rhs_volts(el.chi, bsol) / ew.KE
        q, _ = sv.solve_bordered(e, b, q_sol)
        bsn = ew.neutral_form_bsol(bsol, el.xyz, io.xyz[f], io.q[f], el.box, g, slab)
        b_n = ew.rhs_volts(el.chi, bsn)
        bs.append(bsol)
        bn.append(b_n)
        qs.append(q_sol)
        qq.append(q)
        qb.append(np.linalg.solve(en, b_n / ew.KE))
    return OracleCase(work, g, rc, eps, e, en, np.array(bs), np.array(bn), np.array(qq),
                      np.array(qb), d, c, np.array(qs))


@functools.lru_cache(maxsize=None)
def small_cell_oracle() -> OracleCase:
    return oracle_case(wl.small_cell())


def tiny_two_sheet(nx=3, ny=2, n_ion=8, seed=7, q_sol=0):
    """A 48-atom two-sheet cell with a handful of ions (fast oracle cases)."""
    el = wl.two_sheet_electrode(nx, ny)
    rng = np.random.default_rng(seed)
    n_cat = (n_ion + q_sol) // 2
    ions, q = wl.random_ions(rng, n_cat, n_ion - n_cat, el.box, min_sep=1.0)
    return wl.Workload("tiny", el, wl.Electrolyte(ions[None], q[None]))


def dc_setup(work: wl.Workload, g_dc=wl.G_DC, rcut=wl.RCUT_DC):
    el = work.electrode
    return pc.dc_preconditioner(el.xyz, el.alpha, el.box, g_dc, rcut)
