"""The host plan of the k-space sum (cpm_plan_kspace; host arithmetic only, no GPU).

* The k-vector table is the oracle's (Eq. 13, Eq. 20): the same half-space vectors and
  weights, in order of decreasing weight.
* The tensor-core tail's schedule keeps its stated error budget: every format's region
  of K-blocks sums to a bound 64 max W_K times that format's error per product within
  1e-8, region ends are even (whole [cos | sin] pairs), each block's power-of-two scale
  puts its largest operand value where the format needs it, and chunks hold one scale.
* At the 12,800-atom cell the plan is the one the GPU build reports (474 six-product,
  1,984 three-product and 4,340 one-product K-blocks, 2,270 of them in FP8; a 256-column
  head; 896 head columns for the FP32 SIMT build).
"""
import math

import numpy as np
import pytest

from oracle import ewald as ew
from paper_2111_06704_gb300 import cpm
from paper_2111_06704_gb300 import workloads as wl

ERR8 = 0.13                   # one E4M3 product of scaled values
ERR1 = 2.0**-10 + 2.0**-23    # one FP16 product
ERR3 = 5 * 2.0**-22           # three FP16 products
BUDGET = 1e-8

BOXES = {
    "512-atom cell": wl.small_cell().electrode.box,
    "12,800-atom cell": wl.two_sheet_electrode(40, 40).box,
    "48-atom cell": wl.two_sheet_electrode(3, 2).box,
}


def _plan(box, **kw):
    return cpm.cpm_plan_kspace(box, **kw)


@pytest.mark.parametrize("name", ["512-atom cell", "48-atom cell"])
def test_table_matches_the_oracle(name):
    box = BOXES[name]
    p = _plan(box)
    hkl, _, w = ew.kvectors(box, wl.G_EWALD, wl.KSPACE_EPS)
    assert p["m"] == len(w) and p["m_pad"] == -(-len(w) // 64) * 64
    assert np.all(np.diff(p["w"]) <= 0)  # decreasing weight
    # the same vectors with the same weights (each key once)
    ref = {tuple(int(x) for x in h): wt for h, wt in zip(hkl, w)}
    got = {tuple(int(x) for x in h): wt for h, wt in zip(p["hkl"], p["w"])}
    assert got.keys() == ref.keys()
    assert max(abs(got[k] - ref[k]) / ref[k] for k in ref) < 1e-13


def _bwm(w, kb_end):
    """64 x the largest weight of each K-block (block b: k-vectors 64 (b // 2) ..)."""
    wp = np.zeros(kb_end * 32)
    wp[:len(w)] = w
    pairs = wp.reshape(-1, 64).max(axis=1) * 64.0
    return np.repeat(pairs, 2)


@pytest.mark.parametrize("name", sorted(BOXES))
def test_tail_schedule_keeps_its_error_budget(name):
    p = _plan(BOXES[name])
    kb0, kb6, kb3, kb8, kbn = (p[k] for k in ("kb_begin", "kb6_end", "kb3_end", "kb8_begin",
                                             "kb_end"))
    assert kb0 * 64 == p["head_cols"] and p["head_cols"] % 128 == 0
    assert kb0 <= kb6 <= kb3 <= kb8 <= kbn == 2 * p["m_pad"] // 64
    for end in (kb0, kb6, kb3, kb8, kbn):
        assert end % 2 == 0
    bwm = _bwm(p["w"], kbn)
    assert bwm[kb8:].sum() * ERR8 <= BUDGET
    assert bwm[kb3:kb8].sum() * ERR1 <= BUDGET
    assert bwm[kb6:kb3].sum() * ERR3 <= BUDGET
    # each region starts as early as the budget allows, up to the rounding of its start
    # to a whole pair: one more pair before it would break the budget
    for start, end, err in ((kb8, kbn, ERR8), (kb3, kb8, ERR1), (kb6, kb3, ERR3)):
        if start - 2 >= kb0:
            assert bwm[start - 2:end].sum() * err > BUDGET
    # scales: FP16 values 2^e sqrt(max W) in [1/2, 1), FP8 ones in [128, 256)
    e = p["kexp"].astype(np.float64)
    top = np.sqrt(bwm / 64.0)
    live = bwm > 0
    fp16 = np.zeros(kbn, bool)
    fp16[kb6:kb8] = True
    fp8 = np.zeros(kbn, bool)
    fp8[kb8:] = True
    x16 = np.ldexp(top, e.astype(int))
    assert np.all((x16[fp16 & live] >= 0.5) & (x16[fp16 & live] < 1.0))
    assert np.all((x16[fp8 & live] >= 128.0) & (x16[fp8 & live] < 256.0))
    assert np.all(p["kexp"][0::2] == p["kexp"][1::2])  # a pair shares its scale


@pytest.mark.parametrize("name", sorted(BOXES))
def test_chunks(name):
    p = _plan(BOXES[name])
    kb0, kb6, kbn = p["kb_begin"], p["kb6_end"], p["kb_end"]
    ends = np.flatnonzero(p["chunk_end"])
    assert len(ends) == p["chunks"] and ends[-1] == kbn - 1 and ends[0] >= kb0
    if kb6 > kb0:
        assert kb6 - 1 in ends
    w = np.zeros(kbn * 32)
    w[:len(p["w"])] = p["w"]
    bw = np.repeat(w.reshape(-1, 64).sum(axis=1), 2)
    start = kb0
    for end in ends:
        blocks = np.arange(start, end + 1)
        if end < kb6:
            # six-product chunks: at most 32 blocks, closed once 5e-3 of weight gathered
            assert len(blocks) <= 32 and bw[start:end].sum() < 5e-3
        else:
            # scaled chunks: whole pairs, one scale, at most 512 blocks
            assert start >= kb6 and len(blocks) <= 512 and (end - start) % 2 == 1
            assert len(set(p["kexp"][start:end + 1])) == 1
        start = end + 1


def test_plan_at_the_12800_atom_cell():
    box = BOXES["12,800-atom cell"]
    p = _plan(box)
    assert p["m"] == 217_619 and p["head_cols"] == 256
    n6 = p["kb6_end"] - p["kb_begin"]
    n3 = p["kb3_end"] - p["kb6_end"]
    n1 = p["kb_end"] - p["kb3_end"]
    assert (n6, n3, n1, p["kb_end"] - p["kb8_begin"]) == (474, 1984, 4340, 2270)
    # the head's k-steps each carry more than 5e-3 of weight (16 operand columns a step;
    # the head is rounded up to whole 128-column groups)
    assert _step_weights(p)[: p["head_cols"] // 16 - 7].min() > 5e-3
    assert _plan(box, precision=cpm.CPM_PREC_FP32)["head_cols"] == 896


def _step_weights(p):
    """Weight of each 16-column k-step: step s holds k-vectors 64 (s // 8) + 16 (s % 4)
    .. + 15, in the cos (s % 8 < 4) or the sin half of its 128 columns."""
    w = np.zeros(p["m_pad"])
    w[:p["m"]] = p["w"]
    quarters = w.reshape(-1, 4, 16).sum(axis=2)     # [64-vector group][quarter]
    return np.concatenate([quarters, quarters], axis=1).reshape(-1)


def test_plan_rejects_what_create_rejects():
    import ctypes
    lib = cpm.load()
    p = cpm.default_params((10.0, 10.0, 30.0), kspace_eps=2.0)
    out = cpm.cpm_kspace_plan()
    assert lib.cpm_plan_kspace(ctypes.byref(p), ctypes.byref(out), None, None, None,
                               None) == cpm.CPM_EINVAL
    p = cpm.default_params((10.0, 10.0, 30.0))
    assert lib.cpm_plan_kspace(ctypes.byref(p), None, None, None, None, None) == cpm.CPM_EINVAL
    assert lib.cpm_plan_kspace(None, ctypes.byref(out), None, None, None, None) == cpm.CPM_EINVAL
    assert math.isfinite(cpm.cpm_plan_kspace((10.0, 10.0, 30.0))["w"][0])


@pytest.mark.parametrize("box,g,m", [
    ((8 * wl.CELL_A, 8 * wl.CELL_B, 90.0), 0.3, 8_645),          # the 512-atom cell
    ((40 * wl.CELL_A, 40 * wl.CELL_B, 90.0), 0.3, 217_619),      # the 12,800-atom cell
    ((90 * wl.CELL_A, 52 * wl.CELL_B, 105.0), 0.3, 742_575),     # the scale point
    ((90 * wl.CELL_A, 52 * wl.CELL_B, 105.0), 0.15, 92_837),     # ... at its g = 0.15
])
def test_table_sizes_of_the_workloads(box, g, m):
    # the k-vector counts of the workloads, counted independently of this library
    assert _plan(box, g_ewald=g)["m"] == m
