"""The tensor-core k-space tail of the BF16X6 build against the FP64 oracle and the FP64
build, on electrodes whose size is not a multiple of the 256 x 256 tile edge.

* 1,144 atoms (padded to 1,152): the last tile row holds one 128-row half, so the
  kernels' half-tile paths run; 3,200 atoms: several full tiles per row.
* The tail sums six BF16 products per heavy K-block and three or one FP16 products of
  power-of-two scaled values per light one, with chunked FP32 accumulation drained into
  hi/lo float pairs; the schedule keeps each reduced group's error below 1e-8 and the
  diagonal takes exact weight sums.  So: every entry within 1e-6 of the largest (the
  parity bar), the off-diagonal RMS difference below 1e-8 (float rounding of E included),
  the diagonal within 1e-7 of the FP64 build on average, and E exactly symmetric.
"""
import numpy as np
import pytest

from oracle import ewald as ew
from oracle import solve as sv
from paper_2111_06704_gb300 import cpm
from paper_2111_06704_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def build(el, precision):
    ctx = cpm.Context(el.box, precision=precision)
    ctx.cpm_build_E(el.xyz, el.alpha)
    e = ctx.cpm_get_E(cpm.CPM_E_STORED)
    info = ctx.cpm_get_info()
    ctx.close()
    return e, info


@pytest.mark.parametrize("cells", [(13, 11), (20, 20)])
def test_tensor_core_tail_against_fp64(cells):
    el = wl.two_sheet_electrode(*cells)
    e64, _ = build(el, cpm.CPM_PREC_FP64)
    e, info = build(el, cpm.CPM_PREC_BF16X6)
    n6, n3, n1 = info["tc_blocks"]
    assert n6 > 0 and n3 > 0 and n1 > 0  # all three product counts take part
    assert 0 < info["tc_blocks_fp8"] < n1  # one-product blocks in FP16 and in FP8
    assert n6 % 2 == 0 and (n6 + n3) % 2 == 0  # region ends hold whole [cos | sin] pairs
    scale = np.abs(e64).max()
    d = e - e64
    off = ~np.eye(el.n, dtype=bool)
    assert np.abs(d).max() < 1e-6 * scale
    assert np.sqrt((d[off] ** 2).mean()) < 1e-8
    assert abs(np.diag(d).mean()) < 1e-7
    assert np.array_equal(e, e.T)


def test_rebuilds_reuse_or_release_the_workspace():
    # one context building electrodes of different sizes in one box, with its workspace
    # kept between builds or released, gives what a fresh context gives, bit for bit
    el = wl.two_sheet_electrode(20, 20)
    part = np.arange(0, el.n, 3)  # a ragged subset (1,067 atoms) in the same box

    def fresh(idx):
        ctx = cpm.Context(el.box)
        ctx.cpm_build_E(el.xyz[idx], el.alpha[idx])
        e = ctx.cpm_get_E(cpm.CPM_E_STORED)
        ctx.close()
        return e

    whole = np.arange(el.n)
    ref = {"whole": fresh(whole), "part": fresh(part)}
    ctx = cpm.Context(el.box)
    for name, idx, release in [("whole", whole, False), ("part", part, False),
                               ("whole", whole, True), ("part", part, True)]:
        ctx.cpm_build_E(el.xyz[idx], el.alpha[idx])
        assert np.array_equal(ctx.cpm_get_E(cpm.CPM_E_STORED), ref[name])
        if release:
            ctx.cpm_release_workspace()
    ctx.close()


def test_multi_tile_tail_against_the_oracle():
    # 1,144 atoms: five tile rows of 256, the last a single 128-row half.  E entry by entry
    # against the oracle's FP64 sums (the factored reciprocal form, pinned to the pairwise
    # difference form on CPU) and the neutral charges of a 446-ion frame against the
    # bordered solve (Eq. 29, Eq. 34)
    el = wl.two_sheet_electrode(13, 11)
    rng = np.random.default_rng(wl.seed_for(2, 11))
    ions, q_ion = wl.random_ions(rng, 223, 223, el.box, min_sep=2.5)
    ctx = cpm.Context(el.box)  # the default BF16X6 build
    ctx.cpm_build_E(el.xyz, el.alpha)
    e_gpu = ctx.cpm_get_E(cpm.CPM_E_PAPER)
    q, it, rel, _, qsol = cpm.charges(ctx, ions[None], q_ion[None], el.chi, tol=1e-10,
                                      maxit=2000)
    ctx.close()
    e_ref = ew.interaction_matrix(el.xyz, el.alpha, el.box, wl.G_EWALD, wl.RCUT_REAL,
                                  wl.KSPACE_EPS, True, kspace="factored")
    assert np.abs(e_gpu - e_ref).max() < 1e-6 * np.abs(e_ref).max()
    off = ~np.eye(el.n, dtype=bool)
    assert np.sqrt(((e_gpu - e_ref)[off] ** 2).mean()) < 1e-8
    bsol = ew.electrolyte_potential(el.xyz, el.alpha, ions, q_ion, el.box, wl.G_EWALD,
                                    wl.RCUT_REAL, wl.KSPACE_EPS, True, kspace="factored")
    q_ref, _ = sv.solve_bordered(e_ref, ew.rhs_volts(el.chi, bsol) / ew.KE, float(q_ion.sum()))
    assert rel[0] <= 1e-10
    err = np.linalg.norm(q[0] - q_ref) / np.linalg.norm(q_ref)
    print(f"1,144 atoms: E max error {np.abs(e_gpu - e_ref).max() / np.abs(e_ref).max():.2e} "
          f"of max|E|, q error {err:.2e}")
    assert err < 1e-6
