"""The tensor-core k-space tail of the BF16X6 build: the default 256 x 256 tile kernels
(six-product K-blocks with two-sum chunk drains, then the three- and one-product ones)
against the 128 x 128 tile kernel with TMEM hi/lo drains (CPM_TC_STRIP=0) and against
the FP64 build, on electrodes whose size is not a multiple of the tile edge.

* 1,144 atoms (padded to 1,152): the last 256-row tile holds one 128-row half, so the
  kernels' half-tile paths run; 3,200 atoms: several full tiles per row.
* The two tensor-core paths sum the same BF16 products in the same order inside each
  chunk and differ only in how chunks are carried (FP32 pair vs TMEM pair) and in the
  light region's accumulation, far below the float rounding of E: they agree to two
  float ulps of the largest entry, with an RMS difference under 1e-8.
* Against the FP64 build: 1e-6 of the largest entry (the parity bar), the diagonal
  within 1e-7 of it on average (the diagonal takes the exact weight sums of the tail).
"""
import numpy as np
import pytest

from paper_2111_06704_gb300 import cpm
from paper_2111_06704_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def build(el, precision=cpm.CPM_PREC_BF16X6):
    ctx = cpm.Context(el.box, precision=precision)
    ctx.cpm_build_E(el.xyz, el.alpha)
    e = ctx.cpm_get_E(cpm.CPM_E_STORED)
    ctx.close()
    return e


@pytest.mark.parametrize("cells", [(13, 11), (20, 20)])
def test_256_tiles_match_128_tiles_and_fp64(cells, monkeypatch):
    el = wl.two_sheet_electrode(*cells)
    e64 = build(el, cpm.CPM_PREC_FP64)
    e256 = build(el)
    monkeypatch.setenv("CPM_TC_STRIP", "0")
    e128 = build(el)
    scale = np.abs(e64).max()
    d = e256 - e128
    assert np.abs(d).max() <= 2 * np.spacing(np.float32(scale))
    assert np.sqrt((d ** 2).mean()) < 1e-8
    for e in (e256, e128):
        assert np.abs(e - e64).max() < 1e-6 * scale
        assert abs(np.diag(e - e64).mean()) < 1e-7
        assert np.array_equal(e, e.T)
