"""Forces on the electrolyte ions from the electrode charges (cpm_ion_forces; Eq. S25
inside the Ewald sums of Eq. 22 / 25) against the FP64 oracle (oracle/forces.py, pinned
by finite differences of its coupling energy), through the C ABI.

The reciprocal part's tail runs on float phasors (about one ulp) with error-free sums and
the head and the real space in FP64: every component within 1e-6 of the largest force.
"""
import numpy as np
import pytest

from oracle import forces as fo
from paper_2111_06704_gb300 import cpm
from paper_2111_06704_gb300 import workloads as wl
from tests import _cases

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

PREC = {"fp64": cpm.CPM_PREC_FP64, "bf16x6": cpm.CPM_PREC_BF16X6}


@pytest.mark.parametrize("prec", ["bf16x6", "fp64"])
def test_forces_on_the_small_cell(small_cell_oracle, prec):
    oc = small_cell_oracle
    el, io = oc.work.electrode, oc.work.electrolyte
    ctx = cpm.Context(el.box, precision=PREC[prec])
    ctx.cpm_build_E(el.xyz, el.alpha)
    q = oc.q  # the oracle's neutral charges of the frame
    f = ctx.cpm_ion_forces(io.xyz, io.q, q)[0]
    ref = fo.forces_on_ions(el.xyz, el.alpha, q[0], io.xyz[0], io.q[0], el.box, wl.G_EWALD,
                            wl.RCUT_REAL, wl.KSPACE_EPS, True)
    assert np.abs(f - ref).max() <= 1e-6 * np.abs(ref).max()
    ctx.close()


def test_forces_with_many_images_and_frames():
    # the 48-atom cell: box edges below 2 r_c (many images of every pair), two frames with
    # different electrode charges, an ion 0.6 A from an electrode atom
    work = _cases.tiny_two_sheet(q_sol=2)
    el, io = work.electrode, work.electrolyte
    rng = np.random.default_rng(9)
    ions = np.stack([io.xyz[0], io.xyz[0] + rng.normal(0.0, 0.3, io.xyz[0].shape)])
    ions[1, 0] = el.xyz[5] + np.array([0.3, -0.2, 0.49])
    q_ion = np.stack([io.q[0], io.q[0]])
    q = rng.normal(0.0, 0.01, (2, el.n))
    ctx = cpm.Context(el.box, rcut_dc=3.0)
    ctx.cpm_build_E(el.xyz, el.alpha)
    f = ctx.cpm_ion_forces(ions, q_ion, q)
    for k in range(2):
        ref = fo.forces_on_ions(el.xyz, el.alpha, q[k], ions[k], q_ion[k], el.box, wl.G_EWALD,
                                wl.RCUT_REAL, wl.KSPACE_EPS, True)
        assert np.abs(f[k] - ref).max() <= 1e-6 * np.abs(ref).max(), k
    ctx.close()
