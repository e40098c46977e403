"""Input recipes (host only): every generator makes what the input recipe states (sizes,
boxes, sheet potentials, ion counts, charges, slit bounds, separations, pinholes), and the
scale point's random walk keeps every ion in its own interlayer gap, at least 2 A from both
sheets, with x and y wrapped into the box."""
import numpy as np

from paper_2111_06704_gb300 import workloads as wl


def test_scale_walk_stays_in_the_gaps():
    base = wl.scale_point(rhs=1)
    walk = wl.scale_walk(4)
    el, io = walk.electrode, walk.electrolyte
    assert el.n == base.electrode.n and np.array_equal(el.xyz, base.electrode.xyz)
    assert io.xyz.shape == (4, base.electrolyte.xyz.shape[1], 3)
    gap0 = np.floor(base.electrolyte.xyz[0][:, 2] / 7.0)
    for f in range(4):
        z = io.xyz[f][:, 2]
        gap = np.floor(z / 7.0)
        assert np.array_equal(gap, gap0)
        assert np.min(np.minimum(z - 7.0 * gap, 7.0 * (gap + 1) - z)) >= 2.0 - 1e-9
        assert np.all((io.xyz[f][:, 0] >= 0) & (io.xyz[f][:, 0] < el.box[0]))
        assert np.all((io.xyz[f][:, 1] >= 0) & (io.xyz[f][:, 1] < el.box[1]))
    # steps of 0.1 A per coordinate: frame-to-frame moves stay small (away from the walls)
    d = io.xyz[1] - io.xyz[0]
    d[:, :2] -= np.round(d[:, :2] / np.asarray(el.box[:2])) * np.asarray(el.box[:2])
    assert np.abs(d).max() < 1.0
    assert np.array_equal(io.q[0], base.electrolyte.q[0])


# ---------------------------------------------------- the recipes of the parity workloads

def _min_separation(xyz, box):
    """Smallest pair distance, minimum image in x and y, plain distance in z."""
    from scipy.spatial import cKDTree
    pts = np.array(xyz, dtype=np.float64)
    pts[:, 0] %= box[0]
    pts[:, 1] %= box[1]
    tree = cKDTree(pts, boxsize=[box[0], box[1], 1e6])
    d, _ = tree.query(pts, k=2)
    return d[:, 1].min()


def _check_two_sheets(el, cells_x, cells_y):
    assert el.n == 8 * cells_x * cells_y
    assert np.allclose(el.box, (cells_x * wl.CELL_A, cells_y * wl.CELL_B, 90.0))
    low = el.xyz[:, 2] == 0.0
    assert np.count_nonzero(low) == el.n // 2 and np.all(el.xyz[~low, 2] == 30.0)
    assert np.all(el.chi[low] == -0.5) and np.all(el.chi[~low] == 0.5)
    assert np.all(el.alpha == wl.ALPHA)


def _check_ions(q, xyz, n_ion, box, min_sep=None):
    assert q.shape == (n_ion,) and np.count_nonzero(q == 1.0) == n_ion // 2
    assert np.count_nonzero(q == -1.0) == n_ion // 2  # Q^sol = 0
    assert np.all((xyz[:, 2] > 3.0) & (xyz[:, 2] < 27.0))
    if min_sep is not None:
        assert _min_separation(xyz, box) >= min_sep


def test_small_cell_recipe():
    w = wl.small_cell()
    _check_two_sheets(w.electrode, 8, 8)
    assert w.electrolyte.xyz.shape == (1, 200, 3)
    _check_ions(w.electrolyte.q[0], w.electrolyte.xyz[0], 200, w.electrode.box, 2.5)
    assert np.array_equal(wl.small_cell().electrolyte.xyz, w.electrolyte.xyz)  # seeded


def test_precision_cell_recipe():
    w = wl.precision_cell()
    _check_two_sheets(w.electrode, 40, 40)
    _check_ions(w.electrolyte.q[0], w.electrolyte.xyz[0], 2000, w.electrode.box, 2.5)


def test_frame_batch_recipe():
    w = wl.frame_batch()
    _check_two_sheets(w.electrode, 8, 8)
    xyz, q = w.electrolyte.xyz, w.electrolyte.q
    assert xyz.shape == (256, 2000, 3) and q.shape == (256, 2000)
    for f in (0, 1, 255):
        _check_ions(q[f], xyz[f], 2000, w.electrode.box)
    # Gaussian perturbations of one base frame: sigma 0.5 A per coordinate (away from
    # the reflecting walls and the periodic wrap)
    d = xyz[2] - xyz[1]
    d[:, :2] -= np.round(d[:, :2] / np.asarray(w.electrode.box[:2])) * w.electrode.box[:2]
    assert 0.6 < d[:, :2].std() < 0.8  # two independent sigma = 0.5 draws: 0.5 sqrt(2)


def test_ragged_systems_recipe():
    systems = wl.ragged_systems()
    assert len(systems) == 32
    sizes = [s.electrode.n for s in systems]
    assert min(sizes) >= 400 and max(sizes) <= 8200 and len(set(sizes)) >= 16  # uneven
    for s in systems:
        n, n_ion = s.electrode.n, s.electrolyte.q.shape[1]
        assert n_ion == 2 * max(1, round(n * 200 / 512 / 2))
        _check_ions(s.electrolyte.q[0], s.electrolyte.xyz[0], n_ion, s.electrode.box)


def test_scale_point_recipe():
    w = wl.scale_point(rhs=2)
    el, io = w.electrode, w.electrolyte
    assert el.n == 106_568 and np.allclose(el.box, (90 * wl.CELL_A, 52 * wl.CELL_B, 105.0))
    full = 4 * 90 * 52
    for s in range(6):
        on = el.xyz[:, 2] == 7.0 * s
        assert np.count_nonzero(on) <= 0.95 * full  # at least 5% cut as pinholes
        assert np.all(el.chi[on] == (0.5 if s % 2 else -0.5))
    assert io.xyz.shape == (2, 20_000, 3)
    q = io.q[0]
    assert np.count_nonzero(q == 1.0) == np.count_nonzero(q == -1.0) == 10_000
    for f in range(2):
        z = io.xyz[f][:, 2]
        gap = np.floor(z / 7.0)
        assert np.array_equal(np.bincount(gap.astype(int)), [4000] * 5)
        assert np.min(np.minimum(z - 7.0 * gap, 7.0 * (gap + 1) - z)) >= 2.0 - 1e-9
    for g in range(5):  # 2.5 A apart within each gap (the base frame)
        sel = np.floor(io.xyz[0][:, 2] / 7.0) == g
        assert _min_separation(io.xyz[0][sel], el.box) >= 2.5
