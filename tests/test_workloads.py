"""Input recipes (host only): the scale point's random walk starts from the scale point's
electrode and ions and keeps every ion in its own interlayer gap, at least 2 A from both
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
