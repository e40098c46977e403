"""The learned guess's file format through the C ABI, on the host (no GPU needed):
cpm_guess_save / cpm_guess_load give back the same parameters, normalisation and target
scale bit for bit, and refuse a damaged, truncated or foreign file with CPM_EIO.
"""
import ctypes
import os

import numpy as np

from paper_2111_06704_gb300 import cpm


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def test_save_load_roundtrip_and_damage(tmp_path):
    lib = cpm.load()
    rng = np.random.default_rng(3)
    params = rng.standard_normal(cpm.CPM_MLP_PARAMS).astype(np.float32)
    norm = rng.standard_normal(64).astype(np.float32)
    path = str(tmp_path / "net.cpmguess")
    assert lib.cpm_guess_save(path.encode(), _p(params), _p(norm), ctypes.c_float(0.25)) == 0
    p2 = np.zeros_like(params)
    n2 = np.zeros_like(norm)
    ts = ctypes.c_float(0.0)
    assert lib.cpm_guess_load(path.encode(), _p(p2), _p(n2), ctypes.byref(ts)) == 0
    assert np.array_equal(p2, params) and np.array_equal(n2, norm) and ts.value == 0.25
    raw = open(path, "rb").read()
    for name, data in [("flipped", raw[:100] + bytes([raw[100] ^ 1]) + raw[101:]),
                       ("truncated", raw[:-9]), ("longer", raw + b"\0"),
                       ("foreign", b"NOTGUESS" + raw[8:])]:
        bad = str(tmp_path / name)
        with open(bad, "wb") as f:
            f.write(data)
        p3 = np.full_like(params, 7.0)
        assert lib.cpm_guess_load(bad.encode(), _p(p3), _p(n2), ctypes.byref(ts)) == cpm.CPM_EIO
        assert np.all(p3 == 7.0)  # nothing written
    missing = str(tmp_path / "missing")
    assert lib.cpm_guess_load(missing.encode(), _p(p2), _p(n2), ctypes.byref(ts)) == cpm.CPM_EIO
    assert not os.path.exists(missing)
