"""Pins of the FP64 learned-guess oracle (no GPU): hand-written backpropagation against
central finite differences of the forward pass, SiLU against its closed-form limits,
and the shell features on lattices whose answer is known by symmetry."""
import math

import numpy as np
import pytest

from oracle import ewald as ew
from oracle import mlp
from paper_2111_06704_gb300 import workloads as wl
from oracle import precond as pc


def test_parameter_count():
    assert mlp.N_PARAMS == 64 * 32 + 64 + 2 * (64 * 64 + 64) + 64 + 1


def test_silu_limits_and_derivative():
    z = np.array([-30.0, -1.0, 0.0, 1.0, 30.0])
    s = mlp.silu(z)
    assert s[2] == 0.0 and s[4] == pytest.approx(30.0) and abs(s[0]) < 1e-11
    assert s[3] == pytest.approx(1.0 / (1.0 + math.exp(-1.0)))
    h = 1e-6
    fd = (mlp.silu(z + h) - mlp.silu(z - h)) / (2 * h)
    assert np.allclose(mlp.silu_grad(z), fd, atol=1e-8)
    assert mlp.silu_grad(np.array([0.0]))[0] == pytest.approx(0.5)


def test_backprop_matches_finite_differences():
    rng = np.random.default_rng(3)
    params = mlp.init_params(rng, scale=0.7)
    params += 0.05 * rng.standard_normal(params.shape)  # non-zero biases too
    x = rng.standard_normal((9, mlp.N_FEATURES))
    t = rng.standard_normal(9)
    loss, grad = mlp.loss_and_grad(params, x, t)
    idx = rng.choice(mlp.N_PARAMS, size=60, replace=False)
    idx = np.concatenate([idx, [mlp.N_PARAMS - 1, 64 * 32, 64 * 32 + 64]])  # biases
    h = 1e-6
    for k in idx:
        e = np.zeros_like(params)
        e[k] = h
        lp, _ = mlp.loss_and_grad(params + e, x, t)
        lm, _ = mlp.loss_and_grad(params - e, x, t)
        fd = (lp - lm) / (2 * h)
        assert grad[k] == pytest.approx(fd, rel=1e-5, abs=1e-9)
    # the loss is zero at the network's own output
    y, _ = mlp.forward(params, x)
    assert mlp.loss_and_grad(params, x, y)[0] == 0.0


def test_shell_features_on_a_uniform_sheet():
    # every site of a perfect sheet is equivalent: uniform b gives uniform shell means,
    # and a change of b on one atom shows up only in its neighbours' matching shell
    el = wl.two_sheet_electrode(7, 4)  # box edges above 2 x 8 A
    nb = pc.neighbours(el.xyz, el.box, 8.0)
    b = np.full(el.n, 0.25)
    p0 = np.zeros((el.n, el.n))  # the P feature is pinned separately below
    f = mlp.features(b, b, el.chi, el.xyz, el.box, nb, p0)
    assert np.allclose(f[:, 0], 0.0) and np.allclose(f[:, 1:9], 0.0)
    assert np.allclose(f[:, 9], 0.25)
    filled = f[:, 10:18] != 0.0
    assert np.allclose(f[:, 10:18][filled], 0.25)
    assert set(np.unique(f[:, 19])) == {-1.0, 1.0}
    b2 = b.copy()
    b2[0] += 1.0
    g = mlp.features(b2, b, el.chi, el.xyz, el.box, nb, p0)
    assert g[0, 0] == 1.0 and np.all(g[0, 1:9] == 0.0)
    # nearest neighbours of atom 0 (1.42 A: shell k = 1) see it in their first shell
    d = el.xyz - el.xyz[0]
    d -= np.asarray(el.box) * np.round(d / np.asarray(el.box))
    r = np.sqrt((d * d).sum(axis=1))
    nn = np.nonzero((r > 0.5) & (r < 1.5))[0]
    assert len(nn) == 3
    for j in nn:
        shell = [k for k in nb[j] if k != j]
        dj = el.xyz[shell] - el.xyz[j]
        dj -= np.asarray(el.box) * np.round(dj / np.asarray(el.box))
        rj = np.sqrt((dj * dj).sum(axis=1))
        members = np.count_nonzero((rj >= 0.5) & (rj < 1.5))
        assert g[j, 1] == pytest.approx(1.0 / members)


def test_dc_feature_is_the_local_inverse_applied_to_the_change():
    # when every neighbourhood holds the whole system, column tau of M_tau^-1 is column
    # tau of the inverse of one global matrix M (Eq. 36 with all atoms), so feature 20,
    # (P Delta b) / k_e, solves M x = Delta b / k_e: check by multiplying back
    rng = np.random.default_rng(4)
    box = (30.0, 30.0, 30.0)
    xyz = rng.uniform(0, 4.0, (9, 3)) + 10.0
    alpha = np.full(9, 1.979)
    p, nb = pc.dc_preconditioner(xyz, alpha, box, 0.083, 14.0)
    assert all(len(x) == 9 for x in nb)
    m = pc.local_matrix(np.arange(9), xyz, alpha, box, 0.083, 14.0)
    b0 = rng.standard_normal(9)
    db = rng.standard_normal(9)
    f = mlp.features(b0 + db, b0, np.zeros(9), xyz, box, nb, p)
    assert np.allclose(m @ f[:, 20], db / ew.KE, rtol=0, atol=1e-12)


def test_splitmix64_published_outputs():
    # the first outputs of the SplitMix64 stream seeded with 0, as published with the
    # generator's reference code (top 53 bits of each as the uniform)
    first = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    u = mlp.splitmix64_uniform(0, [0, 1, 2])
    assert list(u) == [(v >> 11) * 2.0 ** -53 for v in first]


def test_counter_initialisation_layout_and_bounds():
    p = mlp.init_params_counter(20211106)
    assert p.dtype == np.float32 and p.shape == (mlp.N_PARAMS,)
    layers = mlp.unpack(p.astype(np.float64))
    for li, ((w, b), (o, i)) in enumerate(zip(layers, mlp.LAYERS)):
        lim = np.sqrt(6.0 / i) * (0.1 if li == 3 else 1.0)
        assert np.all(b == 0) and np.all(np.abs(w) <= lim)
        if w.size >= 2048:  # a uniform on [-lim, lim): mean ~0, variance lim^2 / 3
            assert abs(w.mean()) < 0.05 * lim
            assert abs(w.var() / (lim * lim / 3.0) - 1.0) < 0.1
    # the seed decides the draw
    assert not np.array_equal(p, mlp.init_params_counter(1))


def test_normalisation_small_case():
    feat = np.zeros((4, mlp.N_FEATURES), dtype=np.float32)
    feat[:, 0] = [1.0, 2.0, 3.0, 4.0]   # mean 2.5, population deviation sqrt(1.25)
    feat[:, 1] = 7.0                    # constant: inverse deviation 0
    norm, ts = mlp.normalisation(feat, [1.0, -1.0, 1.0, -1.0])
    assert norm[0] == 2.5 and norm[1] == 7.0
    assert norm[32] == pytest.approx(1.0 / np.sqrt(1.25)) and norm[33] == 0.0
    assert ts == 1.0
    _, ts0 = mlp.normalisation(feat, np.zeros(4))
    assert ts0 == 1.0


def test_adam_first_steps_closed_form():
    # From zero moments the bias corrections make the first step lr g / (|g| + eps), i.e.
    # lr sign(g) where |g| >> eps; a constant gradient keeps m_hat = g and v_hat = g^2 at
    # every later step, so each step moves by the same amount.
    g = np.array([3.0, -2e-3, 0.0, 1e-9])
    p0 = np.array([1.0, 1.0, 1.0, 1.0])
    p1, m, v = mlp.adam_step(p0, np.zeros(4), np.zeros(4), g, 1, 0.01)
    assert np.allclose(p1, p0 - 0.01 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    assert p1[0] == pytest.approx(0.99, abs=1e-10) and p1[1] == pytest.approx(1.01, abs=1e-7)
    assert p1[2] == 1.0
    p, mm, vv = p0, np.zeros(4), np.zeros(4)
    for step in range(1, 6):
        prev = p
        p, mm, vv = mlp.adam_step(p, mm, vv, g, step, 0.01)
        assert np.allclose(p - prev, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=1e-15)
