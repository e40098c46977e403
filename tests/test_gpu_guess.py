"""Learned initial guess on the GPU against the FP64 oracle (features, forward pass,
gradient), and what the trained network gains over the previous-step guess.

Tolerances: features are float sums of float-rounded potentials (1e-6 of each column's
scale); the forward pass and gradient accumulate in FP32 over 32-64-term dot products and
over the samples, so FP32-weight results match the FP64 oracle to 1e-5 (relative); with BF16
weights the oracle is evaluated at the same BF16-rounded weights and the gap to the FP32
oracle is held to 1e-3, as the BF16 rounding of the weights (2^-9) allows.
"""
import numpy as np
import pytest

from oracle import mlp
from oracle import precond as pc
from paper_2111_06704_gb300 import cpm
from paper_2111_06704_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2111_06704_gb300.guess import LearnedGuess  # noqa: E402


def _dev(a, dtype=torch.float64):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


@pytest.fixture(scope="module")
def walk():
    """The 512-atom electrode, 161 random-walk frames of the 200-ion set, with b and the
    first-step charges q^b of every frame (solved to 1e-10)."""
    work = wl.walk_frames(161, step=0.1, seed=123)
    el, io = work.electrode, work.electrolyte
    ctx = cpm.Context(el.box)
    ctx.cpm_build_E(el.xyz, el.alpha)
    F, n = io.frames, el.n
    b = torch.empty((F, n), dtype=torch.float64, device="cuda")
    qs = torch.empty(F, dtype=torch.float64, device="cuda")
    ctx.cpm_potential(_dev(io.xyz), _dev(io.q), _dev(el.chi), b, qs)
    qb = torch.zeros((F, n), dtype=torch.float64, device="cuda")
    ctx.cpm_solve(b, qb, tol=1e-10, maxit=2000)
    yield ctx, work, b, qb
    ctx.close()


def test_features_match_the_oracle(walk):
    ctx, work, b, _ = walk
    el = work.electrode
    g = LearnedGuess(ctx)
    chi = _dev(el.chi)
    feat = g.features(b[1:4], b[0:3], chi).cpu().numpy()
    p_dc, nb = pc.dc_preconditioner(el.xyz, el.alpha, el.box, wl.G_DC, wl.RCUT_DC)
    bh = b.cpu().numpy()
    for k in range(3):
        ref = mlp.features(bh[k + 1], bh[k], el.chi, el.xyz, el.box, nb, p_dc)
        scale = np.maximum(np.abs(ref).max(axis=0), 1e-30)
        assert np.all(np.abs(feat[k] - ref) <= 1e-6 * scale + 1e-12)


@pytest.mark.parametrize("bf16", [False, True])
def test_forward_and_gradient_match_the_oracle(walk, bf16):
    ctx = walk[0]
    rng = np.random.default_rng(9)
    g = LearnedGuess(ctx, seed=4, bf16=bf16)
    p = mlp.init_params(rng, scale=0.8).astype(np.float32)
    p += (0.05 * rng.standard_normal(p.shape)).astype(np.float32)
    g.params = _dev(p, torch.float32)
    s = 777  # several blocks and a ragged last one
    x = rng.standard_normal((s, mlp.N_FEATURES)).astype(np.float32)
    t = rng.standard_normal(s).astype(np.float32)
    y_gpu = g.forward(_dev(x, torch.float32)).cpu().numpy()
    loss_gpu = g.gradient(_dev(x, torch.float32), _dev(t, torch.float32))
    grad_gpu = g.grad.cpu().numpy()
    p_used = p.astype(np.float64)
    if bf16:
        p_used = torch.tensor(p).bfloat16().float().numpy().astype(np.float64)
    y_ref, _ = mlp.forward(p_used, x.astype(np.float64))
    loss_ref, grad_ref = mlp.loss_and_grad(p_used, x.astype(np.float64), t.astype(np.float64))
    assert np.abs(y_gpu - y_ref).max() <= 1e-5 * np.abs(y_ref).max()
    assert loss_gpu == pytest.approx(loss_ref, rel=1e-5)
    assert np.linalg.norm(grad_gpu - grad_ref) <= 1e-5 * np.linalg.norm(grad_ref)
    if bf16:  # BF16 weights stay within the rounding allowance of the FP32 network
        _, grad_fp32 = mlp.loss_and_grad(p.astype(np.float64), x.astype(np.float64),
                                         t.astype(np.float64))
        assert np.linalg.norm(grad_gpu - grad_fp32) <= 1e-1 * np.linalg.norm(grad_fp32)
        y32, _ = mlp.forward(p.astype(np.float64), x.astype(np.float64))
        assert np.abs(y_gpu - y32).max() <= 1e-3 * np.abs(y32).max() * 20


def test_one_call_training_step_against_the_oracle(walk):
    # cpm_guess_train_step: the gradient of the batch's mean squared error, then one Adam
    # step, against the oracle's backpropagation and Adam step in FP64.  Where a gradient
    # component stands clear of zero the first step is lr sign(g) (closed form of the
    # oracle pin), so the parameters must agree to the gradient's float error; elsewhere
    # each move is at most lr.
    ctx = walk[0]
    rng = np.random.default_rng(11)
    g = LearnedGuess(ctx, seed=5, bf16=False)  # FP32 weights: the oracle's network
    p = mlp.init_params(rng, scale=0.8).astype(np.float32)
    g.params = _dev(p, torch.float32)
    s, lr = 1000, 1e-3
    x = rng.standard_normal((s, mlp.N_FEATURES)).astype(np.float32)
    t = rng.standard_normal(s).astype(np.float32)
    loss = g.train_step(_dev(x, torch.float32), _dev(t, torch.float32), lr)
    p1 = g.params.cpu().numpy().astype(np.float64)
    loss_ref, grad_ref = mlp.loss_and_grad(p.astype(np.float64), x.astype(np.float64),
                                           t.astype(np.float64))
    p_ref, _, _ = mlp.adam_step(p, np.zeros_like(grad_ref), np.zeros_like(grad_ref),
                                grad_ref, 1, lr)
    assert loss == pytest.approx(loss_ref, rel=1e-5)
    # the gradient is good to ~1e-5 of its norm (the gradient test), so a component a
    # hundredth of the largest keeps its sign
    clear = np.abs(grad_ref) > 1e-2 * np.abs(grad_ref).max()
    assert clear.sum() > 100
    assert np.abs(p1 - p_ref)[clear].max() <= 1e-6 + 1e-6 * lr
    assert np.all(np.abs(p1 - p) <= lr * (1 + 1e-5) + 1e-7)
    assert g.step == 1


def test_trained_guess_beats_the_previous_step(walk):
    ctx, work, b, qb = walk
    el = work.electrode
    chi = _dev(el.chi)
    g = LearnedGuess(ctx, seed=1)
    train = slice(1, 121)
    feat = g.features(b[train], b[0:120], chi).reshape(-1, mlp.N_FEATURES).contiguous()
    target = (qb[train] - qb[0:120]).reshape(-1).to(torch.float32).contiguous()
    g.set_normalisation(feat, target)
    losses = g.train(feat, target, epochs=40, batch=8192, lr=3e-3)
    assert losses[-1] < 0.5 * losses[0]
    # held-out frames 121..160: PCG iterations to 1e-6 from both guesses
    test = slice(121, 161)
    prev = qb[120:160].contiguous()
    ft = g.features(b[test], b[120:160], chi)
    q0 = g.guess(ft, prev).reshape(prev.shape).contiguous()
    _, it_prev, _ = ctx.cpm_solve(b[test].contiguous(), prev.clone(), use_guess=True, tol=1e-6)
    _, it_mlp, _ = ctx.cpm_solve(b[test].contiguous(), q0.clone(), use_guess=True, tol=1e-6)
    assert it_mlp.mean() < it_prev.mean()


def test_one_call_guess_equals_the_three_calls(walk):
    ctx, work, b, qb = walk
    chi = _dev(work.electrode.chi)
    g = LearnedGuess(ctx, seed=5)
    feat = g.features(b[1:9], b[0:8], chi)
    g.set_normalisation(feat.reshape(-1, mlp.N_FEATURES),
                        (qb[1:9] - qb[0:8]).reshape(-1).to(torch.float32))
    prev = qb[0:8].contiguous()
    three = g.guess(feat, prev).reshape(prev.shape)
    one = g.guess_frames(b[1:9].contiguous(), b[0:8].contiguous(), chi, prev)
    assert torch.equal(one, three)


def test_library_initialisation_and_normalisation_match_the_oracle(walk, tmp_path):
    ctx, work, b, qb = walk
    chi = _dev(work.electrode.chi)
    g = LearnedGuess(ctx, seed=20211106)
    # the counter-based initialisation, bit for bit
    assert np.array_equal(g.params.cpu().numpy(), mlp.init_params_counter(20211106))
    feat = g.features(b[1:9], b[0:8], chi).reshape(-1, mlp.N_FEATURES).contiguous()
    target = (qb[1:9] - qb[0:8]).reshape(-1).to(torch.float32).contiguous()
    g.set_normalisation(feat, target)
    norm_ref, ts_ref = mlp.normalisation(feat.cpu().numpy(), target.cpu().numpy())
    np.testing.assert_allclose(g.norm.cpu().numpy(), norm_ref, rtol=1e-6, atol=1e-30)
    assert g.target_scale == pytest.approx(ts_ref, rel=1e-6)
    # a trained network survives the file format (device arrays in and out)
    g.train(feat, target, epochs=2, batch=4096, lr=1e-3)
    path = str(tmp_path / "net.cpmguess")
    g.save(path)
    h = LearnedGuess(ctx, seed=1)
    h.load(path)
    assert torch.equal(h.params, g.params) and torch.equal(h.norm, g.norm)
    assert h.target_scale == g.target_scale
    prev = qb[0:8].contiguous()
    assert torch.equal(h.guess_frames(b[1:9].contiguous(), b[0:8].contiguous(), chi, prev),
                       g.guess_frames(b[1:9].contiguous(), b[0:8].contiguous(), chi, prev))
