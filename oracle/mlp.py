"""The learned initial guess in FP64 (test infrastructure only).

The paper is silent on a learned guess; this is the project's definition, written out
plainly so the CUDA kernels can be checked against it.

Network: 32 inputs -> 64 -> 64 -> 64 -> 1, SiLU activations (silu(z) = z sigmoid(z)) on
the three hidden layers, linear output.  Parameters are one flat vector laid out as
[W1 (64x32, row-major), b1 (64), W2 (64x64), b2, W3 (64x64), b3, W4 (64), b4 (1)].
Loss: mean squared error over the samples.

Features (per electrode atom i of frame t, from the neutral-form potentials b (V) of
this frame and the previous one, Delta b = b_t - b_{t-1}):
  0      Delta b_i
  1-8    mean of Delta b over the neighbours j != i with k - 1/2 <= r_ij < k + 1/2,
         k = 1..8 (minimum image, neighbours within the PCG-DC cutoff)
  9      b_i
  10-17  the same shell means of b
  18     chi_i
  19     +1 above the mean electrode height (z_i > mean z), -1 otherwise
  20     (P Delta b)_i / k_e with P the PCG-DC preconditioner of Eq. 36 (its pattern
         entries, no p_gap fill): the local inverses applied to the potential change, a
         local estimate of Delta q^b itself
  21-31  zero
The network predicts the change of the first-step charges, Delta q^b_i, in units of
`target_scale`; features are divided by `feature_scale` beforehand.
"""
from __future__ import annotations

import numpy as np

from oracle.ewald import KE

LAYERS = [(64, 32), (64, 64), (64, 64), (1, 64)]
N_FEATURES = 32
N_PARAMS = sum(o * i + o for o, i in LAYERS)  # 10,497


def unpack(params):
    out, k = [], 0
    for o, i in LAYERS:
        w = params[k:k + o * i].reshape(o, i)
        k += o * i
        b = params[k:k + o]
        k += o
        out.append((w, b))
    return out


def silu(z):
    return z / (1.0 + np.exp(-z))


def silu_grad(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def init_params(rng, scale=1.0):
    """He-style uniform initialisation (project choice)."""
    parts = []
    for o, i in LAYERS:
        lim = scale * np.sqrt(6.0 / i)
        parts.append(rng.uniform(-lim, lim, size=o * i))
        parts.append(np.zeros(o))
    return np.concatenate(parts)


def splitmix64_uniform(seed: int, k):
    """Output numbers k (from 0) of the SplitMix64 stream seeded with `seed` (Steele, Lea
    and Flood, 2014) as doubles uniform in [0, 1) from their top 53 bits."""
    m = (1 << 64) - 1
    k = np.asarray(k, dtype=object)
    out = np.empty(k.shape, dtype=np.float64)
    for idx, kk in np.ndenumerate(k):
        z = (seed + (int(kk) + 1) * 0x9E3779B97F4A7C15) & m
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & m
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & m
        z ^= z >> 31
        out[idx] = (z >> 11) * 2.0 ** -53
    return out


def init_params_counter(seed: int):
    """The library's initialisation (project choice), written out: layer by layer, the
    weights of a layer with i inputs uniform in [-sqrt(6/i), sqrt(6/i)), the output
    layer's times 0.1, biases zero; parameter k takes SplitMix64 output k.  Returned as
    float32, the type the library stores."""
    out, k = [], 0
    for li, (o, i) in enumerate(LAYERS):
        lim = np.sqrt(6.0 / i) * (0.1 if li == len(LAYERS) - 1 else 1.0)
        u = splitmix64_uniform(seed, np.arange(k, k + o * i))
        out.append((lim * (2.0 * u - 1.0)).astype(np.float32))
        k += o * i
        out.append(np.zeros(o, dtype=np.float32))
        k += o
    return np.concatenate(out)


def normalisation(feat, target):
    """Per-feature mean and inverse standard deviation (population; 0 for a constant
    feature) and the target's standard deviation (1 if 0), in FP64."""
    f = np.asarray(feat, dtype=np.float64).reshape(-1, N_FEATURES)
    mu = f.mean(axis=0)
    sd = np.sqrt(((f - mu) ** 2).mean(axis=0))
    inv = np.where(sd > 1e-12, 1.0 / np.where(sd > 1e-12, sd, 1.0), 0.0)
    t = np.asarray(target, dtype=np.float64)
    ts = float(np.sqrt(((t - t.mean()) ** 2).mean()))
    return np.concatenate([mu, inv]), (ts if ts > 0 else 1.0)


def forward(params, x):
    """x [S, 32] -> y [S]; also returns the pre-activations for backprop."""
    layers = unpack(np.asarray(params, dtype=np.float64))
    h = np.asarray(x, dtype=np.float64)
    zs = []
    for li, (w, b) in enumerate(layers):
        z = h @ w.T + b
        zs.append(z)
        h = silu(z) if li < len(layers) - 1 else z
    return h[:, 0], (np.asarray(x, dtype=np.float64), zs)


def loss_and_grad(params, x, target):
    """Mean squared error and its gradient by hand-written backpropagation."""
    params = np.asarray(params, dtype=np.float64)
    y, (x0, zs) = forward(params, x)
    s = x0.shape[0]
    diff = y - np.asarray(target, dtype=np.float64)
    loss = float(np.mean(diff * diff))
    layers = unpack(params)
    grads = []
    dz = (2.0 / s) * diff[:, None]  # dL/dz of the output layer
    for li in range(len(layers) - 1, -1, -1):
        w, _ = layers[li]
        h_in = x0 if li == 0 else silu(zs[li - 1])
        grads.append((dz.T @ h_in, dz.sum(axis=0)))
        if li > 0:
            dz = (dz @ w) * silu_grad(zs[li - 1])
    flat = []
    for gw, gb in reversed(grads):
        flat.append(gw.ravel())
        flat.append(gb)
    return loss, np.concatenate(flat)


def shell_means(values, xyz, box, nbrs):
    """Mean of `values` over neighbour shells k - 1/2 <= r < k + 1/2, k = 1..8."""
    xyz = np.asarray(xyz, dtype=np.float64)
    L = np.asarray(box, dtype=np.float64)
    out = np.zeros((xyz.shape[0], 8))
    for i, idx in enumerate(nbrs):
        d = xyz[idx] - xyz[i]
        d -= L * np.round(d / L)
        r = np.sqrt((d * d).sum(axis=1))
        for k in range(1, 9):
            sel = (idx != i) & (r >= k - 0.5) & (r < k + 0.5)
            if np.any(sel):
                out[i, k - 1] = values[idx[sel]].mean()
    return out


def features(b, b_prev, chi, xyz, box, nbrs, p_dc):
    """The 32 per-atom features of one frame (unscaled); p_dc is the dense PCG-DC
    preconditioner (zero outside its neighbour pattern)."""
    b = np.asarray(b, dtype=np.float64)
    db = b - np.asarray(b_prev, dtype=np.float64)
    n = b.shape[0]
    f = np.zeros((n, N_FEATURES))
    f[:, 0] = db
    f[:, 1:9] = shell_means(db, xyz, box, nbrs)
    f[:, 9] = b
    f[:, 10:18] = shell_means(b, xyz, box, nbrs)
    f[:, 18] = chi
    z = np.asarray(xyz)[:, 2]
    f[:, 19] = np.where(z > z.mean(), 1.0, -1.0)
    f[:, 20] = (np.asarray(p_dc, dtype=np.float64) @ db) / KE
    return f


def adam_step(params, m, v, grad, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (Kingma and Ba, Algorithm 1) in FP64: the moving moments of the
    gradient and its square, their bias corrections for step >= 1, and the update
    lr m_hat / (sqrt(v_hat) + eps).  Returns the new (params, m, v)."""
    g = np.asarray(grad, dtype=np.float64)
    m = beta1 * np.asarray(m, dtype=np.float64) + (1.0 - beta1) * g
    v = beta2 * np.asarray(v, dtype=np.float64) + (1.0 - beta2) * g * g
    m_hat = m / (1.0 - beta1 ** step)
    v_hat = v / (1.0 - beta2 ** step)
    return np.asarray(params, dtype=np.float64) - lr * m_hat / (np.sqrt(v_hat) + eps), m, v
