"""FP64 reference of the learned ray-interval proposal -- TEST INFRASTRUCTURE ONLY.

Plain numpy, float64, no fusion.  The paper has no learned component; this
defines the proposal model that the build layers on the plain ray caster:

Input of one ray (224 values), from its first sample position e (local voxel
coordinates), unit direction d, sample count ns and the max-opacity grid:
  * positional encoding of the 6 scalars (e_x/n_x, e_y/n_y, e_z/n_z, d_x, d_y,
    d_z): for each scalar s and k = 0..15, sin(pi * 2^(k/2) * s) and
    cos(pi * 2^(k/2) * s), in that order (192 values);
  * 32 grid features: the grid value of the macro cell containing
    e + ((i + 1/2)/32 * ns * step) * d, i = 0..31 (cell index clamped).
Network: x -> relu(x W1 + b1) -> relu(. W2 + b2) -> relu(. W3 + b3) -> u = . W4 + b4
with widths 224 -> 64 -> 64 -> 64 -> 3.  te = sigmoid(u0) and tx = sigmoid(u1)
are the start and end of the visible part of the ray as fractions of its
samples, conf = sigmoid(u2).
Targets from the plain march: jf, jl = first and last sample index with
nonzero opacity among the composited samples; ye = jf / ns, yx = (jl + 1)/ns,
or (1, 0) for a ray without any.  Coverage c = 1 when the proposed sample
range [floor(te*ns) - m, ceil(tx*ns) + m) contains [jf, jl] (always 1 for an
empty ray); loss per ray = huber(te - ye) + huber(tx - yx) + lam * BCE(conf, c)
with huber(r) = r^2 / (2 delta) for |r| < delta else |r| - delta / 2; the
batch loss is the mean.  Optimiser: Adam (Kingma & Ba) with bias correction.
"""
from __future__ import annotations

import math

import numpy as np

N_FREQ = 16
N_GRID = 32
N_IN = 6 * 2 * N_FREQ + N_GRID   # 224
WIDTH = 64
N_OUT = 3
SHAPES = [("W1", (N_IN, WIDTH)), ("b1", (WIDTH,)), ("W2", (WIDTH, WIDTH)), ("b2", (WIDTH,)),
          ("W3", (WIDTH, WIDTH)), ("b3", (WIDTH,)), ("W4", (WIDTH, N_OUT)), ("b4", (N_OUT,))]


def freqs():
    return np.pi * 2.0 ** (np.arange(N_FREQ) / 2.0)


def init_params(seed: int = 0) -> dict:
    """He-uniform weights, zero biases (FP64)."""
    rng = np.random.default_rng(seed)
    p = {}
    for name, shape in SHAPES:
        if name.startswith("W"):
            lim = math.sqrt(6.0 / shape[0])
            p[name] = rng.uniform(-lim, lim, shape)
        else:
            p[name] = np.zeros(shape)
    return p


def encode(e_n, d) -> np.ndarray:
    """(N, 192) positional encoding of e/n (N,3) and d (N,3)."""
    s = np.concatenate([np.asarray(e_n, np.float64), np.asarray(d, np.float64)], axis=1)  # (N,6)
    ang = s[:, :, None] * freqs()[None, None, :]                                          # (N,6,16)
    enc = np.stack([np.sin(ang), np.cos(ang)], axis=-1)                                    # (N,6,16,2)
    return enc.reshape(len(s), -1)


def grid_features(e, d, ns, step, grid, cell) -> np.ndarray:
    """(N, 32) grid values along each ray's sampled segment (grid (Gz,Gy,Gx))."""
    e = np.asarray(e, np.float64)
    d = np.asarray(d, np.float64)
    L = np.asarray(ns, np.float64) * step
    frac = (np.arange(N_GRID) + 0.5) / N_GRID
    pos = e[:, None, :] + (frac[None, :, None] * L[:, None, None]) * d[:, None, :]       # (N,32,3)
    G = np.array(grid.shape[::-1])                                                         # (Gx,Gy,Gz)
    idx = np.clip(np.floor(pos / cell).astype(np.int64), 0, G - 1)
    return np.asarray(grid, np.float64)[idx[..., 2], idx[..., 1], idx[..., 0]]


def inputs(e, d, ns, n, step, grid, cell) -> np.ndarray:
    e = np.asarray(e, np.float64)
    e_n = e / np.asarray(n, np.float64)[None, :]
    return np.concatenate([encode(e_n, d), grid_features(e, d, ns, step, grid, cell)], axis=1)


def forward(p, X) -> dict:
    a1 = X @ p["W1"] + p["b1"]
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ p["W2"] + p["b2"]
    h2 = np.maximum(a2, 0.0)
    a3 = h2 @ p["W3"] + p["b3"]
    h3 = np.maximum(a3, 0.0)
    u = h3 @ p["W4"] + p["b4"]
    return {"a1": a1, "h1": h1, "a2": a2, "h2": h2, "a3": a3, "h3": h3, "u": u}


def sigmoid(x):
    return 1.0 / (1.0 + np.exp(-x))


def targets(jf, jl, ns):
    jf, jl, ns = (np.asarray(a, np.float64) for a in (jf, jl, ns))
    empty = jf < 0
    ye = np.where(empty, 1.0, jf / ns)
    yx = np.where(empty, 0.0, (jl + 1.0) / ns)
    return ye, yx, empty


def coverage(te, tx, jf, jl, ns, margin):
    ns = np.asarray(ns, np.float64)
    kb = np.floor(te * ns) - margin
    ke = np.ceil(tx * ns) + margin
    jf, jl = np.asarray(jf), np.asarray(jl)
    return np.where(jf < 0, 1.0, ((kb <= jf) & (ke >= jl + 1)).astype(np.float64))


def huber(r, delta):
    a = np.abs(r)
    return np.where(a < delta, 0.5 * r * r / delta, a - 0.5 * delta)


def dhuber(r, delta):
    return np.where(np.abs(r) < delta, r / delta, np.sign(r))


def loss_and_grads(p, X, jf, jl, ns, margin=2, delta=0.02, lam=0.1):
    """Mean loss over the batch and its gradient for every parameter."""
    f = forward(p, X)
    u = f["u"]
    te, tx, conf = sigmoid(u[:, 0]), sigmoid(u[:, 1]), sigmoid(u[:, 2])
    ye, yx, _ = targets(jf, jl, ns)
    c = coverage(te, tx, jf, jl, ns, margin)            # target, no gradient
    bce = -(c * np.log(conf) + (1 - c) * np.log1p(-conf))
    N = len(X)
    loss = float(np.mean(huber(te - ye, delta) + huber(tx - yx, delta) + lam * bce))
    du = np.zeros_like(u)
    du[:, 0] = dhuber(te - ye, delta) * te * (1 - te)
    du[:, 1] = dhuber(tx - yx, delta) * tx * (1 - tx)
    du[:, 2] = lam * (conf - c)
    du /= N
    g = {"W4": f["h3"].T @ du, "b4": du.sum(0)}
    d3 = (du @ p["W4"].T) * (f["a3"] > 0)
    g["W3"], g["b3"] = f["h2"].T @ d3, d3.sum(0)
    d2 = (d3 @ p["W3"].T) * (f["a2"] > 0)
    g["W2"], g["b2"] = f["h1"].T @ d2, d2.sum(0)
    d1 = (d2 @ p["W2"].T) * (f["a1"] > 0)
    g["W1"], g["b1"] = X.T @ d1, d1.sum(0)
    return loss, g


def adam(p, g, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (t counts from 1); returns new (p, m, v)."""
    p2, m2, v2 = {}, {}, {}
    for k in p:
        m2[k] = b1 * m[k] + (1 - b1) * g[k]
        v2[k] = b2 * v[k] + (1 - b2) * g[k] * g[k]
        mh = m2[k] / (1 - b1 ** t)
        vh = v2[k] / (1 - b2 ** t)
        p2[k] = p[k] - lr * mh / (np.sqrt(vh) + eps)
    return p2, m2, v2


def propose(p, X, ns, margin=2, threshold=0.9, widen=None):
    """Sample range [kb, ke) per ray where conf >= threshold, else [0, ns)."""
    return propose_rule(forward(p, X)["u"], ns, margin, threshold, widen)


def nonzero_samples(e, d, ns, step, grid, cell):
    """Per ray, the sample indices k in [0, ns) whose position e + k*step*d
    lies in a macro cell (floor(position / cell), clamped to the grid) with
    a nonzero grid value (grid shaped (Gz, Gy, Gx))."""
    G = np.array(grid.shape[::-1])
    out = []
    for r in range(len(ns)):
        k = np.arange(int(ns[r]), dtype=np.float64)
        pos = np.asarray(e[r], np.float64)[None, :] + (k * step)[:, None] * np.asarray(d[r], np.float64)[None, :]
        idx = np.clip(np.floor(pos / cell).astype(np.int64), 0, G - 1)
        out.append(np.flatnonzero(np.asarray(grid)[idx[:, 2], idx[:, 1], idx[:, 0]] > 0))
    return out


def propose_rule(u, ns, margin=2, threshold=0.9, widen=None):
    """The proposal's decision from the network outputs u (N, 3).

    widen = dict(e, d, step, grid, cell) of the same rays: a confident ray's
    range then becomes the hull of the network's range (if not empty) and
    every sample in a macro cell with a nonzero grid value (nonzero_samples),
    before it is clipped to the ray."""
    u = np.asarray(u, np.float64)
    te, tx, conf = sigmoid(u[:, 0]), sigmoid(u[:, 1]), sigmoid(u[:, 2])
    ns = np.asarray(ns, np.int64)
    kb = np.floor(te * ns).astype(np.int64) - margin
    ke = np.ceil(tx * ns).astype(np.int64) + margin
    use = conf >= threshold
    if widen is not None:
        keep = nonzero_samples(widen["e"], widen["d"], ns, widen["step"], widen["grid"], widen["cell"])
        for r in range(len(ns)):
            if not use[r] or len(keep[r]) == 0:
                continue
            lo, hi = int(keep[r][0]), int(keep[r][-1]) + 1
            if ke[r] > kb[r]:
                kb[r], ke[r] = min(kb[r], lo), max(ke[r], hi)
            else:
                kb[r], ke[r] = lo, hi
    kb = np.clip(kb, 0, ns)
    ke = np.clip(ke, kb, ns)
    return np.where(use, kb, 0), np.where(use, ke, ns), use
