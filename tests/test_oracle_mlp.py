"""Pins of the FP64 learned-proposal oracle: central finite differences of the
loss, Adam's closed-form first step, exact encoding values, grid features on a
hand-placed occupied cell, the coverage rule."""
import math

import numpy as np
import pytest

from oracle import mlp


def _batch(seed, N=40):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((N, mlp.N_IN))
    ns = rng.integers(10, 200, N)
    jf = np.where(rng.uniform(size=N) < 0.2, -1, rng.integers(0, 5, N))
    jl = np.where(jf < 0, -1, np.minimum(ns - 1, jf + rng.integers(0, 150, N)))
    return X, jf, jl, ns


def test_gradients_match_central_differences():
    p = mlp.init_params(3)
    for k in p:
        if k.startswith("b"):
            p[k] = np.random.default_rng(len(k)).standard_normal(p[k].shape) * 0.1
    X, jf, jl, ns = _batch(1)
    loss, g = mlp.loss_and_grads(p, X, jf, jl, ns)
    rng = np.random.default_rng(7)
    h = 1e-6
    for name, _ in mlp.SHAPES:
        for _ in range(6):
            idx = tuple(rng.integers(0, s) for s in p[name].shape)
            q = {k: v.copy() for k, v in p.items()}
            q[name][idx] += h
            lp, _ = mlp.loss_and_grads(q, X, jf, jl, ns)
            q[name][idx] -= 2 * h
            lm, _ = mlp.loss_and_grads(q, X, jf, jl, ns)
            fd = (lp - lm) / (2 * h)
            assert abs(fd - g[name][idx]) <= 1e-6 * max(1e-3, abs(fd)) + 1e-9, (name, idx, fd, g[name][idx])


def test_adam_first_step_closed_form():
    """After one step from m = v = 0 the bias-corrected update is
    -lr * g / (|g| + eps) for every parameter."""
    p = {"w": np.array([1.0, -2.0, 3.0])}
    g = {"w": np.array([0.5, -4e-3, 7.0])}
    z = {"w": np.zeros(3)}
    p2, m, v = mlp.adam(p, g, z, z, 1, lr=0.01)
    np.testing.assert_allclose(p2["w"] - p["w"], -0.01 * g["w"] / (np.abs(g["w"]) + 1e-8), rtol=1e-12)
    np.testing.assert_allclose(m["w"], 0.1 * g["w"])
    np.testing.assert_allclose(v["w"], 0.001 * g["w"] ** 2)


def test_encoding_exact_values():
    e = np.array([[0.0, 0.5, 1.0]])
    d = np.array([[0.0, 0.0, -1.0]])
    enc = mlp.encode(e, d).reshape(6, mlp.N_FREQ, 2)
    np.testing.assert_allclose(enc[0, :, 0], 0.0, atol=0)          # sin(0)
    np.testing.assert_allclose(enc[0, :, 1], 1.0, atol=0)          # cos(0)
    assert enc[1, 0, 0] == pytest.approx(1.0) and enc[1, 0, 1] == pytest.approx(0.0, abs=1e-15)
    assert enc[1, 2, 0] == pytest.approx(0.0, abs=1e-15) and enc[1, 2, 1] == pytest.approx(-1.0)
    assert enc[5, 0, 1] == pytest.approx(-1.0)                      # cos(-pi)
    assert mlp.freqs()[4] == pytest.approx(4 * math.pi)


def test_grid_features_hit_the_occupied_cell():
    """A ray along +x through the centre of a 4x4x4 grid of 8-cell macro cells
    whose only occupied cell is (2, 1, 1): the features read it exactly for the
    samples between x = 16 and 24."""
    grid = np.zeros((4, 4, 4))
    grid[1, 1, 2] = 0.7                           # (z, y, x)
    e = np.array([[0.25, 12.0, 12.0]])
    d = np.array([[1.0, 0.0, 0.0]])
    f = mlp.grid_features(e, d, [64], 0.5, grid, 8)[0]     # segment length 32 -> x in (0.25, 32.25)
    xs = 0.25 + (np.arange(32) + 0.5) / 32 * 32.0
    np.testing.assert_array_equal(f, np.where((xs >= 16) & (xs < 24), 0.7, 0.0))


def test_coverage_rule():
    te, tx = np.array([0.1, 0.1, 0.5]), np.array([0.5, 0.5, 0.2])
    jf, jl, ns = np.array([12, 8, -1]), np.array([49, 49, -1]), np.array([100, 100, 100])
    # [10-2, 50+2) covers [12, 49] and [8, 49]; the empty ray is always covered
    np.testing.assert_array_equal(mlp.coverage(te, tx, jf, jl, ns, 2), [1.0, 1.0, 1.0])
    # [8, 52) misses the last sample 52
    np.testing.assert_array_equal(mlp.coverage(te[:1], tx[:1], [8], [52], [100], 2), [0.0])
    np.testing.assert_array_equal(mlp.coverage(te[:1], tx[:1], [7], [51], [100], 2), [0.0])
