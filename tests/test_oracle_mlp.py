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


def test_targets_hand_computed():
    """Labels of three rays with 16 samples each: a span [3, 11], a span that
    ends on the last sample [0, 15], and a ray with no visible sample."""
    ye, yx, empty = mlp.targets([3, 0, -1], [11, 15, -1], [16, 16, 16])
    np.testing.assert_array_equal(ye, [3 / 16, 0.0, 1.0])
    np.testing.assert_array_equal(yx, [12 / 16, 1.0, 0.0])
    np.testing.assert_array_equal(empty, [False, False, True])


def test_targets_are_the_tightest_covering_window():
    """Used as a proposal with no margin, a ray's own targets cover its span,
    and moving either end one sample inwards does not (so the end target is
    (jl + 1)/ns, not jl/ns, and the start is jf/ns)."""
    rng = np.random.default_rng(5)
    ns = rng.choice([16, 32, 64, 128, 256], 200)
    jf = (rng.uniform(size=200) * (ns - 1)).astype(int)
    jl = jf + (rng.uniform(size=200) * (ns - jf)).astype(int)
    ye, yx, _ = mlp.targets(jf, jl, ns)
    np.testing.assert_array_equal(mlp.coverage(ye, yx, jf, jl, ns, 0), 1.0)
    np.testing.assert_array_equal(mlp.coverage(ye + 1.0 / ns, yx, jf, jl, ns, 0), 0.0)
    np.testing.assert_array_equal(mlp.coverage(ye, yx - 1.0 / ns, jf, jl, ns, 0), 0.0)


def _hand_params():
    """A network whose output is known in closed form: layer 1 passes x0,
    -x1 and 2*x2 - 1 through ReLU on units 0..2 and ignores every other
    input; layer 2 swaps units 0 and 1 and subtracts 0.25 from unit 0;
    layer 3 triples; the output is (h0 + 0.5, h1 - h2 - 1, 3)."""
    p = {name: np.zeros(shape) for name, shape in mlp.SHAPES}
    p["W1"][0, 0], p["W1"][1, 1], p["W1"][2, 2] = 1.0, -1.0, 2.0
    p["b1"][2] = -1.0
    p["W2"] = np.eye(mlp.WIDTH)
    p["W2"][[0, 1]] = p["W2"][[1, 0]]
    p["b2"][0] = -0.25
    p["W3"] = 3.0 * np.eye(mlp.WIDTH)
    p["W4"][0, 0], p["W4"][1, 1], p["W4"][2, 1] = 1.0, 1.0, -1.0
    p["b4"][:] = (0.5, -1.0, 3.0)
    return p


def test_forward_closed_form():
    X = np.random.default_rng(2).standard_normal((2, mlp.N_IN))   # other inputs must not matter
    X[0, :3] = (0.8, -0.6, 0.3)
    X[1, :3] = (-0.5, 0.4, 0.9)
    f = mlp.forward(_hand_params(), X)
    # row 0: h1 = (0.8, 0.6, 0) -> h2 = (0.35, 0.8, 0) -> h3 = (1.05, 2.4, 0)
    # row 1: h1 = (0, 0, 0.8)   -> h2 = (0, 0, 0.8)   -> h3 = (0, 0, 2.4)
    np.testing.assert_allclose(f["h1"][:, :3], [[0.8, 0.6, 0.0], [0.0, 0.0, 0.8]], atol=1e-15)
    np.testing.assert_allclose(f["h3"][:, :3], [[1.05, 2.4, 0.0], [0.0, 0.0, 2.4]], atol=1e-14)
    np.testing.assert_allclose(f["u"], [[1.55, 1.4, 3.0], [0.5, -3.4, 3.0]], atol=1e-14)
    assert np.all(f["h1"][:, 3:] == 0.0) and np.all(f["h3"][:, 3:] == 0.0)


def _const_params(b4):
    p = {name: np.zeros(shape) for name, shape in mlp.SHAPES}
    p["b4"][:] = b4
    return p


def test_propose_constant_network():
    """A constant network proposes te = sigmoid(b4[0]), tx = sigmoid(b4[1])
    with confidence sigmoid(b4[2]) for every ray."""
    X = np.zeros((3, mlp.N_IN))
    ns = np.array([100, 7, 1])
    # te = tx = 1/2, sure: [floor(ns/2) - 2, ceil(ns/2) + 2) clipped to [0, ns)
    kb, ke, use = mlp.propose(_const_params((0.0, 0.0, 5.0)), X, ns, margin=2)
    np.testing.assert_array_equal(kb, [48, 1, 0])
    np.testing.assert_array_equal(ke, [52, 6, 1])
    assert use.all()
    # unsure (conf 1/2 < 0.9): the whole ray
    kb, ke, use = mlp.propose(_const_params((0.0, 0.0, 0.0)), X, ns, margin=2)
    np.testing.assert_array_equal(kb, [0, 0, 0])
    np.testing.assert_array_equal(ke, ns)
    assert not use.any()
    # te > tx: an empty window at kb (te = 0.8808, tx = 0.1192; ns = 100 -> kb = 86)
    kb, ke, use = mlp.propose(_const_params((2.0, -2.0, 5.0)), X[:1], ns[:1], margin=2)
    assert (kb[0], ke[0], use[0]) == (86, 86, True)
    # the threshold is inclusive
    _, _, use = mlp.propose(_const_params((0.0, 0.0, 0.0)), X[:1], ns[:1], threshold=0.5)
    assert use[0]


def test_propose_agrees_with_coverage():
    """A confident proposal's window contains a span exactly when the coverage
    rule counts the ray as covered (the training target of the confidence)."""
    rng = np.random.default_rng(9)
    for trial in range(20):
        b4 = (rng.normal(0, 2), rng.normal(0, 2), 5.0)
        p = _const_params(b4)
        ns = rng.integers(1, 400, 64)
        jf = (rng.uniform(size=64) * ns).astype(int)
        jl = jf + (rng.uniform(size=64) * (ns - jf)).astype(int)
        kb, ke, use = mlp.propose(p, np.zeros((64, mlp.N_IN)), ns, margin=3)
        te, tx = mlp.sigmoid(b4[0]), mlp.sigmoid(b4[1])
        c = mlp.coverage(np.full(64, te), np.full(64, tx), jf, jl, ns, 3)
        assert use.all()
        np.testing.assert_array_equal((kb <= jf) & (ke >= jl + 1), c == 1.0)


def test_nonzero_samples_along_an_axis():
    """A ray along +x at y = z = 4 in a 4^3 grid of 8-cell macro cells whose
    cells x = 1 and x = 3 (of row y = z = 0) are nonzero: samples k with
    position 0.25 + k/2 in [8, 16) or [24, 32) are kept."""
    grid = np.zeros((4, 4, 4))
    grid[0, 0, 1] = 0.2
    grid[0, 0, 3] = 0.7
    keep = mlp.nonzero_samples([[0.25, 4.0, 4.0]], [[1.0, 0.0, 0.0]], [60], 0.5, grid, 8)[0]
    x = 0.25 + 0.5 * np.arange(60)
    np.testing.assert_array_equal(keep, np.flatnonzero(((x >= 8) & (x < 16)) | ((x >= 24) & (x < 32))))
    # a ray that stays in zero cells keeps nothing; positions beyond the grid clamp to its edge
    assert len(mlp.nonzero_samples([[0.25, 20.0, 4.0]], [[1.0, 0.0, 0.0]], [60], 0.5, grid, 8)[0]) == 0
    keep = mlp.nonzero_samples([[30.0, 4.0, 4.0]], [[1.0, 0.0, 0.0]], [10], 0.5, grid, 8)[0]
    np.testing.assert_array_equal(keep, np.arange(10))


def test_propose_widening_hand_computed():
    """The range becomes the hull of the network's (non-empty) range and the
    samples in nonzero macro cells; an empty network range becomes those
    samples' hull; unsure rays keep the whole ray."""
    grid = np.zeros((4, 4, 4))
    grid[0, 0, 1] = 0.2            # x in [8, 16): samples 16..31 of the rays below
    e = np.array([[0.25, 4.0, 4.0]] * 3)
    d = np.array([[1.0, 0.0, 0.0]] * 3)
    ns = np.array([60, 60, 60])
    w = dict(e=e, d=d, step=0.5, grid=grid, cell=8)
    X = np.zeros((3, mlp.N_IN))
    kb, ke, use = mlp.propose(_const_params((0.0, 0.0, 5.0)), X, ns, margin=2, widen=w)
    assert (kb[0], ke[0]) == (16, 32)                  # the network's [28, 32) widened
    kb, ke, _ = mlp.propose(_const_params((-2.0, -1.0, 5.0)), X, ns, margin=0, widen=w)
    assert (kb[0], ke[0]) == (7, 32)                   # network [7, 17) + [16, 32)
    kb, ke, _ = mlp.propose(_const_params((2.0, -2.0, 5.0)), X, ns, margin=2, widen=w)
    assert (kb[0], ke[0]) == (16, 32)                  # empty network range
    kb, ke, _ = mlp.propose(_const_params((0.0, 0.0, 0.0)), X, ns, margin=2, widen=w)
    assert (kb[0], ke[0]) == (0, 60)                   # unsure
    kb, ke, _ = mlp.propose(_const_params((0.0, 0.0, 5.0)), X, ns, margin=2)
    assert (kb[0], ke[0]) == (28, 32)                  # no widening


def test_propose_widening_keeps_every_nonzero_sample():
    rng = np.random.default_rng(4)
    grid = (rng.uniform(size=(4, 4, 4)) < 0.15) * 0.5
    for _ in range(5):
        N = 40
        e = rng.uniform(0, 32, (N, 3))
        d = rng.normal(size=(N, 3))
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        ns = rng.integers(1, 120, N)
        w = dict(e=e, d=d, step=0.5, grid=grid, cell=8)
        b4 = (rng.normal(0, 2), rng.normal(0, 2), 5.0)
        kb0, ke0, _ = mlp.propose(_const_params(b4), np.zeros((N, mlp.N_IN)), ns, margin=1)
        kb, ke, use = mlp.propose(_const_params(b4), np.zeros((N, mlp.N_IN)), ns, margin=1, widen=w)
        keep = mlp.nonzero_samples(e, d, ns, 0.5, grid, 8)
        assert use.all()
        for r in range(N):
            assert np.all((keep[r] >= kb[r]) & (keep[r] < ke[r]))
            if ke0[r] > kb0[r]:
                assert kb[r] <= kb0[r] and ke0[r] <= ke[r]


def test_huber_closed_form():
    """huber(r) = r^2 / (2 delta) inside |r| < delta, |r| - delta/2 outside:
    continuous with its slope at |r| = delta."""
    d = 0.02
    r = np.array([0.0, 0.01, -0.01, 0.05, -0.3125, 0.02])
    np.testing.assert_allclose(mlp.huber(r, d), [0.0, 0.0025, 0.0025, 0.04, 0.3025, 0.01], rtol=1e-12)
    np.testing.assert_allclose(mlp.dhuber(r, d), [0.0, 0.5, -0.5, 1.0, -1.0, 1.0], rtol=1e-12)


def test_loss_closed_form():
    """A constant network (te = tx = conf = 1/2) on two rays of 16 samples:
    the span [3, 11] gives huber(1/2 - 3/16) + huber(1/2 - 12/16) and, as the
    range [8 - 2, 8 + 2) does not cover it, BCE(1/2, 0) = ln 2; the empty ray
    gives huber(1/2 - 1) + huber(1/2 - 0) and BCE(1/2, 1) = ln 2.  The batch
    loss is the mean with the confidence term weighted 0.1."""
    p = _const_params((0.0, 0.0, 0.0))
    loss, g = mlp.loss_and_grads(p, np.zeros((2, mlp.N_IN)), [3, -1], [11, -1], [16, 16], margin=2)
    ray0 = (0.3125 - 0.01) + (0.25 - 0.01) + 0.1 * math.log(2.0)
    ray1 = (0.5 - 0.01) + (0.5 - 0.01) + 0.1 * math.log(2.0)
    assert loss == pytest.approx((ray0 + ray1) / 2, rel=1e-12)
    # output-bias gradient of the first ray alone: dhuber(te - ye) sigma'(0) =
    # +1/4, dhuber(tx - yx) sigma'(0) = -1/4, 0.1 (conf - c) = 0.05
    _, g = mlp.loss_and_grads(p, np.zeros((1, mlp.N_IN)), [3], [11], [16], margin=2)
    np.testing.assert_allclose(g["b4"], [0.25, -0.25, 0.05], atol=1e-15)
    assert np.all(g["W1"] == 0.0)        # zero inputs and zero hidden units
