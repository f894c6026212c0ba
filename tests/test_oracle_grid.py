"""Pins of the oracle's max-opacity grid: brute force in numpy (no oracle
code), a constant field, an empty transfer function."""
import numpy as np
import pytest

import oracle
from paper_1611_09048_b300 import synth
from scenes_util import const_lut, make_scene, ortho_down_z


def _np_alpha(luts, x, s):
    x = np.clip(np.nan_to_num(x, nan=0.0), 0, 1)
    return np.interp(255 * x, np.arange(256), luts[s][:, 3].astype(np.float64))


@pytest.mark.parametrize("cell", [4, 5, 16])
def test_grid_bruteforce(cell):
    rng = np.random.default_rng(cell)
    n = (13, 9, 11)
    g = 2
    vec = rng.uniform(-1, 1, (n[2] + 2 * g, n[1] + 2 * g, n[0] + 2 * g, 3)).astype(np.float32)
    sca = rng.uniform(0, 2, (n[2], n[1], n[0])).astype(np.float32)
    luts = [synth.lut_from_points(21, alpha_max=0.5), synth.lut_from_points(22, alpha_max=0.5)]
    sc = make_scene([vec[..., :]], [[("length",), ("mul", (0.5,))]], [luts[0]], [0.7], n,
                    ortho_down_z(n, 4, 4), 4, 4, guard=g)
    sc.sources.append(synth.source_from_zyx(sca, 0))
    sc.chains.append([("mul", (0.4,)), ("add", (0.1,))])
    sc.luts = np.stack(luts)
    sc.weights = np.array([0.7, 0.6], np.float32)
    grid = oracle.opacity_grid(sc, cell)
    w = [float(np.float32(0.7)), float(np.float32(0.6))]
    # per-cell blended alpha over [-1, n]^3 (vector source: its guards;
    # scalar source: clamped to the border)
    zz, yy, xx = [np.arange(-1, k + 1) for k in n[::-1]]
    V = vec[np.ix_(zz + g, yy + g, xx + g)].astype(np.float64)
    S = sca[np.ix_(np.clip(zz, 0, n[2] - 1), np.clip(yy, 0, n[1] - 1), np.clip(xx, 0, n[0] - 1))]
    a = w[0] * _np_alpha(luts, np.linalg.norm(V, axis=-1) * 0.5, 0) + \
        w[1] * _np_alpha(luts, S.astype(np.float64) * 0.4 + 0.1, 1)
    a = np.clip(a, 0, 1)
    G = [(k + cell - 1) // cell for k in n]
    want = np.zeros((G[2], G[1], G[0]))
    for k in range(G[2]):
        for j in range(G[1]):
            for i in range(G[0]):
                sl = (slice(k * cell, min((k + 1) * cell, n[2]) + 2),
                      slice(j * cell, min((j + 1) * cell, n[1]) + 2),
                      slice(i * cell, min((i + 1) * cell, n[0]) + 2))
                want[k, j, i] = a[sl].max()
    np.testing.assert_allclose(grid, want, rtol=0, atol=1e-12)


def test_grid_constant_and_empty():
    n = (20, 20, 20)
    field = np.full(n, 42.0, np.float32)
    sc = make_scene([field], [[("mul", (1.0 / 84.0,))]], [const_lut((1, 1, 1, 0.25))], [1.0], n,
                    ortho_down_z(n, 4, 4), 4, 4)
    np.testing.assert_allclose(oracle.opacity_grid(sc, 8), float(np.float32(0.25)), atol=1e-15)
    sc.luts = sc.luts.copy()
    sc.luts[..., 3] = 0.0
    assert np.all(oracle.opacity_grid(sc, 8) == 0.0)


@pytest.mark.parametrize("cell", [3, 8])
def test_range_grid_bruteforce(cell):
    """Per macro cell and component, min and max over the apron box of the
    cells as read (guards for the vector source, clamped border for the
    scalar), written out with numpy slicing -- no oracle code."""
    rng = np.random.default_rng(10 + cell)
    n = (11, 7, 9)
    g = 1
    vec = rng.normal(0, 1, (n[2] + 2 * g, n[1] + 2 * g, n[0] + 2 * g, 3)).astype(np.float32)
    sca = rng.uniform(-3, 3, (n[2], n[1], n[0])).astype(np.float32)
    sc = make_scene([vec], [[("length",)]], [const_lut((1, 1, 1, 0.1))], [1.0], n,
                    ortho_down_z(n, 4, 4), 4, 4, guard=g)
    sc.sources.append(synth.source_from_zyx(sca, 0))
    sc.chains.append([])
    sc.luts = np.stack([sc.luts[0], sc.luts[0]])
    sc.weights = np.array([1.0, 1.0], np.float32)
    got = oracle.range_grid(sc, cell)
    zz, yy, xx = [np.arange(-1, k + 1) for k in n[::-1]]
    V = vec[np.ix_(zz + g, yy + g, xx + g)]
    S = sca[np.ix_(np.clip(zz, 0, n[2] - 1), np.clip(yy, 0, n[1] - 1), np.clip(xx, 0, n[0] - 1))]
    comps = [V[..., 0], V[..., 1], V[..., 2], S]
    G = [(k + cell - 1) // cell for k in n]
    assert got.shape == (G[2], G[1], G[0], 4, 2)
    for k in range(G[2]):
        for j in range(G[1]):
            for i in range(G[0]):
                sl = (slice(k * cell, min((k + 1) * cell, n[2]) + 2),
                      slice(j * cell, min((j + 1) * cell, n[1]) + 2),
                      slice(i * cell, min((i + 1) * cell, n[0]) + 2))
                for c, f in enumerate(comps):
                    assert got[k, j, i, c, 0] == f[sl].min()
                    assert got[k, j, i, c, 1] == f[sl].max()


def test_range_grid_nan_and_mask():
    n = (8, 8, 8)
    f = np.zeros(n, np.float32)
    f[2, 3, 4] = np.nan
    sc = make_scene([f, np.ones(n, np.float32)], [[], []], [const_lut((1, 1, 1, 0.1))] * 2,
                    [1.0, 1.0], n, ortho_down_z(n, 4, 4), 4, 4)
    r = oracle.range_grid(sc, 4)
    assert r.shape == (2, 2, 2, 2, 2)
    assert np.isinf(r[0, 0, 1, 0]).all() and r[0, 0, 1, 0, 0] < 0 < r[0, 0, 1, 0, 1]
    assert (r[1, 1, 0, 0] == 0).all()          # far from the NaN: a plain range
    r1 = oracle.range_grid(sc, 4, mask=0b10)   # only the constant source
    assert r1.shape == (2, 2, 2, 1, 2) and (r1 == 1).all()
