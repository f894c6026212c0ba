"""Pins of the oracle's iso-surface frame: closed forms for linear fields
(trilinear interpolation, the secant refinement and central differences are
all exact on them), the first-sample rule, the nearer of two sources, no
crossing."""
import numpy as np

import oracle
from scenes_util import make_scene, ortho_down_z


def _lut(rgb):
    lut = np.zeros((256, 4), np.float32)
    lut[:, :3] = np.asarray(rgb, np.float32)
    lut[:, 3] = 0.5
    return lut


def _linear(n, a, c, b, guard=2):
    """v = a*x + c*z + b at cell centres (i + 1/2), guards included."""
    S = [k + 2 * guard for k in n]
    z, y, x = np.meshgrid(*(np.arange(s) - guard + 0.5 for s in S[::-1]), indexing="ij")
    return (a * x + c * z + b).astype(np.float32)


def test_tilted_plane_closed_form():
    n = (16, 8, 32)
    a, c, b = 0.0625, -0.125, 4.0          # dyadic: every value exact in float32
    W, H = 16, 8
    sc = make_scene([_linear(n, a, c, b)], [[]], [_lut((0.5, 0.25, 0.75))], [1.0], n,
                    ortho_down_z(n, W, H), W, H, guard=2)
    iso = 2.5
    r = oracle.render_iso(sc, [iso])
    m = r["margin"]
    # pixel (px, py) travels at x = (px + 1/2) * nx / W down from z = nz, entering at t = 1/2
    ndl = abs(c) / np.hypot(a, c)
    rgb = np.clip(np.array([0.5, 0.25, 0.75]) * (0.25 + 0.75 * ndl) + 0.25 * ndl ** 32, 0, 1)
    for px in range(W):
        x = (px + 0.5) * n[0] / W
        z_star = (iso - a * x - b) / c
        assert 2.0 < z_star < n[2] - 2.0
        for py in range(H):
            assert abs(m[py, px, 5] - (0.5 + n[2] - z_star)) < 1e-9
            np.testing.assert_allclose(r["rgba"][py, px, :3], rgb, atol=1e-12)
            assert r["rgba"][py, px, 3] == 1.0
            assert abs(m[py, px, 4] - np.hypot(a, c)) < 1e-12


def test_first_sample_hit_and_no_hit():
    n = (8, 8, 16)
    W, H = 4, 4
    sc = make_scene([_linear(n, 0.0, -0.25, 10.0)], [[]], [_lut((1.0, 0.0, 0.0))], [1.0], n,
                    ortho_down_z(n, W, H), W, H, guard=2)
    sc.bg = (0.125, 0.25, 0.5, 0.75)
    # v = 10 - z/4 >= 6 everywhere: the ray starts inside, the hit is its first sample
    r = oracle.render_iso(sc, [5.0])
    assert np.all(r["margin"][..., 5] == 0.5)
    assert np.all(r["margin"][..., 3] >= oracle.INF)      # no refinement at the first sample
    # v <= 10 everywhere: no crossing, the background shows
    r = oracle.render_iso(sc, [11.0])
    assert np.all(r["margin"][..., 5] == -1.0)
    np.testing.assert_array_equal(r["rgba"], np.broadcast_to(sc.bg, r["rgba"].shape))


def test_nearer_source_wins():
    n = (8, 8, 32)
    W, H = 4, 4
    f0 = _linear(n, 0.0, -0.25, 8.0)      # crosses 4 at z = 16
    f1 = _linear(n, 0.0, -0.5, 16.0)      # crosses 5 at z = 22: nearer to the viewer
    sc = make_scene([f0, f1], [[], []], [_lut((1.0, 0.0, 0.0)), _lut((0.0, 1.0, 0.0))],
                    [1.0, 1.0], n, ortho_down_z(n, W, H), W, H, guard=2)
    r = oracle.render_iso(sc, [4.0, 5.0])
    assert np.allclose(r["margin"][..., 5], 0.5 + 32 - 22)
    assert np.all(r["rgba"][..., 1] == 1.0) and np.all(r["rgba"][..., 0] == 0.25)
    # equal crossings: the lower source index wins
    r = oracle.render_iso(sc, [4.0, 8.0])
    assert np.allclose(r["margin"][..., 5], 0.5 + 32 - 16)
    assert np.all(r["rgba"][..., 0] == 1.0) and np.all(r["rgba"][..., 1] == 0.25)
    # a deactivated source is ignored
    r = oracle.render_iso(sc, [4.0, 5.0], mask=0b01)
    assert np.allclose(r["margin"][..., 5], 0.5 + 32 - 16)
