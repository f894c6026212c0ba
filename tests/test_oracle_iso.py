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


def _iso_split(n, g, declared_guard, iso, seed=5):
    """Whole-volume iso frame and the two halves along x (each reading its
    neighbour's cells through guards; `declared_guard` is the guard width the
    halves declare), composited: the nearest hit of the halves wins."""
    from paper_1611_09048_b300 import synth
    fields = synth.pic_fields(n, g, seed=seed)
    whole = synth.scene_pic(n=n, guard=g, width=48, height=40, seed=seed, fields=fields,
                            dist_factor=1.0)
    whole.bg = (0.0, 0.0, 0.0, 0.0)
    ref = oracle.render_iso(whole, iso)
    parts = []
    for lo in (0, n // 2):
        part = synth.scene_pic(n=n, guard=g, width=48, height=40, seed=seed, fields=fields,
                               dist_factor=1.0)
        part.bg = (0.0, 0.0, 0.0, 0.0)
        part.global_n = (n, n, n)
        part.off = (lo, 0, 0)
        part.n = (n // 2, n, n)
        for s in part.sources:
            s.offset = s.offset + lo * s.strides[0]
            s.guard = declared_guard
        parts.append(oracle.render_iso(part, iso))
    t = np.stack([np.where(r["margin"][..., 5] >= 0, r["margin"][..., 5], np.inf) for r in parts])
    first = np.argmin(t, axis=0)
    pick = lambda key: np.where((first == 0)[..., None], parts[0][key], parts[1][key])  # noqa: E731
    return ref, pick("rgba"), pick("margin"), np.isfinite(t).any(axis=0)


def test_domain_split_iso_equals_whole_with_two_guard_layers():
    """Sec. 3.1/3.2: with two guard layers a sub-volume interpolates every
    gradient position of its hits from its own cells, so the halves of a split
    volume, composited by nearest hit, reproduce the whole volume's iso frame
    -- except where a half's hit is its first sample, which has no previous
    sample in the half for the secant step (the whole refines it)."""
    iso = [0.6, 0.55, 0.5]
    ref, rgba, m, hit = _iso_split(20, 2, 2, iso)
    whole_hit = ref["margin"][..., 5] >= 0
    np.testing.assert_array_equal(hit, whole_hit)
    tie = ref["margin"][..., 2] < 1e-9
    no_secant = (m[..., 3] >= oracle.INF) & (ref["margin"][..., 3] < oracle.INF)
    keep = whole_hit & ~tie & ~no_secant
    assert keep.sum() > 300 and no_secant.sum() < 0.1 * whole_hit.sum()
    np.testing.assert_allclose(rgba[keep], ref["rgba"][keep], rtol=0, atol=1e-9)
    np.testing.assert_allclose(m[keep, 5], ref["margin"][keep, 5], rtol=0, atol=1e-9)


def test_domain_split_iso_with_one_guard_layer_clamps_at_the_face():
    """The same split with one declared guard layer: gradient positions are
    clamped to half a voxel beyond the face, so hits within a voxel of the
    split face shade differently from the whole volume (the data the halves
    could read is the same; only the declared guard width differs)."""
    iso = [0.6, 0.55, 0.5]
    ref, rgba, m, hit = _iso_split(20, 2, 1, iso)
    whole_hit = ref["margin"][..., 5] >= 0
    keep = whole_hit & (ref["margin"][..., 2] >= 1e-9) & (m[..., 3] < oracle.INF)
    diff = np.abs(rgba - ref["rgba"]).max(-1)
    assert (diff[keep] > 1e-6).sum() > 0
    np.testing.assert_allclose(m[keep, 5], ref["margin"][keep, 5], rtol=0, atol=1e-9)
