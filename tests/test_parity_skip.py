"""Classical empty-space skipping (isaac_range_grid + isaac_render_skip).

* the value-range grid equals the oracle's (pinned by brute force) exactly;
* a frame with skipping equals the plain frame bit for bit (RGBA8 and the
  unquantised RGBA), whatever the chains, weights, guards, interpolation and
  lanes per ray, and evaluates fewer samples where the LUT leaves space empty;
* the skipped frame agrees with the FP64 oracle like the plain one.
"""
import numpy as np
import pytest

import oracle
from paper_1611_09048_b300 import isaac, synth
from parity_util import assert_parity, compare
from scenes_util import small_pic_scene

pytestmark = pytest.mark.gpu


def _pic_with_gaps(seed=4, layout="aos"):
    """E, B, rho with transfer functions that are transparent over part of
    their range, and a negative weight on one source."""
    sc = small_pic_scene(n=24, guard=2, width=64, height=48, seed=seed, layout=layout,
                         dist_factor=1.2)
    luts = sc.luts.copy()
    luts[0, :140, 3] = 0.0
    luts[1, 60:, 3] = 0.0
    luts[2, :, 3] = np.where(np.arange(256) < 200, 0.0, luts[2, :, 3])
    sc.luts = luts
    sc.weights = np.array([0.5, -0.2, 0.4], np.float32)
    sc.chains = [[("length",), ("mul", (0.7,)), ("pow", (0.5,))],
                 [("length",), ("log",), ("mul", (0.2,)), ("add", (0.8,))],
                 [("log",), ("mul", (1.0 / 6,)), ("add", (0.5,))]]
    return sc


def _scenes():
    bub = synth.scene_bubble(64, frame=10, seed=1, width=96, height=72, dist_factor=1.0)
    near = synth.scene_bubble(64, frame=30, seed=2, width=80, height=64, dist_factor=1.2)
    near.interp = 0
    return {"bubble": bub, "bubble_nearest": near, "pic": _pic_with_gaps(),
            "pic_soa": _pic_with_gaps(seed=5, layout="soa")}


@pytest.mark.parametrize("name", ["bubble", "pic", "pic_soa"])
@pytest.mark.parametrize("cell", [4, 7, 8, 16])
def test_range_grid_matches_oracle(cuda_ok, name, cell):
    import torch
    sc = _scenes()[name]
    got = isaac.DeviceScene(sc).range_grid(cell)
    torch.cuda.synchronize()
    want = oracle.range_grid(sc, cell)
    assert got.shape == want.shape
    np.testing.assert_array_equal(got.cpu().numpy(), want)


@pytest.mark.parametrize("name", ["bubble", "bubble_nearest", "pic", "pic_soa"])
@pytest.mark.parametrize("cell", [4, 8])
@pytest.mark.parametrize("lanes", [None, 1])
def test_skip_equals_plain(cuda_ok, name, cell, lanes):
    import torch
    sc = _scenes()[name]
    ds = isaac.DeviceScene(sc)
    ranges = ds.range_grid(cell)
    plain = ds.render(want_f32=True, want_nsamp=True, lanes=lanes)
    skip = ds.render_skip(ranges, cell, want_f32=True, want_nsamp=True, lanes=lanes)
    torch.cuda.synchronize()
    assert torch.equal(plain[0], skip[0])
    assert torch.equal(plain[1], skip[1])
    n_plain = int(plain[2].sum())
    n_skip = int(skip[2].sum())
    assert n_skip <= n_plain
    if name.startswith("bubble"):
        assert n_skip < 0.5 * n_plain, (n_skip, n_plain)   # the bubble is mostly empty space


def test_skip_matches_oracle(cuda_ok):
    import torch
    sc = _scenes()["pic"]
    ds = isaac.DeviceScene(sc)
    ranges = ds.range_grid(6)
    out, f32, ns = ds.render_skip(ranges, 6, want_f32=True, want_nsamp=True)
    plain_ns = ds.render(want_nsamp=True)[2]
    torch.cuda.synchronize()
    ref = oracle.render(sc)
    # the sample counts differ by design (skipped samples are not evaluated),
    # so the oracle's counts stand in for them
    rep = compare(f32.cpu().numpy(), out.cpu().numpy(), plain_ns.cpu().numpy(), ref)
    assert_parity(rep, what="skip vs oracle")


def test_skip_rejects_short_ranges(cuda_ok):
    import torch
    sc = _scenes()["pic"]
    ds = isaac.DeviceScene(sc)
    ranges = ds.range_grid(8)
    with pytest.raises(isaac.IsaacError) as e:
        ds.render_skip(ranges[:1], 8)
    assert e.value.code == isaac.EINVAL
    with pytest.raises(isaac.IsaacError):
        ds.render_skip(ranges, 4)   # ranges of another cell size are too short


@pytest.mark.parametrize("guard", [0, 2])
@pytest.mark.parametrize("cell", [5, 8, 16])
def test_range_grid_ragged_with_nan(cuda_ok, guard, cell):
    """A 35 x 22 x 41 scalar volume with a z ramp, NaNs sprinkled in (interior,
    guard layer and borders), with and without guards: bit-exact against the
    oracle for the specialised 8/16-cell walks and the general one."""
    import torch
    from scenes_util import make_scene
    n = (35, 22, 41)
    rng = np.random.default_rng(60 + guard + cell)
    S = (n[2] + 2 * guard, n[1] + 2 * guard, n[0] + 2 * guard)
    ramp = (np.arange(S[0], dtype=np.float32) / S[0])[:, None, None]
    f = (ramp - 0.3 + 0.05 * rng.standard_normal(S)).astype(np.float32)
    idx = rng.integers(0, f.size, 10)
    f.reshape(-1)[idx] = np.nan
    f[0, 0, 0] = np.nan
    f[-1, -1, -1] = np.nan
    cams = synth.random_orbit_camera(n, 16, 16, seed=5)
    sc = make_scene([f], [[]], [synth.lut_from_points(70)], [1.0], n, cams, 16, 16, guard=guard)
    got = isaac.DeviceScene(sc).range_grid(cell)
    torch.cuda.synchronize()
    want = oracle.range_grid(sc, cell)
    assert got.shape == want.shape
    assert np.isinf(want).any()                       # some cell reads a NaN
    np.testing.assert_array_equal(got.cpu().numpy(), want)


def test_range_grid_wide_vector_volume(cuda_ok):
    """A very wide, thin 3-component volume (4000 x 3 x 3) with guards and a
    NaN: bit-exact against the oracle."""
    import torch
    from scenes_util import make_scene
    n = (4000, 3, 3)
    g = 1
    rng = np.random.default_rng(78)
    f = rng.standard_normal((n[2] + 2 * g, n[1] + 2 * g, n[0] + 2 * g, 3)).astype(np.float32)
    f[1, 1, 1500, 2] = np.nan
    cams = synth.random_orbit_camera(n, 16, 16, seed=7)
    sc = make_scene([f], [[("length",)]], [synth.lut_from_points(91)], [1.0], n, cams, 16, 16,
                    guard=g)
    for cell in (16, 5):
        got = isaac.DeviceScene(sc).range_grid(cell)
        torch.cuda.synchronize()
        want = oracle.range_grid(sc, cell)
        assert np.isinf(want).any()
        np.testing.assert_array_equal(got.cpu().numpy(), want)
