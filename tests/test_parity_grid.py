"""GPU parity of isaac_opacity_grid against the FP64 oracle."""
import numpy as np
import pytest

import oracle
from paper_1611_09048_b300 import isaac, synth
from scenes_util import small_pic_scene

pytestmark = pytest.mark.gpu

TOL_ALPHA = 1e-5   # FP32 chain/LUT vs FP64, opacities in [0, 1]


@pytest.mark.parametrize("cell", [4, 7, 16])
def test_grid_pic(cuda_ok, cell):
    import torch
    sc = small_pic_scene(n=24, guard=2, seed=4, layout="soa")
    sc.sources[2] = synth.source_from_zyx(synth.pic_fields(24, 0, seed=9)[2], 0)
    g = isaac.DeviceScene(sc).opacity_grid(cell)
    torch.cuda.synchronize()
    want = oracle.opacity_grid(sc, cell)
    np.testing.assert_allclose(g.cpu().numpy(), want, rtol=0, atol=TOL_ALPHA)


def test_grid_bubble_mask_and_empty(cuda_ok):
    import torch
    sc = synth.scene_bubble(64, frame=3, seed=2, width=32, height=32)
    ds = isaac.DeviceScene(sc)
    g = ds.opacity_grid(8)
    torch.cuda.synchronize()
    want = oracle.opacity_grid(sc, 8)
    np.testing.assert_allclose(g.cpu().numpy(), want, rtol=0, atol=TOL_ALPHA)
    assert (want == 0).mean() > 0.5          # the bubble leaves most macro cells empty
    assert np.array_equal(g.cpu().numpy() == 0, want == 0)
    z = ds.opacity_grid(8, mask=0)
    torch.cuda.synchronize()
    assert torch.count_nonzero(z) == 0


@pytest.mark.parametrize("cell", [2, 5, 40])
def test_grid_non_cubic_two_sources(cuda_ok, cell):
    """A 30 x 13 x 19 volume with two scalar sources (the run-time source
    loop), one with guards and a chain, one without: every macro-cell size
    from 2 (z chunks of many cells) to one larger than the volume."""
    import torch
    from scenes_util import make_scene
    n = (30, 13, 19)
    rng = np.random.default_rng(21)
    f0 = rng.random((n[2] + 2, n[1] + 2, n[0] + 2), np.float32)          # guard 1
    f1 = rng.random((n[2], n[1], n[0]), np.float32) ** 3                  # no guard
    cams = synth.random_orbit_camera(n, 16, 16, seed=3)
    sc = make_scene([f0, f1], [[("mul", (2.0,)), ("add", (-0.5,))], []],
                    [synth.lut_from_points(31), synth.lut_from_points(32)], [0.7, 0.6], n, cams,
                    16, 16)
    sc.sources[0] = synth.source_from_zyx(f0, 1)
    g = isaac.DeviceScene(sc).opacity_grid(cell)
    torch.cuda.synchronize()
    want = oracle.opacity_grid(sc, cell)
    assert want.shape == tuple((k + cell - 1) // cell for k in n[::-1])
    np.testing.assert_allclose(g.cpu().numpy(), want, rtol=0, atol=TOL_ALPHA)


@pytest.mark.parametrize("guard", [0, 1, 3])
@pytest.mark.parametrize("cell", [8, 16])
def test_grid_scalar_identity_ragged(cuda_ok, guard, cell):
    """The scalar identity-chain walk (its own kernel for 8- and 16-cell macro
    cells) on volumes that are not multiples of the cell, with and without
    guard cells, and a negative weight (opacity clamped to 0)."""
    import torch
    from scenes_util import make_scene
    n = (37, 20, 45)
    rng = np.random.default_rng(40 + guard + cell)
    S = (n[2] + 2 * guard, n[1] + 2 * guard, n[0] + 2 * guard)
    # a ramp in z (so each macro cell's maximum depends on exactly which z-cells
    # it covers, aprons included) plus a little noise
    ramp = (np.arange(S[0], dtype=np.float32) / S[0])[:, None, None]
    f = (0.05 + 0.9 * ramp + 0.04 * rng.random(S, np.float32)).astype(np.float32)
    cams = synth.random_orbit_camera(n, 16, 16, seed=4)
    for wgt in (0.8, -0.5):
        sc = make_scene([f], [[]], [synth.lut_from_points(50 + cell)], [wgt], n, cams, 16, 16,
                        guard=guard)
        g = isaac.DeviceScene(sc).opacity_grid(cell)
        torch.cuda.synchronize()
        want = oracle.opacity_grid(sc, cell)
        got = g.cpu().numpy()
        np.testing.assert_allclose(got, want, rtol=0, atol=TOL_ALPHA)
        if wgt < 0:
            assert np.all(got.view(np.uint32) == 0)       # +0, never -0


def test_grid_wide_volume_warp_reduction(cuda_ok):
    """A very wide, thin volume (5000 x 3 x 4): long rows of column maxima
    and macro cells clipped to 3 and 4 cells in y and z."""
    import torch
    from scenes_util import make_scene
    n = (5000, 3, 4)
    rng = np.random.default_rng(77)
    ramp = (np.arange(n[0], dtype=np.float32) / n[0])[None, None, :]
    f = (0.1 + 0.8 * ramp + 0.05 * rng.random((n[2], n[1], n[0]), np.float32)).astype(np.float32)
    cams = synth.random_orbit_camera(n, 16, 16, seed=6)
    sc = make_scene([f], [[]], [synth.lut_from_points(90)], [0.9], n, cams, 16, 16)
    for cell in (16, 7):
        g = isaac.DeviceScene(sc).opacity_grid(cell)
        torch.cuda.synchronize()
        np.testing.assert_allclose(g.cpu().numpy(), oracle.opacity_grid(sc, cell), rtol=0,
                                   atol=TOL_ALPHA)


@pytest.mark.parametrize("cell", [8, 16])
def test_grid_tiled_reductions(cuda_ok, cell):
    """The tiled opacity-grid reduction (64 x 64 columns per block) over several
    tiles in x and y with ragged last tiles: the grid of the float32 field and
    of its BF16 copy (two columns per thread: n_x + 2 even) against the oracle,
    and the value-range grid of the same field.  The field is BF16-representable,
    so the copy holds the same values."""
    import torch
    from scenes_util import make_scene
    n = (150, 97, 21)
    rng = np.random.default_rng(81 + cell)
    x = np.arange(n[0], dtype=np.float32)[None, None, :]
    y = np.arange(n[1], dtype=np.float32)[None, :, None]
    f = 0.5 + 0.3 * np.sin(0.11 * x) * np.cos(0.07 * y) + 0.15 * rng.random((n[2], n[1], n[0]))
    f = f.astype(np.float32)
    f = (f.view(np.uint32) & np.uint32(0xFFFF0000)).view(np.float32)   # BF16 values
    cams = synth.random_orbit_camera(n, 16, 16, seed=8)
    sc = make_scene([f], [[]], [synth.lut_from_points(70 + cell)], [0.9], n, cams, 16, 16)
    ds = isaac.DeviceScene(sc)
    want = oracle.opacity_grid(sc, cell)
    assert want.shape == tuple((k + cell - 1) // cell for k in n[::-1])
    assert len(np.unique(want)) > want.size // 8          # maxima differ from cell to cell
    g = ds.opacity_grid(cell)
    gb = ds.pack("bf16").opacity_grid(cell)
    r = ds.range_grid(cell)
    torch.cuda.synchronize()
    np.testing.assert_allclose(g.cpu().numpy(), want, rtol=0, atol=TOL_ALPHA)
    np.testing.assert_allclose(gb.cpu().numpy(), want, rtol=0, atol=TOL_ALPHA)
    assert np.array_equal(r.cpu().numpy(), oracle.range_grid(sc, cell))
