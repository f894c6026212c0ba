"""The staged march (ISAAC_MARCH_STAGED): one thread per ray, each warp copying
the box of cells its rays' next samples read into shared memory before
gathering from there.  It reads the same corner values and composites in the
same order as the gather march, so its frames must equal the gather march's
bit for bit: RGBA8, the float output and the sample counts.  The gather march
is checked against the FP64 oracle throughout test_parity_render.py; one
staged frame is also checked against the oracle directly here.

The cameras span boxes that fit the per-warp buffer (near cameras, rays
closer than a voxel) and boxes that do not (far cameras: those slabs gather
from global memory), cameras inside the volume, both source layouts, a
scalar field without guard cells, and frames the staged kernel cannot take
(sources with different guard widths), which must fall back unchanged."""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_1611_09048_b300 import isaac, synth
from parity_util import assert_parity, compare
from scenes_util import small_pic_scene

pytestmark = pytest.mark.gpu


def _both(sc, **kw):
    """The frame without and with ISAAC_MARCH_STAGED (host copies)."""
    import torch
    ds = isaac.DeviceScene(sc)
    outs = []
    for staged in (False, True):
        o8, o32, ns = ds.render(want_f32=True, want_nsamp=True, staged=staged, **kw)
        torch.cuda.synchronize()
        outs.append((o8.cpu().numpy(), o32.cpu().numpy(), ns.cpu().numpy()))
    return outs


def _assert_same(outs, min_hit=1000):
    (g8, g32, gns), (s8, s32, sns) = outs
    assert (gns > 0).sum() >= min_hit
    np.testing.assert_array_equal(sns, gns)
    np.testing.assert_array_equal(s32, g32)
    np.testing.assert_array_equal(s8, g8)


@pytest.mark.parametrize("layout", ["aos", "soa"])
@pytest.mark.parametrize("dist", [2.0, 1.0, 0.6, 0.45])
def test_staged_equals_gather_pic(cuda_ok, layout, dist):
    sc = small_pic_scene(n=64, guard=2, width=320, height=240, seed=5, layout=layout,
                         dist_factor=dist)
    _assert_same(_both(sc))


@pytest.mark.parametrize("seed", [0, 1, 2])
@pytest.mark.parametrize("dist", [2.0, 0.7])
def test_staged_equals_gather_scalar_without_guards(cuda_ok, seed, dist):
    """One scalar field of Gaussian blobs, no guard cells (reads clamp to the
    interior), at a far and a near camera."""
    sc = synth.scene_blobs(64, 256, 256, seed=seed, dist_factor=dist)
    _assert_same(_both(sc))


@pytest.mark.parametrize("dist", [2.0, 0.9])
def test_staged_equals_gather_pic256_1080p(cuda_ok, dist):
    """Full 1080p frames over a 256^3 E/B/rho volume with 4 guard cells."""
    sc = synth.scene_pic(n=256, guard=4, width=1920, height=1080, seed=2, dist_factor=dist)
    _assert_same(_both(sc), min_hit=50000)


def test_staged_against_oracle(cuda_ok):
    """A near camera (rays ~0.3 voxels apart, staged boxes) against the FP64
    oracle, element by element."""
    import torch
    sc = small_pic_scene(n=24, guard=2, width=96, height=80, seed=3, dist_factor=0.8)
    ds = isaac.DeviceScene(sc)
    o8, o32, ns = ds.render(want_f32=True, want_nsamp=True, staged=True)
    torch.cuda.synchronize()
    rep = compare(o32.cpu().numpy(), o8.cpu().numpy(), ns.cpu().numpy(), oracle.render(sc),
                  interp=sc.interp)
    assert_parity(rep, 1e-3, "staged near camera")
    assert rep.hit > 2000


def test_staged_falls_back_where_it_cannot_stage(cuda_ok):
    """Sources with different guard widths (no common box), nearest-cell
    sampling and an explicit lane count all keep the gather march's image."""
    sc = small_pic_scene(n=32, guard=2, width=160, height=120, seed=7, dist_factor=0.8)
    _assert_same(_both(sc, lanes=4))
    near = dataclasses.replace(sc, interp=0)
    _assert_same(_both(near))
    E, B, rho = synth.pic_fields(32, 2, seed=7)
    mixed = synth.scene_pic(n=32, guard=2, width=160, height=120, seed=7, fields=(E, B, rho),
                            dist_factor=0.8)
    mixed.sources[2] = synth.source_from_zyx(np.ascontiguousarray(rho[2:-2, 2:-2, 2:-2]), 0,
                                             name="rho")
    _assert_same(_both(mixed))
