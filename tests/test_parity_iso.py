"""GPU parity of the iso-surface frame (isaac_render_iso) against the FP64
oracle's iso-surface reading.

A pixel is compared unless one of its discrete decisions sits at a tie the
two precisions may resolve differently: the entry or exit sample (margins as
in the volume mode), the crossing (|v - iso| below 1e-4 relative at a sample
up to the hit), an ill-conditioned refinement (|v(k) - v(k-1)| < 1e-4) or an
ill-conditioned normal (|gradient| < 1e-2).  Compared pixels agree within
2e-3 per channel before quantisation (FP32 gradients by central differences,
then the 32nd power of n.v) and within 1 LSB after.
"""
import numpy as np
import pytest

import oracle
from paper_1611_09048_b300 import isaac, synth
from scenes_util import make_scene, ortho_down_z, small_pic_scene

pytestmark = pytest.mark.gpu

TOL_ISO = 2e-3


def _compare(sc, iso, g32, g8, max_excluded=0.02):
    ref = oracle.render_iso(sc, iso)
    m = ref["margin"].reshape(-1, 6)
    hit = m[:, 5] >= 0
    scale = 1.0 + np.max(np.abs(iso))
    excl = (m[:, 0] < 1e-6) | (m[:, 1] < 1e-6) | (m[:, 2] < 1e-4 * scale)
    excl |= hit & ((m[:, 3] < 1e-4) | (m[:, 4] < 1e-2))
    keep = ~excl
    e = np.abs(np.asarray(g32, np.float64).reshape(-1, 4) - ref["rgba"].reshape(-1, 4)).max(-1)
    d8 = np.abs(np.asarray(g8).reshape(-1, 4).astype(int) - ref["rgba8"].reshape(-1, 4).astype(int)).max(-1)
    assert excl.mean() <= max_excluded, excl.mean()
    assert e[keep].max(initial=0.0) <= TOL_ISO, e[keep].max()
    assert d8[keep].max(initial=0) <= 1
    return int(hit.sum())


def _gpu(sc, iso):
    import torch
    out, f32, ns = isaac.DeviceScene(sc).render_iso(iso, want_f32=True, want_nsamp=True)
    torch.cuda.synchronize()
    return out.cpu().numpy(), f32.cpu().numpy(), ns.cpu().numpy()


def test_iso_bubble(cuda_ok):
    sc = synth.scene_bubble(64, frame=10, seed=1, width=96, height=72, dist_factor=1.0)
    g8, g32, _ = _gpu(sc, [0.4])
    assert _compare(sc, [0.4], g32, g8) > 80


@pytest.mark.parametrize("layout", ["aos", "soa"])
def test_iso_pic_three_sources(cuda_ok, layout):
    sc = small_pic_scene(n=24, guard=2, width=64, height=48, seed=6, layout=layout, dist_factor=1.2)
    iso = [0.6, 0.55, 0.5]
    g8, g32, _ = _gpu(sc, iso)
    assert _compare(sc, iso, g32, g8) > 300


def test_iso_nearest_and_clip(cuda_ok):
    sc = synth.scene_bubble(64, frame=40, seed=3, width=80, height=64, dist_factor=1.2)
    sc.interp = 0
    sc.clip = [(0.0, 0.0, 1.0, -30.0)]
    g8, g32, _ = _gpu(sc, [0.35])
    _compare(sc, [0.35], g32, g8, max_excluded=0.05)


def test_iso_linear_field_closed_form(cuda_ok):
    """v = x/16 - z/8 + 4: the crossing, the normal and the colour are exact
    closed forms (the oracle's pin); the GPU matches them within FP32."""
    n = (16, 8, 32)
    S = [k + 4 for k in n]
    z, y, x = np.meshgrid(*(np.arange(s) - 2 + 0.5 for s in S[::-1]), indexing="ij")
    f = (x / 16 - z / 8 + 4).astype(np.float32)
    lut = np.zeros((256, 4), np.float32)
    lut[:, :3] = (0.5, 0.25, 0.75)
    lut[:, 3] = 0.5
    sc = make_scene([f], [[]], [lut], [1.0], n, ortho_down_z(n, 16, 8), 16, 8, guard=2)
    g8, g32, ns = _gpu(sc, [2.5])
    ndl = 0.125 / np.hypot(0.0625, 0.125)
    rgb = np.clip(np.array([0.5, 0.25, 0.75]) * (0.25 + 0.75 * ndl) + 0.25 * ndl ** 32, 0, 1)
    np.testing.assert_allclose(g32[..., :3], np.broadcast_to(rgb, g32[..., :3].shape), atol=2e-6)
    assert np.all(g32[..., 3] == 1.0)
    assert np.all(ns > 0)


def test_iso_rejects_nonfinite_threshold(cuda_ok):
    sc = synth.scene_bubble(32, frame=0, seed=0, width=16, height=16)
    with pytest.raises(isaac.IsaacError) as e:
        isaac.DeviceScene(sc).render_iso([float("nan")])
    assert e.value.code == isaac.EINVAL


def test_domain_split_iso_composites_to_whole(cuda_ok):
    """Two halves along x with two guard layers, each an iso frame on the GPU
    with a zero background and the depth output, composited by isaac_composite
    (the nearest layer with a hit wins, alpha 1): the oracle's whole-volume
    iso frame, except where a half's hit is its own first sample (no previous
    sample in the half for the secant step) and at decision ties."""
    import torch
    n, g = 20, 2
    iso = [0.6, 0.55, 0.5]
    fields = synth.pic_fields(n, g, seed=5)
    whole = synth.scene_pic(n=n, guard=g, width=48, height=40, seed=5, fields=fields,
                            dist_factor=1.0)
    whole.bg = (0.0, 0.0, 0.0, 0.0)
    ref = oracle.render_iso(whole, iso)
    layers, no_secant = [], np.zeros((40, 48), bool)
    for lo in (0, n // 2):
        part = synth.scene_pic(n=n, guard=g, width=48, height=40, seed=5, fields=fields,
                               dist_factor=1.0)
        part.bg = (0.0, 0.0, 0.0, 0.0)
        part.global_n = (n, n, n)
        part.off = (lo, 0, 0)
        part.n = (n // 2, n, n)
        for s in part.sources:
            s.offset = s.offset + lo * s.strides[0]
        pm = oracle.render_iso(part, iso)["margin"]
        no_secant |= (pm[..., 5] >= 0) & (pm[..., 3] >= oracle.INF)
        f32 = torch.empty((40, 48, 4), dtype=torch.float32, device="cuda")
        dep = torch.empty((40, 48), dtype=torch.float32, device="cuda")
        isaac.DeviceScene(part).render_iso(iso, rgba32=f32, depth=dep)
        layers.append((f32, dep))
    out8 = torch.empty((40, 48, 4), dtype=torch.uint8, device="cuda")
    out32 = torch.empty((40, 48, 4), dtype=torch.float32, device="cuda")
    isaac.composite(layers, bg=(0.0, 0.0, 0.0, 0.0), out=out8, rgba32=out32)
    torch.cuda.synchronize()
    m = ref["margin"]
    hit = m[..., 5] >= 0
    excl = (m[..., 0] < 1e-6) | (m[..., 1] < 1e-6) | (m[..., 2] < 1e-4 * 1.6)
    excl |= hit & ((m[..., 3] < 1e-4) | (m[..., 4] < 1e-2))
    keep = ~excl & ~(no_secant & (m[..., 3] < oracle.INF))
    got = out32.cpu().numpy().astype(np.float64)
    assert hit.sum() > 300 and keep.mean() > 0.9
    assert np.abs(got - ref["rgba"])[keep].max() <= TOL_ISO
    assert np.abs(out8.cpu().numpy().astype(int) - ref["rgba8"].astype(int))[keep].max() <= 1
