"""Sort-last compositing on the GPU (isaac_composite, Sec. 3.4): a volume
split into four sub-volumes with guards, each rendered on its own on the
global sample grid with a zero background and the depth output, composited
per pixel in depth order, equals the oracle's frame of the whole volume
(termination off); and equals the over operator applied in numpy to the same
layers in the order their depths give."""
import numpy as np
import pytest

import oracle
from paper_1611_09048_b300 import isaac, synth
from parity_util import TOL_F32

pytestmark = pytest.mark.gpu


def _split_scene(n, g, lo, size, fields, seed=5, bg=(0.0, 0.0, 0.0, 0.0)):
    sc = synth.scene_pic(n=n, guard=g, width=48, height=40, seed=seed, fields=fields,
                         dist_factor=1.0)
    sc.term = 2.0
    sc.bg = bg
    sc.global_n = (n, n, n)
    sc.off = tuple(lo)
    sc.n = tuple(size)
    for s in sc.sources:
        s.offset = s.offset + lo[0] * s.strides[0] + lo[1] * s.strides[1] + lo[2] * s.strides[2]
    return sc


def test_four_way_split_composites_to_whole(cuda_ok):
    import torch
    n, g = 20, 2
    fields = synth.pic_fields(n, g, seed=5)
    bg = (0.1, 0.2, 0.3, 1.0)
    whole = synth.scene_pic(n=n, guard=g, width=48, height=40, seed=5, fields=fields, dist_factor=1.0)
    whole.term = 2.0
    whole.bg = bg
    ref = oracle.render(whole)
    layers = []
    for lo in ((0, 0, 0), (n // 2, 0, 0), (0, 0, n // 2), (n // 2, 0, n // 2)):
        size = (n // 2, n, n // 2)
        part = _split_scene(n, g, lo, size, fields)
        ds = isaac.DeviceScene(part)
        H, W = part.height, part.width
        f32 = torch.empty((H, W, 4), dtype=torch.float32, device="cuda")
        dep = torch.empty((H, W), dtype=torch.float32, device="cuda")
        ds.render(rgba32=f32, depth=dep)
        layers.append((f32, dep))
    out8 = torch.empty((40, 48, 4), dtype=torch.uint8, device="cuda")
    out32 = torch.empty((40, 48, 4), dtype=torch.float32, device="cuda")
    isaac.composite(layers, bg=bg, out=out8, rgba32=out32)
    torch.cuda.synchronize()
    got = out32.cpu().numpy().astype(np.float64)
    assert (ref["nsamp"] > 0).sum() > 300
    assert np.abs(got - ref["rgba"]).max() <= 4 * TOL_F32
    assert np.abs(out8.cpu().numpy().astype(int) - ref["rgba8"].astype(int)).max() <= 1
    # the same layers, over-composited in numpy in depth order
    L = [(c.cpu().numpy().astype(np.float64), d.cpu().numpy()) for c, d in layers]
    D = np.stack([d for _, d in L])
    order = np.argsort(D, axis=0, kind="stable")
    C = np.zeros((40, 48, 3))
    A = np.zeros((40, 48, 1))
    for m in range(len(L)):
        idx = order[m]
        c = np.take_along_axis(np.stack([x for x, _ in L]), idx[None, ..., None], 0)[0]
        C += (1 - A) * c[..., :3]
        A += (1 - A) * c[..., 3:4]
    want = np.concatenate([C + (1 - A) * np.asarray(bg[:3]), A + (1 - A) * bg[3]], -1)
    assert np.abs(got - want).max() <= 1e-6


def test_depth_is_first_sample_distance(cuda_ok):
    """Two halves along x seen from +x: where both are hit, the near half's
    depth is smaller; missed pixels carry +inf."""
    import torch
    n, g = 20, 2
    fields = synth.pic_fields(n, g, seed=7)
    deps = []
    for lo in ((0, 0, 0), (n // 2, 0, 0)):
        part = _split_scene(n, g, lo, (n // 2, n, n), fields, seed=7)
        mv, proj = synth.orbit_camera(part.gn, 48, 40, np.pi / 2, 0.1, dist_factor=1.5)
        ds = isaac.DeviceScene(part)
        dep = torch.empty((40, 48), dtype=torch.float32, device="cuda")
        ds.render(mv, proj, depth=dep)
        deps.append(dep.cpu().numpy())
    torch.cuda.synchronize()
    both = np.isfinite(deps[0]) & np.isfinite(deps[1])
    assert both.sum() > 100
    assert np.all(deps[1][both] < deps[0][both])     # the camera is on the +x side
    assert np.isinf(deps[0]).any()


def _over_numpy(L, bg):
    D = np.stack([np.where(np.isnan(d), np.inf, d) for _, d in L])
    order = np.argsort(D, axis=0, kind="stable")
    H, W = D.shape[1:]
    C = np.zeros((H, W, 3), np.float32)
    A = np.zeros((H, W, 1), np.float32)
    S = np.stack([x for x, _ in L]).astype(np.float32)
    for m in range(len(L)):
        c = np.take_along_axis(S, order[m][None, ..., None], 0)[0]
        C = (1 - A) * c[..., :3] + C
        A = (1 - A) * c[..., 3:4] + A
    return np.concatenate([C + (1 - A) * np.asarray(bg[:3], np.float32),
                           A + (1 - A) * np.float32(bg[3])], -1)


@pytest.mark.parametrize("n_layers", [1, 2, 5, 8, 16])
def test_ties_nan_and_every_layer_count(cuda_ok, n_layers):
    """Depths drawn from a few values (many ties), with NaN and +inf mixed in,
    at every layer count the kernel is specialised for: the result equals the
    over operator in stable depth order (NaN as +inf), on a ragged image."""
    import torch
    H, W = 37, 53
    rng = np.random.default_rng(100 + n_layers)
    L = []
    for _ in range(n_layers):
        a = rng.random((H, W, 1), np.float32) * 0.6
        c = np.concatenate([rng.random((H, W, 3), np.float32) * a, a], -1)
        d = rng.choice(np.array([1.0, 2.0, 3.0, np.inf, np.nan], np.float32), size=(H, W))
        L.append((c, d))
    bg = (0.2, 0.1, 0.4, 1.0)
    layers = [(torch.from_numpy(np.ascontiguousarray(c)).cuda(),
               torch.from_numpy(np.ascontiguousarray(d)).cuda()) for c, d in L]
    out8 = torch.empty((H, W, 4), dtype=torch.uint8, device="cuda")
    out32 = torch.empty((H, W, 4), dtype=torch.float32, device="cuda")
    isaac.composite(layers, bg=bg, out=out8, rgba32=out32)
    torch.cuda.synchronize()
    want = _over_numpy(L, bg)
    got = out32.cpu().numpy()
    assert np.abs(got - want).max() <= 2e-6
    q = np.minimum(255, np.floor(255 * np.clip(want.astype(np.float64), 0, 1) + 0.5)).astype(int)
    assert np.abs(out8.cpu().numpy().astype(int) - q).max() <= 1
