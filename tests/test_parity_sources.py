"""Sources whose memory is not persistent (Sec. 3.2) on the GPU.

* isaac_copy_source writes exactly the cells a frame can read (the interior
  and one guard layer when the source has guards), components adjacent, for
  AoS, SoA and guard-free layouts; bit for bit against numpy slicing.
* A frame of the copies equals the frame of the originals after the
  originals were overwritten: bitwise where the layout is unchanged (AoS),
  and within the FP32 tolerance of the oracle where the copy changes the
  layout (SoA -> AoS selects another specialisation).
* The paper's use case: two derived fields computed in turn into ONE scratch
  buffer by the per-source update callback, each copied before the next
  source's update reuses the buffer, render exactly like two persistent
  fields; without the copy both sources would show the last field.
"""
import numpy as np
import pytest

import oracle
from paper_1611_09048_b300 import isaac, synth
from parity_util import assert_parity, compare

pytestmark = pytest.mark.gpu


def _expected_copy(arr, field_guard, g, n):
    """(z, y, x[, c]) array with ``field_guard`` layers -> the flat AoS copy of
    cells [-g, n+g) per axis."""
    lo, hi = field_guard - g, field_guard + n + g
    sub = arr[lo:hi, lo:hi, lo:hi]
    return np.ascontiguousarray(sub, np.float32).reshape(-1)


@pytest.mark.parametrize("layout,guard", [("aos", 2), ("soa", 4), ("aos", 0)])
def test_copy_is_the_reachable_region(cuda_ok, layout, guard):
    import torch
    n = 13
    rng = np.random.default_rng(7)
    arr = rng.standard_normal((n + 2 * guard,) * 3 + (3,)).astype(np.float32)
    src = synth.source_from_zyx(arr, guard, layout)
    dev = torch.from_numpy(src.data).cuda()
    d = isaac.Source()
    d.ptr, d.extent, d.offset = dev.data_ptr(), dev.numel(), src.offset
    for a in range(3):
        d.stride[a] = src.strides[a]
    d.comp_stride, d.f_dim, d.guard = src.cstride, 3, guard
    g = 1 if guard >= 1 else 0
    buf = torch.full((isaac.copy_bytes((n, n, n), 3, guard) // 4 + 64,), -7.0, device="cuda")
    out = isaac.copy_source(d, (n, n, n), buf)
    torch.cuda.synchronize()
    want = _expected_copy(arr, guard, g, n)
    got = buf.cpu().numpy()
    assert np.array_equal(got[:want.size].view(np.uint32), want.view(np.uint32))
    assert np.all(got[want.size:] == -7.0)                  # nothing written past the copy
    X = n + 2 * g
    assert (out.f_dim, out.guard, out.comp_stride) == (3, g, 1)
    assert tuple(out.stride) == (3, 3 * X, 3 * X * X)
    assert out.offset == g * (3 + 3 * X + 3 * X * X) and out.extent == want.size


def _render(ds):
    import torch
    out, f32, ns = ds.render(want_f32=True, want_nsamp=True)
    torch.cuda.synchronize()
    return out.cpu().numpy(), f32.cpu().numpy(), ns.cpu().numpy()


def test_copies_render_like_originals_aos(cuda_ok):
    sc = synth.scene_pic(n=20, guard=2, width=48, height=40, seed=3, dist_factor=1.2)
    ds = isaac.DeviceScene(sc)
    ref = _render(ds)
    originals = list(ds.data)
    for s in range(len(sc.sources)):
        ds.copy_source(s)
    for t in originals:
        t.fill_(float("nan"))                                # the application reuses them
    got = _render(ds)
    assert (ref[2] > 0).sum() > 300
    for a, b in zip(ref, got):
        assert np.array_equal(a.view(np.uint8), b.view(np.uint8))


def test_copies_render_like_originals_soa(cuda_ok):
    sc = synth.scene_pic(n=20, guard=3, width=48, height=40, seed=4, layout="soa",
                         dist_factor=1.2)
    ds = isaac.DeviceScene(sc)
    for s in range(len(sc.sources)):
        ds.copy_source(s)
    ds.data[0].zero_()
    g8, g32, gns = _render(ds)
    rep = compare(g32, g8, gns, oracle.render(sc))
    assert_parity(rep, 1e-3, "SoA sources copied to AoS")
    assert rep.hit > 200


def _scalar_scene(fields, n, g):
    srcs = [synth.source_from_zyx(f, g) for f in fields]
    base = synth.scene_blobs(n, 64, 48, seed=2)
    return synth.Scene(n=(n, n, n), sources=srcs, chains=[[], []],
                       luts=np.stack([synth.lut_from_points(11), synth.lut_from_points(12)]),
                       weights=np.array([0.5, 0.5], np.float32), modelview=base.modelview,
                       projection=base.projection, width=64, height=48)


def test_update_callback_with_one_scratch_buffer(cuda_ok):
    import torch
    n, g = 24, 1
    rng = np.random.default_rng(9)
    fields = [rng.random((n + 2 * g,) * 3, dtype=np.float32) ** (3 + 2 * k) for k in range(2)]
    persistent = isaac.DeviceScene(_scalar_scene(fields, n, g))
    ref = _render(persistent)
    assert (ref[2] > 0).sum() > 150

    # both sources are described on one scratch buffer, which the update
    # callback fills with the source's derived field right before it is read
    sc = _scalar_scene([np.zeros_like(fields[0])] * 2, n, g)
    ds = isaac.DeviceScene(sc)
    scratch = ds.data[0]
    scratch_desc = isaac.Source.from_buffer_copy(ds.sources[0])
    ds.sources[1] = isaac.Source.from_buffer_copy(scratch_desc)
    dev_fields = [torch.from_numpy(f.reshape(-1)).cuda() for f in fields]
    nb = isaac.copy_bytes((n, n, n), 1, g) // 4
    copies = [torch.empty(nb, device="cuda") for _ in fields]
    calls = []

    def update(s, enabled, copy=True):
        calls.append((s, enabled))
        scratch.copy_(dev_fields[s])                         # the derived field of source s
        if copy:
            ds.sources[s] = isaac.copy_source(scratch_desc, (n, n, n), copies[s])
        else:
            ds.sources[s] = isaac.Source.from_buffer_copy(scratch_desc)

    isaac.set_update_hook(update)
    try:
        got = _render(ds)
        assert calls == [(0, True), (1, True)]
        for a, b in zip(ref, got):
            assert np.array_equal(a.view(np.uint8), b.view(np.uint8))
        # the same frame without the copy: source 0 reads the last field written
        isaac.set_update_hook(lambda s, en: update(s, en, copy=False))
        shared = _render(ds)
    finally:
        isaac.set_update_hook(None)
    last = isaac.DeviceScene(_scalar_scene([fields[1], fields[1]], n, g))
    want = _render(last)
    for a, b in zip(want, shared):
        assert np.array_equal(a.view(np.uint8), b.view(np.uint8))
    assert not np.array_equal(shared[1], ref[1])


def _slab_scene(field, guard, n, width=64, height=48, term=0.99):
    """One scalar source over an n[0] x n[1] x n[2] box, seen obliquely."""
    from scenes_util import make_scene
    cams = synth.random_orbit_camera(n, width, height, seed=17, dist_factor=1.4)
    return make_scene([field], [[("mul", (1.5,))]], [synth.lut_from_points(88, alpha_max=0.4)],
                      [1.0], n, cams, width, height, guard=guard, term=term)


@pytest.mark.parametrize("guard", [0, 1])
def test_two_dimensional_source(cuda_ok, guard):
    """A 2D field (n_z = 1) is a volume one cell thick: its frame equals the
    oracle's, with guards (the layers above and below are read) and without
    (z clamps to the one layer)."""
    n = (40, 28, 1)
    rng = np.random.default_rng(3 + guard)
    f = rng.random((1 + 2 * guard, 28 + 2 * guard, 40 + 2 * guard), np.float32)
    sc = _slab_scene(f, guard, n)
    g8, g32, gns = _render(isaac.DeviceScene(sc))
    rep = compare(g32, g8, gns, oracle.render(sc))
    assert_parity(rep, 1e-3, f"2D source, guard {guard}")
    assert rep.hit > 100


def test_time_series_as_z(cuda_ok):
    """Time steps of a 2D field stacked along z (time-as-z) form an ordinary
    source: its frame equals the oracle's."""
    T, ny, nx = 12, 20, 36
    t = np.arange(T, dtype=np.float32)[:, None, None]
    y = np.arange(ny, dtype=np.float32)[None, :, None]
    x = np.arange(nx, dtype=np.float32)[None, None, :]
    stack = (0.5 + 0.4 * np.sin(0.3 * x + 0.2 * y - 0.5 * t)).astype(np.float32)
    sc = _slab_scene(stack, 0, (nx, ny, T))
    g8, g32, gns = _render(isaac.DeviceScene(sc))
    rep = compare(g32, g8, gns, oracle.render(sc))
    assert_parity(rep, 1e-3, "time-as-z stack")
    assert rep.hit > 200
