"""Transfer functions passed in host memory (isaac_render_opts.flags =
ISAAC_LUTS_HOST): the frame and the opacity grid equal those of the same LUTs
in device memory bit for bit; the call copies the LUTs before it returns, so
the caller may overwrite its array at once; the pinned staging ring (8 slots
per stream) wraps without mixing frames; unknown flag bits are rejected."""
import ctypes as C

import numpy as np
import pytest

from paper_1611_09048_b300 import isaac, synth
from scenes_util import small_pic_scene

pytestmark = pytest.mark.gpu


def _scene():
    return small_pic_scene(n=24, guard=2, width=96, height=64, seed=8, dist_factor=1.0)


def test_host_luts_frame_equals_device_luts(cuda_ok):
    import torch
    sc = _scene()
    ds = isaac.DeviceScene(sc)
    want = ds.render(want_f32=True, want_nsamp=True)
    host = np.ascontiguousarray(sc.luts, np.float32).copy()
    got = ds.render(want_f32=True, want_nsamp=True, luts=host)
    host[:] = 0.0                     # the call has copied them: this must not show
    torch.cuda.synchronize()
    assert int((want[2] > 0).sum()) > 500
    for a, b in zip(want, got):
        assert torch.equal(a, b)


def test_host_luts_staging_ring_wraps(cuda_ok):
    """20 frames on one stream, the LUT array rewritten after every call
    (alternating two LUT sets): each frame equals the device-LUT frame of the
    set it was called with."""
    import torch
    sc = _scene()
    ds = isaac.DeviceScene(sc)
    sets = [np.ascontiguousarray(sc.luts, np.float32).copy(),
            np.stack([synth.lut_from_points(77 + s) for s in range(len(sc.sources))])]
    want = []
    for L in sets:
        ds.set_luts(L)
        want.append(ds.render(want_f32=True)[1].clone())
    ds.set_luts(sets[0])
    host = np.empty_like(sets[0])
    outs = []
    for i in range(20):
        host[:] = sets[i % 2]
        outs.append(ds.render(want_f32=True, luts=host)[1])
    torch.cuda.synchronize()
    assert not torch.equal(want[0], want[1])
    for i, o in enumerate(outs):
        assert torch.equal(o, want[i % 2]), i


def test_host_luts_opacity_grid(cuda_ok):
    import torch
    sc = _scene()
    ds = isaac.DeviceScene(sc)
    a = ds.opacity_grid(8)
    b = ds.opacity_grid(8, host_luts=np.ascontiguousarray(sc.luts, np.float32))
    torch.cuda.synchronize()
    assert float(a.max()) > 0.0
    assert torch.equal(a, b)


def test_unknown_flag_bits_are_rejected(cuda_ok):
    import torch
    sc = _scene()
    ds = isaac.DeviceScene(sc)
    o8 = torch.zeros((sc.height, sc.width, 4), dtype=torch.uint8, device=ds.device)
    args, keep = ds.prepare(out=o8)
    args[8]._obj.flags = 0x4
    lib = isaac.load()
    assert lib.isaac_render(*args, C.c_void_p(0)) == isaac.EINVAL
    assert "flags" in lib.isaac_last_error().decode()


def _with_host_luts(args, lut_index, opts_index, host):
    """The same call's arguments with the LUT pointer replaced by a host array
    and ISAAC_LUTS_HOST set in its options."""
    a = list(args)
    a[lut_index] = host.ctypes.data
    a[opts_index]._obj.flags = isaac.LUTS_HOST
    return a


def test_host_luts_in_skip_iso_learned_and_packed_frames(cuda_ok):
    """Every other frame entry point that reads LUTs gives the device-LUT image
    bit for bit with host LUTs: empty-space skipping (whose empty flags read
    the LUTs before the march), iso surfaces, the learned frame (widened
    proposal) and the packed BF16 frame."""
    import torch
    sc = _scene()
    ds = isaac.DeviceScene(sc)
    host = np.ascontiguousarray(sc.luts, np.float32).copy()
    lib = isaac.load()
    H, W = sc.height, sc.width

    def pair(prep_fn, launch, lut_i, opts_i):
        outs = []
        for use_host in (False, True):
            o8 = torch.zeros((H, W, 4), dtype=torch.uint8, device=ds.device)
            f32 = torch.zeros((H, W, 4), dtype=torch.float32, device=ds.device)
            args, keep = prep_fn(o8, f32)
            if use_host:
                args = _with_host_luts(args, lut_i, opts_i, host)
            assert launch(*args, C.c_void_p(0)) == 0, lib.isaac_last_error().decode()
            torch.cuda.synchronize()
            outs.append((o8.cpu().numpy(), f32.cpu().numpy()))
        np.testing.assert_array_equal(outs[0][0], outs[1][0])
        np.testing.assert_array_equal(outs[0][1], outs[1][1])
        return outs[0]

    ranges = ds.range_grid(8)
    pair(lambda o8, f32: ds.prepare_skip(ranges, 8, out=o8, rgba32=f32), lib.isaac_render_skip, 3, 8)
    iso = [0.6, 0.55, 0.5]
    pair(lambda o8, f32: ds.prepare_iso(iso, out=o8, rgba32=f32), lib.isaac_render_iso, 3, 8)
    grid = ds.opacity_grid(8)
    model = isaac.MLPModel(isaac.pack_mlp_params(synth.mlp_params(2, bias_scale=0.3)), train=False)
    prop = model.proposal(grid, 8, threshold=0.5, margin=2)
    img = pair(lambda o8, f32: ds.prepare_learned(prop, out=o8, rgba32=f32), lib.isaac_render_learned, 3, 8)
    assert (img[1][..., 3] > 0).sum() > 300
    pv = ds.pack("bf16")
    pair(lambda o8, f32: pv.prepare(out=o8, rgba32=f32), lib.isaac_render_packed, 2, 7)
