"""isaac_render_noalloc: the render entry point for callers that must not
allocate device memory (for example a simulation that owns all of the GPU's
memory through its own pool, or a time-step loop where cudaMalloc's possible
device synchronisation is not allowed).  It keeps the frame's ray list in a
fixed array compiled into the library instead of a cudaMalloc'd workspace.

These tests call it through the C ABI and compare it with isaac_render on
the same inputs, for two calls in a row (the array keeps the previous call's
contents, so the second call checks that the reset between calls works).
Both entry points pick the same kernel (lanes per ray from the same corner
size) and so give the same image bit for bit.

The file name sorts last so that a run stopping at its first failure has run
every other test before this one; the tests depend on no earlier test and
pass in a fresh process as well."""
import ctypes as C

import numpy as np
import pytest

from paper_1611_09048_b300 import isaac, synth
from scenes_util import small_pic_scene

pytestmark = pytest.mark.gpu


def _frames(ds, cams, entry):
    """Render each camera with the given C entry point; returns host copies."""
    import torch
    lib = isaac.load()
    fn = getattr(lib, entry)
    W, H = ds.scene.width, ds.scene.height
    outs = []
    stream = torch.cuda.current_stream()
    for mv, proj in cams:
        o8 = torch.zeros((H, W, 4), dtype=torch.uint8, device=ds.device)
        o32 = torch.zeros((H, W, 4), dtype=torch.float32, device=ds.device)
        ns = torch.zeros((H, W), dtype=torch.int32, device=ds.device)
        args, keep = ds.prepare(mv, proj, o8, o32, ns)
        rc = fn(*args, C.c_void_p(stream.cuda_stream))
        assert rc == 0, lib.isaac_last_error().decode()
        torch.cuda.synchronize()
        outs.append((o8.cpu().numpy(), o32.cpu().numpy(), ns.cpu().numpy()))
        del keep
    return outs


def test_noalloc_matches_render_on_two_calls_in_a_row(cuda_ok):
    sc = small_pic_scene(n=32, guard=2, width=160, height=120, seed=12, dist_factor=1.0)
    ds = isaac.DeviceScene(sc)
    n = sc.n
    cams = [synth.random_orbit_camera(n, sc.width, sc.height, seed=s, dist_factor=1.0)
            for s in (31, 32)]
    got = _frames(ds, cams, "isaac_render_noalloc")
    want = _frames(ds, cams, "isaac_render")
    for (g8, g32, gns), (w8, w32, wns) in zip(got, want):
        assert (wns > 0).sum() > 1000
        # the same kernel on the same inputs: the same image bit for bit
        np.testing.assert_array_equal(g32, w32)
        np.testing.assert_array_equal(g8, w8)
        np.testing.assert_array_equal(gns, wns)


def test_noalloc_rejects_a_rectangle_beyond_its_array(cuda_ok):
    """A camera close enough to fill a 1024x1024 image needs more ray records
    than the fixed array holds: the call fails on the host with ENOMEM."""
    import torch
    sc = small_pic_scene(n=32, guard=2, width=1024, height=1024, seed=12, dist_factor=0.6)
    ds = isaac.DeviceScene(sc)
    o8 = torch.zeros((1024, 1024, 4), dtype=torch.uint8, device=ds.device)
    args, keep = ds.prepare(out=o8)
    lib = isaac.load()
    rc = lib.isaac_render_noalloc(*args, C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == isaac.ENOMEM
    assert "at most 262144 rays" in lib.isaac_last_error().decode()
    torch.cuda.synchronize()
    assert int(o8.sum()) == 0          # nothing was launched


def test_noalloc_rejects_host_luts(cuda_ok):
    """Host LUTs need pinned staging that the library allocates, so this entry
    point refuses them on the host (nothing launched)."""
    import torch
    sc = small_pic_scene(n=16, guard=2, width=64, height=48, seed=3, dist_factor=1.0)
    ds = isaac.DeviceScene(sc)
    host_luts = np.ascontiguousarray(sc.luts, np.float32)
    o8 = torch.zeros((48, 64, 4), dtype=torch.uint8, device=ds.device)
    args, keep = ds.prepare(out=o8)
    args = list(args)
    args[3] = host_luts.ctypes.data
    opts = args[8]._obj
    opts.flags = isaac.LUTS_HOST
    lib = isaac.load()
    rc = lib.isaac_render_noalloc(*args, C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == isaac.EINVAL
    assert "host LUTs" in lib.isaac_last_error().decode()
