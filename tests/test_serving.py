"""The serving loop (isaac_server_*): continuous batching of render requests
of different sizes, cameras and steering updates against one resident volume.

* every request's image is bitwise the same rendered alone and in a mix;
* it equals isaac_render / isaac_render_packed on the same arguments;
* the zero-copy server's 8-bit output agrees with the FP64 oracle;
* admission by memory budget: a small budget still finishes every request
  (in smaller batches) and an oversize request is rejected at submit.
"""
import dataclasses
import math

import numpy as np
import pytest

import oracle
from paper_1611_09048_b300 import isaac, synth
from scenes_util import small_pic_scene

pytestmark = pytest.mark.gpu

SIZES = [(64, 48), (96, 64), (33, 17), (128, 96), (80, 80), (1, 1), (150, 40), (48, 112)]


def _requests(sc, seed=0):
    """(mv, proj, W, H, luts or None, chains or None) per request: seeded orbit
    cameras (one looks away from the volume), every third request steers."""
    rng = np.random.default_rng(seed)
    out = []
    for i, (W, H) in enumerate(SIZES):
        theta, phi = rng.uniform(0, 2 * math.pi), rng.uniform(-0.6, 0.6)
        mv, proj = synth.orbit_camera(sc.n, W, H, theta, phi, dist_factor=1.2 + 0.3 * (i % 3))
        if i == 4:      # looking away from the box: every pixel is background
            eye = np.array([0.0, 0.0, 2.0 * max(sc.n)])
            mv = synth.look_at(eye, 2.0 * eye, (0.0, 1.0, 0.0))
        luts = chains = None
        if i % 3 == 1:
            luts = np.stack([synth.lut_from_points(seed=100 + 7 * i + s) for s in range(len(sc.sources))])
        if i % 3 == 2:
            chains = [list(c) for c in sc.chains]
            chains[0] = [("length",), ("mul", (0.9 / (1 + i),)), ("add", (0.05,)), ("pow", (0.5,))]
        out.append((np.asarray(mv, np.float64), np.asarray(proj, np.float64), W, H, luts, chains))
    return out


def _pinned(W, H):
    import torch
    return torch.zeros((H, W, 4), dtype=torch.uint8).pin_memory()


def _serve(target, reqs, order, together, **cfg):
    """Submit requests ``order``; all at once or each after the previous finished."""
    outs = {i: _pinned(r[2], r[3]) for i, r in enumerate(reqs)}
    res = {}
    with isaac.Server(target, **cfg) as srv:
        tags = {}
        for i in order:
            mv, proj, W, H, luts, chains = reqs[i]
            tags[srv.submit(mv, proj, W, H, outs[i], luts=luts, chains=chains)] = i
            if not together:
                for r in srv.drain():
                    res[tags[r["tag"]]] = r
        for r in srv.drain():
            res[tags[r["tag"]]] = r
    assert all(r["status"] == 0 for r in res.values()), res
    return {i: o.numpy().copy() for i, o in outs.items()}, res


def _serve_batched(target, sc, reqs, n_streams, max_batch):
    """Serve ``reqs`` submitted together so that they are batched: first one
    1920x1080 request per stream (a few ms each on the GPU), then ``reqs``,
    which queue while the large ones render and are admitted max_batch at a
    time as streams free up.  The submits are host calls, so a host pause
    between them could still let the queue drain; the collector is off
    across them and the case gets up to three attempts.  Returns the images
    and results of ``reqs`` (the large requests are left out)."""
    import gc
    mv, proj = synth.orbit_camera(sc.n, 1920, 1080, 0.7, 0.25, dist_factor=0.8)
    big = (np.asarray(mv, np.float64), np.asarray(proj, np.float64), 1920, 1080, None, None)
    allr = [big] * n_streams + list(reqs)
    order = list(range(len(allr)))
    for attempt in range(3):
        gc.collect()
        gc.disable()
        try:
            outs, res = _serve(target, allr, order, True, n_streams=n_streams, max_batch=max_batch)
        finally:
            gc.enable()
        mine = {i - n_streams: res[i] for i in range(n_streams, len(allr))}
        if max(r["batch_size"] for r in mine.values()) > 1:
            break
    return {i - n_streams: outs[i] for i in range(n_streams, len(allr))}, mine


def _direct(sc, req, packed=None):
    """The same request through isaac_render (or isaac_render_packed)."""
    import torch
    mv, proj, W, H, luts, chains = req
    s2 = dataclasses.replace(sc, width=W, height=H)
    if luts is not None:
        s2.luts = luts.astype(np.float32)
    if chains is not None:
        s2.chains = chains
    ds = isaac.DeviceScene(s2)
    tgt = ds.pack("bf16") if packed else ds
    out, _, _ = tgt.render(mv, proj)
    torch.cuda.synchronize()
    return out.cpu().numpy(), s2


def _check_u8_vs_oracle(g8, s2, mv, proj):
    s3 = dataclasses.replace(s2, modelview=mv, projection=proj)
    o = oracle.render(s3)
    g = g8.reshape(-1, 4).astype(np.int64)
    u8 = o["rgba8"].reshape(-1, 4).astype(np.int64)
    u8a = o["rgba8_alt"].reshape(-1, 4).astype(np.int64)
    m = o["margin"].reshape(-1, 4)
    keep = (m[:, 0] >= 1e-6) & (m[:, 1] >= 1e-6)
    ok = (np.abs(g - u8).max(-1) <= 1) | ((m[:, 2] < 1e-3) & (np.abs(g - u8a).max(-1) <= 1))
    assert int((~ok & keep).sum()) == 0
    return int((o["nsamp"] > 0).sum())


@pytest.fixture(scope="module")
def pic():
    return small_pic_scene(n=24, guard=2, width=64, height=48, seed=11)


def test_alone_equals_mix_zero_copy(cuda_ok, pic):
    import torch
    ds = isaac.DeviceScene(pic)
    reqs = _requests(pic)
    order = list(range(len(reqs)))
    alone, _ = _serve(ds, reqs, order, together=False, n_streams=2, max_batch=8)
    mix, res = _serve_batched(ds, pic, reqs, n_streams=1, max_batch=8)
    assert max(r["batch_size"] for r in res.values()) > 1
    for i in order:
        np.testing.assert_array_equal(alone[i], mix[i], err_msg=f"request {i}")
    torch.cuda.synchronize()
    hits = 0
    for i in order:
        direct, s2 = _direct(pic, reqs[i])
        np.testing.assert_array_equal(mix[i], direct, err_msg=f"request {i} vs isaac_render")
        if i in (0, 1, 2, 7):
            hits += _check_u8_vs_oracle(mix[i], s2, reqs[i][0], reqs[i][1])
    assert hits > 500
    assert alone[4][..., 3].max() == 0   # the camera looking away sees background only


def test_alone_equals_mix_packed_bf16(cuda_ok, pic):
    ds = isaac.DeviceScene(pic)
    pv = ds.pack("bf16")
    reqs = _requests(pic, seed=5)
    order = list(range(len(reqs)))
    alone, _ = _serve(pv, reqs, order, together=False, n_streams=1, max_batch=4)
    mix, res = _serve_batched(pv, pic, reqs, n_streams=3, max_batch=3)
    assert max(r["batch_size"] for r in res.values()) > 1
    for i in order:
        np.testing.assert_array_equal(alone[i], mix[i], err_msg=f"request {i}")
        direct, _ = _direct(pic, reqs[i], packed=True)
        np.testing.assert_array_equal(mix[i], direct, err_msg=f"request {i} vs isaac_render_packed")


def test_budget_admission(cuda_ok, pic):
    """A 1 MiB budget holds about one 128x96 request (image + ray list) at a
    time; everything still finishes, in order of admission, with the same
    images as with a large budget."""
    ds = isaac.DeviceScene(pic)
    reqs = _requests(pic, seed=9)
    order = list(range(len(reqs))) * 2
    reqs2 = [reqs[i] for i in order]
    small, res_s = _serve(ds, reqs2, list(range(len(reqs2))), together=True, budget=1 << 20,
                          n_streams=2, max_batch=16)
    big, res_b = _serve(ds, reqs2, list(range(len(reqs2))), together=True, budget=64 << 20,
                        n_streams=2, max_batch=16)
    for i in range(len(reqs2)):
        np.testing.assert_array_equal(small[i], big[i])
    assert max(r["batch_size"] for r in res_s.values()) < max(r["batch_size"] for r in res_b.values())
    launches = sorted(res_s.values(), key=lambda r: r["t_launch"])
    assert all(r["t_submit"] <= r["t_launch"] <= r["t_done"] for r in launches)


def test_submit_rejections(cuda_ok, pic):
    import torch
    ds = isaac.DeviceScene(pic)
    mv, proj = synth.orbit_camera(pic.n, 64, 48, 0.3, 0.2)
    with isaac.Server(ds, budget=1 << 20, n_streams=1, max_batch=4) as srv:
        big = _pinned(1024, 1024)           # 4 MiB image: over the 1 MiB budget
        with pytest.raises(isaac.IsaacError) as e:
            srv.submit(mv, proj, 1024, 1024, big)
        assert e.value.code == isaac.ENOMEM
        pageable = torch.zeros((48, 64, 4), dtype=torch.uint8)
        with pytest.raises(isaac.IsaacError) as e:
            srv.submit(mv, proj, 64, 48, pageable)
        assert e.value.code == isaac.EINVAL
        bad = np.full((len(pic.sources), 256, 4), np.nan, np.float32)
        with pytest.raises(isaac.IsaacError) as e:
            srv.submit(mv, proj, 64, 48, _pinned(64, 48), luts=bad)
        assert e.value.code == isaac.EINVAL
        dev_out = torch.zeros((48, 64, 4), dtype=torch.uint8, device="cuda")
        srv.submit(mv, proj, 64, 48, dev_out)
        (r,) = srv.drain()
        assert r["status"] == 0
        direct, _ = _direct(pic, (mv, proj, 64, 48, None, None))
        np.testing.assert_array_equal(dev_out.cpu().numpy(), direct)
        assert srv.outstanding() == 0


def test_requests_on_two_streams_overlap_on_the_device(cuda_ok):
    """Two 1080p requests submitted together to a server with two streams and
    batches of one: they run as two batches on different streams whose
    device-clock intervals (CUDA events around each batch) overlap, and each
    image is bitwise the one the request gets when it is served alone.

    "Together" means the second request is queued while the first is still on
    the GPU (a few ms).  The submits are two host calls, so a pause of the
    host thread between them (a garbage collection in a long test process)
    can let the first batch finish first; the second then reuses its stream,
    which is correct serving but not this case.  The collector is off across
    the submits and the case gets up to three attempts."""
    import gc
    sc = small_pic_scene(n=48, guard=2, width=64, height=64, seed=31, dist_factor=1.0)
    ds = isaac.DeviceScene(sc)
    reqs = []
    for k in range(2):
        mv, proj = synth.orbit_camera(sc.n, 1920, 1080, 0.4 + 1.3 * k, 0.2, dist_factor=0.9)
        reqs.append((np.asarray(mv, np.float64), np.asarray(proj, np.float64), 1920, 1080, None, None))
    for attempt in range(3):
        gc.collect()
        gc.disable()
        try:
            together, res = _serve(ds, reqs, [0, 1], True, n_streams=2, max_batch=1)
        finally:
            gc.enable()
        a, b = res[0], res[1]
        assert a["batch_size"] == 1 and b["batch_size"] == 1, (a, b)
        if a["stream"] != b["stream"]:
            break
    assert a["stream"] != b["stream"], (a, b)
    assert 0.0 <= a["t_gpu_start"] < a["t_gpu_end"] and 0.0 <= b["t_gpu_start"] < b["t_gpu_end"]
    assert max(a["t_gpu_start"], b["t_gpu_start"]) < min(a["t_gpu_end"], b["t_gpu_end"]), (a, b)
    for i in range(2):
        alone, _ = _serve(ds, reqs, [i], False, n_streams=2, max_batch=1)
        np.testing.assert_array_equal(together[i], alone[i])


def test_host_side_faults(cuda_ok, pic):
    """Faults injected on the host, none on the GPU: a poll that waits on an
    empty server times out with no result; a steering update with a malformed
    functor chain is refused at submit and leaves the queue as it was; a
    server destroyed with requests still queued finishes them and returns
    (their results are dropped), and a new server then serves normally."""
    import time
    ds = isaac.DeviceScene(pic)
    mv, proj = synth.orbit_camera(pic.n, 64, 48, 0.3, 0.2)
    with isaac.Server(ds, budget=8 << 20, n_streams=2, max_batch=4) as srv:
        t0 = time.perf_counter()
        assert srv.poll(wait=0.05) == []
        assert 0.04 <= time.perf_counter() - t0 < 5.0
        assert srv.outstanding() == 0
        bad = [list(c) for c in pic.chains]
        bad[0] = [("pow", (0.5, 1.0))]                     # pow takes one argument
        with pytest.raises(isaac.IsaacError) as e:
            srv.submit(mv, proj, 64, 48, _pinned(64, 48), chains=bad)
        assert e.value.code == isaac.EINVAL
        assert srv.outstanding() == 0
        out = _pinned(64, 48)
        srv.submit(mv, proj, 64, 48, out)
        (r,) = srv.drain()
        assert r["status"] == 0
    srv = isaac.Server(ds, budget=8 << 20, n_streams=1, max_batch=1)
    outs = [_pinned(64, 48) for _ in range(6)]
    for o in outs:
        srv.submit(mv, proj, 64, 48, o)
    srv.close()                                              # six queued, none polled
    with isaac.Server(ds, budget=8 << 20, n_streams=2, max_batch=4) as srv2:
        again = _pinned(64, 48)
        srv2.submit(mv, proj, 64, 48, again)
        (r,) = srv2.drain()
        assert r["status"] == 0
    direct, _ = _direct(pic, (mv, proj, 64, 48, None, None))
    np.testing.assert_array_equal(again.numpy(), direct)
    np.testing.assert_array_equal(out.numpy(), direct)
