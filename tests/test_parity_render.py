"""GPU parity: isaac_render (CUDA, through the C ABI) against the FP64 oracle,
element by element on the same seeded inputs."""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_1611_09048_b300 import isaac, synth
from parity_util import TOL_F32, assert_parity, compare
from scenes_util import const_lut, make_scene, ortho_down_z, small_pic_scene

pytestmark = pytest.mark.gpu


def _gpu(scene, **kw):
    import torch
    ds = isaac.DeviceScene(scene)
    out, f32, ns = ds.render(want_f32=True, want_nsamp=True, **kw)
    torch.cuda.synchronize()
    return out.cpu().numpy(), f32.cpu().numpy(), ns.cpu().numpy()


def _check(scene, what, max_excluded=1e-3, **cmp):
    g8, g32, gns = _gpu(scene)
    r = oracle.render(scene)
    rep = compare(g32, g8, gns, r, interp=scene.interp, **cmp)
    assert_parity(rep, max_excluded, what)
    return rep, r, (g8, g32, gns)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_blobs_64_full_frame(cuda_ok, seed):
    """One scalar 64^3 field of Gaussian blobs, 256x256, trilinear, step 0.5,
    termination at 0.99, black background."""
    sc = synth.scene_blobs(64, 256, 256, seed=seed)
    rep, r, _ = _check(sc, f"blobs seed {seed}")
    assert rep.hit > 1000


@pytest.mark.parametrize("layout", ["aos", "soa"])
@pytest.mark.parametrize("dist", [2.0, 1.0, 0.45])
def test_pic_small(cuda_ok, layout, dist):
    """E, B (3 components) and density with guards, functor chains, three
    LUTs, weights, a clip plane; AoS and component-plane layouts; far, near
    and inside-the-box cameras (the last covers the whole screen)."""
    sc = small_pic_scene(n=24, guard=2, width=53, height=37, seed=3, layout=layout,
                         dist_factor=dist)
    rep, _, _ = _check(sc, f"pic {layout} {dist}")
    assert rep.hit > 50


def test_pic_nearest(cuda_ok):
    sc = small_pic_scene(n=24, guard=2, width=64, height=48, seed=4, dist_factor=1.0)
    sc.interp = 0
    # nearest-cell sampling flips cells where FP32 positions sit within
    # rounding of a boundary; those pixels are excluded and counted
    rep, _, _ = _check(sc, "nearest", max_excluded=0.2)
    assert rep.hit - rep.excluded > 200


def test_generic_kernel_four_sources_mixed_guards(cuda_ok):
    """Four sources (f_dim 2, 4, 1, 3), one without guards, run the generic
    kernel (run-time f_dim, per-source border handling)."""
    rng = np.random.default_rng(11)
    n = (20, 18, 22)
    g = [1, 0, 2, 1]
    fd = [2, 4, 1, 3]
    fields = []
    for gi, f in zip(g, fd):
        shape = tuple(k + 2 * gi for k in n[::-1]) + ((f,) if f > 1 else ())
        fields.append(rng.uniform(-1, 1, shape).astype(np.float32))
    srcs = [synth.source_from_zyx(fl, gi) for fl, gi in zip(fields, g)]
    chains = [[("length",), ("mul", (0.6,))], [("mul", (0.5, 1.0, 0.25, 2.0)), ("sum",),
                                                 ("add", (0.5,))],
              [("add", (1.0,)), ("pow", (1.5,)), ("mul", (0.3,))], [("pow", (2.0, 1.0, 0.5)), ("sum",), ("log",), ("add", (1.0,))]]
    luts = np.stack([synth.lut_from_points(40 + i, alpha_max=0.08) for i in range(4)])
    mv, proj = synth.random_orbit_camera(n, 61, 47, seed=9, dist_factor=1.2)
    sc = synth.Scene(n=n, sources=srcs, chains=chains, luts=luts,
                     weights=np.array([0.3, 0.3, 0.2, 0.2], np.float32), modelview=mv,
                     projection=proj, width=61, height=47, clip=[(0.3, -0.5, 0.2, 3.0)])
    rep, _, _ = _check(sc, "generic 4 sources")
    assert rep.hit > 300


def test_disabled_source_poisoned_on_gpu(cuda_ok):
    sc = small_pic_scene(dist_factor=1.0)
    sc.active_mask = 0b101
    sc.sources[1].data = np.full_like(sc.sources[1].data, np.nan)
    rep, _, _ = _check(sc, "mask 101 with NaN in the disabled source")
    assert rep.hit > 100


def test_single_active_of_three(cuda_ok):
    sc = small_pic_scene(dist_factor=1.0)
    sc.active_mask = 0b010
    _check(sc, "mask 010")


def test_domain_split_on_gpu(cuda_ok):
    """Two halves rendered separately on the GPU on the same global sample
    grid, over-composited, equal the oracle's whole-volume image."""
    n, g = 20, 2
    E, B, rho = synth.pic_fields(n, g, seed=5)
    whole = synth.scene_pic(n=n, guard=g, width=40, height=32, seed=5, fields=(E, B, rho),
                            dist_factor=1.0)
    whole.term = 2.0
    ref = oracle.render(whole)
    parts = []
    for lo in (0, n // 2):
        part = synth.scene_pic(n=n, guard=g, width=40, height=32, seed=5, fields=(E, B, rho),
                               dist_factor=1.0)
        part.term = 2.0
        part.global_n = (n, n, n)
        part.off = (lo, 0, 0)
        part.n = (n // 2, n, n)
        for s in part.sources:
            s.offset = s.offset + lo * s.strides[0]
        g8, g32, gns = _gpu(part)
        po = oracle.render(part)
        assert_parity(compare(g32, g8, gns, po), 1e-3, f"half at {lo}")
        parts.append((g32.astype(np.float64), po["kfirst"]))
    first0 = (parts[0][1] >= 0) & ((parts[1][1] < 0) | (parts[0][1] < parts[1][1]))
    f = np.where(first0[..., None], parts[0][0], parts[1][0])
    b = np.where(first0[..., None], parts[1][0], parts[0][0])
    comp = f + (1 - f[..., 3:4]) * b
    assert np.abs(comp - ref["rgba"]).max() <= 2 * TOL_F32


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_far_camera_deep_domain_split(cuda_ok, seed):
    """Large coordinates for the float-float ray setup: a 24 x 20 x 16 local box
    deep inside a 4096 x 3000 x 2048 global volume, seen from ~6000 voxels
    away through a 0.5-degree field of view, so ray parameters are ~1e4 voxels
    and the first sample index counts from a global entry thousands of voxels
    before the local box.  With termination off, every pixel's sample count
    and colour must match the oracle (near-ties excluded)."""
    rng = np.random.default_rng(seed)
    n, g = (24, 20, 16), 1
    gn, off = (4096, 3000, 2048), (2500, 1200, 900)
    f = (0.2 + 0.6 * rng.random((n[2] + 2 * g, n[1] + 2 * g, n[0] + 2 * g))).astype(np.float32)
    centre = np.asarray(off, np.float64) + np.asarray(n) / 2.0 - np.asarray(gn) / 2.0
    d = rng.normal(size=3)
    d /= np.linalg.norm(d)
    up = (0.0, 1.0, 0.0) if abs(d[1]) < 0.9 else (1.0, 0.0, 0.0)
    W, H = 64, 48
    cam = (synth.look_at(centre + 6000.0 * d, centre, up), synth.perspective(0.5, W / H, 5000.0, 7000.0))
    sc = make_scene([f], [[]], [synth.lut_from_points(30 + seed, alpha_max=0.2)], [1.0], n, cam,
                    W, H, guard=g)
    sc.global_n, sc.off, sc.term = gn, off, 2.0
    g8, g32, gns = _gpu(sc)
    r = oracle.render(sc)
    rep = compare(g32, g8, gns, r)
    assert_parity(rep, 1e-3, f"far camera, seed {seed}")
    assert rep.hit > 300
    assert r["kfirst"].max() > 1000             # samples counted from the far global entry


def test_edge_cases(cuda_ok):
    base = small_pic_scene(n=16, guard=1, width=37, height=23, dist_factor=1.0)
    # ragged image size, 1x1 image, a single huge step, termination disabled
    for kw in ({}, {"width": 1, "height": 1}, {"step": 40.0}, {"term": 2.0},
               {"bg": (0.2, 0.4, 0.6, 1.0)}):
        sc = dataclasses.replace(base, **kw)
        _check(sc, f"edge {kw}")
    # no active source: background only
    sc = dataclasses.replace(base, active_mask=0, bg=(0.1, 0.2, 0.3, 0.5))
    g8, g32, gns = _gpu(sc)
    assert np.all(gns == 0)
    np.testing.assert_allclose(g32, np.broadcast_to(np.float32([0.1, 0.2, 0.3, 0.5]), g32.shape))
    # camera looking away from the volume: every pixel misses
    mv = synth.look_at((0.0, 0.0, 60.0), (0.0, 0.0, 120.0), (0.0, 1.0, 0.0))
    sc = dataclasses.replace(base, modelview=mv)
    g8, g32, gns = _gpu(sc)
    assert np.all(gns == 0) and np.all(g8 == 0)


def test_constant_slab_closed_form_on_gpu(cuda_ok):
    """The closed form A = 1 - (1-a)^n checked directly on the GPU output."""
    n = (8, 8, 8)
    a = float(np.float32(0.05))
    field = np.full(n[::-1], 42.0, np.float32)
    sc = make_scene([field], [[("mul", (1.0 / 84.0,))]], [const_lut((0.25, 0.5, 0.75, a))], [1.0],
                    n, ortho_down_z(n, 8, 8), 8, 8, term=2.0, step=0.5,
                    clip=[(0.0, 0.0, 1.0, -2.3)])
    g8, g32, gns = _gpu(sc)
    assert np.all(gns == 12)
    np.testing.assert_allclose(g32[..., 3], 1 - (1 - a) ** 12, rtol=0, atol=1e-6)


@pytest.mark.parametrize("fmt", [None, "bf16", "e4m3"])
@pytest.mark.parametrize("layout", ["aos", "soa"])
def test_lanes_per_ray_do_not_change_the_image(cuda_ok, fmt, layout):
    """1, 2, 4, 8 or 16 threads per ray composite the same samples in the same
    order: the images (and sample counts) are bit-identical."""
    import torch
    sc = small_pic_scene(n=24, guard=2, width=70, height=52, seed=8, layout=layout,
                         dist_factor=1.0)
    ds = isaac.DeviceScene(sc)
    target = ds if fmt is None else ds.pack(fmt)
    outs = [target.render(want_f32=True, want_nsamp=True, lanes=rl) for rl in (1, 2, 4, 8, 16)]
    torch.cuda.synchronize()
    for o in outs[1:]:
        for a, b in zip(outs[0], o):
            assert torch.equal(a, b)


def test_pic_256_1080p_sampled(cuda_ok):
    """PIConGPU-shaped frame at full size (256^3 + 4 guards, 1920x1080):
    the whole frame on the GPU, the oracle on sampled pixels."""
    sc = synth.scene_pic(n=256, guard=4, width=1920, height=1080, seed=0)
    g8, g32, gns = _gpu(sc)
    rng = np.random.default_rng(0)
    hit = np.flatnonzero(gns.reshape(-1) > 0)
    assert hit.size > 50000
    pix = np.concatenate([rng.choice(hit, 2500, replace=False),
                          rng.choice(gns.size, 500, replace=False)])
    r = oracle.render(sc, pixels=pix)
    rep = compare(g32, g8, gns, r, sel=pix)
    assert_parity(rep, 2e-3, "pic 256 1080p sampled")


@pytest.mark.parametrize("clip", [
    [(1.0, 0.0, 0.0, -16.0), (0.0, 0.0, -1.0, 9.0)],          # keep x >= 16 and z <= 9
    [(-2.0, 0.0, 0.0, 10.0), (0.3, -0.5, 0.2, 3.0)],          # keep x <= 5, plus an oblique plane
    [(0.0, 1.0, 0.0, -24.0)],                                 # keep y >= 24: one face only
    [(0.0, 0.0, 1.0, -40.0)],                                 # keep z >= 40: nothing
])
def test_axis_aligned_clip_planes_shrink_the_rectangle(cuda_ok, clip):
    """Axis-aligned clip planes cut the box whose projection bounds the pixels
    that get a ray; every frame still equals the oracle's, pixel for pixel
    (the pixels cut away are background on both sides)."""
    sc = dataclasses.replace(small_pic_scene(n=24, guard=2, width=64, height=48, seed=6,
                                             dist_factor=1.3), clip=clip)
    rep, r, (g8, g32, gns) = _check(sc, f"clip {clip}")
    if clip[0][3] <= -24.0:
        assert rep.hit == 0 and np.all(gns == 0)
    else:
        assert rep.hit > 100


@pytest.fixture(scope="module")
def pic512_device():
    """The bench's headline workload: 512^3 + 4 guards E/B/rho, 1920x1080."""
    sc = synth.scene_pic(n=512, guard=4, width=1920, height=1080, seed=0)
    return sc, isaac.DeviceScene(sc)


@pytest.mark.parametrize("cam", [3, 20])
def test_pic_512_1080p_sampled_bench_cameras(cuda_ok, pic512_device, cam):
    """Full size, in the launch configuration the bench times (default lanes
    per ray, one of its 32 Fibonacci cameras): the whole frame on the GPU,
    the oracle on sampled pixels."""
    import torch
    sc, ds = pic512_device
    mv, proj = synth.fibonacci_cameras((512, 512, 512), 1920, 1080, count=32, seed=0)[cam]
    out, f32, ns = ds.render(mv, proj, want_f32=True, want_nsamp=True)
    torch.cuda.synchronize()
    g8, g32, gns = out.cpu().numpy(), f32.cpu().numpy(), ns.cpu().numpy()
    rng = np.random.default_rng(cam)
    hit = np.flatnonzero(gns.reshape(-1) > 0)
    assert hit.size > 50000
    pix = np.concatenate([rng.choice(hit, 2500, replace=False),
                          rng.choice(gns.size, 500, replace=False)])
    r = oracle.render(sc.with_camera(mv, proj), pixels=pix)
    rep = compare(g32, g8, gns, r, sel=pix)
    assert_parity(rep, 2e-3, f"pic 512 1080p camera {cam}")


def test_pic_512_reduced_precision_error_32_cameras(cuda_ok, pic512_device):
    """The reduced-precision copies at full size over the bench's 32 cameras
    on the sphere: per-channel max and mean abs error against the FP64 oracle
    on the original float32 fields (400 hit pixels per camera).  16-bit
    storage stays within 2e-3 before quantisation; every format within 1 LSB
    mean after it."""
    import json
    import torch
    sc, ds = pic512_device
    cams = synth.fibonacci_cameras((512, 512, 512), 1920, 1080, count=32, seed=0)
    packs = {fmt: ds.pack(fmt) for fmt in ("bf16", "f16", "e4m3")}
    errs = {fmt: [] for fmt in packs}
    lsbs = {fmt: [] for fmt in packs}
    rng = np.random.default_rng(512)
    for ci, (mv, proj) in enumerate(cams):
        outs = {}
        for fmt, pv in packs.items():
            o8, o32, ons = pv.render(mv, proj, want_f32=True, want_nsamp=True)
            outs[fmt] = (o8, o32, ons)
        torch.cuda.synchronize()
        ns0 = outs["bf16"][2].cpu().numpy().reshape(-1)
        hit = np.flatnonzero(ns0 > 0)
        pix = rng.choice(hit, min(400, hit.size), replace=False)
        ref = oracle.render(sc.with_camera(mv, proj), pixels=pix)
        keep = ref["nsamp"] > 0
        for fmt, (o8, o32, _) in outs.items():
            g = o32.cpu().numpy().reshape(-1, 4)[pix].astype(np.float64)
            e = np.minimum(np.abs(g - ref["rgba"]), np.abs(g - ref["rgba_alt"]))[keep]
            l8 = o8.cpu().numpy().reshape(-1, 4)[pix].astype(np.int64)
            errs[fmt].append(e)
            lsbs[fmt].append(np.abs(l8 - ref["rgba8"].astype(np.int64))[keep])
    report = {}
    for fmt in packs:
        e = np.concatenate(errs[fmt])
        lsb = np.concatenate(lsbs[fmt])
        report[fmt] = {"pixels": int(e.shape[0]), "max_abs_rgba": e.max(0).round(6).tolist(),
                       "mean_abs_rgba": e.mean(0).round(7).tolist(), "mean_lsb": float(lsb.mean())}
        assert lsb.mean() <= 1.0, (fmt, report[fmt])
        if fmt != "e4m3":
            assert e.max() <= 2e-3, (fmt, report[fmt])
    print("reduced-precision error vs FP64 oracle, pic512 1080p, 32 cameras:", json.dumps(report))


@pytest.mark.parametrize("chains", [
    [[("length",), ("mul", (0.5,))], [("log",)], [("mul", (2.0,)), ("add", (-0.3,))],
     [("length",), ("log",), ("mul", (0.1,)), ("add", (0.6,))]],
    [[], [("length",)], [("log",), ("mul", (0.2,)), ("add", (0.5,))],
     [("length",), ("mul", (0.4,)), ("add", (0.1,)), ("pow", (0.5,))]],
])
def test_every_chain_shape_against_oracle(cuda_ok, chains):
    """Each folded chain shape the kernels run as straight-line code (identity,
    affine, length, length+affine, length+affine+sqrt, log, log+affine) and a
    chain they interpret op by op, on four sources of one frame."""
    from scenes_util import make_scene
    n = (22, 18, 20)
    rng = np.random.default_rng(31)
    fields = [rng.random((n[2], n[1], n[0], 3), np.float32) * 0.6,
              rng.random((n[2], n[1], n[0]), np.float32) + 0.05,
              rng.random((n[2], n[1], n[0]), np.float32),
              rng.random((n[2], n[1], n[0], 2), np.float32)]
    if chains[0] == []:
        fields[0] = fields[0][..., 0].copy()
        fields[1] = rng.random((n[2], n[1], n[0], 3), np.float32)
        fields[2] = fields[2] + 0.05
        fields[3] = rng.random((n[2], n[1], n[0], 3), np.float32)
    cams = synth.random_orbit_camera(n, 56, 44, seed=12, dist_factor=1.3)
    luts = [synth.lut_from_points(200 + i, alpha_max=0.15) for i in range(4)]
    sc = make_scene(fields, chains, luts, [0.3, 0.3, 0.2, 0.2], n, cams, 56, 44)
    rep, _, _ = _check(sc, f"chains {chains}")
    assert rep.hit > 300


def test_prepared_frame_reads_the_given_lut_buffer(cuda_ok):
    """A frame prepared with another LUT buffer reads that buffer: a copy of the
    scene's LUTs gives the same image bit for bit, an all-transparent table the
    background alone (the binding only passes the pointer)."""
    import torch
    sc = small_pic_scene()
    ds = isaac.DeviceScene(sc)
    out = torch.empty((sc.height, sc.width, 4), dtype=torch.uint8, device="cuda")
    ds.launch(ds.prepare(out=out))
    torch.cuda.synchronize()
    ref = out.clone()
    assert (ref[..., 3] > 0).sum() > 100
    same = ds.luts.clone()
    ds.launch(ds.prepare(out=out, luts=same))
    torch.cuda.synchronize()
    assert torch.equal(out, ref)
    clear = torch.zeros_like(ds.luts)
    ds.launch(ds.prepare(out=out, luts=clear))
    torch.cuda.synchronize()
    bg = np.clip(np.floor(255.0 * np.asarray(sc.bg, np.float32) + 0.5), 0, 255).astype(np.uint8)
    assert np.all(out.cpu().numpy() == bg)
    with pytest.raises(ValueError):
        ds.prepare(out=out, luts=torch.zeros(7, device="cuda"))
