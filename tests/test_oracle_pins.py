"""Pins of the FP64 oracle against closed forms, brute force and invariants.

None of these compares the oracle with itself: every expected value comes from
the paper's worked examples, from a closed form, from a library routine on a
special case, or from a brute-force evaluation that contains no ray code.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_1611_09048_b300 import synth
from scenes_util import const_lut, make_scene, ortho_down_z, ramp_lut, small_pic_scene

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------- camera

def test_invert4_matches_lapack():
    rng = np.random.default_rng(0)
    mats = [rng.standard_normal((4, 4)) + 4 * np.eye(4) for _ in range(5)]
    mv, proj = synth.random_orbit_camera((64, 64, 64), 256, 256, seed=7)
    mats.append((proj.reshape(4, 4).T @ mv.reshape(4, 4).T))
    # a matrix whose first pivot must be swapped
    mats.append(np.array([[0.0, 2, 0, 0], [1, 0, 0, 0], [0, 0, 3, 1], [0, 0, 0, 1]]))
    for m in mats:
        cm = m.T.reshape(16)                      # column-major
        inv = oracle.invert4(cm).reshape(4, 4).T  # back to row-major
        np.testing.assert_allclose(inv, np.linalg.inv(m), rtol=1e-12, atol=1e-12)


# ---------------------------------------------------------------- functors

def test_functor_chains_golden():
    with open(os.path.join(GOLDEN, "functor_chains.json")) as f:
        g = json.load(f)
    for case in g["cases"]:
        chain = [tuple([c[0]] + ([tuple(c[1])] if len(c) > 1 else [])) for c in case["chain"]]
        got = oracle.chain_eval(chain, case["input"])
        assert got == pytest.approx(case["expected"], rel=1e-14, abs=1e-14), case["what"]
    for case in g["invalid"]:
        chain = [tuple([c[0]] + ([tuple(c[1])] if len(c) > 1 else [])) for c in case["chain"]]
        with pytest.raises(ValueError):
            oracle.chain_eval(chain, [1.0] * case["dim"])


def test_classify_is_linear_between_entries():
    rng = np.random.default_rng(1)
    lut = rng.uniform(0, 1, (256, 4)).astype(np.float32)
    for j in (0, 1, 17, 128, 254, 255):
        np.testing.assert_allclose(oracle.classify(lut, j / 255.0), lut[j], rtol=0, atol=1e-12)
    for x in rng.uniform(0, 1, 20):
        want = [np.interp(x * 255.0, np.arange(256), lut[:, c].astype(np.float64)) for c in range(4)]
        np.testing.assert_allclose(oracle.classify(lut, x), want, rtol=0, atol=1e-12)
    np.testing.assert_allclose(oracle.classify(lut, -3.0), lut[0], atol=0)
    np.testing.assert_allclose(oracle.classify(lut, 7.0), lut[255], atol=0)
    np.testing.assert_allclose(oracle.classify(lut, float("nan")), lut[0], atol=0)


# ------------------------------------------------------ compositing closed form

@pytest.mark.parametrize("a,step,clip_z,term", [
    (0.05, 0.5, 2.3, 2.0),     # n = #{k : 0.5 k < 5.7} = 12
    (0.2, 0.3, 0.0, 2.0),      # no clip: n = ceil(8 / 0.3) = 27
    (0.2, 0.3, 0.0, 0.99),     # termination: n = ceil(ln 0.01 / ln 0.8) = 21
    (0.013, 0.25, 1.1, 0.9),
])
def test_constant_source_slab(a, step, clip_z, term):
    """Sec. 3.2's homogeneous source (42 everywhere) with one LUT colour of
    opacity a: the ray composites n equal samples, so A = 1 - (1 - a)^n and
    C = rgb * A, n counted from the slab thickness or from the threshold."""
    n = (8, 8, 8)
    rgb = (0.25, 0.5, 0.75)
    field = np.full(n[::-1], 42.0, np.float32)
    sc = make_scene([field], [[("mul", (1.0 / 84.0,))]], [const_lut(rgb + (a,))], [1.0], n,
                    ortho_down_z(n, 8, 8), 8, 8, term=term, step=step,
                    clip=[(0.0, 0.0, 1.0, -clip_z)] if clip_z else [])
    r = oracle.render(sc)
    a = float(np.float32(a))                     # the LUT stores float32
    rgb = tuple(float(np.float32(c)) for c in rgb)
    thickness = n[2] - clip_z
    n_slab = math.ceil(thickness / step)
    n_term = math.ceil(math.log(1.0 - term) / math.log(1.0 - a)) if term < 1 else n_slab
    ns = min(n_slab, n_term)
    A = 1.0 - (1.0 - a) ** ns
    assert np.all(r["nsamp"] == ns)
    # entry not raised by a plane -> no entry decision; exit margin is the
    # distance of thickness/step to the nearest integer
    assert np.all(r["margin"][..., 0] == oracle.oracle.INF)
    x = thickness / step
    np.testing.assert_allclose(r["margin"][..., 1], abs(x - round(x)), atol=1e-9)
    np.testing.assert_allclose(r["rgba"][..., 3], A, rtol=0, atol=1e-13)
    for c in range(3):
        np.testing.assert_allclose(r["rgba"][..., c], rgb[c] * A, rtol=0, atol=1e-13)


@pytest.mark.parametrize("step,top", [(0.5, 5.7), (0.3, 6.0), (0.25, 1.3)])
def test_clip_plane_raises_entry_on_global_grid(step, top):
    """Keep z <= top (normal (0,0,-1)): rays travelling -z enter the box at
    z = 8 but start sampling at the first grid point t0 + k*step past the
    plane, k = ceil((8 - top)/step); the count is #{k : 8-top <= k step < 8}."""
    n = (8, 8, 8)
    a = float(np.float32(0.05))
    field = np.full(n[::-1], 42.0, np.float32)
    sc = make_scene([field], [[("mul", (1.0 / 84.0,))]], [const_lut((1.0, 1.0, 1.0, a))], [1.0],
                    n, ortho_down_z(n, 8, 8), 8, 8, term=2.0, step=step,
                    clip=[(0.0, 0.0, -1.0, top)])
    r = oracle.render(sc)
    kf = math.ceil((8 - top) / step)
    ke = math.ceil(8 / step)
    assert np.all(r["kfirst"] == kf)
    assert np.all(r["nsamp"] == ke - kf)
    x = (8 - top) / step
    np.testing.assert_allclose(r["margin"][..., 0], abs(x - round(x)), atol=1e-9)
    np.testing.assert_allclose(r["rgba"][..., 3], 1 - (1 - a) ** (ke - kf), rtol=0, atol=1e-13)


def test_visible_span_closed_form():
    """A slab of opacity a between z = 2 and z = 5 inside an empty volume:
    rays along -z enter at z = 8, so with step 0.5 and nearest-cell sampling
    the first sample with opacity is the one at z = 4.5 (index 7) and the last
    the one at z = 2.0 (index 12)."""
    n = (8, 8, 8)
    field = np.zeros(n[::-1], np.float32)
    field[2:5] = 1.0
    lut = np.zeros((256, 4), np.float32)
    lut[128:, :] = (1.0, 1.0, 1.0, 0.1)
    sc = make_scene([field], [[]], [lut], [1.0], n, ortho_down_z(n, 8, 8), 8, 8, interp=0,
                    step=0.5, term=2.0)
    r = oracle.render(sc)
    # samples at z = 8 - 0.5k; cells 2..4 hold the slab: 4.5 (k=7) ... 2.0 (k=12)
    assert np.all(r["jspan"][..., 0] == 7) and np.all(r["jspan"][..., 1] == 12)
    sc.luts = np.zeros_like(sc.luts)
    assert np.all(oracle.render(sc)["jspan"] == -1)


def test_empty_transfer_function_gives_background():
    sc = small_pic_scene()
    sc.luts = sc.luts.copy()
    sc.luts[..., 3] = 0.0
    sc.bg = (0.1, 0.2, 0.3, 0.4)
    r = oracle.render(sc)
    assert (r["nsamp"] > 0).sum() > 100
    np.testing.assert_array_equal(r["rgba"], np.broadcast_to(np.array(sc.bg), r["rgba"].shape))


# ----------------------------------------------------------- interpolation

def _linear_field(n, guard, a, b):
    S = [k + 2 * guard for k in n]
    z, y, x = np.meshgrid(*[np.arange(s, dtype=np.float64) - guard + 0.5 for s in S[::-1]],
                          indexing="ij")
    return (a[0] * x + a[1] * y + a[2] * z + b).astype(np.float64)


def test_trilinear_reproduces_linear_field_with_guards():
    """A linear field is reproduced exactly by trilinear interpolation
    everywhere when the guards carry its continuation (Sec. 3.1 guards): the
    first sample of every ray sits on the entry face z = nz at a known x, y."""
    n = (8, 6, 5)
    a, b = (1 / 64, -1 / 128, 1 / 32), 0.25
    field = _linear_field(n, 1, a, b)
    assert np.array_equal(field.astype(np.float32).astype(np.float64), field)
    W, H = 13, 11
    sc = make_scene([field], [[]], [ramp_lut(1.0)], [1.0], n, ortho_down_z(n, W, H), W, H,
                    guard=1)
    r = oracle.render(sc)
    px, py = np.meshgrid(np.arange(W), np.arange(H))
    x = (px + 0.5) * n[0] / W
    y = n[1] - (py + 0.5) * n[1] / H
    want = a[0] * x + a[1] * y + a[2] * n[2] + b
    assert np.all(r["nsamp"] == 1)
    np.testing.assert_allclose(r["rgba"][..., 0], want, rtol=0, atol=1e-7)   # float32 LUT entries


def test_trilinear_without_guards_clamps_to_border():
    """guard = 0: indices clamp to the border cell, so the entry-face sample at
    z = nz averages cell nz-1 with itself and reads the field at nz - 1/2."""
    n = (8, 6, 5)
    a, b = (1 / 64, -1 / 128, 1 / 32), 0.25
    field = _linear_field(n, 0, a, b)
    W, H = 13, 11
    sc = make_scene([field], [[]], [ramp_lut(1.0)], [1.0], n, ortho_down_z(n, W, H), W, H)
    r = oracle.render(sc)
    px, py = np.meshgrid(np.arange(W), np.arange(H))
    x = np.clip((px + 0.5) * n[0] / W, 0.5, n[0] - 0.5)
    y = np.clip(n[1] - (py + 0.5) * n[1] / H, 0.5, n[1] - 0.5)
    want = a[0] * x + a[1] * y + a[2] * (n[2] - 0.5) + b
    np.testing.assert_allclose(r["rgba"][..., 0], want, rtol=0, atol=1e-7)


def test_camera_centre_ray_enters_face_centre():
    """Perspective camera on the +z axis: the centre pixel's ray enters the
    box at the centre of the face z = nz and crosses a chord of length nz."""
    n = (10, 10, 10)
    a, b = (0.0, 0.0, 1 / 32), 0.125
    field = _linear_field(n, 1, a, b)
    W = H = 9
    mv = synth.look_at((0.0, 0.0, 40.0), (0.0, 0.0, 0.0), (0.0, 1.0, 0.0))
    proj = synth.perspective(30.0, 1.0, 0.1, 100.0)
    sc = make_scene([field], [[]], [ramp_lut(1 / 128)], [1.0], n, (mv, proj), W, H, guard=1,
                    term=2.0, step=0.5)
    r = oracle.render(sc)
    c = r["rgba"][4, 4]
    assert r["nsamp"][4, 4] == 20 and r["kfirst"][4, 4] == 0
    # closed form of the composite over a linear red ramp with constant alpha
    alphas = np.full(20, 1 / 128)
    z = 10.0 - 0.5 * np.arange(20)
    T = np.concatenate([[1.0], np.cumprod(1 - alphas)[:-1]])
    # red entries are float32(j/255): the ramp reproduces x to ~1e-8
    np.testing.assert_allclose(c[0], np.sum(T * alphas * (a[2] * z + b)), rtol=0, atol=1e-8)
    np.testing.assert_allclose(c[3], 1 - (1 - 1 / 128) ** 20, rtol=0, atol=1e-13)


# ------------------------------------------------------------ brute force

def _composite(rgba_samples, term=2.0):
    """Closed-form front-to-back composite: C = sum_k T_k a_k rgb_k with
    T_k = prod_{j<k} (1 - a_j), A = 1 - prod (1 - a_k)."""
    a = np.clip(rgba_samples[:, 3], 0, 1)
    T = np.concatenate([[1.0], np.cumprod(1 - a)[:-1]])
    A_run = 1 - np.cumprod(1 - a)
    stop = np.nonzero(A_run >= term)[0]
    m = stop[0] + 1 if stop.size else len(a)
    C = (T[:m, None] * a[:m, None] * rgba_samples[:m, :3]).sum(0)
    return np.concatenate([C, [A_run[m - 1]]]), m


def _np_classify(lut, x):
    x = np.clip(np.nan_to_num(x, nan=0.0), 0, 1)
    return np.stack([np.interp(255 * x, np.arange(256), lut[:, c].astype(np.float64))
                     for c in range(4)], axis=-1)


@pytest.mark.parametrize("interp", [0, 1])
@pytest.mark.parametrize("n", [(4, 4, 4), (6, 5, 7), (8, 8, 8)])
def test_bruteforce_tiny_volume_columns(interp, n):
    """Whole pipeline on tiny volumes: orthographic rays along -z through
    voxel centres.  The expected pixel is computed column by column with no
    ray code: nearest mode samples cells floor(nz - 0.37k), trilinear mode with
    step 1 averages cells nz-k-1 and nz-k (clamped), two sources (a vector
    field through length|mul and a scalar through mul|add), weights, LUTs."""
    rng = np.random.default_rng(sum(n) + 10 * interp)
    nx, ny, nz = n
    vec = rng.uniform(-1, 1, (nz, ny, nx, 3)).astype(np.float32)
    sca = rng.uniform(0, 2, (nz, ny, nx)).astype(np.float32)
    luts = [synth.lut_from_points(5, alpha_max=0.3), synth.lut_from_points(6, alpha_max=0.3)]
    chains = [[("length",), ("mul", (0.5,))], [("mul", (0.4,)), ("add", (0.1,))]]
    w = [0.6, 0.5]
    step = 0.37 if interp == 0 else 1.0
    sc = make_scene([vec, sca], chains, luts, w, n, ortho_down_z(n, nx, ny), nx, ny,
                    step=step, interp=interp, term=0.95)
    r = oracle.render(sc)
    w = [float(np.float32(x)) for x in w]       # the scene stores float32 weights
    ks = np.arange(int(math.ceil(nz / step)))
    if interp == 0:
        # nearest-cell margin: distance of a sample to the closest boundary
        # between two interior cells (x, y sit on cell centres: 0.5)
        pz = nz - step * ks
        near_int = np.floor(pz + 0.5)
        inner = (near_int > 0) & (near_int < nz)
        want_m = min(0.5, float(np.abs(pz - near_int)[inner].min()))
        stopped = r["nsamp"] < len(ks)
        np.testing.assert_allclose(r["margin"][..., 3][~stopped], want_m, rtol=0, atol=1e-9)
    else:
        assert np.all(r["margin"][..., 3] == oracle.oracle.INF)
    for py in range(ny):
        iy = ny - 1 - py
        for px in range(nx):
            if interp == 0:
                cells = np.minimum(np.floor(nz - step * ks).astype(int), nz - 1)
                vv = vec[cells, iy, px].astype(np.float64)
                ss = sca[cells, iy, px].astype(np.float64)
            else:
                lo = nz - ks - 1
                hi = np.minimum(nz - ks, nz - 1)
                vv = 0.5 * (vec[lo, iy, px].astype(np.float64) + vec[hi, iy, px])
                ss = 0.5 * (sca[lo, iy, px].astype(np.float64) + sca[hi, iy, px])
            x0 = np.linalg.norm(vv, axis=1) * 0.5
            x1 = ss * 0.4 + 0.1
            samp = w[0] * _np_classify(luts[0], x0) + w[1] * _np_classify(luts[1], x1)
            want, m = _composite(samp, term=0.95)
            assert r["nsamp"][py, px] == m
            np.testing.assert_allclose(r["rgba"][py, px], want, rtol=0, atol=1e-12)


# ------------------------------------------------------------- invariants

def test_single_weight_reproduces_single_source():
    sc = small_pic_scene()
    single = make_scene([np.zeros((1, 1, 1), np.float32)], [[]], [sc.luts[0]], [1.0], sc.n,
                        (sc.modelview, sc.projection), sc.width, sc.height)
    single.sources = [sc.sources[0]]
    single.chains = [sc.chains[0]]
    single.clip = sc.clip
    sc.weights = np.array([1.0, 0.0, 0.0], np.float32)
    a = oracle.render(sc)
    b = oracle.render(single)
    np.testing.assert_array_equal(a["rgba"], b["rgba"])


def test_disabled_source_is_never_read():
    """Sec. 3.2: a deactivated source is not touched at all; NaN poison in it
    cannot change the image, which equals the image without that source."""
    sc = small_pic_scene()
    sc.active_mask = 0b101
    ref = oracle.render(sc)
    poisoned = small_pic_scene()
    poisoned.active_mask = 0b101
    poisoned.sources[1].data = np.full_like(poisoned.sources[1].data, np.nan)
    got = oracle.render(poisoned)
    np.testing.assert_array_equal(ref["rgba"], got["rgba"])
    two = small_pic_scene()
    two.sources = [two.sources[0], two.sources[2]]
    two.chains = [two.chains[0], two.chains[2]]
    two.luts = two.luts[[0, 2]]
    two.weights = two.weights[[0, 2]]
    np.testing.assert_array_equal(ref["rgba"], oracle.render(two)["rgba"])


def test_guards_only_matter_with_interpolation():
    sc = small_pic_scene(layout="soa")
    base = {i: oracle.render(dataclasses_replace(sc, interp=i))["rgba"] for i in (0, 1)}
    S = sc.n[0] + 2 * sc.sources[0].guard
    g = sc.sources[0].guard
    for s in sc.sources:
        arr = s.data.reshape((-1, S, S, S))
        mask = np.ones((S, S, S), bool)
        mask[g:S - g, g:S - g, g:S - g] = False
        arr[:, mask] = np.float32(7.5)
    after = {i: oracle.render(dataclasses_replace(sc, interp=i))["rgba"] for i in (0, 1)}
    np.testing.assert_array_equal(base[0], after[0])
    assert np.abs(base[1] - after[1]).max() > 1e-3


def dataclasses_replace(sc, **kw):
    import dataclasses
    return dataclasses.replace(sc, **kw)


def test_domain_split_composites_to_whole():
    """Sec. 3.1 / Sec. 3.4: two nodes each own half of the global volume with
    guards from the neighbour; their images, over-composited in visibility
    order, equal the image of the whole volume (same global sample grid)."""
    n, g = 20, 2
    E, B, rho = synth.pic_fields(n, g, seed=5)
    whole = synth.scene_pic(n=n, guard=g, width=40, height=32, seed=5, fields=(E, B, rho),
                            dist_factor=1.0)
    whole.term = 2.0
    ref = oracle.render(whole)
    halves = []
    for lo in (0, n // 2):
        part = synth.scene_pic(n=n, guard=g, width=40, height=32, seed=5, fields=(E, B, rho),
                               dist_factor=1.0)
        part.term = 2.0
        part.global_n = (n, n, n)
        part.off = (lo, 0, 0)
        part.n = (n // 2, n, n)
        for s in part.sources:
            s.offset = s.offset + lo * s.strides[0]
        halves.append(oracle.render(part))
    k0, k1 = halves[0]["kfirst"], halves[1]["kfirst"]
    first0 = (k0 >= 0) & ((k1 < 0) | (k0 < k1))
    f = np.where(first0[..., None], halves[0]["rgba"], halves[1]["rgba"])
    b = np.where(first0[..., None], halves[1]["rgba"], halves[0]["rgba"])
    comp = f + (1 - f[..., 3:4]) * b
    assert (ref["nsamp"] > 0).sum() > 200
    np.testing.assert_array_equal(ref["nsamp"], halves[0]["nsamp"] + halves[1]["nsamp"])
    np.testing.assert_allclose(comp, ref["rgba"], rtol=0, atol=1e-12)


def test_termination_alternative_and_margins():
    sc = small_pic_scene()
    sc.term = 2.0
    r = oracle.render(sc)
    np.testing.assert_array_equal(r["rgba"], r["rgba_alt"])
    sc.term = 0.5
    r = oracle.render(sc)
    hit = r["nsamp"] > 0
    diff = np.abs(r["rgba"] - r["rgba_alt"]).max(-1)
    # the alternative differs by at most one sample's share of the remaining transparency
    assert np.all(diff[hit] <= 1 - 0.5 + 1e-12)
    assert np.all(np.abs(r["nsamp"] - r["nsamp_alt"])[hit] >= 0)
    stopped = hit & (r["rgba"][..., 3] >= 0.5)
    assert stopped.sum() > 10
    assert np.all(r["margin"][..., 2][stopped] <= 0.5)


def test_pixel_subset_matches_full_frame():
    sc = small_pic_scene()
    full = oracle.render(sc)
    rng = np.random.default_rng(2)
    pix = rng.choice(sc.width * sc.height, 97, replace=False)
    sub = oracle.render(sc, pixels=pix)
    for k in ("rgba", "nsamp", "margin", "rgba8"):
        np.testing.assert_array_equal(sub[k], full[k].reshape((-1,) + full[k].shape[2:])[pix])


def test_quantisation_round_half_up():
    sc = make_scene([np.full((4, 4, 4), 0.5, np.float32)], [[]],
                    [const_lut((0.5 / 255 * 3, 1.0, 0.0, 1.0))], [1.0], (4, 4, 4),
                    ortho_down_z((4, 4, 4), 4, 4), 4, 4)
    r = oracle.render(sc)
    # 255 * (1.5/255) + 0.5 = 2.0 exactly -> 2; alpha 1 -> 255; 0 -> 0
    assert np.all(r["rgba8"][..., 0] == 2) and np.all(r["rgba8"][..., 1] == 255)
    assert np.all(r["rgba8"][..., 2] == 0) and np.all(r["rgba8"][..., 3] == 255)
