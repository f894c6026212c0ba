"""GPU parity where a march step has nothing to composite.

A lane group (or a long-ray window) whose samples all have opacity 0 and
finite colours leaves C and A bit for bit as they are (Sec. 3.2's front-to-back
compositing adds (1 - A) * 0 * c = +0), so the march only counts those
samples.  These cases check that against the FP64 oracle on sparse frames
(sample counts exact), and the two cases where such samples still matter: a
termination threshold <= 0 (the first sample ends the ray) and a colour that
is not finite (0 * inf is NaN, in the oracle as on the GPU).
"""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_1611_09048_b300 import isaac, synth
from parity_util import assert_parity, compare

pytestmark = pytest.mark.gpu


def _bubble(**kw):
    sc = synth.scene_bubble(64, frame=7, seed=4, width=200, height=150, dist_factor=1.1)
    return dataclasses.replace(sc, **kw)


def _render(sc, lanes=None):
    import torch
    out, f32, ns = isaac.DeviceScene(sc).render(want_f32=True, want_nsamp=True, lanes=lanes)
    torch.cuda.synchronize()
    return out.cpu().numpy(), f32.cpu().numpy(), ns.cpu().numpy()


@pytest.mark.parametrize("lanes", [1, 4, 8, 16])
def test_sparse_bubble_matches_oracle(cuda_ok, lanes):
    """The bubble's transfer function is zero below a threshold, so most
    groups of a ray's samples composite nothing."""
    sc = _bubble()
    g8, g32, gns = _render(sc, lanes)
    ref = oracle.render(sc)
    rep = compare(g32, g8, gns, ref)
    assert_parity(rep, 1e-3, f"sparse bubble, {lanes} lanes per ray")
    assert rep.hit > 5000
    assert np.all(gns[ref["nsamp"] > 0] > 0)


def test_long_ray_windows_match_oracle(cuda_ok):
    """A full-window proposal sends every ray of more than 96 samples to the
    long-ray march, whose 64-sample windows over empty space composite
    nothing: against the oracle, not only against the plain march."""
    import torch
    sc = _bubble()
    ds = isaac.DeviceScene(sc)
    grid = ds.opacity_grid(8)
    p = synth.mlp_params(0)
    for k in ("W1", "W2", "W3", "W4"):
        p[k] = np.zeros_like(p[k])
    p["b4"] = np.asarray((-30.0, 30.0, 30.0), np.float32)       # te = 0, tx = 1, sure
    model = isaac.MLPModel(isaac.pack_mlp_params(p), train=False)
    out, f32, ns = ds.render_learned(model.proposal(grid, 8, threshold=0.9, margin=2),
                                     want_f32=True, want_nsamp=True)
    torch.cuda.synchronize()
    gns = ns.cpu().numpy()
    assert int((gns > 96).sum()) > 1000
    rep = compare(f32.cpu().numpy(), out.cpu().numpy(), gns, oracle.render(sc))
    assert_parity(rep, 1e-3, "long-ray windows")


@pytest.mark.parametrize("term", [0.0, -1.0])
def test_nonpositive_threshold_ends_every_ray_at_its_first_sample(cuda_ok, term):
    sc = _bubble(term=term)
    for lanes in (1, 8):
        g8, g32, gns = _render(sc, lanes)
        ref = oracle.render(sc)
        hit = ref["nsamp"] > 0
        assert hit.sum() > 5000
        assert np.all(gns[hit] == 1) and np.all(gns[~hit] == 0)
        assert_parity(compare(g32, g8, gns, ref), 1e-3, f"term {term}, {lanes} lanes")


def test_infinite_colour_at_zero_opacity_poisons_the_pixel(cuda_ok):
    """Opacity 0 everywhere, red = +inf: every composited sample adds
    0 * inf = NaN to red, so every hit pixel's red is NaN (oracle and GPU);
    green, blue and opacity stay 0."""
    lut = np.zeros((1, 256, 4), np.float32)
    lut[..., 0] = np.inf
    sc = _bubble(luts=lut)
    ref = oracle.render(sc)
    hit = ref["nsamp"] > 0
    # pixels whose first or last sample sits on a decision tie are left out
    keep = (ref["margin"][..., 0] >= 1e-6) & (ref["margin"][..., 1] >= 1e-6)
    assert hit.sum() > 5000 and (~keep).sum() < 1e-3 * hit.sum()
    assert np.array_equal(np.isnan(ref["rgba"][..., 0]), hit)
    for lanes in (4, 16):
        g8, g32, gns = _render(sc, lanes)
        assert np.array_equal(np.isnan(g32[..., 0])[keep], hit[keep])
        assert not g32[..., 1:].any()
        np.testing.assert_array_equal(gns[keep], ref["nsamp"][keep])


@pytest.mark.parametrize("fmt", ["bf16", "e4m3"])
def test_sparse_bubble_packed_matches_oracle_on_dequantised_copy(cuda_ok, fmt):
    """The packed single-source kernels take the same vote: the sparse bubble
    from its BF16 / E4M3 copy against the oracle run on the oracle's own
    dequantised copy of the field (one-cell apron as guard cells)."""
    import torch
    sc = _bubble()
    pv = isaac.DeviceScene(sc).pack(fmt)
    vals, _ = oracle.lowp_copy(sc.sources[0], sc.n, fmt)
    deq = dataclasses.replace(sc, sources=[synth.source_from_zyx(vals[..., 0], 1)])
    ref = oracle.render(deq)
    for lanes in (4, 16):
        out, f32, ns = pv.render(want_f32=True, want_nsamp=True, lanes=lanes)
        torch.cuda.synchronize()
        rep = compare(f32.cpu().numpy(), out.cpu().numpy(), ns.cpu().numpy(), ref)
        assert_parity(rep, 1e-3, f"sparse bubble {fmt}, {lanes} lanes per ray")
        assert rep.hit > 5000
