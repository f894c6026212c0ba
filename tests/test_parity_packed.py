"""GPU parity of the reduced-precision path (isaac_pack / isaac_render_packed).

* the packed codes equal the oracle's own quantisation bit for bit;
* rendering the packed copy matches the FP64 oracle run on the dequantised
  copy within the FP32 tolerance (arithmetic error only);
* a float32 packed copy renders bit-identically to the zero-copy path;
* against the original float32 data the storage error is reported and held
  to the reduced-precision tolerance.
"""
import numpy as np
import pytest

import oracle
from paper_1611_09048_b300 import isaac, synth
from parity_util import assert_parity, compare

pytestmark = pytest.mark.gpu

TOL_16 = 2e-3      # max abs per channel, 16-bit storage vs FP64 on the original data


def _mixed_scene(n=20, width=56, height=44, seed=7, dist=1.0):
    """E (AoS, 2 guards), B (component planes, 2 guards), rho (no guards)."""
    E, B, _ = synth.pic_fields(n, 2, seed=seed)
    rho = synth.pic_fields(n, 0, seed=seed + 1)[2]
    sc = synth.scene_pic(n=n, guard=2, width=width, height=height, seed=seed,
                         fields=(E, B, rho[:1, :1, :1]), dist_factor=dist)
    sc.sources = [synth.source_from_zyx(E, 2, "aos"), synth.source_from_zyx(B, 2, "soa"),
                  synth.source_from_zyx(rho, 0)]
    return sc


def _decode(pv, fmt, n):
    import torch
    P = [k + 2 for k in n]
    pad = pv.desc.pad
    raw = pv.data.cpu()
    cells = P[0] * P[1] * P[2]
    if fmt == "f32":
        v = raw[: cells * pad * 4].view(torch.float32)
    elif fmt == "bf16":
        v = raw[: cells * pad * 2].view(torch.bfloat16).float()
    elif fmt == "f16":
        v = raw[: cells * pad * 2].view(torch.float16).float()
    else:
        v = raw[: cells * pad].view(torch.float8_e4m3fn).float()
    v = v.numpy().reshape(P[2], P[1], P[0], pad)
    sc = None
    if fmt == "e4m3":
        Bk = [(p + 7) // 8 for p in P]
        sc = pv.scales.cpu().numpy()[: Bk[0] * Bk[1] * Bk[2] * pad].reshape(Bk[2], Bk[1], Bk[0], pad)
        full = np.repeat(np.repeat(np.repeat(sc, 8, 0), 8, 1), 8, 2)[: P[2], : P[1], : P[0]]
        v = (v * full).astype(np.float32)
    return v, sc


def _expected(scene, fmt):
    vals, scales = [], []
    for s in scene.sources:
        v, sc = oracle.lowp_copy(s, scene.n, fmt)
        vals.append(v)
        scales.append(sc)
    return np.concatenate(vals, -1), (np.concatenate(scales, -1) if fmt == "e4m3" else None)


@pytest.mark.parametrize("fmt", ["f32", "bf16", "f16", "e4m3"])
def test_pack_matches_oracle_bit_exact(cuda_ok, fmt):
    import torch
    sc = _mixed_scene()
    ds = isaac.DeviceScene(sc)
    pv = ds.pack(fmt)
    torch.cuda.synchronize()
    got, got_scales = _decode(pv, fmt, sc.n)
    want, want_scales = _expected(sc, fmt)
    nc = want.shape[-1]
    assert pv.desc.n_comp == nc == 7 and pv.desc.pad == 8
    np.testing.assert_array_equal(got[..., :nc], want)
    if fmt == "e4m3":
        np.testing.assert_array_equal(got_scales[..., :nc], want_scales)


def _dequantised_scene(sc, fmt, mask=None):
    """The same frame over the oracle's dequantised copy (one-cell apron as
    guard cells)."""
    import dataclasses
    srcs = []
    for s in sc.sources:
        v, _ = oracle.lowp_copy(s, sc.n, fmt)
        srcs.append(synth.source_from_zyx(v if v.shape[-1] > 1 else v[..., 0], 1))
    return dataclasses.replace(sc, sources=srcs, active_mask=mask)


@pytest.mark.parametrize("fmt", ["f32", "bf16", "f16", "e4m3"])
@pytest.mark.parametrize("interp", [1, 0])
def test_render_packed_matches_oracle_on_dequantised_copy(cuda_ok, fmt, interp):
    import torch
    sc = _mixed_scene()
    sc.interp = interp
    pv = isaac.DeviceScene(sc).pack(fmt)
    out, f32, ns = pv.render(want_f32=True, want_nsamp=True)
    torch.cuda.synchronize()
    ref = oracle.render(_dequantised_scene(sc, fmt))
    rep = compare(f32.cpu().numpy(), out.cpu().numpy(), ns.cpu().numpy(), ref, interp=interp)
    assert_parity(rep, 1e-3 if interp else 0.3, f"packed {fmt} interp {interp}")
    assert rep.hit > 300


def test_packed_subset_uses_generic_kernel(cuda_ok):
    import torch
    sc = _mixed_scene()
    pv = isaac.DeviceScene(sc).pack("bf16")
    out, f32, ns = pv.render(mask=0b101, want_f32=True, want_nsamp=True)
    torch.cuda.synchronize()
    ref = oracle.render(_dequantised_scene(sc, "bf16", mask=0b101))
    assert_parity(compare(f32.cpu().numpy(), out.cpu().numpy(), ns.cpu().numpy(), ref),
                  1e-3, "packed subset")


def test_pack_single_scalar_tight_record(cuda_ok):
    """A lone scalar source packs into 1-component records (2 bytes in bf16)."""
    import torch
    sc = synth.scene_blobs(32, 64, 64, seed=3, dist_factor=1.0)
    pv = isaac.DeviceScene(sc).pack("bf16")
    assert pv.desc.pad == 1 and pv.data.numel() >= 34 ** 3 * 2
    out, f32, ns = pv.render(want_f32=True, want_nsamp=True)
    torch.cuda.synchronize()
    ref = oracle.render(_dequantised_scene(sc, "bf16"))
    assert_parity(compare(f32.cpu().numpy(), out.cpu().numpy(), ns.cpu().numpy(), ref), 1e-3,
                  "blobs bf16")


def test_f32_packed_is_bitwise_equal_to_zero_copy(cuda_ok):
    import torch
    sc = _mixed_scene()
    ds = isaac.DeviceScene(sc)
    a8, a32, ans = ds.render(want_f32=True, want_nsamp=True)
    b8, b32, bns = ds.pack("f32").render(want_f32=True, want_nsamp=True)
    torch.cuda.synchronize()
    assert torch.equal(a8, b8) and torch.equal(ans, bns)
    assert torch.equal(a32, b32)


@pytest.mark.parametrize("fmt", ["bf16", "f16", "e4m3"])
def test_storage_error_against_original_data(cuda_ok, fmt):
    """Reduced-precision frame vs the FP64 oracle on the original float32
    fields: 16-bit storage stays within the stated tolerance; E4M3 is
    reported (mean and max per channel) and held to 1 LSB mean."""
    import torch
    sc = _mixed_scene(n=32, width=96, height=72)
    pv = isaac.DeviceScene(sc).pack(fmt)
    out, f32, ns = pv.render(want_f32=True, want_nsamp=True)
    torch.cuda.synchronize()
    ref = oracle.render(sc)
    g = f32.cpu().numpy().astype(np.float64)
    err = np.minimum(np.abs(g - ref["rgba"]), np.abs(g - ref["rgba_alt"]))
    hit = ref["nsamp"] > 0
    e = err[hit]
    lsb = np.abs(out.cpu().numpy().astype(np.int64) - ref["rgba8"].astype(np.int64))[hit]
    print(f"{fmt}: max abs per channel {e.max(0)}, mean {e.mean(0)}, mean LSB {lsb.mean():.4f}")
    assert lsb.mean() <= 1.0
    if fmt != "e4m3":
        assert e.max() <= TOL_16, e.max(0)


@pytest.mark.parametrize("fmt", ["f32", "bf16", "f16", "e4m3"])
@pytest.mark.parametrize("cell", [4, 7])
def test_opacity_grid_of_packed_copy(cuda_ok, fmt, cell):
    """isaac_opacity_grid_packed equals the oracle's grid of the dequantised
    copy; over the float32 copy it equals the zero-copy grid bit for bit (the
    same values through the same arithmetic)."""
    import torch
    sc = _mixed_scene()
    ds = isaac.DeviceScene(sc)
    pv = ds.pack(fmt)
    g = pv.opacity_grid(cell)
    torch.cuda.synchronize()
    want = oracle.opacity_grid(_dequantised_scene(sc, fmt), cell)
    np.testing.assert_allclose(g.cpu().numpy(), want, rtol=0, atol=1e-5)
    if fmt == "f32":
        z = ds.opacity_grid(cell)
        torch.cuda.synchronize()
        assert torch.equal(g, z)
    sub = pv.opacity_grid(cell, mask=0b101)
    torch.cuda.synchronize()
    want_sub = oracle.opacity_grid(_dequantised_scene(sc, fmt, mask=0b101), cell)
    np.testing.assert_allclose(sub.cpu().numpy(), want_sub, rtol=0, atol=1e-5)


@pytest.mark.parametrize("fmt", ["f32", "bf16", "f16", "e4m3"])
@pytest.mark.parametrize("n", [64, 62, 61])
def test_opacity_grid_of_packed_scalar_bubble(cuda_ok, fmt, n):
    """The learned workload's shape (one scalar source, identity chain): its
    own walk for 8- and 16-cell macro cells (float32 records, and 16-bit
    records one column per thread when the padded row n + 2 is odd, two when
    it is even; 62 leaves a ragged last macro cell), the general one for other
    cells and for E4M3."""
    import torch
    sc = synth.scene_bubble(n, frame=4, seed=3, width=32, height=32)
    pv = isaac.DeviceScene(sc).pack(fmt)
    deq = _dequantised_scene(sc, fmt)
    for cell in (8, 16, 5):
        g = pv.opacity_grid(cell)
        torch.cuda.synchronize()
        want = oracle.opacity_grid(deq, cell)
        np.testing.assert_allclose(g.cpu().numpy(), want, rtol=0, atol=1e-5)
        assert (want > 0).any() and (want == 0).any()
