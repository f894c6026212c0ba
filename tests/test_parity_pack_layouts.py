"""isaac_pack across record widths, layouts and box shapes, bit for bit
against the oracle's own quantisation (Sec. 3.2's sources, stored at reduced
precision; the paper has no such copy).

* one scalar (1-slot records), two scalars (2), a scalar and a vector (4),
  E/B/rho (8), and a source set without a specialised record (8, generic);
* guard cells and clamped borders, component-interleaved and planar storage;
* boxes that are not cubes and whose edges end inside an 8^3 brick and
  inside a warp's 32 cells of a row; rows of an odd and of an even number
  of records (2-byte records of an even row are stored in pairs);
* at full size, the 512^3 bubble: sampled cells against the oracle's
  quantiser (BF16, FP16) and sampled interior bricks against the oracle's
  copy of that brick (E4M3 codes and scales).
"""
import numpy as np
import pytest

import oracle
from paper_1611_09048_b300 import isaac, synth

pytestmark = pytest.mark.gpu

FORMATS = ["f32", "bf16", "f16", "e4m3"]

# name: (n (x, y, z), [(f_dim, guard, layout), ...], expected record slots)
CASES = {
    "scalar_clamped": ((45, 21, 19), [(1, 0, "aos")], 1),
    "scalar_guards": ((33, 40, 17), [(1, 2, "aos")], 1),
    "scalar_even_rows": ((38, 27, 17), [(1, 1, "aos")], 1),   # 40-record rows: paired stores
    "two_scalars": ((29, 23, 31), [(1, 0, "aos"), (1, 3, "aos")], 2),
    "scalar_vector": ((26, 35, 18), [(1, 0, "aos"), (3, 1, "soa")], 4),
    "e_b_rho": ((41, 19, 22), [(3, 2, "aos"), (3, 2, "soa"), (1, 0, "aos")], 8),
    "generic": ((27, 22, 20), [(2, 1, "aos"), (1, 0, "aos")], 8),
}


def _field(rng, n, fdim, guard):
    """Values whose magnitude changes from brick to brick (so E4M3 scales
    differ) with exact zeros in places (all-zero bricks get scale 1)."""
    S = (n[2] + 2 * guard, n[1] + 2 * guard, n[0] + 2 * guard)
    shape = S + ((fdim,) if fdim > 1 else ())
    v = rng.standard_normal(shape)
    zz, yy, xx = np.meshgrid(*[np.arange(s) for s in S], indexing="ij")
    mag = 10.0 ** (((xx // 8 + 2 * (yy // 8) + 3 * (zz // 8)) % 7) - 4.0)
    if fdim > 1:
        mag = mag[..., None]
    v = v * mag
    v[:, : min(9, S[1]), : min(9, S[2])] = 0.0
    return v.astype(np.float32)


def _scene(name, seed=0):
    n, specs, _ = CASES[name]
    rng = np.random.default_rng(seed)
    srcs = [synth.source_from_zyx(_field(rng, n, fd, g), g, lay) for fd, g, lay in specs]
    mv, proj = synth.orbit_camera(n, 32, 32, 0.4, 0.3, dist_factor=1.0)
    k = len(srcs)
    return synth.Scene(n=n, sources=srcs, chains=[[] for _ in range(k)],
                       luts=np.zeros((k, 256, 4), np.float32),
                       weights=np.ones(k, np.float32), modelview=mv, projection=proj,
                       width=32, height=32)


def _decode(pv, fmt, n):
    """The copy's codes as float32 (E4M3: the codes' values, unscaled) and
    the E4M3 scales, shaped (z, y, x, slot) and (bz, by, bx, slot)."""
    import torch
    P = [k + 2 for k in n]
    pad = pv.desc.pad
    cells = P[0] * P[1] * P[2]
    raw = pv.data.cpu()
    if fmt == "f32":
        v = raw[: cells * pad * 4].view(torch.float32)
    elif fmt == "bf16":
        v = raw[: cells * pad * 2].view(torch.bfloat16).float()
    elif fmt == "f16":
        v = raw[: cells * pad * 2].view(torch.float16).float()
    else:
        v = raw[: cells * pad].view(torch.float8_e4m3fn).float()
    v = v.numpy().reshape(P[2], P[1], P[0], pad)
    scales = None
    if fmt == "e4m3":
        Bk = [(p + 7) // 8 for p in P]
        scales = pv.scales.cpu().numpy()[: Bk[0] * Bk[1] * Bk[2] * pad].reshape(
            Bk[2], Bk[1], Bk[0], pad)
    return v, scales


@pytest.mark.parametrize("fmt", FORMATS)
@pytest.mark.parametrize("name", sorted(CASES))
def test_pack_codes_match_oracle(cuda_ok, name, fmt):
    import torch
    sc = _scene(name)
    ds = isaac.DeviceScene(sc)
    pv = ds.pack(fmt)
    torch.cuda.synchronize()
    got, got_scales = _decode(pv, fmt, sc.n)
    assert pv.desc.pad == CASES[name][2]
    want = np.concatenate([oracle.lowp_copy(s, sc.n, fmt)[0] for s in sc.sources], -1)
    nc = want.shape[-1]
    if fmt != "e4m3":
        np.testing.assert_array_equal(got[..., :nc], want)
        assert not got[..., nc:].any()      # unused slots hold zeros
        return
    want_scales = np.concatenate([oracle.lowp_copy(s, sc.n, fmt)[1] for s in sc.sources], -1)
    np.testing.assert_array_equal(got_scales[..., :nc], want_scales)
    np.testing.assert_array_equal(got_scales[..., nc:], 1.0)
    full = np.repeat(np.repeat(np.repeat(got_scales, 8, 0), 8, 1), 8, 2)
    P = [k + 2 for k in sc.n]
    deq = (got * full[: P[2], : P[1], : P[0]]).astype(np.float32)
    # the oracle's stored value is quantize(v / scale) * scale, both in float32
    np.testing.assert_array_equal(deq[..., :nc], want)


def test_repack_is_idempotent(cuda_ok):
    """The per-time-step refresh into the same buffers gives the same bytes."""
    import torch
    for fmt in FORMATS:
        sc = _scene("e_b_rho", seed=3)
        pv = isaac.DeviceScene(sc).pack(fmt)
        a = pv.data.clone()
        sa = pv.scales.clone() if pv.scales is not None else None
        pv.repack()
        torch.cuda.synchronize()
        assert torch.equal(a, pv.data)
        if sa is not None:
            assert torch.equal(sa, pv.scales)


def test_pack_bubble512_sampled(cuda_ok):
    """Full size: the 512^3 float32 bubble (one scalar, clamped borders).
    BF16 and FP16 records of 40,000 random cells against the oracle's
    quantiser; E4M3 codes and scales of 48 random interior bricks against the
    oracle's copy of that brick alone (a 6^3 box with one guard layer is
    exactly one brick, counted from cell -1, like the brick in the volume)."""
    import torch
    n = 512
    dev = "cuda"
    field = synth.bubble_field(n, 40, 0, noise=synth.value_noise(n, 77, device=dev), device=dev)
    sc = synth.scene_bubble(n, frame=40, seed=1, width=64, height=64, field=field)
    ds = isaac.DeviceScene(sc, device=dev)
    vol = field.reshape(n, n, n).float().cpu().numpy()          # (z, y, x)
    rng = np.random.default_rng(11)
    P = n + 2
    idx = rng.integers(0, P, size=(40000, 3))                    # packed (z, y, x)
    src = np.clip(idx - 1, 0, n - 1)                             # clamped border reads
    vals = vol[src[:, 0], src[:, 1], src[:, 2]]
    lin = (idx[:, 0] * P + idx[:, 1]) * P + idx[:, 2]
    for fmt, tdt in (("bf16", torch.bfloat16), ("f16", torch.float16)):
        pv = ds.pack(fmt)
        torch.cuda.synchronize()
        assert pv.desc.pad == 1
        got = pv.data[: P ** 3 * 2].view(tdt)[torch.as_tensor(lin, device=dev)].float().cpu().numpy()
        np.testing.assert_array_equal(got, oracle.quantize(vals, fmt))
        del pv
    pv = ds.pack("e4m3")
    torch.cuda.synchronize()
    B = (P + 7) // 8
    codes = pv.data[: P ** 3]
    scales = pv.scales[: B ** 3].cpu().numpy().reshape(B, B, B)
    for bz, by, bx in rng.integers(1, B - 2, size=(48, 3)):
        c0 = np.array([bz, by, bx]) * 8 - 1                      # cell of the brick's corner
        block = vol[c0[0]: c0[0] + 8, c0[1]: c0[1] + 8, c0[2]: c0[2] + 8]
        want, want_s = oracle.lowp_copy(synth.source_from_zyx(block, 1), (6, 6, 6), "e4m3")
        assert scales[bz, by, bx] == want_s.reshape(-1)[0]
        zz, yy, xx = np.meshgrid(*[np.arange(8) + b * 8 for b in (bz, by, bx)], indexing="ij")
        sel = torch.as_tensor(((zz * P + yy) * P + xx).reshape(-1), device=dev)
        got = codes[sel].cpu().view(torch.float8_e4m3fn).float().numpy().reshape(8, 8, 8)
        got = got * scales[bz, by, bx]
        np.testing.assert_array_equal(got.astype(np.float32), want[..., 0])


def _e4m3_rounding_points():
    """The positive E4M3 values up to 416 and the midpoints between
    neighbours (subnormals k 2^-9, normals (1 + j/8) 2^e, e = -6..8), plus
    2^-11 and 2^-12 below the smallest midpoint; all exact in float32."""
    vals = [k * 2.0 ** -9 for k in range(8)]
    vals += [(1 + j / 8) * 2.0 ** e for e in range(-6, 9) for j in range(8)]
    vals = sorted(v for v in vals if v <= 448.0)
    mids = [(a + b) / 2 for a, b in zip(vals[:-1], vals[1:])]
    return [v for v in vals + mids + [2.0 ** -11, 2.0 ** -12] if v <= 432.0]


def test_e4m3_quotients_at_rounding_points(cuda_ok):
    """E4M3 codes where v / scale falls on, or one or two float32 ulps from,
    a rounding point of the format (its values and the midpoints between
    them, where ties go to even), over scales from 2^-61 to 2^61, with signed
    zeros, the smallest subnormal float and an all-zero brick.  A block of
    four bricks whose scales all lie in [2^-60, 2^60] takes the reciprocal
    and residual quotient, the others the division; both must give the
    oracle's float32 division and rounding bit for bit, signs of zero
    included."""
    import torch
    n = (30, 14, 14)                     # packed box 32 x 16 x 16: 4 x 2 x 2 bricks
    P = (n[0] + 2, n[1] + 2, n[2] + 2)
    targets = {                          # (bz, by): scales of the row's 4 bricks
        (0, 0): [1 / 448, 2.0 ** -20, 2.0 ** -59.5, 2.0 ** 59.5],
        (0, 1): [3.7e-3, 0.37, 1234.5, 2.0 ** -59.99],
        (1, 0): [2.0 ** -61, 1.0, 2.0 ** 61, 5e-7],      # two scales out of range
        (1, 1): [7.77e-12, 2.0 ** 40, 9.1e9, 0.0],        # 0: an all-zero brick
    }
    pts = np.array(_e4m3_rounding_points(), np.float32)
    rng = np.random.default_rng(5)
    Q = np.zeros((P[2], P[1], P[0]), np.float32)         # packed (z, y, x)
    for (bz, by), row in targets.items():
        for bx, t in enumerate(row):
            blk = np.zeros((8, 8, 8), np.float32)
            if t == 0.0:
                blk[:] = np.where(rng.random((8, 8, 8)) < 0.5, np.float32(-0.0), np.float32(0.0))
            else:
                A = np.float32(t * 448.0)
                s = np.float32(A) / np.float32(448.0)
                base = pts * s
                cand = [base]
                for direction in (np.float32(np.inf), np.float32(-np.inf)):
                    c = base
                    for _ in range(2):
                        c = np.nextafter(c, direction)
                        cand.append(c)
                cand = np.concatenate(cand)
                cand = np.concatenate([cand, -cand, np.float32([0.0, -0.0, 1e-45, -1e-45])])
                cand = cand[np.abs(cand) <= A]
                blk.reshape(-1)[:] = rng.choice(cand, 512, replace=len(cand) < 512)
                blk[3, 3, 3] = A                          # the brick's absmax
            Q[bz * 8: bz * 8 + 8, by * 8: by * 8 + 8, bx * 8: bx * 8 + 8] = blk
    field = np.ascontiguousarray(Q[1:-1, 1:-1, 1:-1])   # cells [-1, n] of the source
    src = synth.source_from_zyx(field, 0)
    mv, proj = synth.orbit_camera(n, 32, 32, 0.4, 0.3, dist_factor=1.0)
    sc = synth.Scene(n=n, sources=[src], chains=[[]], luts=np.zeros((1, 256, 4), np.float32),
                     weights=np.ones(1, np.float32), modelview=mv, projection=proj,
                     width=32, height=32)
    pv = isaac.DeviceScene(sc).pack("e4m3")
    torch.cuda.synchronize()
    got, got_scales = _decode(pv, "e4m3", n)
    want, want_scales = oracle.lowp_copy(src, n, "e4m3")
    np.testing.assert_array_equal(got_scales, want_scales)
    full = np.repeat(np.repeat(np.repeat(got_scales, 8, 0), 8, 1), 8, 2)
    deq = (got * full).astype(np.float32)
    np.testing.assert_array_equal(deq, want)
    np.testing.assert_array_equal(np.signbit(deq), np.signbit(want))
    # the cases are really there: codes on both sides of many midpoints
    assert len(np.unique(got)) > 200
