"""Pins of the oracle's reduced-precision storage against independent
library conversions (numpy float16, torch bfloat16 / float8_e4m3fn on the CPU)
and against brute-force brick scales."""
import numpy as np
import pytest
import torch

import oracle
from paper_1611_09048_b300 import synth


def _probe_values(rng):
    v = [0.0, -0.0, 1.0, -1.0, 3.0, 0.1, 1e-3, 65504.0, 65519.0, 65520.0, 1e5, 6e-5, 6e-8, 3e-8,
         1e-9, 448.0, 464.0, 0.0078125, 0.001953125, 0.00048828125, 2.0 ** -10, 2.0 ** -9]
    # exact ties between neighbouring representable values
    v += [1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, 1.0 + 2.0 ** -11, 1.0 + 3 * 2.0 ** -11,
          1.0 + 2.0 ** -4, 1.0 + 3 * 2.0 ** -4, 2.0 ** -7 * 1.0625, 2.0 ** -7 * 1.1875]
    v += list(rng.standard_normal(300) * 10.0 ** rng.uniform(-6, 3, 300))
    v = np.array(v, np.float32)
    return np.concatenate([v, -v])


def test_bf16_matches_torch():
    v = _probe_values(np.random.default_rng(0))
    want = torch.from_numpy(v).to(torch.bfloat16).to(torch.float32).numpy()
    np.testing.assert_array_equal(oracle.quantize(v, "bf16"), want)


def test_f16_matches_numpy():
    v = _probe_values(np.random.default_rng(1))
    with np.errstate(over="ignore"):        # values past 65504 become +-inf on purpose
        want = v.astype(np.float16).astype(np.float32)
    np.testing.assert_array_equal(oracle.quantize(v, "f16"), want)


def test_e4m3_matches_torch_in_range_and_saturates():
    v = _probe_values(np.random.default_rng(2))
    v = v[np.abs(v) <= 448.0]
    want = torch.from_numpy(v).to(torch.float8_e4m3fn).to(torch.float32).numpy()
    np.testing.assert_array_equal(oracle.quantize(v, "e4m3"), want)
    sat = oracle.quantize(np.array([464.0, 1e6, -500.0, 449.0], np.float32), "e4m3")
    np.testing.assert_array_equal(sat, [448.0, 448.0, -448.0, 448.0])
    # spacing of E4M3: 3 mantissa bits -> 1.125 representable, 1.0625 is a tie -> 1.0 (even)
    np.testing.assert_array_equal(oracle.quantize(np.array([1.0625, 1.1875], np.float32), "e4m3"),
                                  [1.0, 1.25])


@pytest.mark.parametrize("guard", [0, 2])
@pytest.mark.parametrize("fmt", ["bf16", "f16", "e4m3"])
def test_lowp_copy_apron_and_scales(guard, fmt):
    """The copy covers cells [-1, n]: guard cells when present, otherwise the
    border cell repeated (what clamping reads); e4m3 brick scales are the brick
    absmax / 448 and values round-trip through torch's own e4m3 conversion."""
    rng = np.random.default_rng(3)
    n = (13, 9, 11)
    S = [k + 2 * guard for k in n]
    arr = (rng.standard_normal((S[2], S[1], S[0], 3)) * np.exp(rng.uniform(-4, 2, (S[2], 1, 1, 1))))
    arr = arr.astype(np.float32)
    src = synth.source_from_zyx(arr, guard)
    vals, scales = oracle.lowp_copy(src, n, fmt)
    idx = [np.clip(np.arange(-1, k + 1), 0, k - 1) if guard == 0 else np.arange(-1, k + 1)
           for k in n]
    ref = arr[np.ix_(idx[2] + guard, idx[1] + guard, idx[0] + guard)]
    if fmt == "bf16":
        want = torch.from_numpy(ref).to(torch.bfloat16).float().numpy()
    elif fmt == "f16":
        want = ref.astype(np.float16).astype(np.float32)
    else:
        P = [k + 2 for k in n]
        B = [(p + 7) // 8 for p in P]
        want = np.zeros_like(ref)
        for bz in range(B[2]):
            for by in range(B[1]):
                for bx in range(B[0]):
                    sl = (slice(8 * bz, 8 * bz + 8), slice(8 * by, 8 * by + 8),
                          slice(8 * bx, 8 * bx + 8))
                    blk = ref[sl]
                    amax = np.abs(blk).reshape(-1, 3).max(0)
                    sc = np.where(amax > 0, amax / np.float32(448.0), np.float32(1.0)).astype(np.float32)
                    np.testing.assert_array_equal(scales[bz, by, bx], sc)
                    q = torch.from_numpy((blk / sc).astype(np.float32)).to(torch.float8_e4m3fn).float()
                    want[sl] = (q.numpy() * sc).astype(np.float32)
    np.testing.assert_array_equal(vals, want)
