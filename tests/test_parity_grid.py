"""GPU parity of isaac_opacity_grid against the FP64 oracle."""
import numpy as np
import pytest

import oracle
from paper_1611_09048_b300 import isaac, synth
from scenes_util import small_pic_scene

pytestmark = pytest.mark.gpu

TOL_ALPHA = 1e-5   # FP32 chain/LUT vs FP64, opacities in [0, 1]


@pytest.mark.parametrize("cell", [4, 7, 16])
def test_grid_pic(cuda_ok, cell):
    import torch
    sc = small_pic_scene(n=24, guard=2, seed=4, layout="soa")
    sc.sources[2] = synth.source_from_zyx(synth.pic_fields(24, 0, seed=9)[2], 0)
    g = isaac.DeviceScene(sc).opacity_grid(cell)
    torch.cuda.synchronize()
    want = oracle.opacity_grid(sc, cell)
    np.testing.assert_allclose(g.cpu().numpy(), want, rtol=0, atol=TOL_ALPHA)


def test_grid_bubble_mask_and_empty(cuda_ok):
    import torch
    sc = synth.scene_bubble(64, frame=3, seed=2, width=32, height=32)
    ds = isaac.DeviceScene(sc)
    g = ds.opacity_grid(8)
    torch.cuda.synchronize()
    want = oracle.opacity_grid(sc, 8)
    np.testing.assert_allclose(g.cpu().numpy(), want, rtol=0, atol=TOL_ALPHA)
    assert (want == 0).mean() > 0.5          # the bubble leaves most macro cells empty
    assert np.array_equal(g.cpu().numpy() == 0, want == 0)
    z = ds.opacity_grid(8, mask=0)
    torch.cuda.synchronize()
    assert torch.count_nonzero(z) == 0
