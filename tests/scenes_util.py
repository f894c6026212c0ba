"""Small hand-built scenes for pins and parity tests (test-side helpers).

Only input construction lives here: fields, LUTs and cameras whose geometry is
known in closed form, so that tests can state expected values without any ray
code."""
from __future__ import annotations

import numpy as np

from paper_1611_09048_b300 import synth


def ortho_down_z(n, width, height, near=0.5, extra=2.0):
    """Orthographic camera looking along -z whose image covers exactly the
    x-y extent of the (global) box ``n``.  Pixel (px, py) then travels along
    voxel x = (px + 0.5) * nx / width, y = ny - (py + 0.5) * ny / height and
    enters the box at z = nz."""
    nx, ny, nz = n
    eye = (0.0, 0.0, nz / 2.0 + near)
    mv = synth.look_at(eye, (0.0, 0.0, 0.0), (0.0, 1.0, 0.0))
    proj = synth.orthographic(-nx / 2.0, nx / 2.0, -ny / 2.0, ny / 2.0, 0.0, nz + near + extra)
    return mv, proj


def const_lut(rgba):
    return np.tile(np.asarray(rgba, np.float32), (256, 1))


def ramp_lut(alpha=1.0):
    """Red channel equals the classified scalar (entry j = j/255)."""
    lut = np.zeros((256, 4), np.float32)
    lut[:, 0] = np.arange(256, dtype=np.float64) / 255.0
    lut[:, 3] = alpha
    return lut


def make_scene(fields, chains, luts, weights, n, camera, width, height, guard=0, **kw):
    """``fields``: list of (S,S,S) or (S,S,S,C) arrays with S = n + 2*guard."""
    srcs = [synth.source_from_zyx(np.asarray(f, np.float32), guard) for f in fields]
    return synth.Scene(n=tuple(n), sources=srcs, chains=chains,
                       luts=np.stack([np.asarray(l, np.float32) for l in luts]),
                       weights=np.asarray(weights, np.float32), modelview=camera[0],
                       projection=camera[1], width=width, height=height, **kw)


def small_pic_scene(n=24, guard=2, width=48, height=40, seed=3, layout="aos", clip=True,
                    dist_factor=2.0):
    """E, B, rho scene at a size the oracle renders in well under a second."""
    return synth.scene_pic(n=n, guard=guard, width=width, height=height, seed=seed,
                           layout=layout, clip=clip, dist_factor=dist_factor)
