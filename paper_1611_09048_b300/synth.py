"""Seeded synthetic inputs for the ISAAC volume ray caster.

This module only *generates inputs*: scalar and vector fields shaped like
particle-in-cell output (Sec. 4.1 renders the electric field and a current
density of a PIConGPU run), transfer-function LUTs, camera matrices and functor
chains.  It holds none of the ray caster's arithmetic (no ray setup, no
interpolation, no classification, no compositing), so both the CUDA path and
the FP64 oracle can consume the very same arrays without sharing method code.

Every generator takes an explicit seed and uses ``numpy.random.default_rng``.

Conventions shared by every scene (the readings of the paper's silent points):

* A field lives on the interior grid of ``n = (nx, ny, nz)`` cells plus
  ``guard`` ghost cells per side (Sec. 3.1 guard cells).  Cell ``i`` holds the
  value at voxel coordinate ``i + 0.5``; the interior box is ``[0, n)``.
* World coordinates are voxel coordinates shifted so that the box centre is the
  origin: ``world = voxel - n / 2``.  Camera matrices are OpenGL-style,
  column-major (element ``(r, c)`` at index ``4 * c + r``).
* Storage is a flat float32 array; ``offset`` is the element index of interior
  cell (0,0,0) component 0 and ``strides``/``cstride`` are element steps, so any
  pitch or axis order can be described without a copy (Sec. 3.1 accessors).
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence, Tuple

import numpy as np

__all__ = [
    "Source", "Scene", "lut_from_points", "look_at", "perspective",
    "orbit_camera", "random_orbit_camera", "fibonacci_cameras",
    "gaussian_blobs", "pic_fields", "scene_blobs", "scene_pic",
    "source_from_zyx", "sphere_camera",
]


@dataclasses.dataclass
class Source:
    """One data source (Sec. 3.2): a scalar or up-to-4-component vector field."""

    data: np.ndarray            # flat storage (float32 for the plain path)
    fdim: int                   # feature dimension, 1..4
    offset: int                 # element index of interior cell (0,0,0), comp 0
    strides: Tuple[int, int, int]  # elements between neighbouring cells in x, y, z
    cstride: int                # elements between components
    guard: int                  # ghost cells per side present in the storage
    name: str = ""


@dataclasses.dataclass
class Scene:
    """Everything one frame needs; plain data only."""

    n: Tuple[int, int, int]
    sources: List[Source]
    chains: List[list]          # per source: [("length",), ("mul", (a,)), ...]
    luts: np.ndarray            # (n_src, 256, 4) float32 RGBA in [0, 1]
    weights: np.ndarray         # (n_src,) float32
    modelview: np.ndarray       # (16,) float64 column-major
    projection: np.ndarray      # (16,) float64 column-major
    width: int
    height: int
    clip: List[Tuple[float, float, float, float]] = dataclasses.field(default_factory=list)
    step: float = 0.5
    interp: int = 1
    term: float = 0.99
    bg: Tuple[float, float, float, float] = (0.0, 0.0, 0.0, 0.0)
    active_mask: Optional[int] = None
    # Sec. 3.1 domain decomposition: this volume is the cuboid [off, off + n)
    # of a global volume of ``global_n`` cells (None = the volume is global).
    global_n: Optional[Tuple[int, int, int]] = None
    off: Tuple[int, int, int] = (0, 0, 0)

    @property
    def gn(self) -> Tuple[int, int, int]:
        return tuple(self.n) if self.global_n is None else tuple(self.global_n)

    @property
    def mask(self) -> int:
        if self.active_mask is None:
            return (1 << len(self.sources)) - 1
        return int(self.active_mask)

    def with_camera(self, mv: np.ndarray, proj: np.ndarray) -> "Scene":
        return dataclasses.replace(self, modelview=np.asarray(mv, np.float64),
                                   projection=np.asarray(proj, np.float64))


# --------------------------------------------------------------------------
# transfer functions
# --------------------------------------------------------------------------

def lut_from_points(seed: int, n_points: int = 4, alpha_max: float = 0.1) -> np.ndarray:
    """256-entry RGBA LUT, piecewise linear through seeded control points.

    Control-point positions are sorted U(0,1) with the first pinned to 0 and
    the last to 1; RGB is U(0,1) and alpha U(0, alpha_max) so that rays stay
    translucent for many samples.  Entry j holds the curve at j / 255.
    """
    rng = np.random.default_rng(seed)
    xs = np.sort(rng.uniform(0.0, 1.0, n_points))
    xs[0], xs[-1] = 0.0, 1.0
    rgb = rng.uniform(0.0, 1.0, (n_points, 3))
    a = rng.uniform(0.0, alpha_max, (n_points, 1))
    pts = np.concatenate([rgb, a], axis=1)
    grid = np.arange(256, dtype=np.float64) / 255.0
    lut = np.stack([np.interp(grid, xs, pts[:, c]) for c in range(4)], axis=1)
    return lut.astype(np.float32)


# --------------------------------------------------------------------------
# cameras
# --------------------------------------------------------------------------

def look_at(eye, center, up) -> np.ndarray:
    eye = np.asarray(eye, np.float64)
    f = np.asarray(center, np.float64) - eye
    f /= np.linalg.norm(f)
    s = np.cross(f, np.asarray(up, np.float64))
    s /= np.linalg.norm(s)
    u = np.cross(s, f)
    m = np.eye(4)
    m[0, :3], m[1, :3], m[2, :3] = s, u, -f
    m[0, 3], m[1, 3], m[2, 3] = -s @ eye, -u @ eye, f @ eye
    return m.T.reshape(16).copy()      # column-major


def perspective(fovy_deg: float, aspect: float, near: float, far: float) -> np.ndarray:
    f = 1.0 / math.tan(math.radians(fovy_deg) / 2.0)
    m = np.zeros((4, 4))
    m[0, 0] = f / aspect
    m[1, 1] = f
    m[2, 2] = (far + near) / (near - far)
    m[2, 3] = 2.0 * far * near / (near - far)
    m[3, 2] = -1.0
    return m.T.reshape(16).copy()


def orthographic(left, right, bottom, top, near, far) -> np.ndarray:
    m = np.eye(4)
    m[0, 0] = 2.0 / (right - left)
    m[1, 1] = 2.0 / (top - bottom)
    m[2, 2] = -2.0 / (far - near)
    m[0, 3] = -(right + left) / (right - left)
    m[1, 3] = -(top + bottom) / (top - bottom)
    m[2, 3] = -(far + near) / (far - near)
    return m.T.reshape(16).copy()


def _diag(n) -> float:
    return float(np.linalg.norm(np.asarray(n, np.float64)))


def sphere_camera(n, width, height, direction, dist_factor=2.0, fovy=60.0, up=(0.0, 1.0, 0.0)):
    """Perspective camera on a sphere of radius ``dist_factor * diag`` about
    the box centre, looking at it.  ``direction`` is a unit vector."""
    diag = _diag(n)
    eye = np.asarray(direction, np.float64) * dist_factor * diag
    up = np.asarray(up, np.float64)
    if abs(np.dot(eye / np.linalg.norm(eye), up)) > 0.999:
        up = np.array([0.0, 0.0, 1.0])
    mv = look_at(eye, (0.0, 0.0, 0.0), up)
    proj = perspective(fovy, width / height, 0.1, (dist_factor + 2.0) * diag)
    return mv, proj


def orbit_camera(n, width, height, theta, phi, dist_factor=2.0, fovy=60.0):
    """Orbit angle ``theta`` about +y and elevation ``phi`` (radians)."""
    d = (math.cos(phi) * math.sin(theta), math.sin(phi), math.cos(phi) * math.cos(theta))
    return sphere_camera(n, width, height, d, dist_factor, fovy)


def random_orbit_camera(n, width, height, seed, dist_factor=2.0, fovy=60.0):
    rng = np.random.default_rng(seed)
    theta = rng.uniform(0.0, 2.0 * math.pi)
    phi = rng.uniform(-math.pi / 4.0, math.pi / 4.0)
    return orbit_camera(n, width, height, theta, phi, dist_factor, fovy)


def fibonacci_cameras(n, width, height, count=32, seed=0, dist_factor=2.0, fovy=60.0):
    """``count`` cameras on a Fibonacci sphere with a seeded rotation about +y."""
    rng = np.random.default_rng(seed)
    rot = rng.uniform(0.0, 2.0 * math.pi)
    golden = math.pi * (3.0 - math.sqrt(5.0))
    cams = []
    for i in range(count):
        y = 1.0 - 2.0 * (i + 0.5) / count
        r = math.sqrt(max(0.0, 1.0 - y * y))
        th = golden * i + rot
        cams.append(sphere_camera(n, width, height, (r * math.cos(th), y, r * math.sin(th)),
                                  dist_factor, fovy))
    return cams


# --------------------------------------------------------------------------
# fields
# --------------------------------------------------------------------------

def gaussian_blobs(n: int = 64, seed: int = 0, n_blobs: int = 3) -> np.ndarray:
    """Sum of isotropic Gaussian blobs sampled at cell centres, shape (z, y, x).

    Centres uniform in the box, sigma U(4, 12) voxels, amplitude U(0.5, 1)."""
    rng = np.random.default_rng(seed)
    c = np.arange(n, dtype=np.float64) + 0.5
    out = np.zeros((n, n, n), np.float64)
    for _ in range(n_blobs):
        ctr = rng.uniform(0.0, n, 3)
        sig = rng.uniform(4.0, 12.0)
        amp = rng.uniform(0.5, 1.0)
        gx = np.exp(-((c - ctr[0]) ** 2) / (2 * sig * sig))
        gy = np.exp(-((c - ctr[1]) ** 2) / (2 * sig * sig))
        gz = np.exp(-((c - ctr[2]) ** 2) / (2 * sig * sig))
        out += amp * gz[:, None, None] * gy[None, :, None] * gx[None, None, :]
    return out.astype(np.float32)


def _plane_wave_field(rng, n: int, guard: int, n_waves: int = 4, noise: float = 0.01) -> np.ndarray:
    """3-component field: sum of plane waves plus Gaussian noise, shape
    (S, S, S, 3) with S = n + 2*guard, guards holding the analytic continuation."""
    S = n + 2 * guard
    pos = np.arange(S, dtype=np.float64) - guard + 0.5
    out = np.zeros((S, S, S, 3), np.float32)
    waves = []
    for _ in range(n_waves):
        kmag = rng.uniform(2.0, 16.0)
        u = rng.standard_normal(3)
        u /= np.linalg.norm(u)
        pol = rng.standard_normal(3)
        pol -= (pol @ u) * u
        pol /= np.linalg.norm(pol)
        amp = rng.uniform(0.5, 1.0)
        phase = rng.uniform(0.0, 2.0 * math.pi)
        waves.append((2.0 * math.pi * kmag / n * u, pol * amp, phase))
    for kv, pa, ph in waves:
        axy = kv[0] * pos[None, :] + kv[1] * pos[:, None]          # (y, x)
        sa, ca = np.sin(axy), np.cos(axy)
        bz = kv[2] * pos + ph
        sb, cb = np.sin(bz), np.cos(bz)
        for z in range(S):
            s = (sa * cb[z] + ca * sb[z]).astype(np.float32)
            out[z] += s[:, :, None] * pa.astype(np.float32)[None, None, :]
    rms = float(np.sqrt(np.mean(out[::4, ::4, ::4].astype(np.float64) ** 2)))
    for z0 in range(0, S, 32):
        z1 = min(S, z0 + 32)
        out[z0:z1] += (noise * rms) * rng.standard_normal(out[z0:z1].shape, dtype=np.float32)
    return out


def _density_field(rng, n: int, guard: int) -> np.ndarray:
    """Log-normal (mu 0, sigma 1) per cell, smoothed by a 3-cell box filter;
    shape (S, S, S)."""
    S = n + 2 * guard
    raw = np.exp(rng.standard_normal((S + 2, S + 2, S + 2), dtype=np.float32))
    out = raw.astype(np.float64)
    for ax in range(3):
        c = np.cumsum(out, axis=ax)
        zero = np.zeros_like(np.take(c, [0], axis=ax))
        c = np.concatenate([zero, c], axis=ax)
        hi = np.take(c, np.arange(3, c.shape[ax]), axis=ax)
        lo = np.take(c, np.arange(0, c.shape[ax] - 3), axis=ax)
        out = (hi - lo) / 3.0
    return out.astype(np.float32)


def pic_fields(n: int = 256, guard: int = 4, seed: int = 0):
    """E, B (vector, (S,S,S,3)) and rho (scalar, (S,S,S)) with S = n + 2 guard."""
    rng = np.random.default_rng(seed)
    E = _plane_wave_field(rng, n, guard)
    B = _plane_wave_field(rng, n, guard)
    rho = _density_field(rng, n, guard)
    return E, B, rho


def source_from_zyx(arr: np.ndarray, guard: int, layout: str = "aos", name: str = "") -> Source:
    """Describe a (S,S,S[,C]) z-major array as a strided source without copying
    (``aos``: components innermost) or as component planes (``soa``)."""
    fdim = 1 if arr.ndim == 3 else arr.shape[3]
    S = tuple(int(s) for s in arr.shape[:3])
    if not isinstance(arr, np.ndarray) and hasattr(arr, "contiguous"):   # a torch tensor
        if layout != "aos" and fdim > 1:
            raise ValueError("tensor sources are described in place (AoS) only")
        data = arr.contiguous().reshape(-1)
        sx, sy, sz, cs = fdim, fdim * S[2], fdim * S[2] * S[1], 1
        return Source(data=data, fdim=fdim, offset=guard * (sx + sy + sz), strides=(sx, sy, sz),
                      cstride=cs, guard=guard, name=name)
    if layout == "aos" or fdim == 1:
        data = np.ascontiguousarray(arr, dtype=np.float32).reshape(-1)
        sx, sy, sz, cs = fdim, fdim * S[2], fdim * S[2] * S[1], 1
    elif layout == "soa":
        data = np.ascontiguousarray(np.moveaxis(arr, 3, 0), dtype=np.float32).reshape(-1)
        sx, sy, sz, cs = 1, S[2], S[2] * S[1], S[0] * S[1] * S[2]
    else:
        raise ValueError(layout)
    off = guard * (sx + sy + sz)
    return Source(data=data, fdim=fdim, offset=off, strides=(sx, sy, sz), cstride=cs,
                  guard=guard, name=name)


def value_noise(n: int, seed: int, octaves=((64, 0.5), (32, 0.3), (16, 0.2)), device=None):
    """Smooth seeded noise in [0, 1): random lattice values every L cells,
    trilinearly upsampled, summed over octaves with the given weights.  A numpy
    array, or a torch tensor on `device` when one is given (same values up to
    float rounding of the upsampling)."""
    import torch
    rng = np.random.default_rng(seed)
    dev = torch.device(device) if device is not None else torch.device("cpu")
    out = torch.zeros((n, n, n), dtype=torch.float32, device=dev)
    for L, w in octaves:
        L = max(2, min(L, n))
        m = n // L + 2
        lat = torch.from_numpy(rng.uniform(0.0, 1.0, (1, 1, m, m, m)).astype(np.float32)).to(dev)
        up = torch.nn.functional.interpolate(lat, size=(m - 1) * L, mode="trilinear",
                                             align_corners=True)[0, 0, :n, :n, :n]
        out += w * up
    return out if device is not None else out.numpy()


def bubble_field(n: int = 512, frame: int = 0, seed: int = 0, noise=None,
                 thickness: float = 6.0, speed: float = 2.0, device=None):
    """Laser-wakefield-like bubble: an ellipsoidal shell (semi-axes 60/60/90
    cells at n = 512, scaled with n) of Gaussian profile and the given
    thickness, centred on the x-y axis and moving +z by `speed` cells per frame
    from z = 150 (scaled), plus 0.1 * seeded value noise.  Shape (z, y, x);
    numpy float32, or a torch tensor on `device` when one is given."""
    import torch
    dev = torch.device(device) if device is not None else torch.device("cpu")
    s = n / 512.0
    ax, ay, az = 60.0 * s, 60.0 * s, 90.0 * s
    cz = (150.0 + speed * frame) * s
    c = torch.arange(n, dtype=torch.float32, device=dev) + 0.5
    z, y, x = c[:, None, None], c[None, :, None], c[None, None, :]
    r = torch.sqrt(((x - n / 2) / ax) ** 2 + ((y - n / 2) / ay) ** 2 + ((z - cz) / az) ** 2)
    d = (r - 1.0) * min(ax, ay, az)
    sig = max(thickness * s, 1.0) / 2.0
    shell = torch.exp(-(d * d) / (2.0 * sig * sig))
    if noise is None:
        noise = value_noise(n, seed + 77, device=device)
    noise_t = noise if isinstance(noise, torch.Tensor) else torch.from_numpy(np.asarray(noise))
    f = shell + 0.1 * noise_t.to(dev)
    return f if device is not None else f.numpy().astype(np.float32)


def bubble_lut(seed: int, alpha_max: float = 0.3) -> np.ndarray:
    """TF for the bubble: fully transparent below a seeded threshold in
    U(0.15, 0.35) (so the 0.1-amplitude background noise is empty space), then
    piecewise linear through 3 seeded points with alpha U(0.02, alpha_max)."""
    rng = np.random.default_rng(seed)
    thr = rng.uniform(0.15, 0.35)
    xs = np.concatenate([[0.0, thr], np.sort(rng.uniform(thr + 0.02, 1.0, 2)), [1.0]])
    rgb = rng.uniform(0.0, 1.0, (5, 3))
    a = np.concatenate([[0.0, 0.0], rng.uniform(0.02, alpha_max, 3)])
    pts = np.concatenate([rgb, a[:, None]], axis=1)
    grid = np.arange(256, dtype=np.float64) / 255.0
    lut = np.stack([np.interp(grid, xs, pts[:, c]) for c in range(4)], axis=1)
    lut[grid <= thr, 3] = 0.0
    return lut.astype(np.float32)


def scene_bubble(n: int = 512, frame: int = 0, seed: int = 0, width: int = 1920,
                 height: int = 1080, field=None, lut_seed=None, dist_factor: float = 2.0) -> Scene:
    """One frame of the bubble: scalar field, identity chain, seeded TF."""
    f = bubble_field(n, frame, seed) if field is None else field
    src = source_from_zyx(f, 0, name="bubble")
    mv, proj = random_orbit_camera((n, n, n), width, height, seed + 1000 + frame, dist_factor)
    lut = bubble_lut(seed + 4000 if lut_seed is None else lut_seed)
    return Scene(n=(n, n, n), sources=[src], chains=[[]], luts=lut[None],
                 weights=np.ones(1, np.float32), modelview=mv, projection=proj, width=width,
                 height=height)


def mlp_params(seed: int = 0, bias_scale: float = 0.0) -> dict:
    """Seeded initial weights of the 224-64-64-64-3 proposal MLP: He-uniform
    weights (input-major), biases U(-bias_scale, bias_scale)."""
    rng = np.random.default_rng(seed)
    shapes = [("W1", (224, 64)), ("b1", (64,)), ("W2", (64, 64)), ("b2", (64,)),
              ("W3", (64, 64)), ("b3", (64,)), ("W4", (64, 3)), ("b4", (3,))]
    out = {}
    for name, shape in shapes:
        if name.startswith("W"):
            lim = math.sqrt(6.0 / shape[0])
            out[name] = rng.uniform(-lim, lim, shape).astype(np.float32)
        else:
            out[name] = rng.uniform(-bias_scale, bias_scale, shape).astype(np.float32)
    return out


def random_rays(n_rays: int, n, seed: int = 0, ns_range=(20, 400)):
    """Seeded synthetic ray records: first sample inside the box, unit
    direction, sample count, and a visible span [jf, jl] (-1 for ~20% empty
    rays).  Returns a dict of arrays."""
    rng = np.random.default_rng(seed)
    e = rng.uniform(0.0, 1.0, (n_rays, 3)) * np.asarray(n, np.float64)
    d = rng.standard_normal((n_rays, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    ns = rng.integers(ns_range[0], ns_range[1], n_rays)
    jf = rng.integers(0, ns // 2 + 1)
    jl = np.minimum(ns - 1, jf + rng.integers(0, ns // 2 + 1))
    empty = rng.uniform(size=n_rays) < 0.2
    jf = np.where(empty, -1, jf)
    jl = np.where(empty, -1, jl)
    return {"e": e.astype(np.float32), "d": d.astype(np.float32), "nsteps": ns.astype(np.int32),
            "jf": jf.astype(np.int32), "jl": jl.astype(np.int32)}


# --------------------------------------------------------------------------
# whole scenes
# --------------------------------------------------------------------------

def scene_blobs(n: int = 64, width: int = 256, height: int = 256, seed: int = 0,
                dist_factor: float = 2.0) -> Scene:
    """One scalar field of Gaussian blobs, identity chain, one LUT, no guard."""
    f = gaussian_blobs(n, seed)
    src = source_from_zyx(f, 0, name="blobs")
    mv, proj = random_orbit_camera((n, n, n), width, height, seed + 1000, dist_factor)
    return Scene(n=(n, n, n), sources=[src], chains=[[]],
                 luts=lut_from_points(seed + 2000)[None], weights=np.ones(1, np.float32),
                 modelview=mv, projection=proj, width=width, height=height)


def _pct_length(v: np.ndarray, guard: int, rng) -> float:
    S = v.shape[0]
    idx = rng.integers(guard, S - guard, size=(200000, 3))
    s = v[idx[:, 0], idx[:, 1], idx[:, 2]].astype(np.float64)
    return float(np.percentile(np.sqrt((s * s).sum(axis=1)), 99.9))


def scene_pic(n: int = 256, guard: int = 4, width: int = 1920, height: int = 1080,
              seed: int = 0, layout: str = "aos", fields=None, clip: bool = True,
              dist_factor: float = 2.0) -> Scene:
    """E and B (3-component) plus density (scalar), PIConGPU-shaped.

    Chains: E, B -> length | mul(1/L) | add(0) | pow(0.5) with L the 99.9th
    percentile of the field's length; density -> log | mul(1/6) | add(0.5).
    Three seeded LUTs, weights 0.4/0.3/0.3, one clip plane x >= n/2 - 20
    (scaled for small n), 0.5-voxel steps."""
    if fields is None:
        fields = pic_fields(n, guard, seed)
    E, B, rho = fields
    rng = np.random.default_rng(seed + 17)
    LE, LB = _pct_length(E, guard, rng), _pct_length(B, guard, rng)
    srcs = [source_from_zyx(E, guard, layout, "E"), source_from_zyx(B, guard, layout, "B"),
            source_from_zyx(rho, guard, layout, "rho")]
    chains = [
        [("length",), ("mul", (1.0 / LE,)), ("add", (0.0,)), ("pow", (0.5,))],
        [("length",), ("mul", (1.0 / LB,)), ("add", (0.0,)), ("pow", (0.5,))],
        [("log",), ("mul", (1.0 / 6.0,)), ("add", (0.5,))],
    ]
    luts = np.stack([lut_from_points(seed + 3000 + i) for i in range(3)])
    mv, proj = random_orbit_camera((n, n, n), width, height, seed + 1000, dist_factor)
    planes = [(1.0, 0.0, 0.0, -(n / 2.0 - 20.0 * n / 256.0))] if clip else []
    return Scene(n=(n, n, n), sources=srcs, chains=chains, luts=luts,
                 weights=np.array([0.4, 0.3, 0.3], np.float32), modelview=mv,
                 projection=proj, width=width, height=height, clip=planes)
