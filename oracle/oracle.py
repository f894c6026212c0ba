"""ctypes binding of ``isaac_oracle.c`` (FP64 reference ray caster).

TEST INFRASTRUCTURE ONLY -- see the package docstring.  The C library is
compiled with gcc on first use into ``oracle/_build/``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "isaac_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

MAX_OPS = 16
MAX_CLIP = 16
INF = 1.0e300

# Functor op codes of this oracle (Sec. 3.3, Table 1, plus the user functor log).
OP_CODES = {"add": 1, "mul": 2, "length": 3, "sum": 4, "pow": 5, "log": 6}


class _Source(C.Structure):
    _fields_ = [("data", C.c_void_p), ("offset", C.c_int64), ("stride", C.c_int64 * 3),
                ("cstride", C.c_int64), ("fdim", C.c_int32), ("guard", C.c_int32)]


class _Functor(C.Structure):
    _fields_ = [("op", C.c_int32), ("nargs", C.c_int32), ("arg", C.c_double * 4)]


class _Chain(C.Structure):
    _fields_ = [("nops", C.c_int32), ("ops", _Functor * MAX_OPS)]


class _Params(C.Structure):
    _fields_ = [("n", C.c_int64 * 3), ("gn", C.c_int64 * 3), ("off", C.c_int64 * 3),
                ("modelview", C.c_double * 16),
                ("projection", C.c_double * 16), ("width", C.c_int32), ("height", C.c_int32),
                ("n_clip", C.c_int32), ("clip", (C.c_double * 4) * MAX_CLIP),
                ("step", C.c_double), ("interp", C.c_int32), ("term", C.c_double),
                ("bg", C.c_double * 4), ("active_mask", C.c_uint32)]


class _Outputs(C.Structure):
    _fields_ = [("rgba", C.c_void_p), ("rgba_alt", C.c_void_p), ("rgba8", C.c_void_p),
                ("rgba8_alt", C.c_void_p), ("nsamp", C.c_void_p), ("nsamp_alt", C.c_void_p),
                ("margin", C.c_void_p), ("kfirst", C.c_void_p), ("jspan", C.c_void_p)]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fast-math, no FMA contraction)."""
    with _lock:
        if force or not os.path.exists(_LIB_PATH) or \
                os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
            os.makedirs(_OUT_DIR, exist_ok=True)
            tmp = _LIB_PATH + f".{os.getpid()}.tmp"
            cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
                   "-o", tmp, _SRC, "-lm"]
            subprocess.run(cmd, check=True)
            os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        lib = C.CDLL(build())
        lib.orc_render.restype = C.c_int
        lib.orc_render.argtypes = [C.POINTER(_Params), C.POINTER(_Source), C.POINTER(_Chain),
                                   C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p, C.c_int64,
                                   C.POINTER(_Outputs), C.c_int32]
        lib.orc_invert4.restype = C.c_int
        lib.orc_invert4.argtypes = [C.c_void_p, C.c_void_p]
        lib.orc_max_threads.restype = C.c_int
        lib.orc_chain_eval.restype = C.c_int
        lib.orc_chain_eval.argtypes = [C.POINTER(_Chain), C.c_void_p, C.c_int32, C.c_void_p]
        lib.orc_classify_eval.restype = None
        lib.orc_classify_eval.argtypes = [C.c_void_p, C.c_double, C.c_void_p]
        lib.orc_quantize_value.restype = C.c_float
        lib.orc_quantize_value.argtypes = [C.c_float, C.c_int32]
        lib.orc_opacity_grid.restype = C.c_int
        lib.orc_opacity_grid.argtypes = [C.POINTER(_Source), C.POINTER(_Chain), C.c_void_p,
                                         C.c_void_p, C.c_int32, C.c_void_p, C.c_uint32,
                                         C.c_int32, C.c_void_p, C.c_int32]
        lib.orc_range_grid.restype = C.c_int
        lib.orc_range_grid.argtypes = [C.POINTER(_Source), C.c_int32, C.c_void_p, C.c_uint32,
                                       C.c_int32, C.c_void_p, C.c_int32]
        lib.orc_render_iso.restype = C.c_int
        lib.orc_render_iso.argtypes = [C.POINTER(_Params), C.POINTER(_Source), C.POINTER(_Chain),
                                       C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p,
                                       C.c_void_p, C.c_int32]
        lib.orc_lowp_copy.restype = C.c_int
        lib.orc_lowp_copy.argtypes = [C.POINTER(_Source), C.c_void_p, C.c_int32, C.c_void_p,
                                      C.c_void_p]
        _lib = lib
    return _lib


def max_threads() -> int:
    return int(_load().orc_max_threads())


def invert4(m) -> np.ndarray:
    """Column-major 4x4 inverse by the oracle's Gauss-Jordan routine."""
    m = np.ascontiguousarray(np.asarray(m, np.float64).reshape(16))
    out = np.zeros(16, np.float64)
    if _load().orc_invert4(m.ctypes.data, out.ctypes.data):
        raise ValueError("singular matrix")
    return out


def chain_eval(spec, v) -> float:
    """Apply a functor chain (list of (name, args) tuples) to one value."""
    v = np.zeros(4, np.float64) + 0.0 if v is None else np.asarray(v, np.float64).reshape(-1)
    dim = v.size
    buf = np.zeros(4, np.float64)
    buf[:dim] = v
    out = C.c_double()
    if _load().orc_chain_eval(C.byref(_chain(spec, dim)), buf.ctypes.data, dim, C.byref(out)):
        raise ValueError("invalid chain for this dimension")
    return float(out.value)


def classify(lut, x: float) -> np.ndarray:
    """RGBA of scalar ``x`` through one (256, 4) float32 LUT."""
    lut = np.ascontiguousarray(lut, np.float32).reshape(256, 4)
    out = np.zeros(4, np.float64)
    _load().orc_classify_eval(lut.ctypes.data, float(x), out.ctypes.data)
    return out


def range_grid(scene, cell: int = 16, threads: int = 0, mask=None) -> np.ndarray:
    """Value-range grid of ``scene``'s active sources: shape (ceil(nz/cell),
    ceil(ny/cell), ceil(nx/cell), slots, 2), float32 (min, max) per active
    component in source order, over the same boxes as ``opacity_grid``."""
    lib = _load()
    n_src = len(scene.sources)
    srcs = (_Source * n_src)()
    keep = []
    for s, src in enumerate(scene.sources):
        data = np.ascontiguousarray(src.data, dtype=np.float32)
        keep.append(data)
        srcs[s].data = data.ctypes.data
        srcs[s].offset = int(src.offset)
        for a in range(3):
            srcs[s].stride[a] = int(src.strides[a])
        srcs[s].cstride = int(src.cstride)
        srcs[s].fdim = int(src.fdim)
        srcs[s].guard = int(src.guard)
    m = int(scene.mask if mask is None else mask)
    slots = sum(int(src.fdim) for s, src in enumerate(scene.sources) if (m >> s) & 1)
    n = np.asarray(scene.n, np.int64)
    G = [(int(k) + cell - 1) // cell for k in scene.n]
    out = np.zeros((G[2], G[1], G[0], slots, 2), np.float32)
    rc = lib.orc_range_grid(srcs, n_src, n.ctypes.data, m, int(cell), out.ctypes.data, int(threads))
    if rc:
        raise ValueError("oracle rejected the range-grid request")
    return out


def opacity_grid(scene, cell: int = 16, threads: int = 0, mask=None) -> np.ndarray:
    """Max-opacity grid of ``scene``'s active sources, shape
    (ceil(nz/cell), ceil(ny/cell), ceil(nx/cell)), float64."""
    lib = _load()
    n_src = len(scene.sources)
    srcs = (_Source * n_src)()
    chains = (_Chain * n_src)()
    keep = []
    for s, src in enumerate(scene.sources):
        data = np.ascontiguousarray(src.data, dtype=np.float32)
        keep.append(data)
        srcs[s].data = data.ctypes.data
        srcs[s].offset = int(src.offset)
        for a in range(3):
            srcs[s].stride[a] = int(src.strides[a])
        srcs[s].cstride = int(src.cstride)
        srcs[s].fdim = int(src.fdim)
        srcs[s].guard = int(src.guard)
        chains[s] = _chain(scene.chains[s], src.fdim)
    luts = np.ascontiguousarray(scene.luts, dtype=np.float32).reshape(n_src, 256, 4)
    w = np.ascontiguousarray(scene.weights, dtype=np.float64).reshape(n_src)
    n = np.asarray(scene.n, np.int64)
    G = [(int(k) + cell - 1) // cell for k in scene.n]
    out = np.zeros((G[2], G[1], G[0]), np.float64)
    rc = lib.orc_opacity_grid(srcs, chains, luts.ctypes.data, w.ctypes.data, n_src, n.ctypes.data,
                              int(scene.mask if mask is None else mask), int(cell),
                              out.ctypes.data, int(threads))
    if rc:
        raise ValueError("oracle rejected the opacity-grid request")
    return out


FORMATS = {"f32": 0, "bf16": 1, "f16": 2, "e4m3": 3}


def quantize(values, fmt: str) -> np.ndarray:
    """Value each float32 takes after storage in ``fmt`` (bf16, f16, e4m3;
    round to nearest even; e4m3 saturates at +-448)."""
    lib = _load()
    v = np.asarray(values, np.float32).reshape(-1)
    code = FORMATS[fmt]
    return np.array([lib.orc_quantize_value(float(x), code) for x in v], np.float32)


def lowp_copy(src, n, fmt: str):
    """Reduced-precision copy of one ``synth.Source`` over cells [-1, n]^3.

    Returns (values, scales): values (nz+2, ny+2, nx+2, fdim) float32 holding
    what the stored codes represent; scales per 8^3 brick and component for
    e4m3 (else None)."""
    lib = _load()
    data = np.ascontiguousarray(src.data, dtype=np.float32)
    s = _Source()
    s.data = data.ctypes.data
    s.offset = int(src.offset)
    for a in range(3):
        s.stride[a] = int(src.strides[a])
    s.cstride = int(src.cstride)
    s.fdim = int(src.fdim)
    s.guard = int(src.guard)
    nn = np.asarray(n, np.int64)
    P = [int(k) + 2 for k in n]
    out = np.zeros((P[2], P[1], P[0], src.fdim), np.float32)
    B = [(p + 7) // 8 for p in P]
    scales = np.zeros((B[2], B[1], B[0], src.fdim), np.float32) if fmt == "e4m3" else None
    rc = lib.orc_lowp_copy(C.byref(s), nn.ctypes.data, FORMATS[fmt], out.ctypes.data,
                           scales.ctypes.data if scales is not None else None)
    if rc:
        raise ValueError("oracle rejected the low-precision copy")
    return out, scales


def _chain(spec, fdim: int) -> _Chain:
    ch = _Chain()
    if len(spec) > MAX_OPS:
        raise ValueError("chain too long for the oracle")
    ch.nops = len(spec)
    for i, f in enumerate(spec):
        name = f[0]
        args = tuple(f[1]) if len(f) > 1 else ()
        ch.ops[i].op = OP_CODES[name]
        ch.ops[i].nargs = len(args)
        for j, a in enumerate(args[:4]):
            ch.ops[i].arg[j] = float(a)
    return ch


def _frame_args(scene, mask=None):
    """(params, sources, chains, luts, keepalive) of ``scene`` for the C side."""
    n_src = len(scene.sources)
    P = _Params()
    for a in range(3):
        P.n[a] = int(scene.n[a])
        P.gn[a] = int(scene.gn[a])
        P.off[a] = int(scene.off[a])
    for i in range(16):
        P.modelview[i] = float(scene.modelview[i])
        P.projection[i] = float(scene.projection[i])
    P.width, P.height = int(scene.width), int(scene.height)
    if len(scene.clip) > MAX_CLIP:
        raise ValueError("too many clip planes for the oracle")
    P.n_clip = len(scene.clip)
    for i, pl in enumerate(scene.clip):
        for j in range(4):
            P.clip[i][j] = float(pl[j])
    P.step = float(scene.step)
    P.interp = int(scene.interp)
    P.term = float(scene.term)
    for j in range(4):
        P.bg[j] = float(scene.bg[j])
    P.active_mask = int(scene.mask if mask is None else mask)
    srcs = (_Source * n_src)()
    chains = (_Chain * n_src)()
    keep = []
    for s, src in enumerate(scene.sources):
        data = np.ascontiguousarray(src.data, dtype=np.float32)
        keep.append(data)
        srcs[s].data = data.ctypes.data
        srcs[s].offset = int(src.offset)
        for a in range(3):
            srcs[s].stride[a] = int(src.strides[a])
        srcs[s].cstride = int(src.cstride)
        srcs[s].fdim = int(src.fdim)
        srcs[s].guard = int(src.guard)
        chains[s] = _chain(scene.chains[s], src.fdim)
    luts = np.ascontiguousarray(scene.luts, dtype=np.float32).reshape(n_src, 256, 4)
    return P, srcs, chains, luts, keep


def render_iso(scene, iso, threads: int = 0, mask=None) -> dict:
    """Iso-surface frame of ``scene`` in FP64 (the reading stated at
    orc_render_iso): ``iso`` holds one threshold per source.  Returns ``rgba``
    (float64, (H, W, 4)), ``rgba8`` (uint8) and ``margin`` (float64,
    (H, W, 6): entry, exit, |v - iso|, refinement slope, |gradient|, t_hit)."""
    lib = _load()
    P, srcs, chains, luts, keep = _frame_args(scene, mask)
    n_src = len(scene.sources)
    iso = np.ascontiguousarray(iso, dtype=np.float64).reshape(n_src)
    H, W = int(scene.height), int(scene.width)
    rgba = np.zeros((H, W, 4), np.float64)
    rgba8 = np.zeros((H, W, 4), np.uint8)
    margin = np.zeros((H, W, 6), np.float64)
    rc = lib.orc_render_iso(C.byref(P), srcs, chains, luts.ctypes.data, iso.ctypes.data, n_src,
                            rgba.ctypes.data, rgba8.ctypes.data, margin.ctypes.data, int(threads))
    if rc:
        raise ValueError("oracle rejected the iso-surface frame")
    return {"rgba": rgba, "rgba8": rgba8, "margin": margin}


def render(scene, pixels=None, threads: int = 0, mask=None) -> dict:
    """Render ``scene`` (a ``synth.Scene``) in FP64.

    ``pixels``: optional 1-D array of row-major pixel indices; outputs then
    have one entry per listed pixel.  Returns a dict with ``rgba`` (float64,
    (..., 4)), ``rgba_alt``, ``rgba8``, ``rgba8_alt`` (uint8), ``nsamp``,
    ``nsamp_alt``, ``kfirst`` (int32) and ``margin`` (float64, (..., 4):
    entry and exit in steps, termination in A, nearest-cell in voxels)."""
    lib = _load()
    n_src = len(scene.sources)
    P = _Params()
    for a in range(3):
        P.n[a] = int(scene.n[a])
        P.gn[a] = int(scene.gn[a])
        P.off[a] = int(scene.off[a])
    for i in range(16):
        P.modelview[i] = float(scene.modelview[i])
        P.projection[i] = float(scene.projection[i])
    P.width, P.height = int(scene.width), int(scene.height)
    if len(scene.clip) > MAX_CLIP:
        raise ValueError("too many clip planes for the oracle")
    P.n_clip = len(scene.clip)
    for i, pl in enumerate(scene.clip):
        for j in range(4):
            P.clip[i][j] = float(pl[j])
    P.step = float(scene.step)
    P.interp = int(scene.interp)
    P.term = float(scene.term)
    for j in range(4):
        P.bg[j] = float(scene.bg[j])
    P.active_mask = int(scene.mask if mask is None else mask)

    srcs = (_Source * n_src)()
    chains = (_Chain * n_src)()
    keep = []
    for s, src in enumerate(scene.sources):
        data = np.ascontiguousarray(src.data, dtype=np.float32)
        keep.append(data)
        srcs[s].data = data.ctypes.data
        srcs[s].offset = int(src.offset)
        for a in range(3):
            srcs[s].stride[a] = int(src.strides[a])
        srcs[s].cstride = int(src.cstride)
        srcs[s].fdim = int(src.fdim)
        srcs[s].guard = int(src.guard)
        chains[s] = _chain(scene.chains[s], src.fdim)
    luts = np.ascontiguousarray(scene.luts, dtype=np.float32).reshape(n_src, 256, 4)
    w = np.ascontiguousarray(scene.weights, dtype=np.float64).reshape(n_src)

    if pixels is None:
        count = scene.width * scene.height
        pix_ptr = None
        shape = (scene.height, scene.width)
    else:
        pix = np.ascontiguousarray(pixels, dtype=np.int64).reshape(-1)
        if pix.size and (pix.min() < 0 or pix.max() >= scene.width * scene.height):
            raise ValueError("pixel index out of range")
        keep.append(pix)
        count = pix.size
        pix_ptr = pix.ctypes.data
        shape = (count,)
    res = {
        "rgba": np.zeros(shape + (4,), np.float64),
        "rgba_alt": np.zeros(shape + (4,), np.float64),
        "rgba8": np.zeros(shape + (4,), np.uint8),
        "rgba8_alt": np.zeros(shape + (4,), np.uint8),
        "nsamp": np.zeros(shape, np.int32),
        "nsamp_alt": np.zeros(shape, np.int32),
        "margin": np.zeros(shape + (4,), np.float64),
        "kfirst": np.zeros(shape, np.int32),
        "jspan": np.zeros(shape + (2,), np.int32),
    }
    O = _Outputs(*(res[k].ctypes.data for k in
                   ("rgba", "rgba_alt", "rgba8", "rgba8_alt", "nsamp", "nsamp_alt", "margin",
                    "kfirst", "jspan")))
    if count == 0:
        return res
    rc = lib.orc_render(C.byref(P), srcs, chains, luts.ctypes.data, w.ctypes.data, n_src,
                        pix_ptr, count, C.byref(O), int(threads))
    if rc != 0:
        raise ValueError(f"oracle rejected the scene (rc={rc})")
    return res
