"""Thin ctypes binding of ``libisaac_b300.so`` (the C ABI in include/isaac_b300.h).

Argument marshalling only: every step of a frame runs in the library's CUDA
kernels.  PyTorch provides device memory and streams.  The binding refuses to
run without the compiled library -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libisaac_b300.so")

MAX_SOURCES = 8
MAX_ACTIVE = 4
MAX_FUNCTORS = 8
MAX_CLIP = 6

OK, EINVAL, EGUARD, ENOMEM, ECUDA, ENOTSUP = 0, -1, -2, -3, -4, -5
F32, BF16, F16, E4M3 = 0, 1, 2, 3
LUTS_HOST = 1   # isaac_render_opts.flags: `luts` is a host array
MARCH_STAGED = 2   # isaac_render_opts.flags: staged march where the frame allows it
OPS = {"add": 1, "mul": 2, "length": 3, "sum": 4, "pow": 5, "log": 6}

# every C symbol declared in include/isaac_b300.h
EXPORTS = ("isaac_render", "isaac_last_error", "isaac_abi_version", "isaac_pack_layout",
           "isaac_pack", "isaac_render_packed", "isaac_release_workspaces",
           "isaac_opacity_grid", "isaac_render_noalloc", "isaac_trace", "isaac_render_learned",
           "isaac_render_packed_learned", "isaac_mlp_sync", "isaac_mlp_features",
           "isaac_mlp_forward", "isaac_mlp_train_step", "isaac_server_create",
           "isaac_server_submit", "isaac_server_poll", "isaac_server_outstanding",
           "isaac_server_destroy", "isaac_time_march", "isaac_range_grid", "isaac_render_skip",
           "isaac_render_iso", "isaac_probe_read", "isaac_composite", "isaac_copy_source",
           "isaac_set_update_hook", "isaac_opacity_grid_packed", "isaac_mlp_create",
           "isaac_mlp_destroy", "isaac_mlp_checkpoint_bytes", "isaac_mlp_save", "isaac_mlp_load")

# fn(source, enabled, user) of isaac_set_update_hook
UPDATE_FN = C.CFUNCTYPE(None, C.c_int32, C.c_int32, C.c_void_p)

# lanes per ray used when a call does not pass one (0 = the library chooses)
LANES_PER_RAY = int(os.environ.get("ISAAC_LANES_PER_RAY", "0"))


class Source(C.Structure):
    _fields_ = [("ptr", C.c_void_p), ("extent", C.c_int64), ("offset", C.c_int64),
                ("stride", C.c_int64 * 3), ("comp_stride", C.c_int64), ("f_dim", C.c_int32),
                ("guard", C.c_int32)]


class Functor(C.Structure):
    _fields_ = [("op", C.c_int32), ("n_args", C.c_int32), ("arg", C.c_float * 4)]


class Chain(C.Structure):
    _fields_ = [("n_ops", C.c_int32), ("ops", Functor * MAX_FUNCTORS)]


class Plane(C.Structure):
    _fields_ = [("n", C.c_double * 3), ("d", C.c_double)]


class Camera(C.Structure):
    _fields_ = [("modelview", C.c_double * 16), ("projection", C.c_double * 16),
                ("width", C.c_int32), ("height", C.c_int32)]


class RenderOpts(C.Structure):
    _fields_ = [("n", C.c_int64 * 3), ("global_n", C.c_int64 * 3), ("offset", C.c_int64 * 3),
                ("step", C.c_float), ("interp", C.c_int32), ("term_alpha", C.c_float),
                ("bg", C.c_float * 4), ("active_mask", C.c_uint32), ("lanes_per_ray", C.c_int32),
                ("flags", C.c_uint32)]


class Framebuffer(C.Structure):
    _fields_ = [("rgba8", C.c_void_p), ("rgba32", C.c_void_p), ("nsamples", C.c_void_p),
                ("touched", C.c_void_p), ("depth", C.c_void_p)]


class Packed(C.Structure):
    _fields_ = [("data", C.c_void_p), ("scales", C.c_void_p), ("n", C.c_int64 * 3),
                ("dtype", C.c_int32), ("n_src", C.c_int32), ("f_dim", C.c_int32 * MAX_ACTIVE),
                ("n_comp", C.c_int32), ("pad", C.c_int32)]


DTYPES = {"f32": F32, "bf16": BF16, "f16": F16, "e4m3": E4M3}

MLP_PARAMS, MLP_HALF, MLP_INPUTS = 22915, 32256, 224
# public parameter layout: name, shape (input-major weights)
MLP_LAYOUT = [("W1", (224, 64)), ("b1", (64,)), ("W2", (64, 64)), ("b2", (64,)),
              ("W3", (64, 64)), ("b3", (64,)), ("W4", (64, 3)), ("b4", (3,))]
RAY_INTS = 12   # isaac_ray = 48 bytes


class Mlp(C.Structure):
    _fields_ = [("params", C.c_void_p), ("grads", C.c_void_p), ("adam_m", C.c_void_p),
                ("adam_v", C.c_void_p), ("half_w", C.c_void_p), ("step", C.c_int32)]


class Proposal(C.Structure):
    _fields_ = [("model", C.POINTER(Mlp)), ("grid", C.c_void_p), ("cell", C.c_int32),
                ("threshold", C.c_float), ("margin", C.c_int32), ("stats", C.c_void_p),
                ("widen", C.c_int32)]


class ServerConfig(C.Structure):
    _fields_ = [("budget_bytes", C.c_int64), ("n_streams", C.c_int32), ("max_batch", C.c_int32)]


class ServerRequest(C.Structure):
    _fields_ = [("camera", Camera), ("luts", C.c_void_p), ("chains", C.POINTER(Chain)),
                ("out", C.c_void_p), ("tag", C.c_int64)]


class ServerResult(C.Structure):
    _fields_ = [("tag", C.c_int64), ("status", C.c_int32), ("batch_size", C.c_int32),
                ("t_submit", C.c_double), ("t_launch", C.c_double), ("t_done", C.c_double),
                ("t_gpu_start", C.c_double), ("t_gpu_end", C.c_double), ("stream", C.c_int32),
                ("reserved", C.c_int32)]


def pack_mlp_params(named) -> np.ndarray:
    """Named arrays -> the flat float32 layout of the C ABI."""
    return np.concatenate([np.asarray(named[k], np.float32).reshape(-1) for k, _ in MLP_LAYOUT])


def unpack_mlp_params(flat) -> dict:
    flat = np.asarray(flat)
    out, o = {}, 0
    for k, shape in MLP_LAYOUT:
        size = int(np.prod(shape))
        out[k] = flat[o:o + size].reshape(shape)
        o += size
    return out


class IsaacError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"isaac error {code}: {msg}")
        self.code = code


_lib = None


def load(path: Optional[str] = None):
    """Load the CUDA library; raises if it was not built."""
    global _lib
    if _lib is None:
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"{p} is missing: build it with "
                               "`python -m paper_1611_09048_b300.build` (no CPU fallback exists)")
        lib = C.CDLL(p)
        lib.isaac_render.restype = C.c_int
        lib.isaac_render.argtypes = [C.POINTER(Source), C.POINTER(Chain), C.c_int32, C.c_void_p,
                                     C.c_void_p, C.POINTER(Camera), C.POINTER(Plane), C.c_int32,
                                     C.POINTER(RenderOpts), C.POINTER(Framebuffer), C.c_void_p]
        lib.isaac_pack_layout.restype = C.c_int
        lib.isaac_pack_layout.argtypes = [C.POINTER(Source), C.c_int32, C.c_uint32, C.c_void_p,
                                          C.c_int32, C.POINTER(Packed), C.POINTER(C.c_int64),
                                          C.POINTER(C.c_int64)]
        lib.isaac_pack.restype = C.c_int
        lib.isaac_pack.argtypes = [C.POINTER(Source), C.c_int32, C.c_uint32, C.c_void_p,
                                   C.c_int32, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64,
                                   C.POINTER(Packed), C.c_void_p]
        lib.isaac_render_packed.restype = C.c_int
        lib.isaac_render_packed.argtypes = [C.POINTER(Packed), C.POINTER(Chain), C.c_void_p,
                                            C.c_void_p, C.POINTER(Camera), C.POINTER(Plane),
                                            C.c_int32, C.POINTER(RenderOpts),
                                            C.POINTER(Framebuffer), C.c_void_p]
        lib.isaac_opacity_grid.restype = C.c_int
        lib.isaac_opacity_grid.argtypes = [C.POINTER(Source), C.POINTER(Chain), C.c_int32,
                                           C.c_void_p, C.c_void_p, C.POINTER(RenderOpts),
                                           C.c_int32, C.c_void_p, C.c_int64, C.c_void_p]
        lib.isaac_release_workspaces.restype = C.c_int
        lib.isaac_render_noalloc.restype = C.c_int
        lib.isaac_render_noalloc.argtypes = lib.isaac_render.argtypes
        render_args = list(lib.isaac_render.argtypes[:-1])
        lib.isaac_trace.restype = C.c_int
        lib.isaac_trace.argtypes = render_args + [C.POINTER(Proposal), C.c_void_p, C.c_int64,
                                                  C.c_void_p, C.c_void_p]
        lib.isaac_render_learned.restype = C.c_int
        lib.isaac_render_learned.argtypes = render_args + [C.POINTER(Proposal), C.c_void_p]
        lib.isaac_render_packed_learned.restype = C.c_int
        lib.isaac_render_packed_learned.argtypes = list(lib.isaac_render_packed.argtypes[:-1]) + \
            [C.POINTER(Proposal), C.c_void_p]
        lib.isaac_mlp_sync.restype = C.c_int
        lib.isaac_mlp_sync.argtypes = [C.POINTER(Mlp), C.c_void_p]
        lib.isaac_mlp_create.restype = C.c_int
        lib.isaac_mlp_create.argtypes = [C.POINTER(Mlp), C.c_int32, C.c_uint64, C.c_void_p]
        lib.isaac_mlp_destroy.restype = C.c_int
        lib.isaac_mlp_destroy.argtypes = [C.POINTER(Mlp)]
        lib.isaac_mlp_checkpoint_bytes.restype = C.c_int64
        lib.isaac_mlp_checkpoint_bytes.argtypes = [C.c_int32]
        lib.isaac_mlp_save.restype = C.c_int
        lib.isaac_mlp_save.argtypes = [C.POINTER(Mlp), C.c_uint64, C.c_void_p, C.c_int64, C.c_void_p]
        lib.isaac_mlp_load.restype = C.c_int
        lib.isaac_mlp_load.argtypes = [C.POINTER(Mlp), C.c_void_p, C.c_int64, C.POINTER(C.c_uint64),
                                       C.c_void_p]
        lib.isaac_mlp_features.restype = C.c_int
        lib.isaac_mlp_features.argtypes = [C.c_void_p, C.c_int64, C.c_void_p, C.c_float, C.c_void_p,
                                           C.c_int32, C.c_void_p, C.c_void_p]
        lib.isaac_mlp_forward.restype = C.c_int
        lib.isaac_mlp_forward.argtypes = [C.POINTER(Mlp), C.c_void_p, C.c_int64, C.c_void_p,
                                          C.c_void_p]
        lib.isaac_mlp_train_step.restype = C.c_int
        lib.isaac_mlp_train_step.argtypes = [C.POINTER(Mlp), C.c_void_p, C.c_void_p, C.c_int64,
                                             C.c_float, C.c_int32, C.c_void_p, C.c_void_p]
        lib.isaac_server_create.restype = C.c_int
        lib.isaac_server_create.argtypes = [C.POINTER(Source), C.POINTER(Chain), C.c_int32,
                                            C.c_void_p, C.c_void_p, C.POINTER(Packed),
                                            C.POINTER(RenderOpts), C.POINTER(Plane), C.c_int32,
                                            C.POINTER(ServerConfig), C.POINTER(C.c_void_p)]
        lib.isaac_server_submit.restype = C.c_int
        lib.isaac_server_submit.argtypes = [C.c_void_p, C.POINTER(ServerRequest)]
        lib.isaac_server_poll.restype = C.c_int
        lib.isaac_server_poll.argtypes = [C.c_void_p, C.POINTER(ServerResult), C.c_int32, C.c_double]
        lib.isaac_server_outstanding.restype = C.c_int
        lib.isaac_server_outstanding.argtypes = [C.c_void_p]
        lib.isaac_server_destroy.restype = C.c_int
        lib.isaac_server_destroy.argtypes = [C.c_void_p]
        lib.isaac_range_grid.restype = C.c_int
        lib.isaac_range_grid.argtypes = [C.POINTER(Source), C.c_int32, C.POINTER(RenderOpts),
                                         C.c_int32, C.c_void_p, C.c_int64, C.c_void_p]
        lib.isaac_render_skip.restype = C.c_int
        lib.isaac_render_skip.argtypes = list(lib.isaac_render.argtypes[:-1]) + \
            [C.c_void_p, C.c_int64, C.c_int32, C.c_void_p]
        lib.isaac_render_iso.restype = C.c_int
        lib.isaac_render_iso.argtypes = [C.POINTER(Source), C.POINTER(Chain), C.c_int32, C.c_void_p,
                                         C.c_void_p, C.POINTER(Camera), C.POINTER(Plane), C.c_int32,
                                         C.POINTER(RenderOpts), C.POINTER(Framebuffer), C.c_void_p]
        lib.isaac_composite.restype = C.c_int
        lib.isaac_composite.argtypes = [C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.c_int32,
                                        C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
        lib.isaac_probe_read.restype = C.c_int
        lib.isaac_probe_read.argtypes = [C.c_void_p, C.c_int64, C.c_int32, C.c_void_p, C.c_void_p]
        lib.isaac_opacity_grid_packed.restype = C.c_int
        lib.isaac_opacity_grid_packed.argtypes = [C.POINTER(Packed), C.POINTER(Chain), C.c_void_p,
                                                  C.c_void_p, C.POINTER(RenderOpts), C.c_int32,
                                                  C.c_void_p, C.c_int64, C.c_void_p]
        lib.isaac_copy_source.restype = C.c_int
        lib.isaac_copy_source.argtypes = [C.POINTER(Source), C.POINTER(C.c_int64), C.c_void_p,
                                          C.c_int64, C.POINTER(Source), C.c_void_p]
        lib.isaac_set_update_hook.restype = C.c_int
        lib.isaac_set_update_hook.argtypes = [UPDATE_FN, C.c_void_p]
        lib.isaac_time_march.restype = C.c_int
        lib.isaac_time_march.argtypes = [C.c_void_p, C.c_void_p]
        lib.isaac_last_error.restype = C.c_char_p
        lib.isaac_abi_version.restype = C.c_int
        _lib = lib
    return _lib


def check(rc: int):
    if rc != OK:
        raise IsaacError(rc, load().isaac_last_error().decode())


# ----------------------------------------------------------- marshalling

def make_chain(spec) -> Chain:
    """[("length",), ("mul", (a,)), ...] -> Chain (Sec. 3.3)."""
    ch = Chain()
    if len(spec) > MAX_FUNCTORS:
        raise ValueError(f"chain longer than {MAX_FUNCTORS}")
    ch.n_ops = len(spec)
    for i, f in enumerate(spec):
        args = tuple(f[1]) if len(f) > 1 else ()
        ch.ops[i].op = OPS[f[0]]
        ch.ops[i].n_args = len(args)
        for j, a in enumerate(args[:4]):
            ch.ops[i].arg[j] = float(a)
    return ch


def make_camera(mv, proj, width, height) -> Camera:
    cam = Camera()
    for i in range(16):
        cam.modelview[i] = float(mv[i])
        cam.projection[i] = float(proj[i])
    cam.width, cam.height = int(width), int(height)
    return cam


def make_opts(scene, mask=None, lanes=None) -> RenderOpts:
    o = RenderOpts()
    o.lanes_per_ray = LANES_PER_RAY if lanes is None else int(lanes)
    for a in range(3):
        o.n[a] = int(scene.n[a])
        o.global_n[a] = int(scene.gn[a])
        o.offset[a] = int(scene.off[a])
    o.step = float(scene.step)
    o.interp = int(scene.interp)
    o.term_alpha = float(scene.term)
    for c in range(4):
        o.bg[c] = float(scene.bg[c])
    o.active_mask = int(scene.mask if mask is None else mask)
    return o


def make_planes(clip):
    if len(clip) > MAX_CLIP:
        raise ValueError(f"more than {MAX_CLIP} clip planes")
    arr = (Plane * max(1, len(clip)))()
    for i, pl in enumerate(clip):
        arr[i].n[0], arr[i].n[1], arr[i].n[2] = (float(v) for v in pl[:3])
        arr[i].d = float(pl[3])
    return arr, len(clip)


def time_march(start=None, stop=None):
    """Record torch.cuda.Event ``start``/``stop`` around the march kernel of
    this thread's next frames (None, None: stop).  The events must have been
    recorded once before, so that their CUDA handles exist."""
    check(load().isaac_time_march(C.c_void_p(start.cuda_event) if start is not None else None,
                                  C.c_void_p(stop.cuda_event) if stop is not None else None))


def composite(layers, bg=(0.0, 0.0, 0.0, 0.0), out=None, rgba32=None, stream=None):
    """Sort-last compositing (isaac_composite) of ``layers``: a list of
    (rgba32, depth) device tensors of shape (H, W, 4) and (H, W)."""
    import torch
    H, W = layers[0][1].shape
    n = len(layers)
    rp = (C.c_void_p * n)(*[l[0].data_ptr() for l in layers])
    dp = (C.c_void_p * n)(*[l[1].data_ptr() for l in layers])
    if out is None:
        out = torch.empty((H, W, 4), dtype=torch.uint8, device=layers[0][0].device)
    bga = (C.c_float * 4)(*[float(v) for v in bg])
    check(load().isaac_composite(rp, dp, n, W, H, bga, out.data_ptr(),
                                 rgba32.data_ptr() if rgba32 is not None else None,
                                 _stream_handle(stream)))
    return out, rgba32


_update_keep = {}


def set_update_hook(fn):
    """Install ``fn(source, enabled)`` as this thread's per-source update
    callback (isaac_set_update_hook); None removes it."""
    import threading
    tid = threading.get_ident()
    if fn is None:
        check(load().isaac_set_update_hook(UPDATE_FN(), None))
        _update_keep.pop(tid, None)
        return
    cb = UPDATE_FN(lambda s, en, _u: fn(int(s), bool(en)))
    _update_keep[tid] = cb            # the C side keeps only the pointer
    check(load().isaac_set_update_hook(cb, None))


def copy_bytes(n, fdim, guard):
    """Bytes isaac_copy_source writes for an n-cell source."""
    g = 1 if guard >= 1 else 0
    return 4 * fdim * (n[0] + 2 * g) * (n[1] + 2 * g) * (n[2] + 2 * g)


def copy_source(src: "Source", n, dst, stream=None) -> "Source":
    """Copy a (non-persistent) source into device tensor ``dst``
    (isaac_copy_source); returns the descriptor of the copy."""
    out = Source()
    nn = (C.c_int64 * 3)(*[int(v) for v in n])
    check(load().isaac_copy_source(C.byref(src), nn, dst.data_ptr(),
                                   dst.numel() * dst.element_size(), C.byref(out),
                                   _stream_handle(stream)))
    return out


def probe_read(buf, passes, sink, stream=None):
    """Read device tensor ``buf`` ``passes`` times (isaac_probe_read)."""
    check(load().isaac_probe_read(buf.data_ptr(), buf.numel() * buf.element_size(), int(passes),
                                  sink.data_ptr(), _stream_handle(stream)))


def _stream_handle(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


class DeviceScene:
    """A synth.Scene whose sources and LUTs are resident in device memory.

    The fields are copied to the GPU once (standing in for simulation data that
    already lives there); ``render`` then launches frames against them."""

    def __init__(self, scene, device="cuda"):
        import torch
        self.scene = scene
        self.device = torch.device(device)
        self.data = []
        n_src = len(scene.sources)
        self.sources = (Source * n_src)()
        self.chains = (Chain * n_src)()
        for s, src in enumerate(scene.sources):
            if isinstance(src.data, torch.Tensor):       # already resident: used in place
                t = src.data.to(self.device, torch.float32).contiguous().reshape(-1)
            else:
                t = torch.from_numpy(np.ascontiguousarray(src.data, np.float32)).to(self.device)
            self.data.append(t)
            self._describe(s, src, t)
            self.chains[s] = make_chain(scene.chains[s])
        self.luts = torch.from_numpy(np.ascontiguousarray(scene.luts, np.float32)).to(self.device)
        self.weights = (C.c_float * n_src)(*[float(w) for w in scene.weights])

    def _describe(self, s, src, t):
        d = self.sources[s]
        d.ptr = t.data_ptr()
        d.extent = t.numel()
        d.offset = int(src.offset)
        for a in range(3):
            d.stride[a] = int(src.strides[a])
        d.comp_stride = int(src.cstride)
        d.f_dim = int(src.fdim)
        d.guard = int(src.guard)

    def copy_source(self, s, stream=None):
        """Replace source ``s`` by a copy made through its accessor
        (isaac_copy_source); the copy's buffer is kept with the scene."""
        import torch
        src = self.sources[s]
        nb = copy_bytes(self.scene.n, src.f_dim, src.guard)
        buf = torch.empty(nb // 4, dtype=torch.float32, device=self.device)
        self.sources[s] = copy_source(src, self.scene.n, buf, stream)
        self.data.append(buf)
        return buf

    def set_luts(self, luts):
        self.luts.copy_(self.luts.new_tensor(np.asarray(luts, np.float32)).reshape(self.luts.shape))

    def set_chain(self, s, spec):
        self.chains[s] = make_chain(spec)

    def footprint_words(self):
        nx, ny, nz = self.scene.n
        return ((nx + 2) * (ny + 2) * (nz + 2) + 31) // 32

    def prepare(self, mv=None, proj=None, out=None, rgba32=None, nsamples=None, mask=None,
                touched=None, lanes=None, depth=None, luts=None, staged=False):
        """Marshal one frame's arguments (camera, opts, framebuffer) once; the
        returned tuple can be launched repeatedly with ``launch``.  ``luts``: a
        device float32 tensor shaped like ``self.luts`` to read the transfer
        functions from instead (e.g. one of two buffers a pipeline uploads into
        in turn).  ``staged``: set ISAAC_MARCH_STAGED."""
        sc = self.scene
        cam = make_camera(sc.modelview if mv is None else mv,
                          sc.projection if proj is None else proj, sc.width, sc.height)
        planes, n_clip = make_planes(sc.clip)
        fb = Framebuffer(out.data_ptr(), rgba32.data_ptr() if rgba32 is not None else None,
                         nsamples.data_ptr() if nsamples is not None else None,
                         touched.data_ptr() if touched is not None else None,
                         depth.data_ptr() if depth is not None else None)
        opts = make_opts(sc, mask, lanes)
        if luts is None:
            luts = self.luts
            lut_ptr = luts.data_ptr()
        elif isinstance(luts, np.ndarray):     # host LUTs: copied by the call
            if luts.dtype != np.float32 or luts.size != self.luts.numel() or not luts.flags.c_contiguous:
                raise ValueError("host luts must be a contiguous float32 array of the scene's LUT size")
            opts.flags = LUTS_HOST
            lut_ptr = luts.ctypes.data
        elif luts.shape != self.luts.shape or luts.dtype != self.luts.dtype or not luts.is_contiguous() \
                or luts.device != self.luts.device:
            raise ValueError("luts must be a contiguous float32 tensor shaped like the scene's, on its device")
        else:
            lut_ptr = luts.data_ptr()
        if staged:
            opts.flags |= MARCH_STAGED
        keep = (cam, planes, fb, opts, luts)
        return (self.sources, self.chains, len(sc.sources), lut_ptr,
                C.cast(self.weights, C.c_void_p), C.byref(cam), planes, n_clip, C.byref(opts),
                C.byref(fb)), keep

    @staticmethod
    def launch(prepared, stream=None):
        args, _keep = prepared
        check(load().isaac_render(*args, _stream_handle(stream)))

    def render(self, mv=None, proj=None, out=None, rgba32=None, nsamples=None, stream=None,
               mask=None, want_f32=False, want_nsamp=False, touched=None, lanes=None,
               depth=None, luts=None, staged=False):
        """Enqueue one frame; returns (rgba8, rgba32 or None, nsamples or None)
        as device tensors (``depth``: optional (H, W) float32 output; ``luts``:
        a device tensor, or a host float32 array copied by the call)."""
        import torch
        W, H = self.scene.width, self.scene.height
        if out is None:
            out = torch.empty((H, W, 4), dtype=torch.uint8, device=self.device)
        if rgba32 is None and want_f32:
            rgba32 = torch.empty((H, W, 4), dtype=torch.float32, device=self.device)
        if nsamples is None and want_nsamp:
            nsamples = torch.empty((H, W), dtype=torch.int32, device=self.device)
        self.launch(self.prepare(mv, proj, out, rgba32, nsamples, mask, touched, lanes, depth, luts,
                                 staged), stream)
        return out, rgba32, nsamples


    def opacity_grid(self, cell=16, mask=None, stream=None, out=None, host_luts=None):
        """Max-opacity grid (Gz, Gy, Gx) float32 on the device (``host_luts``:
        a host float32 array to read the transfer functions from instead)."""
        import torch
        sc = self.scene
        G = [(int(k) + cell - 1) // cell for k in sc.n]
        if out is None:
            out = torch.empty((G[2], G[1], G[0]), dtype=torch.float32, device=self.device)
        opts = make_opts(sc, mask)
        lut_ptr = self.luts.data_ptr()
        if host_luts is not None:
            opts.flags = LUTS_HOST
            lut_ptr = np.ascontiguousarray(host_luts, np.float32).ctypes.data
        check(load().isaac_opacity_grid(self.sources, self.chains, len(sc.sources),
                                        lut_ptr, C.cast(self.weights, C.c_void_p),
                                        C.byref(opts), int(cell), out.data_ptr(), out.numel(),
                                        _stream_handle(stream)))
        return out

    def range_grid(self, cell=16, mask=None, stream=None, out=None):
        """Value-range grid (Gz, Gy, Gx, components, 2) float32 on the device."""
        import torch
        sc = self.scene
        m = int(sc.mask if mask is None else mask)
        slots = sum(int(src.fdim) for i, src in enumerate(sc.sources) if (m >> i) & 1)
        G = [(int(k) + cell - 1) // cell for k in sc.n]
        if out is None:
            out = torch.empty((G[2], G[1], G[0], slots, 2), dtype=torch.float32, device=self.device)
        opts = make_opts(sc, m)
        check(load().isaac_range_grid(self.sources, len(sc.sources), C.byref(opts), int(cell),
                                      out.data_ptr(), out.numel(), _stream_handle(stream)))
        return out

    def prepare_skip(self, ranges, cell, mv=None, proj=None, out=None, rgba32=None, nsamples=None,
                     mask=None, lanes=None):
        args, keep = self.prepare(mv, proj, out, rgba32, nsamples, mask, None, lanes)
        return args + (ranges.data_ptr(), ranges.numel(), int(cell)), keep + (ranges,)

    @staticmethod
    def launch_skip(prepared, stream=None):
        args, _keep = prepared
        check(load().isaac_render_skip(*args, _stream_handle(stream)))

    def render_skip(self, ranges, cell=16, mv=None, proj=None, out=None, stream=None, mask=None,
                    want_f32=False, want_nsamp=False, lanes=None):
        """isaac_render with empty-space skipping over ``ranges`` (range_grid)."""
        import torch
        W, H = self.scene.width, self.scene.height
        if out is None:
            out = torch.empty((H, W, 4), dtype=torch.uint8, device=self.device)
        f32 = torch.empty((H, W, 4), dtype=torch.float32, device=self.device) if want_f32 else None
        ns = torch.empty((H, W), dtype=torch.int32, device=self.device) if want_nsamp else None
        self.launch_skip(self.prepare_skip(ranges, cell, mv, proj, out, f32, ns, mask, lanes), stream)
        return out, f32, ns

    def prepare_iso(self, iso, mv=None, proj=None, out=None, rgba32=None, nsamples=None, mask=None,
                    depth=None):
        """Marshal one iso-surface frame (``iso``: one threshold per source)."""
        sc = self.scene
        cam = make_camera(sc.modelview if mv is None else mv,
                          sc.projection if proj is None else proj, sc.width, sc.height)
        planes, n_clip = make_planes(sc.clip)
        fb = Framebuffer(out.data_ptr(), rgba32.data_ptr() if rgba32 is not None else None,
                         nsamples.data_ptr() if nsamples is not None else None, None,
                         depth.data_ptr() if depth is not None else None)
        opts = make_opts(sc, mask)
        iso_arr = (C.c_float * len(sc.sources))(*[float(v) for v in iso])
        keep = (cam, planes, fb, opts, iso_arr)
        return (self.sources, self.chains, len(sc.sources), self.luts.data_ptr(),
                C.cast(iso_arr, C.c_void_p), C.byref(cam), planes, n_clip, C.byref(opts),
                C.byref(fb)), keep

    @staticmethod
    def launch_iso(prepared, stream=None):
        args, _keep = prepared
        check(load().isaac_render_iso(*args, _stream_handle(stream)))

    def render_iso(self, iso, mv=None, proj=None, out=None, stream=None, mask=None,
                   want_f32=False, want_nsamp=False, rgba32=None, depth=None):
        import torch
        W, H = self.scene.width, self.scene.height
        if out is None:
            out = torch.empty((H, W, 4), dtype=torch.uint8, device=self.device)
        f32 = rgba32
        if f32 is None and want_f32:
            f32 = torch.empty((H, W, 4), dtype=torch.float32, device=self.device)
        ns = torch.empty((H, W), dtype=torch.int32, device=self.device) if want_nsamp else None
        self.launch_iso(self.prepare_iso(iso, mv, proj, out, f32, ns, mask, depth), stream)
        return out, f32, ns

    def trace(self, mv=None, proj=None, out=None, proposal=None, capacity=None, stream=None,
              lanes=None, want_f32=False, want_nsamp=False):
        """Render and return the frame's ray list: (rays (cap, 12) int32
        records, count (1,) int32 on the device, rgba8, rgba32, nsamples)."""
        import torch
        W, H = self.scene.width, self.scene.height
        if out is None:
            out = torch.empty((H, W, 4), dtype=torch.uint8, device=self.device)
        f32 = torch.empty((H, W, 4), dtype=torch.float32, device=self.device) if want_f32 else None
        ns = torch.empty((H, W), dtype=torch.int32, device=self.device) if want_nsamp else None
        rays, count, _ = _trace(self, mv, proj, out, proposal, capacity, stream, lanes, f32, ns)
        return rays, count, out, f32, ns

    def prepare_learned(self, proposal, mv=None, proj=None, out=None, rgba32=None, nsamples=None,
                        lanes=None):
        args, keep = self.prepare(mv, proj, out, rgba32, nsamples, lanes=lanes)
        return args + (C.byref(proposal),), keep + (proposal,)

    @staticmethod
    def launch_learned(prepared, stream=None):
        args, _keep = prepared
        check(load().isaac_render_learned(*args, _stream_handle(stream)))

    def render_learned(self, proposal, mv=None, proj=None, out=None, stream=None, lanes=None,
                       want_f32=False, want_nsamp=False):
        import torch
        W, H = self.scene.width, self.scene.height
        if out is None:
            out = torch.empty((H, W, 4), dtype=torch.uint8, device=self.device)
        f32 = torch.empty((H, W, 4), dtype=torch.float32, device=self.device) if want_f32 else None
        ns = torch.empty((H, W), dtype=torch.int32, device=self.device) if want_nsamp else None
        self.launch_learned(self.prepare_learned(proposal, mv, proj, out, f32, ns, lanes), stream)
        return out, f32, ns

    # ----------------------------------------------------- packed copies

    def pack(self, dtype="bf16", mask=None, stream=None):
        """Packed copy of the active sources (device buffers owned by the
        returned PackedVolume)."""
        import torch
        sc = self.scene
        mask = sc.mask if mask is None else int(mask)
        n = (C.c_int64 * 3)(*[int(v) for v in sc.n])
        lay = Packed()
        db, sb = C.c_int64(), C.c_int64()
        lib = load()
        check(lib.isaac_pack_layout(self.sources, len(sc.sources), mask, C.cast(n, C.c_void_p),
                                    DTYPES[dtype], C.byref(lay), C.byref(db), C.byref(sb)))
        data = torch.empty(max(16, db.value), dtype=torch.uint8, device=self.device)
        scales = torch.empty(max(4, sb.value // 4), dtype=torch.float32, device=self.device) \
            if sb.value else None
        out = Packed()
        check(lib.isaac_pack(self.sources, len(sc.sources), mask, C.cast(n, C.c_void_p),
                             DTYPES[dtype], data.data_ptr(), db.value,
                             scales.data_ptr() if scales is not None else None, sb.value,
                             C.byref(out), _stream_handle(stream)))
        srcs = [s for i, s in enumerate(range(len(sc.sources))) if (mask >> i) & 1]
        pv = PackedVolume(self, out, data, scales, srcs)
        pv.mask, pv.dtype = mask, dtype
        return pv


class PackedVolume:
    """A packed (reduced-precision) copy of a DeviceScene's active sources."""

    def __init__(self, ds, desc, data, scales, src_index):
        self.ds, self.desc, self.data, self.scales = ds, desc, data, scales
        self.src_index = src_index      # original source index of each packed source
        n = len(src_index)
        self.chains = (Chain * n)(*[ds.chains[i] for i in src_index])
        self.weights = (C.c_float * n)(*[ds.weights[i] for i in src_index])
        self.luts = ds.luts[src_index].contiguous()

    def repack(self, stream=None):
        """Pack the scene's current source data again into this copy's buffers
        (the per-time-step refresh; allocates nothing)."""
        sc = self.ds.scene
        n = (C.c_int64 * 3)(*[int(v) for v in sc.n])
        out = Packed()
        check(load().isaac_pack(self.ds.sources, len(sc.sources), self.mask, C.cast(n, C.c_void_p),
                                DTYPES[self.dtype], self.data.data_ptr(), self.data.numel(),
                                self.scales.data_ptr() if self.scales is not None else None,
                                self.scales.numel() * 4 if self.scales is not None else 0,
                                C.byref(out), _stream_handle(stream)))
        self.desc = out
        return self

    def opacity_grid(self, cell=16, mask=None, stream=None, out=None):
        """Max-opacity grid of this copy (isaac_opacity_grid_packed), (Gz, Gy, Gx)
        float32 on the device: the grid of the dequantised fields."""
        import torch
        sc = self.ds.scene
        G = [(int(k) + cell - 1) // cell for k in sc.n]
        if out is None:
            out = torch.empty((G[2], G[1], G[0]), dtype=torch.float32, device=self.ds.device)
        opts = make_opts(sc, (1 << len(self.src_index)) - 1 if mask is None else mask)
        check(load().isaac_opacity_grid_packed(C.byref(self.desc), self.chains, self.luts.data_ptr(),
                                               C.cast(self.weights, C.c_void_p), C.byref(opts),
                                               int(cell), out.data_ptr(), out.numel(),
                                               _stream_handle(stream)))
        return out

    def prepare(self, mv=None, proj=None, out=None, rgba32=None, nsamples=None, mask=None,
                lanes=None):
        sc = self.ds.scene
        cam = make_camera(sc.modelview if mv is None else mv,
                          sc.projection if proj is None else proj, sc.width, sc.height)
        planes, n_clip = make_planes(sc.clip)
        fb = Framebuffer(out.data_ptr(), rgba32.data_ptr() if rgba32 is not None else None,
                         nsamples.data_ptr() if nsamples is not None else None, None)
        opts = make_opts(sc, (1 << len(self.src_index)) - 1 if mask is None else mask, lanes)
        keep = (cam, planes, fb, opts)
        return (C.byref(self.desc), self.chains, self.luts.data_ptr(),
                C.cast(self.weights, C.c_void_p), C.byref(cam), planes, n_clip, C.byref(opts),
                C.byref(fb)), keep

    @staticmethod
    def launch(prepared, stream=None):
        args, _keep = prepared
        check(load().isaac_render_packed(*args, _stream_handle(stream)))

    def prepare_learned(self, proposal, mv=None, proj=None, out=None, rgba32=None, nsamples=None,
                        mask=None, lanes=None):
        args, keep = self.prepare(mv, proj, out, rgba32, nsamples, mask, lanes)
        return args + (C.byref(proposal),), keep + (proposal,)

    @staticmethod
    def launch_learned(prepared, stream=None):
        args, _keep = prepared
        check(load().isaac_render_packed_learned(*args, _stream_handle(stream)))

    def render_learned(self, proposal, mv=None, proj=None, out=None, stream=None, want_f32=False,
                       want_nsamp=False, lanes=None):
        import torch
        W, H = self.ds.scene.width, self.ds.scene.height
        dev = self.ds.device
        if out is None:
            out = torch.empty((H, W, 4), dtype=torch.uint8, device=dev)
        f32 = torch.empty((H, W, 4), dtype=torch.float32, device=dev) if want_f32 else None
        ns = torch.empty((H, W), dtype=torch.int32, device=dev) if want_nsamp else None
        self.launch_learned(self.prepare_learned(proposal, mv, proj, out, f32, ns, None, lanes), stream)
        return out, f32, ns

    def render(self, mv=None, proj=None, out=None, stream=None, mask=None, want_f32=False,
               want_nsamp=False, lanes=None, rgba32=None):
        import torch
        W, H = self.ds.scene.width, self.ds.scene.height
        dev = self.ds.device
        if out is None:
            out = torch.empty((H, W, 4), dtype=torch.uint8, device=dev)
        f32 = rgba32
        if f32 is None and want_f32:
            f32 = torch.empty((H, W, 4), dtype=torch.float32, device=dev)
        ns = torch.empty((H, W), dtype=torch.int32, device=dev) if want_nsamp else None
        self.launch(self.prepare(mv, proj, out, f32, ns, mask, lanes), stream)
        return out, f32, ns


# ---------------------------------------------------------------- serving

class Server:
    """Continuous-batching render server over one DeviceScene (zero-copy
    sources) or PackedVolume (BF16 packed copy); see isaac_server_create.

    ``submit`` queues one request and returns its tag; the request's ``out``
    (a pinned host or device uint8 tensor of shape (H, W, 4)) is kept alive
    here until ``poll`` reports the request finished."""

    def __init__(self, target, budget=256 << 20, n_streams=4, max_batch=16, lanes=None):
        self.target = target
        lib = load()
        handle = C.c_void_p()
        cfg = ServerConfig(int(budget), int(n_streams), int(max_batch))
        if isinstance(target, PackedVolume):
            sc = target.ds.scene
            self.n_src = len(target.src_index)
            opts = make_opts(sc, (1 << self.n_src) - 1, lanes)
            planes, n_clip = make_planes(sc.clip)
            check(lib.isaac_server_create(None, target.chains, self.n_src, target.luts.data_ptr(),
                                          C.cast(target.weights, C.c_void_p), C.byref(target.desc),
                                          C.byref(opts), planes, n_clip, C.byref(cfg),
                                          C.byref(handle)))
        else:
            sc = target.scene
            self.n_src = len(sc.sources)
            opts = make_opts(sc, None, lanes)
            planes, n_clip = make_planes(sc.clip)
            check(lib.isaac_server_create(target.sources, target.chains, self.n_src,
                                          target.luts.data_ptr(), C.cast(target.weights, C.c_void_p),
                                          None, C.byref(opts), planes, n_clip, C.byref(cfg),
                                          C.byref(handle)))
        self.handle = handle
        self._live = {}
        self._next_tag = 0

    def submit(self, mv, proj, width, height, out, luts=None, chains=None):
        """Queue a request; ``luts`` (n_src, 256, 4) float32 host array and
        ``chains`` (list of n_src chain specs) override the server's."""
        rq = ServerRequest()
        rq.camera = make_camera(mv, proj, width, height)
        keep = [out]
        if luts is not None:
            la = np.ascontiguousarray(luts, np.float32).reshape(-1)
            if la.size != self.n_src * 256 * 4:
                raise ValueError(f"luts must hold {self.n_src} x 256 x 4 floats")
            keep.append(la)
            rq.luts = la.ctypes.data
        if chains is not None:
            if len(chains) != self.n_src:
                raise ValueError(f"chains must list {self.n_src} chains")
            ca = (Chain * self.n_src)(*[make_chain(c) for c in chains])
            keep.append(ca)
            rq.chains = ca
        rq.out = out.data_ptr()
        rq.tag = self._next_tag
        check(load().isaac_server_submit(self.handle, C.byref(rq)))
        self._live[rq.tag] = keep
        self._next_tag += 1
        return rq.tag

    def poll(self, max_results=256, wait=0.0):
        """Finished requests as dicts (tag, status, batch_size, t_submit,
        t_launch, t_done: host clock; t_gpu_start, t_gpu_end: device clock of
        the request's batch; stream; times in seconds since the server
        started)."""
        buf = (ServerResult * max_results)()
        n = load().isaac_server_poll(self.handle, buf, max_results, float(wait))
        if n < 0:
            check(n)
        out = []
        for i in range(n):
            r = buf[i]
            self._live.pop(r.tag, None)
            out.append({"tag": r.tag, "status": r.status, "batch_size": r.batch_size,
                        "t_submit": r.t_submit, "t_launch": r.t_launch, "t_done": r.t_done,
                        "t_gpu_start": r.t_gpu_start, "t_gpu_end": r.t_gpu_end,
                        "stream": r.stream})
        return out

    def outstanding(self):
        n = load().isaac_server_outstanding(self.handle)
        if n < 0:
            check(n)
        return n

    def drain(self, timeout=60.0):
        """Poll until every submitted request has finished; returns the results."""
        import time
        res, t_end = [], time.time() + timeout
        while self._live and time.time() < t_end:
            res += self.poll(wait=0.05)
        if self._live:
            raise TimeoutError(f"{len(self._live)} requests still outstanding")
        return res

    def close(self):
        if self.handle:
            check(load().isaac_server_destroy(self.handle))
            self.handle = None
            self._live.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------- learned proposal

class MLPModel:
    """Device buffers of the interval-proposal MLP (float32 master weights,
    gradients, Adam moments, FP16 kernel copy)."""

    def __init__(self, params_flat, device="cuda", train=True):
        import torch
        self.device = torch.device(device)
        flat = np.asarray(params_flat, np.float32).reshape(-1)
        assert flat.size == MLP_PARAMS
        self.params = torch.from_numpy(flat.copy()).to(self.device)
        z = lambda: torch.zeros(MLP_PARAMS, dtype=torch.float32, device=self.device)  # noqa: E731
        self.grads, self.m, self.v = (z(), z(), z()) if train else (None, None, None)
        self.half = torch.empty(MLP_HALF, dtype=torch.float16, device=self.device)
        self.desc = Mlp(self.params.data_ptr(), self.grads.data_ptr() if train else None,
                        self.m.data_ptr() if train else None, self.v.data_ptr() if train else None,
                        self.half.data_ptr(), 0)
        check(load().isaac_mlp_sync(C.byref(self.desc), None))

    @property
    def step(self):
        return self.desc.step

    def named(self):
        return unpack_mlp_params(self.params.cpu().numpy())

    def save(self, tag=0, stream=None) -> bytes:
        """Checkpoint image (header, parameters, Adam moments when training)."""
        return checkpoint_save(self.desc, tag, stream)

    def load(self, image, stream=None) -> int:
        """Restore from a checkpoint image; returns its tag."""
        return checkpoint_load(self.desc, image, stream)


    def forward(self, X, stream=None):
        import torch
        U = torch.empty((X.shape[0], 3), dtype=torch.float32, device=self.device)
        check(load().isaac_mlp_forward(C.byref(self.desc), X.data_ptr(), X.shape[0], U.data_ptr(),
                                       _stream_handle(stream)))
        return U

    def train_step(self, X, rays, lr=1e-3, margin=2, loss_sum=None, stream=None):
        check(load().isaac_mlp_train_step(C.byref(self.desc), X.data_ptr(), rays.data_ptr(),
                                          X.shape[0], float(lr), int(margin),
                                          loss_sum.data_ptr() if loss_sum is not None else None,
                                          _stream_handle(stream)))

    def proposal(self, grid, cell, threshold=0.9, margin=2, stats=None, widen=True):
        p = Proposal(C.pointer(self.desc), grid.data_ptr(), int(cell), float(threshold), int(margin),
                     stats.data_ptr() if stats is not None else None, 1 if widen else 0)
        p._keep = (grid, stats)
        return p


def grid_proposal(grid, cell, stats=None):
    """A proposal without a network: every ray marches the hull of its samples
    in macro cells whose max-opacity grid value is nonzero."""
    p = Proposal(None, grid.data_ptr(), int(cell), 0.0, 0,
                 stats.data_ptr() if stats is not None else None, 1)
    p._keep = (grid, stats)
    return p


def checkpoint_save(desc, tag=0, stream=None) -> bytes:
    lib = load()
    n = lib.isaac_mlp_checkpoint_bytes(1 if desc.adam_m and desc.adam_v else 0)
    buf = (C.c_ubyte * n)()
    check(lib.isaac_mlp_save(C.byref(desc), int(tag), buf, n, _stream_handle(stream)))
    return bytes(buf)


def checkpoint_load(desc, image, stream=None) -> int:
    tag = C.c_uint64(0)
    data = bytes(image)
    check(load().isaac_mlp_load(C.byref(desc), data, len(data), C.byref(tag), _stream_handle(stream)))
    return int(tag.value)


class LibraryMLP:
    """A proposal network whose buffers the library allocates
    (isaac_mlp_create) and frees (close / isaac_mlp_destroy)."""

    def __init__(self, train=True, seed=0, stream=None):
        self.desc = Mlp()
        check(load().isaac_mlp_create(C.byref(self.desc), 1 if train else 0, int(seed),
                                      _stream_handle(stream)))

    @property
    def step(self):
        return self.desc.step

    def params(self) -> np.ndarray:
        out = np.empty(MLP_PARAMS, np.float32)
        C.memmove(out.ctypes.data, self.save()[64:64 + 4 * MLP_PARAMS], 4 * MLP_PARAMS)
        return out

    def train_step(self, X, rays, lr=1e-3, margin=2, loss_sum=None, stream=None):
        check(load().isaac_mlp_train_step(C.byref(self.desc), X.data_ptr(), rays.data_ptr(),
                                          X.shape[0], float(lr), int(margin),
                                          loss_sum.data_ptr() if loss_sum is not None else None,
                                          _stream_handle(stream)))

    def save(self, tag=0, stream=None) -> bytes:
        return checkpoint_save(self.desc, tag, stream)

    def load(self, image, stream=None) -> int:
        return checkpoint_load(self.desc, image, stream)

    def close(self):
        if self.desc.params:
            check(load().isaac_mlp_destroy(C.byref(self.desc)))


def mlp_features(rays, n_rays, vol_n, step, grid, cell, stream=None):
    """Inputs (n_rays, 224) FP16 of ray records (tensor (N, 12) int32)."""
    import torch
    X = torch.empty((max(1, n_rays), MLP_INPUTS), dtype=torch.float16, device=rays.device)
    nn_ = (C.c_int64 * 3)(*[int(v) for v in vol_n])
    check(load().isaac_mlp_features(rays.data_ptr(), int(n_rays), C.cast(nn_, C.c_void_p), float(step),
                                    grid.data_ptr(), int(cell), X.data_ptr(), _stream_handle(stream)))
    return X[:n_rays]


def _trace(ds, mv, proj, out, proposal, capacity, stream, lanes, rgba32=None, nsamples=None):
    import torch
    sc = ds.scene
    if capacity is None:
        capacity = sc.width * sc.height
    rays = torch.zeros((max(1, capacity), RAY_INTS), dtype=torch.int32, device=ds.device)
    count = torch.zeros(1, dtype=torch.int32, device=ds.device)
    args, keep = ds.prepare(mv, proj, out, rgba32, nsamples, lanes=lanes)
    check(load().isaac_trace(*args, C.byref(proposal) if proposal is not None else None,
                             rays.data_ptr(), capacity, count.data_ptr(), _stream_handle(stream)))
    return rays, count, keep


def render(scene, **kw):
    """One-shot convenience: upload ``scene`` and render it on the current GPU."""
    return DeviceScene(scene).render(**kw)
