"""The C-ABI library loads, exports every symbol the header declares, and
rejects malformed calls on the host (no GPU work is issued by these calls)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_1611_09048_b300 import isaac

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*[A-Za-z_][\w\s\*]*?\b(isaac_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


def test_library_exports_every_declared_symbol():
    lib = isaac.load()
    declared = _declared_functions()
    assert "isaac_render" in declared
    for name in declared:
        assert hasattr(lib, name), name
    assert set(isaac.EXPORTS) <= declared


def test_abi_version():
    assert isaac.load().isaac_abi_version() == 3


def test_struct_sizes_match_header_layout():
    # sizes implied by the header's field order on LP64
    assert C.sizeof(isaac.Source) == 8 + 8 + 8 + 24 + 8 + 4 + 4
    assert C.sizeof(isaac.Functor) == 4 + 4 + 16
    assert C.sizeof(isaac.Chain) == 4 + 24 * isaac.MAX_FUNCTORS
    assert C.sizeof(isaac.Camera) == 256 + 8
    assert C.sizeof(isaac.Framebuffer) == 5 * 8
    # 9 int64, step, interp, term_alpha, bg[4], active_mask, lanes_per_ray, flags -> 112
    assert C.sizeof(isaac.RenderOpts) == 112
    assert isaac.RenderOpts.flags.offset == 108


FAKE = 0x7F0000000000  # never dereferenced: every call below fails validation first


def _valid_call_args(n=8, fdim=1, guard=0, width=16, height=16):
    S = n + 2 * guard
    src = (isaac.Source * 1)()
    src[0].ptr = FAKE
    src[0].extent = S ** 3 * fdim
    src[0].offset = guard * (fdim + fdim * S + fdim * S * S)
    src[0].stride[0], src[0].stride[1], src[0].stride[2] = fdim, fdim * S, fdim * S * S
    src[0].comp_stride = 1
    src[0].f_dim = fdim
    src[0].guard = guard
    chains = (isaac.Chain * 1)()
    weights = (C.c_float * 1)(1.0)
    mv = np.eye(4).reshape(16)
    mv[14] = -3.0 * n
    from paper_1611_09048_b300 import synth
    proj = synth.perspective(60.0, 1.0, 0.1, 10.0 * n)
    cam = isaac.make_camera(mv, proj, width, height)
    opts = isaac.RenderOpts()
    for a in range(3):
        opts.n[a] = n
    opts.step = 0.5
    opts.interp = 1
    opts.term_alpha = 0.99
    opts.active_mask = 1
    fb = isaac.Framebuffer(FAKE, None, None, None)
    return dict(src=src, chains=chains, n_src=1, luts=FAKE, weights=weights, cam=cam,
                clip=None, n_clip=0, opts=opts, fb=fb)


def _call(a):
    lib = isaac.load()
    return lib.isaac_render(a["src"], a["chains"], a["n_src"], a["luts"],
                            C.cast(a["weights"], C.c_void_p), C.byref(a["cam"]), a["clip"],
                            a["n_clip"], C.byref(a["opts"]), C.byref(a["fb"]), None)


def _expect(a, code, fragment):
    rc = _call(a)
    msg = isaac.load().isaac_last_error().decode()
    assert rc == code, (rc, msg)
    assert fragment in msg, msg


def test_rejects_bad_fdim():
    a = _valid_call_args()
    a["src"][0].f_dim = 5
    _expect(a, isaac.EINVAL, "f_dim")


def test_rejects_guard_beyond_allocation():
    a = _valid_call_args(guard=0)
    a["src"][0].guard = 2          # declares guards the storage does not hold
    _expect(a, isaac.EGUARD, "extent")


def test_rejects_extent_too_small():
    a = _valid_call_args()
    a["src"][0].extent -= 1
    _expect(a, isaac.EGUARD, "extent")


def test_rejects_chain_argument_count():
    a = _valid_call_args(fdim=3)
    a["chains"][0] = isaac.make_chain([("mul", (1.0, 2.0))])
    _expect(a, isaac.EINVAL, "arguments")


def test_rejects_unknown_functor():
    a = _valid_call_args()
    a["chains"][0].n_ops = 1
    a["chains"][0].ops[0].op = 42
    _expect(a, isaac.EINVAL, "unknown op")


def test_rejects_nan_weight():
    a = _valid_call_args()
    a["weights"][0] = float("nan")
    _expect(a, isaac.EINVAL, "weight")


def test_rejects_singular_camera():
    a = _valid_call_args()
    for i in range(16):
        a["cam"].projection[i] = 0.0
    _expect(a, isaac.EINVAL, "singular")


def test_rejects_bad_step_and_sizes():
    a = _valid_call_args()
    a["opts"].step = 0.0
    _expect(a, isaac.EINVAL, "step")
    a = _valid_call_args()
    a["cam"].width = 0
    _expect(a, isaac.EINVAL, "image size")
    a = _valid_call_args()
    a["opts"].global_n[0], a["opts"].global_n[1], a["opts"].global_n[2] = 8, 8, 8
    a["opts"].offset[0] = 1
    _expect(a, isaac.EINVAL, "global size")


def test_rejects_mask_bits_beyond_sources():
    a = _valid_call_args()
    a["opts"].active_mask = 0b11
    _expect(a, isaac.EINVAL, "active_mask")


def test_rejects_too_many_active_sources():
    a = _valid_call_args()
    n = 5
    src = (isaac.Source * n)(*[a["src"][0]] * n)
    a["src"] = src
    a["chains"] = (isaac.Chain * n)()
    a["weights"] = (C.c_float * n)(*([1.0] * n))
    a["n_src"] = n
    a["opts"].active_mask = (1 << n) - 1
    _expect(a, isaac.ENOTSUP, "active sources")


def test_disabled_source_may_be_null():
    """A NULL inactive source passes validation (it is never read); the call
    then fails only on the deliberately missing framebuffer."""
    a = _valid_call_args()
    src = (isaac.Source * 2)(a["src"][0], isaac.Source())
    a["src"] = src
    a["chains"] = (isaac.Chain * 2)()
    a["weights"] = (C.c_float * 2)(1.0, 1.0)
    a["n_src"] = 2
    a["opts"].active_mask = 0b01
    a["fb"] = isaac.Framebuffer(None, None, None, None)
    _expect(a, isaac.EINVAL, "rgba8")


def test_rejects_misaligned_lut():
    a = _valid_call_args()
    a["luts"] = FAKE + 4
    _expect(a, isaac.EINVAL, "16-byte")


def test_rejects_unknown_opts_flags():
    a = _valid_call_args()
    a["opts"].flags = 0x6
    _expect(a, isaac.EINVAL, "flags")


# ------------------------------------------------------------ serving loop

def test_server_struct_sizes():
    assert C.sizeof(isaac.ServerConfig) == 8 + 4 + 4
    assert C.sizeof(isaac.ServerRequest) == (256 + 8) + 8 + 8 + 8 + 8
    assert C.sizeof(isaac.ServerResult) == 8 + 4 + 4 + 5 * 8 + 4 + 4


def _server_create(a, cfg, vol=None):
    lib = isaac.load()
    h = C.c_void_p()
    rc = lib.isaac_server_create(a["src"], a["chains"], a["n_src"], a["luts"],
                                 C.cast(a["weights"], C.c_void_p), vol, C.byref(a["opts"]),
                                 a["clip"], a["n_clip"], C.byref(cfg), C.byref(h))
    return rc, h, lib.isaac_last_error().decode()


@pytest.mark.parametrize("cfg,fragment", [
    ((1 << 20, 0, 4), "n_streams"),
    ((1 << 20, 9, 4), "n_streams"),
    ((1 << 20, 2, 0), "max_batch"),
    ((1 << 20, 2, 65), "max_batch"),
    ((1 << 19, 2, 4), "budget"),
])
def test_server_create_rejects_bad_config(cfg, fragment):
    rc, h, msg = _server_create(_valid_call_args(), isaac.ServerConfig(*cfg))
    assert rc == isaac.EINVAL and fragment in msg and not h.value, (rc, msg)


def test_server_create_rejects_bad_sources_before_any_allocation():
    a = _valid_call_args(fdim=5)
    rc, h, msg = _server_create(a, isaac.ServerConfig(1 << 20, 1, 4))
    assert rc == isaac.EINVAL and "f_dim" in msg and not h.value
    a = _valid_call_args()
    a["luts"] = FAKE + 4
    rc, h, msg = _server_create(a, isaac.ServerConfig(1 << 20, 1, 4))
    assert rc == isaac.EINVAL and "16-byte" in msg and not h.value


def test_server_calls_reject_null_handles():
    lib = isaac.load()
    rq = isaac.ServerRequest()
    assert lib.isaac_server_submit(None, C.byref(rq)) == isaac.EINVAL
    res = (isaac.ServerResult * 4)()
    assert lib.isaac_server_poll(None, res, 4, 0.0) == isaac.EINVAL
    assert lib.isaac_server_outstanding(None) == isaac.EINVAL
    assert lib.isaac_server_destroy(None) == isaac.OK


def test_time_march_wants_both_events_or_neither():
    lib = isaac.load()
    assert lib.isaac_time_march(C.c_void_p(FAKE), None) == isaac.EINVAL
    assert "both" in lib.isaac_last_error().decode()
    assert lib.isaac_time_march(None, None) == isaac.OK


def test_range_grid_and_skip_validate_before_any_launch():
    lib = isaac.load()
    a = _valid_call_args()
    assert lib.isaac_range_grid(a["src"], 1, C.byref(a["opts"]), 1, FAKE, 1 << 20, None) == isaac.EINVAL
    assert "cell" in lib.isaac_last_error().decode()
    # 8 x 8 x 8 cells, cell 4: 2^3 macro cells x 1 component x 2 floats
    assert lib.isaac_range_grid(a["src"], 1, C.byref(a["opts"]), 4, FAKE, 15, None) == isaac.ENOMEM
    rc = lib.isaac_render_skip(a["src"], a["chains"], 1, a["luts"], C.cast(a["weights"], C.c_void_p),
                               C.byref(a["cam"]), None, 0, C.byref(a["opts"]), C.byref(a["fb"]),
                               FAKE, 15, 4, None)
    assert rc == isaac.EINVAL and "ranges holds 15" in lib.isaac_last_error().decode()


def test_composite_validates_before_any_launch():
    lib = isaac.load()
    one = (C.c_void_p * 1)(FAKE)
    bg = (C.c_float * 4)(0, 0, 0, 0)
    assert lib.isaac_composite(one, one, 0, 4, 4, bg, FAKE, None, None) == isaac.EINVAL
    assert lib.isaac_composite(one, one, 17, 4, 4, bg, FAKE, None, None) == isaac.EINVAL
    bad = (C.c_void_p * 1)(FAKE + 4)
    assert lib.isaac_composite(bad, one, 1, 4, 4, bg, FAKE, None, None) == isaac.EINVAL
    assert "misaligned" in lib.isaac_last_error().decode()
    nan = (C.c_float * 4)(float("nan"), 0, 0, 0)
    assert lib.isaac_composite(one, one, 1, 4, 4, nan, FAKE, None, None) == isaac.EINVAL


def test_opacity_grid_packed_validates_before_any_launch():
    lib = isaac.load()
    a = _valid_call_args(n=8)
    vol = isaac.Packed()
    vol.data = FAKE
    vol.n[0] = vol.n[1] = vol.n[2] = 8
    vol.dtype = isaac.BF16
    vol.n_src = 1
    vol.f_dim[0] = 1
    vol.n_comp = 1
    vol.pad = 1

    def call(v, cell=4, grid_len=8, opts=None):
        return lib.isaac_opacity_grid_packed(C.byref(v) if v is not None else None, a["chains"], FAKE,
                                             C.cast(a["weights"], C.c_void_p),
                                             C.byref(opts or a["opts"]), cell, FAKE, grid_len, None)
    assert call(None) == isaac.EINVAL
    assert call(vol, cell=1) == isaac.EINVAL
    rc = call(vol, grid_len=7)
    assert rc == isaac.ENOMEM and "grid holds 7" in lib.isaac_last_error().decode()
    bad = isaac.Packed.from_buffer_copy(vol)
    bad.pad = 3
    assert call(bad) == isaac.EINVAL
    other = isaac.RenderOpts.from_buffer_copy(a["opts"])
    other.n[0] = 9
    rc = call(vol, opts=other)
    assert rc == isaac.EINVAL and "differs" in lib.isaac_last_error().decode()
    e4 = isaac.Packed.from_buffer_copy(vol)
    e4.dtype = isaac.E4M3
    assert call(e4) == isaac.EINVAL                       # E4M3 without scales
