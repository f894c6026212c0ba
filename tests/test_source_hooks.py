"""The rest of the source contract of Sec. 3.2 on the host, no GPU work: the
per-source update callback runs for every source in order, with its active
bit, before the descriptors are read (a descriptor the callback rewrites is
the one validated), and isaac_copy_source rejects malformed copies before
enqueuing anything."""
import ctypes as C

import pytest

from paper_1611_09048_b300 import isaac
from test_abi import FAKE, _call, _valid_call_args


@pytest.fixture
def hook_calls():
    calls = []
    yield calls
    isaac.set_update_hook(None)


def _three_sources(a):
    src = (isaac.Source * 3)(a["src"][0], isaac.Source(), a["src"][0])
    a["src"] = src
    a["chains"] = (isaac.Chain * 3)()
    a["weights"] = (C.c_float * 3)(1.0, 1.0, 1.0)
    a["n_src"] = 3
    a["opts"].active_mask = 0b101
    return a


def test_update_hook_runs_for_every_source_in_order(hook_calls):
    a = _three_sources(_valid_call_args())
    a["fb"] = isaac.Framebuffer(None, None, None, None)     # fails after the sources
    isaac.set_update_hook(lambda s, en: hook_calls.append((s, en)))
    assert _call(a) == isaac.EINVAL
    assert "rgba8" in isaac.load().isaac_last_error().decode()
    assert hook_calls == [(0, True), (1, False), (2, True)]


def test_update_hook_sees_descriptors_before_validation(hook_calls):
    """The callback rewrites source 2's descriptor (a derived field placed in a
    fresh buffer); the call validates the rewritten one."""
    a = _three_sources(_valid_call_args())

    def upd(s, en):
        hook_calls.append(s)
        if s == 2:
            a["src"][2].f_dim = 6
    isaac.set_update_hook(upd)
    assert _call(a) == isaac.EINVAL
    msg = isaac.load().isaac_last_error().decode()
    assert "source 2" in msg and "f_dim 6" in msg, msg
    assert hook_calls == [0, 1, 2]


def test_update_hook_removed_and_skipped_on_early_failure(hook_calls):
    a = _three_sources(_valid_call_args())
    isaac.set_update_hook(lambda s, en: hook_calls.append(s))
    a["opts"].step = -1.0                                    # camera/options fail first
    assert _call(a) == isaac.EINVAL and hook_calls == []
    a["opts"].step = 0.5
    isaac.set_update_hook(None)
    a["fb"] = isaac.Framebuffer(None, None, None, None)
    assert _call(a) == isaac.EINVAL and hook_calls == []


def test_update_hook_is_per_thread(hook_calls):
    import threading
    isaac.set_update_hook(lambda s, en: hook_calls.append(("main", s)))
    a = _three_sources(_valid_call_args())
    a["fb"] = isaac.Framebuffer(None, None, None, None)
    t = threading.Thread(target=lambda: _call(a))
    t.start()
    t.join()
    assert hook_calls == []
    _call(a)
    assert hook_calls == [("main", 0), ("main", 1), ("main", 2)]


def test_opacity_grid_and_pack_call_the_hook(hook_calls):
    lib = isaac.load()
    a = _three_sources(_valid_call_args())
    isaac.set_update_hook(lambda s, en: hook_calls.append(s))
    rc = lib.isaac_opacity_grid(a["src"], a["chains"], 3, FAKE, C.cast(a["weights"], C.c_void_p),
                                C.byref(a["opts"]), 4, FAKE, 0, None)
    assert rc == isaac.ENOMEM and hook_calls == []          # size checks precede the sources
    a["weights"][0] = float("nan")                           # fails on the first source read
    rc = lib.isaac_opacity_grid(a["src"], a["chains"], 3, FAKE, C.cast(a["weights"], C.c_void_p),
                                C.byref(a["opts"]), 4, FAKE, 8, None)
    assert rc == isaac.EINVAL and "weight 0" in lib.isaac_last_error().decode()
    assert hook_calls == [0, 1, 2]
    del hook_calls[:]
    n = (C.c_int64 * 3)(8, 8, 8)
    out = isaac.Packed()
    rc = lib.isaac_pack(a["src"], 3, 0b101, n, isaac.BF16, FAKE, 0, None, 0, C.byref(out), None)
    assert rc == isaac.ENOMEM and hook_calls == [0, 1, 2]


def _copy(src, n, dst, nbytes):
    lib = isaac.load()
    out = isaac.Source()
    nn = (C.c_int64 * 3)(*n)
    rc = lib.isaac_copy_source(C.byref(src), nn, dst, nbytes, C.byref(out), None)
    return rc, isaac.load().isaac_last_error().decode()


def test_copy_source_validates_before_enqueuing():
    src = _valid_call_args(n=8, fdim=3, guard=2)["src"][0]
    need = isaac.copy_bytes((8, 8, 8), 3, 2)
    assert need == 4 * 3 * 10 ** 3
    lib = isaac.load()
    assert lib.isaac_copy_source(None, (C.c_int64 * 3)(8, 8, 8), FAKE, need, None, None) == isaac.EINVAL
    assert _copy(src, (8, 0, 8), FAKE, need)[0] == isaac.EINVAL
    rc, msg = _copy(src, (8, 8, 8), FAKE + 4, need)
    assert rc == isaac.EINVAL and "16-byte" in msg
    rc, msg = _copy(src, (8, 8, 8), FAKE, need - 4)
    assert rc == isaac.ENOMEM and str(need) in msg
    # the highest element a trilinear frame reads: cell (8, 8, 8) (one guard
    # layer past the interior), last component
    hi = src.offset + 8 * (src.stride[0] + src.stride[1] + src.stride[2]) + 2
    src.extent = hi                                          # one element short
    rc, msg = _copy(src, (8, 8, 8), FAKE, need)
    assert rc == isaac.EGUARD, msg
    src.f_dim = 0
    assert _copy(src, (8, 8, 8), FAKE, need)[0] == isaac.EINVAL


def test_copy_bytes_guard_rule():
    assert isaac.copy_bytes((4, 5, 6), 1, 0) == 4 * 4 * 5 * 6
    assert isaac.copy_bytes((4, 5, 6), 2, 1) == 4 * 2 * 6 * 7 * 8
    assert isaac.copy_bytes((4, 5, 6), 2, 4) == 4 * 2 * 6 * 7 * 8   # one guard layer at most
