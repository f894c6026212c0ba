"""Checkpoint / resume of the proposal network (isaac_mlp_save/load,
isaac_mlp_create/destroy) and bitwise-reproducible training: N steps, save,
M more steps equals N steps, load into a fresh model, M more steps, bit for
bit (parameters, Adam moments and step)."""
import ctypes as C
import struct
import zlib

import numpy as np
import pytest

from paper_1611_09048_b300 import isaac, synth

HEADER = 64


def _image(n_params=isaac.MLP_PARAMS, adam=False, step=7, tag=99, version=1, magic=b"ISAACMLP"):
    payload = np.random.default_rng(1).standard_normal(n_params * (3 if adam else 1)).astype("<f4")
    body = payload.tobytes()
    head = struct.pack("<8sIIiIQI", magic, version, n_params, step, 1 if adam else 0, tag,
                       zlib.crc32(body))
    return head + b"\0" * (HEADER - len(head)) + body


def _load_rc(image):
    lib = isaac.load()
    desc = isaac.Mlp()                      # no buffers: a valid image fails only at the model check
    tag = C.c_uint64(0)
    rc = lib.isaac_mlp_load(C.byref(desc), image, len(image), C.byref(tag), None)
    return rc, lib.isaac_last_error().decode()


def test_checkpoint_sizes():
    lib = isaac.load()
    assert lib.isaac_mlp_checkpoint_bytes(0) == HEADER + 4 * isaac.MLP_PARAMS
    assert lib.isaac_mlp_checkpoint_bytes(1) == HEADER + 12 * isaac.MLP_PARAMS


def test_load_validates_the_image_on_the_host():
    """Every check runs before any device work: a well-formed image whose
    CRC was computed by zlib passes the checksum (and fails only at the
    missing model buffers); each corruption is named."""
    good = _image()
    rc, msg = _load_rc(good)
    assert rc == isaac.EINVAL and "model params" in msg
    rc, msg = _load_rc(_image(adam=True))
    assert rc == isaac.EINVAL and "model params" in msg
    bad = bytearray(good)
    bad[HEADER + 100] ^= 0x01
    assert _load_rc(bytes(bad)) == (isaac.EINVAL, "checkpoint checksum mismatch (corrupt image)")
    assert "not a proposal-network" in _load_rc(_image(magic=b"ISAACXXX"))[1]
    assert "version" in _load_rc(_image(version=2))[1]
    assert "parameters" in _load_rc(_image(n_params=1000))[1]
    assert "truncated" in _load_rc(good[:-4])[1]
    assert "shorter than the header" in _load_rc(good[:10])[1]


def _records(rays):
    N = len(rays["nsteps"])
    rec = np.zeros((N, 12), np.int32)
    f = rec.view(np.float32)
    f[:, 0:3] = rays["e"]
    rec[:, 3] = rays["nsteps"]
    f[:, 4:7] = rays["d"]
    rec[:, 7] = np.arange(N)
    rec[:, 9] = rays["jf"]
    rec[:, 10] = rays["jl"]
    return rec


def _batches(k, n=3000, seed=0):
    import torch
    out = []
    for i in range(k):
        rr = synth.random_rays(n, (64, 64, 64), seed=seed + i)
        X = np.random.default_rng(1000 + seed + i).uniform(-1, 1, (n, 224)).astype(np.float16)
        out.append((torch.from_numpy(X).cuda(), torch.from_numpy(_records(rr)).cuda()))
    return out


def _state(model):
    return (model.params.cpu().numpy().copy(), model.m.cpu().numpy().copy(),
            model.v.cpu().numpy().copy(), model.step)


@pytest.mark.gpu
def test_training_is_bitwise_reproducible(cuda_ok):
    import torch
    flat = isaac.pack_mlp_params(synth.mlp_params(4, bias_scale=0.1))
    data = _batches(4)
    states = []
    for _ in range(2):
        model = isaac.MLPModel(flat)
        loss = torch.zeros(1, dtype=torch.float32, device="cuda")
        for X, R in data:
            model.train_step(X, R, lr=2e-3, margin=2, loss_sum=loss)
        torch.cuda.synchronize()
        states.append(_state(model) + (float(loss.item()),))
    for a, b in zip(states[0], states[1]):
        if isinstance(a, np.ndarray):
            np.testing.assert_array_equal(a, b)
        else:
            assert a == b


@pytest.mark.gpu
def test_resume_from_checkpoint_equals_uninterrupted_run(cuda_ok, tmp_path):
    import torch
    flat = isaac.pack_mlp_params(synth.mlp_params(5, bias_scale=0.1))
    data = _batches(6, seed=20)
    a = isaac.MLPModel(flat)
    for X, R in data[:3]:
        a.train_step(X, R, lr=2e-3)
    image = a.save(tag=3)
    (tmp_path / "proposal.ckpt").write_bytes(image)
    for X, R in data[3:]:
        a.train_step(X, R, lr=2e-3)
    torch.cuda.synchronize()
    want = _state(a)
    # a fresh model with other weights, restored from the file
    b = isaac.MLPModel(isaac.pack_mlp_params(synth.mlp_params(99)))
    assert b.load((tmp_path / "proposal.ckpt").read_bytes()) == 3
    assert b.step == 3
    for X, R in data[3:]:
        b.train_step(X, R, lr=2e-3)
    torch.cuda.synchronize()
    got = _state(b)
    for x, y in zip(want, got):
        if isinstance(x, np.ndarray):
            np.testing.assert_array_equal(x, y)
        else:
            assert x == y
    assert want[3] == 6
    # the image holds what the model held at save time
    p3 = np.frombuffer(image[HEADER:HEADER + 4 * isaac.MLP_PARAMS], "<f4")
    assert not np.array_equal(p3, want[0])


@pytest.mark.gpu
def test_create_destroy_and_inference_checkpoint(cuda_ok):
    import torch
    m1 = isaac.LibraryMLP(train=True, seed=11)
    m2 = isaac.LibraryMLP(train=False, seed=11)
    p1, p2 = m1.params(), m2.params()
    np.testing.assert_array_equal(p1, p2)
    w1 = isaac.unpack_mlp_params(p1)
    lim = np.sqrt(6.0 / 224)
    assert np.abs(w1["W1"]).max() <= lim and np.abs(w1["W1"]).max() > 0.9 * lim
    assert np.all(w1["b1"] == 0) and np.all(w1["b4"] == 0)
    assert not np.array_equal(isaac.LibraryMLP(train=False, seed=12).params(), p1)
    # a training image restores the parameters of an inference model
    X, R = _batches(1, seed=40)[0]
    m1.train_step(X, R, lr=1e-3)
    img = m1.save(tag=5)
    assert len(img) == isaac.load().isaac_mlp_checkpoint_bytes(1)
    assert m2.load(img) == 5
    np.testing.assert_array_equal(m2.params(), m1.params())
    # inference model images are smaller; loading one into a training model resets Adam
    img2 = m2.save()
    assert len(img2) == isaac.load().isaac_mlp_checkpoint_bytes(0)
    m1.load(img2)
    assert m1.step == 0
    torch.cuda.synchronize()
    m1.close()
    m2.close()
    assert not m1.desc.params
    # a caller-owned model is not the library's to free
    own = isaac.MLPModel(isaac.pack_mlp_params(synth.mlp_params(1)))
    lib = isaac.load()
    assert lib.isaac_mlp_destroy(C.byref(own.desc)) == isaac.EINVAL
