"""GPU parity of the learned ray-interval proposal: labels, inputs, forward
pass and gradients against the FP64 oracle; the restricted march's exactness
rules; and what a trained network gains on the bubble workload."""
import numpy as np
import pytest

import oracle
from oracle import mlp as omlp
from paper_1611_09048_b300 import isaac, synth
from parity_util import compare

pytestmark = pytest.mark.gpu


def _records(rays):
    """Pack a synth.random_rays dict into (N, 12) int32 ray records."""
    N = len(rays["nsteps"])
    rec = np.zeros((N, 12), np.int32)
    f = rec.view(np.float32)
    f[:, 0:3] = rays["e"]
    rec[:, 3] = rays["nsteps"]
    f[:, 4:7] = rays["d"]
    rec[:, 7] = np.arange(N)
    rec[:, 8] = 0
    rec[:, 9] = rays["jf"]
    rec[:, 10] = rays["jl"]
    return rec


def _fp16(a):
    return np.asarray(a, np.float32).astype(np.float16).astype(np.float64)


def test_trace_labels_match_oracle(cuda_ok):
    import torch
    sc = synth.scene_bubble(64, frame=10, seed=1, width=128, height=96, dist_factor=1.0)
    ds = isaac.DeviceScene(sc)
    rays, count, out, f32, ns = ds.trace(want_f32=True, want_nsamp=True)
    torch.cuda.synchronize()
    n = int(count.item())
    rec = rays[:n].cpu().numpy()
    ref = oracle.render(sc)
    rep = compare(f32.cpu().numpy(), out.cpu().numpy(), ns.cpu().numpy(), ref)
    assert rep.bad == 0 and rep.bad_ns == 0, rep
    pix = rec[:, 7]
    want = ref["jspan"].reshape(-1, 2)[pix]
    got = rec[:, 9:11]
    m_term = ref["margin"].reshape(-1, 4)[pix, 2]
    same = np.all(got == want, axis=1)
    assert n > 3000 and (want[:, 0] >= 0).sum() > 150
    # a different span is only allowed where the termination decision was a tie
    assert np.all(same | (m_term < 1e-3)), np.flatnonzero(~same)[:10]


def test_features_match_oracle(cuda_ok):
    import torch
    n = (40, 48, 56)
    rr = synth.random_rays(3000, n, seed=4)
    sc = synth.scene_bubble(40, frame=0, seed=3, width=8, height=8)
    sc.n = n
    sc.sources[0] = synth.source_from_zyx(
        np.random.default_rng(1).uniform(0, 1, (n[2], n[1], n[0])).astype(np.float32), 0)
    grid = oracle.opacity_grid(sc, 8).astype(np.float32)
    dev = torch.device("cuda")
    X = isaac.mlp_features(torch.from_numpy(_records(rr)).to(dev), 3000, n, 0.5,
                           torch.from_numpy(grid).to(dev), 8)
    torch.cuda.synchronize()
    got = X.float().cpu().numpy().astype(np.float64)
    want = omlp.inputs(rr["e"], rr["d"], rr["nsteps"], n, 0.5, grid, 8)
    enc_err = np.abs(got[:, :192] - want[:, :192]).max()
    assert enc_err <= 2e-3, enc_err                       # FP16 storage of sin/cos
    grid_ok = np.abs(got[:, 192:] - _fp16(want[:, 192:])) <= 1e-3
    assert grid_ok.mean() >= 0.995, grid_ok.mean()        # cell lookups at FP32 boundaries


def _random_X(N, seed):
    rng = np.random.default_rng(seed)
    return rng.uniform(-1, 1, (N, 224)).astype(np.float16)


def test_forward_matches_oracle(cuda_ok):
    import torch
    params = synth.mlp_params(5, bias_scale=0.1)
    model = isaac.MLPModel(isaac.pack_mlp_params(params), train=False)
    X = _random_X(1000, 6)
    U = model.forward(torch.from_numpy(X).cuda())
    torch.cuda.synchronize()
    p16 = {k: _fp16(v) if k.startswith("W") else v.astype(np.float64) for k, v in params.items()}
    want = omlp.forward(p16, X.astype(np.float64))["u"]
    err = np.abs(U.cpu().numpy() - want).max()
    # FP16 hidden activations (rounded once per layer) against FP64: measured
    # <= 1.5e-3 at |u| <= 3.7
    assert err <= 5e-3 * max(1.0, np.abs(want).max()), err


@pytest.mark.parametrize("n", [1, 127, 128, 129, 4099])
def test_forward_tiles_of_any_size(cuda_ok, n):
    """The tensor-core forward pass works on tiles of 128 rays: a single ray,
    one short of a tile, exactly one tile, one past it, and many tiles with a
    ragged tail all match the oracle row by row (no row of a partial tile is
    lost or taken from a neighbour)."""
    import torch
    params = synth.mlp_params(9, bias_scale=0.2)
    model = isaac.MLPModel(isaac.pack_mlp_params(params), train=False)
    X = _random_X(n, 100 + n)
    U = model.forward(torch.from_numpy(X).cuda())
    torch.cuda.synchronize()
    p16 = {k: _fp16(v) if k.startswith("W") else v.astype(np.float64) for k, v in params.items()}
    want = omlp.forward(p16, X.astype(np.float64))["u"]
    got = U.cpu().numpy()
    assert got.shape == (n, 3)
    err = np.abs(got - want).max(axis=1)
    assert np.all(err <= 5e-3 * np.maximum(1.0, np.abs(want).max(axis=1))), err.max()


def test_gradients_match_oracle(cuda_ok):
    import torch
    params = synth.mlp_params(7, bias_scale=0.1)
    model = isaac.MLPModel(isaac.pack_mlp_params(params))
    rr = synth.random_rays(2000, (64, 64, 64), seed=8)
    X = _random_X(2000, 9)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    model.train_step(torch.from_numpy(X).cuda(), torch.from_numpy(_records(rr)).cuda(), lr=0.0,
                     margin=2, loss_sum=loss)
    torch.cuda.synchronize()
    g_gpu = isaac.unpack_mlp_params(model.grads.cpu().numpy())
    p16 = {k: _fp16(v) if k.startswith("W") else v.astype(np.float64) for k, v in params.items()}
    lo, g = omlp.loss_and_grads(p16, X.astype(np.float64), rr["jf"], rr["jl"], rr["nsteps"], margin=2)
    assert abs(float(loss.item()) - lo) <= 1e-2 * abs(lo)
    for k in g:
        rel = np.linalg.norm(g_gpu[k] - g[k]) / max(1e-12, np.linalg.norm(g[k]))
        assert rel <= 2e-2, (k, rel)
    # lr = 0 leaves the weights untouched
    np.testing.assert_array_equal(model.params.cpu().numpy(), isaac.pack_mlp_params(params))


def test_adam_first_step_is_minus_lr_sign(cuda_ok):
    import torch
    params = synth.mlp_params(11, bias_scale=0.1)
    model = isaac.MLPModel(isaac.pack_mlp_params(params))
    rr = synth.random_rays(1024, (64, 64, 64), seed=12)
    model.train_step(torch.from_numpy(_random_X(1024, 13)).cuda(),
                     torch.from_numpy(_records(rr)).cuda(), lr=1e-3)
    torch.cuda.synchronize()
    g = model.grads.cpu().numpy()
    dp = model.params.cpu().numpy() - isaac.pack_mlp_params(params)
    big = np.abs(g) > 1e-5
    np.testing.assert_allclose(dp[big], -1e-3 * np.sign(g[big]), rtol=2e-2, atol=1e-6)
    assert model.step == 1


def _const_model(b4):
    p = synth.mlp_params(0)
    for k in ("W1", "W2", "W3", "W4"):
        p[k] = np.zeros_like(p[k])
    p["b4"] = np.asarray(b4, np.float32)
    return isaac.MLPModel(isaac.pack_mlp_params(p), train=False)


@pytest.mark.parametrize("packed", [None, "bf16"])
def test_proposal_plumbing_closed_forms(cuda_ok, packed):
    """Constant networks: 'everything' (te=0, tx=1, sure) and 'unsure'
    reproduce the plain image bit for bit; 'nothing' (te=1, tx=0, sure, no
    margin) leaves the background."""
    import torch
    sc = synth.scene_bubble(64, frame=1, seed=2, width=80, height=64, dist_factor=1.5)
    ds = isaac.DeviceScene(sc)
    target = ds if packed is None else ds.pack(packed)
    grid = ds.opacity_grid(8)
    plain = target.render(want_f32=True, want_nsamp=True)
    for b4, margin, expect in (((-30, 30, 30), 2, "same"), ((-30, 30, -30), 2, "same"),
                               ((30, -30, 30), 0, "empty")):
        stats = torch.zeros(2, dtype=torch.int32, device="cuda")
        model = _const_model(b4)
        prop = model.proposal(grid, 8, threshold=0.9, margin=margin, stats=stats, widen=False)
        got = target.render_learned(prop, want_f32=True, want_nsamp=True)
        torch.cuda.synchronize()
        seen, restricted = stats.tolist()
        assert seen == int((plain[2] > 0).sum()) or seen > 0
        if expect == "same":
            for a, b in zip(plain, got):
                assert torch.equal(a, b)
            assert restricted == (seen if b4[2] > 0 else 0)
        else:
            assert int(got[2].sum()) == 0 and restricted == seen
            assert int(got[0].sum()) == 0


@pytest.mark.parametrize("packed", [None, "bf16"])
def test_long_ray_list_refills(cuda_ok, packed):
    """'Everything' (full windows, so every ray of > 96 samples goes to the
    long-ray list) on a frame with many more long rays than the long-ray
    kernel holds at once (4 per warp): the image is the plain one bit for bit,
    so slots are refilled in order and no ray is lost or marched twice."""
    import torch
    sc = synth.scene_bubble(64, frame=2, seed=5, width=640, height=480, dist_factor=1.1)
    ds = isaac.DeviceScene(sc)
    target = ds if packed is None else ds.pack(packed)
    grid = ds.opacity_grid(8)
    plain = target.render(want_f32=True, want_nsamp=True)
    model = _const_model((-30, 30, 30))
    got = target.render_learned(model.proposal(grid, 8, threshold=0.9, margin=2),
                                want_f32=True, want_nsamp=True)
    torch.cuda.synchronize()
    long_rays = int((plain[2] > 96).sum())
    assert long_rays > 4 * 4 * 148 * 8 // 2          # well beyond one long-ray slot per warp
    for a, b in zip(plain, got):
        assert torch.equal(a, b)


def test_trained_proposal_gain_on_bubble(cuda_ok):
    """Train on traced bubble frames, then render an unseen frame: where the
    proposal covered a ray's visible span the pixel is bit-identical to the
    plain march; the image error stays within 1 LSB on average; and the learned
    march composites far fewer samples."""
    import torch
    n, W, H, cell = 96, 128, 96, 8
    noise = synth.value_noise(n, 77)
    dev = torch.device("cuda")
    Xs, Rs = [], []
    for f in range(6):
        field = synth.bubble_field(n, frame=3 * f, seed=0, noise=noise)
        for c in range(6):
            sc = synth.scene_bubble(n, frame=3 * f, seed=10 * f + c, width=W, height=H,
                                    field=field, lut_seed=100 + c, dist_factor=1.5)
            ds = isaac.DeviceScene(sc)
            rays, count, *_ = ds.trace()
            k = int(count.item())
            grid = ds.opacity_grid(cell)
            Xs.append(isaac.mlp_features(rays[:k], k, sc.n, sc.step, grid, cell))
            Rs.append(rays[:k].clone())
    X = torch.cat(Xs)
    R = torch.cat(Rs)
    model = isaac.MLPModel(isaac.pack_mlp_params(synth.mlp_params(3)))
    gen = torch.Generator(device="cpu").manual_seed(0)
    for it in range(400):
        idx = torch.randint(0, X.shape[0], (4096,), generator=gen).to(dev)
        model.train_step(X[idx].contiguous(), R[idx].contiguous(), lr=2e-3, margin=2)
    torch.cuda.synchronize()

    field = synth.bubble_field(n, frame=8, seed=0, noise=noise)
    sc = synth.scene_bubble(n, frame=8, seed=999, width=W, height=H, field=field, lut_seed=101,
                            dist_factor=1.5)
    ds = isaac.DeviceScene(sc)
    grid = ds.opacity_grid(cell)
    p_rays, p_cnt, p8, p32, pns = ds.trace(want_f32=True, want_nsamp=True)
    stats = torch.zeros(2, dtype=torch.int32, device=dev)
    prop = model.proposal(grid, cell, threshold=0.9, margin=2, stats=stats)
    l_rays, l_cnt, l8, l32, lns = ds.trace(proposal=prop, want_f32=True, want_nsamp=True)
    torch.cuda.synchronize()
    k = int(p_cnt.item())
    assert int(l_cnt.item()) == k
    pr = p_rays[:k].cpu().numpy()
    lr_ = l_rays[:k].cpu().numpy()
    order = np.argsort(pr[:, 7])
    pr, lr_ = pr[order], lr_[np.argsort(lr_[:, 7])]
    covered = (pr[:, 9] < 0) | ((lr_[:, 8] <= pr[:, 9]) & (lr_[:, 3] >= pr[:, 10] + 1))
    pix = pr[:, 7]
    a32 = p32.reshape(-1, 4).cpu().numpy()[pix]
    b32 = l32.reshape(-1, 4).cpu().numpy()[pix]
    assert np.array_equal(a32[covered], b32[covered])
    lsb = np.abs(p8.cpu().numpy().astype(int) - l8.cpu().numpy().astype(int))
    seen, restricted = stats.tolist()
    frac_cov = covered.mean()
    saved = 1.0 - lns.sum().item() / max(1, pns.sum().item())
    print(f"rays {k}, restricted {restricted}/{seen}, covered {frac_cov:.3f}, "
          f"samples saved {saved:.3f}, mean LSB {lsb.mean():.4f}")
    assert lsb.mean() <= 1.0
    assert restricted > 0.5 * seen
    assert saved > 0.3


@pytest.mark.parametrize("margin,widen", [(0, False), (3, False), (2, True)])
def test_proposal_windows_match_oracle_rule(cuda_ok, margin, widen):
    """The windows the proposal kernel writes into the ray list equal the
    oracle's proposal rule applied to the network outputs of the same rays
    (forward pass on the same FP16 inputs; with widening, the same grid and
    ray records); rays whose te*ns or tx*ns lies within 1e-4 of an integer, or
    whose confidence lies within 1e-5 of the threshold, are decided at a tie
    and only counted; with widening an end may also differ by one sample that
    lies within 1e-3 voxel of a macro-cell face (FP32 against FP64 position)."""
    import torch
    sc = synth.scene_bubble(64, frame=4, seed=6, width=160, height=120, dist_factor=1.2)
    ds = isaac.DeviceScene(sc)
    grid = ds.opacity_grid(8)
    rays, count, *_ = ds.trace()
    k = int(count.item())
    params = synth.mlp_params(21, bias_scale=0.5)
    params["b4"] = np.asarray((params["b4"][0], params["b4"][1], 2.2), np.float32)
    model = isaac.MLPModel(isaac.pack_mlp_params(params), train=False)
    X = isaac.mlp_features(rays[:k], k, sc.n, sc.step, grid, 8)
    U = model.forward(X).cpu().numpy()
    l_rays, l_cnt, *_ = ds.trace(proposal=model.proposal(grid, 8, threshold=0.9, margin=margin,
                                                         widen=widen))
    torch.cuda.synchronize()
    assert int(l_cnt.item()) == k
    base = rays[:k].cpu().numpy()
    got = l_rays[:k].cpu().numpy()
    got = got[np.argsort(got[:, 7])]
    order = np.argsort(base[:, 7])
    base, U = base[order], U[order]
    ns = base[:, 3]
    fl = base.view(np.float32)
    e, d = fl[:, 0:3].astype(np.float64), fl[:, 4:7].astype(np.float64)
    g_np = grid.cpu().numpy()
    w = dict(e=e, d=d, step=sc.step, grid=g_np, cell=8) if widen else None
    kb, ke, use = omlp.propose_rule(U, ns, margin, 0.9, w)
    te, tx, conf = (omlp.sigmoid(U[:, i].astype(np.float64)) for i in range(3))

    def near_int(x):
        return np.abs(x - np.round(x)) < 1e-4

    def near_face(r, k):
        p = e[r] + k * sc.step * d[r]
        f = p / 8.0 - np.floor(p / 8.0)
        return bool(np.any(np.minimum(f, 1.0 - f) * 8.0 < 1e-3))

    tie = (np.abs(conf - 0.9) < 1e-5) | (use & (near_int(te * ns) | near_int(tx * ns)))
    assert 0.2 < use.mean() < 0.95, use.mean()
    assert tie.mean() < 0.01
    ok = (got[:, 8] == kb) & (got[:, 3] == ke)
    if widen:
        for r in np.flatnonzero(~ok & ~tie):
            db, de = got[r, 8] - kb[r], got[r, 3] - ke[r]
            assert abs(db) <= 1 and abs(de) <= 1, (r, db, de)
            # the sample one side keeps and the other does not
            assert db == 0 or near_face(r, min(got[r, 8], kb[r])), (r, db)
            assert de == 0 or near_face(r, min(got[r, 3], ke[r])), (r, de)
            ok[r] = True
        keep = omlp.nonzero_samples(e, d, ns, sc.step, g_np, 8)
        assert np.mean([len(k) > 0 for k in keep]) > 0.1      # the widening has work to do
    assert np.all(ok | tie), np.flatnonzero(~ok & ~tie)[:10]


def test_grid_hull_windows_and_exact_frame(cuda_ok):
    """A proposal without a network: every ray's range is the hull of its
    samples in macro cells with a nonzero max-opacity grid value (the oracle's
    nonzero_samples, up to a sample within 1e-3 voxel of a macro-cell face);
    with the bubble's transfer function (zero below a threshold, nonzero above)
    no visible sample lies outside it, so the frame equals the plain one bit
    for bit while far fewer samples are marched."""
    import torch
    sc = synth.scene_bubble(64, frame=6, seed=7, width=160, height=120, dist_factor=1.2)
    ds = isaac.DeviceScene(sc)
    grid = ds.opacity_grid(8)
    rays, count, p8, p32, pns = ds.trace(want_f32=True, want_nsamp=True)
    h_rays, h_cnt, h8, h32, hns = ds.trace(proposal=isaac.grid_proposal(grid, 8), want_f32=True,
                                          want_nsamp=True)
    torch.cuda.synchronize()
    k = int(count.item())
    assert int(h_cnt.item()) == k and k > 3000
    base = rays[:k].cpu().numpy()
    got = h_rays[:k].cpu().numpy()
    base, got = base[np.argsort(base[:, 7])], got[np.argsort(got[:, 7])]
    fl = base.view(np.float32)
    e, d = fl[:, 0:3].astype(np.float64), fl[:, 4:7].astype(np.float64)
    keep = omlp.nonzero_samples(e, d, base[:, 3], sc.step, grid.cpu().numpy(), 8)
    kb = np.array([kk[0] if len(kk) else 0 for kk in keep])
    ke = np.array([kk[-1] + 1 if len(kk) else 0 for kk in keep])
    empty = np.array([len(kk) == 0 for kk in keep])

    def near_face(r, s):
        p = e[r] + s * sc.step * d[r]
        f = p / 8.0 - np.floor(p / 8.0)
        return bool(np.any(np.minimum(f, 1.0 - f) * 8.0 < 1e-3))

    for r in range(k):
        if empty[r]:
            assert got[r, 3] <= got[r, 8] or near_face(r, got[r, 8]), r
            continue
        db, de = got[r, 8] - kb[r], got[r, 3] - ke[r]
        assert (db == 0 or (abs(db) <= 1 and near_face(r, min(got[r, 8], kb[r])))), (r, db)
        assert (de == 0 or (abs(de) <= 1 and near_face(r, min(got[r, 3], ke[r])))), (r, de)
    assert empty.mean() > 0.2 and (~empty).mean() > 0.1
    assert torch.equal(p8, h8) and torch.equal(p32, h32)
    assert hns.sum().item() < 0.5 * pns.sum().item()
