"""GPU checks of the transport surrogate: bf16 tcgen05 forward and backward
against the FP64 oracle (with the same bf16 storage points), Adam training
against the oracle's, the fused surrogate shading, and what the trained
network gives against the stored-transport method."""
import math

import numpy as np
import pytest

import synth
from oracle import haar as oh
from oracle import mlp as om
from oracle import shift as osh
from oracle import transport as otr
from tests.helpers import rel_l2

pytestmark = pytest.mark.gpu


def _t(x, dtype=None):
    import torch
    return torch.tensor(np.ascontiguousarray(x), dtype=dtype, device="cuda")


def _flat(params):
    return np.concatenate([np.concatenate([W.ravel(), b]) for W, b in params])


def _unflat(flat):
    out, o = [], 0
    for fi, fo in zip(om.SIZES[:-1], om.SIZES[1:]):
        W = flat[o:o + fo * fi].reshape(fo, fi)
        o += fo * fi
        b = flat[o:o + fo]
        o += fo
        out.append((W, b))
    return out


def _raw(rng, B):
    p = rng.uniform(-1.4, 1.4, (B, 3))
    n = rng.standard_normal((B, 3))
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    v = rng.standard_normal((B, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return np.concatenate([p, n, v], axis=1).astype(np.float32).astype(np.float64)


def _f32_params(rng):
    P = om.init(rng)
    P = [(W.astype(np.float32).astype(np.float64), (rng.standard_normal(b.shape) * 0.05).astype(np.float32)
          .astype(np.float64)) for W, b in P]
    return P


# The encoded inputs are stored as bf16: sin/cos of arguments up to pi 2^7.5
# (~570 rad) carry ~ulp(570) = 6e-5 of FP32 argument rounding, which flips the
# bf16 rounding of ~1.5% of the high-frequency features by one bf16 ulp
# (2^-8 relative); a 5-layer network turns that into ~1e-3; bound 1e-2.
FWD_TOL = 1e-2


def test_param_count(hs):
    assert int(hs.lib().haar_mlp_param_count()) == sum(fo * fi + fo for fi, fo in zip(om.SIZES[:-1], om.SIZES[1:]))


def test_forward_matches_oracle(hs):
    rng = np.random.default_rng(0)
    P = _f32_params(rng)
    raw = _raw(rng, 512)
    net = hs.Surrogate(max_batch=512, max_rows=512, max_groups=4)
    net.set_params(_t(_flat(P), None).float())
    out = net.forward(_t(raw, None).float()).cpu().numpy()
    ref, _ = om.forward(P, om.encode(raw), bf16=True)
    assert rel_l2(out, ref) <= FWD_TOL
    assert net.status() == 0
    net.close()


def test_gradients_match_oracle(hs):
    rng = np.random.default_rng(1)
    P = _f32_params(rng)
    raw = _raw(rng, 1024)
    tgt = rng.standard_normal((1024, 512)).astype(np.float32).astype(np.float64)
    net = hs.Surrogate(max_batch=1024, max_rows=128, max_groups=1)
    net.set_params(_t(_flat(P), None).float())
    g, loss = net.grads(_t(raw, None).float(), _t(tgt, None).float())
    g = _unflat(g.cpu().numpy().astype(np.float64))
    out, cache = om.forward(P, om.encode(raw), bf16=True)
    ref = om.backward(P, cache, out, tgt, bf16=True)
    assert float(loss.item()) == pytest.approx(om.mse(out, tgt), rel=1e-3)
    for li in range(5):
        assert rel_l2(g[li][0], ref[li][0]) <= 2e-2, (li, rel_l2(g[li][0], ref[li][0]))
        assert rel_l2(g[li][1], ref[li][1]) <= 2e-2, (li, rel_l2(g[li][1], ref[li][1]))
    net.close()


def test_training_tracks_oracle(hs):
    rng = np.random.default_rng(2)
    P = _f32_params(rng)
    raw = _raw(rng, 512)
    # a smooth target the network can fit
    tgt = np.tanh(raw @ rng.standard_normal((9, 512)) * 0.5)
    net = hs.Surrogate(max_batch=512, max_rows=128, max_groups=1)
    net.set_params(_t(_flat(P), None).float())
    R, T = _t(raw, None).float(), _t(tgt, None).float()
    gpu = [float(net.train_step(R, T, 1e-3).item()) for _ in range(25)]
    X = om.encode(raw)
    st, Pc, ref = {}, P, []
    for _ in range(25):
        out, cache = om.forward(Pc, X, bf16=True)
        ref.append(om.mse(out, tgt))
        Pc, st = om.adam(Pc, om.backward(Pc, cache, out, tgt, bf16=True), st, lr=1e-3)
    assert gpu[-1] < 0.5 * gpu[0]
    for a, b in zip(gpu, ref):
        assert abs(a - b) <= 0.05 * b, (gpu, ref)
    net.close()


def test_captured_training_step_replays_eager(hs):
    # the Adam step count lives on the device, so a captured step replays exactly
    import torch
    rng = np.random.default_rng(5)
    flat = _t(_flat(_f32_params(rng)), None).float()
    batches = [(_t(_raw(rng, 256), None).float(), _t(rng.standard_normal((256, 512)), None).float())
               for _ in range(4)]
    eager = hs.Surrogate(max_batch=256, max_rows=128, max_groups=1)
    eager.set_params(flat)
    want = [float(eager.train_step(r, t, 1e-3).item()) for r, t in batches]
    net = hs.Surrogate(max_batch=256, max_rows=128, max_groups=1)
    net.set_params(flat)
    R = torch.empty_like(batches[0][0])
    T = torch.empty_like(batches[0][1])
    graph, loss = net.capture_train_step(R, T, 1e-3)
    got = []
    for r, t in batches:
        R.copy_(r)
        T.copy_(t)
        graph.replay()
        got.append(float(loss.item()))
    # the loss is summed with float atomics (order varies); the update itself is deterministic
    assert np.allclose(got, want, rtol=1e-5, atol=0)
    assert torch.equal(net.get_params(), eager.get_params())
    eager.close()
    net.close()


def test_fused_shade_matches_oracle(hs):
    import torch
    rng = np.random.default_rng(3)
    P = _f32_params(rng)
    V, S, C, H, W = 300, 5, 3, 32, 64
    sc = synth.scene(4, V=V, S=S, H=H, W=W)
    pos, nrm, cams = [x.astype(np.float32).astype(np.float64) for x in (sc["pos"], sc["nrm"], sc["cams"])]
    L = oh.forward(sc["light"]).astype(np.float32).astype(np.float64)
    Ls = osh.haar_shift(L, H, W, osh.ROTATE_EULER, sc["params"]).astype(np.float32).astype(np.float64)  # [S,C,N]
    idx = np.sort(rng.choice(H * W, 512, replace=False)).astype(np.int32)
    mu = rng.standard_normal(512).astype(np.float32).astype(np.float64) * 0.01
    sg = (rng.random(512) * 0.02 + 0.001).astype(np.float32).astype(np.float64)
    net = hs.Surrogate(max_batch=128, max_rows=512, max_groups=S)
    net.set_params(_t(_flat(P), None).float())
    R = net.shade(_t(pos).float(), _t(nrm).float(), _t(cams).float(), _t(mu).float(), _t(sg).float(),
                  _t(idx, torch.int32), _t(Ls).float(), C, (C * H * W, H * W, 1)).cpu().numpy()
    ref = np.zeros((V, S, C))
    for s in range(S):
        view = cams[s][None] - pos
        view /= np.linalg.norm(view, axis=1, keepdims=True)
        out, _ = om.forward(P, om.encode(np.concatenate([pos, nrm, view], axis=1)), bf16=True)
        ref[:, s] = om.shade_from_outputs(out, mu, sg, Ls[s][:, idx])
    assert rel_l2(R, ref) <= FWD_TOL
    net.close()
    # the layer-by-layer path (taken when the per-vertex table does not fit the
    # inference buffers) gives the same result within bf16 storage
    small = hs.Surrogate(max_batch=128, max_rows=128, max_groups=S)
    small.set_params(_t(_flat(P), None).float())
    R2 = small.shade(_t(pos).float(), _t(nrm).float(), _t(cams).float(), _t(mu).float(), _t(sg).float(),
                     _t(idx, torch.int32), _t(Ls).float(), C, (C * H * W, H * W, 1)).cpu().numpy()
    assert rel_l2(R2, ref) <= FWD_TOL
    assert rel_l2(R2, R) <= FWD_TOL
    small.close()


def _glossy_dataset(n, seed, device="cuda", chunk=8192):
    """(raw [n, 9], T [n, 8192]) for random (vertex, camera) pairs of the
    glossy torus scene: Phong transfer on the 64x128 grid, projected by the
    oracle (coefficients of the 256x512 map; finer levels are zero)."""
    sc = synth.scene(4, V=100000, S=1)
    rng = np.random.default_rng(seed)
    vid = rng.integers(0, sc["V"], n)
    cams = synth.cameras(rng, n)
    pos, nrm, expo = sc["pos"][vid], sc["nrm"][vid], sc["expo"][vid]
    view = cams - pos
    view /= np.linalg.norm(view, axis=1, keepdims=True)
    Ts = []
    for a in range(0, n, chunk):
        w = synth.transport_weights(pos[a:a + chunk], nrm[a:a + chunk], sc["occ_c"], sc["occ_r"], 64, 128,
                                    view=view[a:a + chunk], expo=expo[a:a + chunk], device=device)
        Ts.append(oh.forward(w.double().cpu().numpy()) / 4.0)
    raw = np.concatenate([pos, nrm, view], axis=1).astype(np.float32)
    return raw, np.concatenate(Ts), sc, (vid, cams)


def test_trained_surrogate_against_stored_transport(hs):
    # Train the surrogate on oracle transports (S8), then compare, on held-out
    # (vertex, camera) pairs under rotated lighting, three ways of shading
    # against the transport at the exact view, untruncated:
    #   the surrogate (512 coefficients at a fixed index set),
    #   the plain stored method (16 view bins x top-512 FP16 per vertex),
    #   the mean transport (no network).
    # The view binning costs the stored method far more than the network
    # costs the surrogate (glossy lobes up to s = 128 move between bins), so
    # the surrogate must beat it clearly; its own error stays above the
    # 512-index set's truncation floor.
    import torch
    from oracle import transport as otr2
    from paper_1705_07272_gb300 import training
    n_train, n_test = 131072, 4096
    raw, T, sc, (vid, cams) = _glossy_dataset(n_train + n_test, 7)
    Ttr = T[:n_train]
    idx = np.sort(np.argsort(-np.abs(Ttr).mean(axis=0), kind="stable")[:512])
    mu = Ttr[:, idx].mean(axis=0)
    # one scale for all outputs: the loss then weighs each coefficient by its
    # share of the transport's energy, as the shading error does
    sg = np.full(512, Ttr[:, idx].std() + 1e-12)
    Y = ((T[:, idx] - mu) / sg).astype(np.float32)
    net = hs.Surrogate(max_batch=4096, max_rows=4096, max_groups=8)
    net.set_params(_t(_flat(om.init(np.random.default_rng(11))), None).float())
    training.fit(net, _t(raw[:n_train]), _t(Y[:n_train]), epochs=120, batch=4096, lr=(2e-3, 6e-4, 2e-4))
    out = net.forward(_t(raw[n_train:])).cpu().numpy().astype(np.float64)
    assert net.status() == 0
    # the plain method's stored row for each test pair: the bin the camera
    # falls in, its transport at the bin's direction, top-512 in FP16
    te = slice(n_train, None)
    pos, nrm = sc["pos"][vid[te]], sc["nrm"][vid[te]]
    dirs = synth.view_bin_dirs(16)
    bins = np.array([otr2.view_bins(pos[k:k + 1], nrm[k:k + 1], cams[te][k:k + 1], dirs)[0][0, 0]
                     for k in range(n_test)])
    bview = synth.bin_view_world(nrm, 16)[np.arange(n_test), bins]
    w = synth.transport_weights(pos, nrm, sc["occ_c"], sc["occ_r"], 64, 128, view=bview,
                                expo=sc["expo"][vid[te]], device="cuda")
    Tb = oh.forward(w.double().cpu().numpy()) / 4.0
    bv, bi, bp = otr2.topk_csr(Tb, 512)
    Tbin = otr2.csr_dense(otr2.to_f16(bv), bi, bp, 8192)
    # shading under 3 rotations of the c4 lighting
    H, W = 256, 512
    L = oh.forward(sc["light"])
    eul = synth.euler_angles(np.random.default_rng(3), 3)
    Ls = osh.haar_shift(L, H, W, osh.ROTATE_EULER, eul)[..., :8192]         # [3, C, 8192]
    Tte = T[n_train:]
    exact = np.einsum("nk,sck->nsc", Tte, Ls)
    plain = np.einsum("nk,sck->nsc", Tbin, Ls)
    floor = np.einsum("nk,sck->nsc", Tte[:, idx], Ls[..., idx])
    mean_only = np.einsum("k,sck->sc", mu, Ls[..., idx])[None].repeat(n_test, 0)
    sur = np.einsum("nk,sck->nsc", mu + sg * out, Ls[..., idx])
    e_sur, e_plain = rel_l2(sur, exact), rel_l2(plain, exact)
    e_floor, e_mean = rel_l2(floor, exact), rel_l2(mean_only, exact)
    print(f"against the exact-view transport: surrogate {e_sur:.3e}, 16-bin stored transport {e_plain:.3e}, "
          f"512-index floor {e_floor:.3e}, mean transport {e_mean:.3e}")
    stored = 100000 * 16 * 512 * 6
    weights = int(hs.lib().haar_mlp_param_count()) * 2
    assert stored / weights > 1000
    # measured: surrogate 0.21, stored 0.50, floor 0.051, mean 0.80
    assert e_floor <= e_sur <= 0.25
    assert e_sur < 0.6 * e_plain
    assert e_sur < 0.5 * e_mean
    net.close()
