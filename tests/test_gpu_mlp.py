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
