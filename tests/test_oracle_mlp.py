"""Pins of the surrogate oracle: gradients against central finite
differences (FP64), GELU against its closed form, encoding layout, Adam
against a hand-computed first step."""
import math

import numpy as np
import pytest

from oracle import mlp


def _small_params(rng, sizes=(6, 5, 4, 3)):
    return [(rng.standard_normal((o, i)) * 0.5, rng.standard_normal(o) * 0.1)
            for i, o in zip(sizes[:-1], sizes[1:])]


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(0)
    P = _small_params(rng)
    X = rng.standard_normal((7, 6))
    Y = rng.standard_normal((7, 3))
    out, cache = mlp.forward(P, X)
    grads = mlp.backward(P, cache, out, Y)
    h = 1e-6
    for li, (W, b) in enumerate(P):
        for arr, g in ((W, grads[li][0]), (b, grads[li][1])):
            it = np.nditer(arr, flags=["multi_index"])
            for _ in it:
                idx = it.multi_index
                old = arr[idx]
                arr[idx] = old + h
                lp = mlp.mse(mlp.forward(P, X)[0], Y)
                arr[idx] = old - h
                lm = mlp.mse(mlp.forward(P, X)[0], Y)
                arr[idx] = old
                fd = (lp - lm) / (2 * h)
                assert abs(fd - g[idx]) <= 1e-6 * max(1.0, abs(fd)), (li, idx, fd, g[idx])


def test_gelu_closed_form():
    z = np.array([-3.0, -1.0, 0.0, 0.5, 2.0])
    ref = [0.5 * x * (1 + math.tanh(math.sqrt(2 / math.pi) * (x + 0.044715 * x ** 3))) for x in z]
    assert np.allclose(mlp.gelu(z), ref, rtol=1e-15, atol=1e-300)
    # the tanh form stays within 2e-3 of the erf form x (1 + erf(x / sqrt 2)) / 2
    xs = np.linspace(-6, 6, 241)
    erf_form = np.array([0.5 * x * (1 + math.erf(x / math.sqrt(2))) for x in xs])
    assert np.abs(mlp.gelu(xs) - erf_form).max() < 2e-3
    h = 1e-6
    assert np.allclose(mlp.gelu_grad(z), (mlp.gelu(z + h) - mlp.gelu(z - h)) / (2 * h), rtol=1e-8, atol=1e-9)
    assert mlp.gelu(np.array([0.0]))[0] == 0.0


def test_encoding_layout():
    raw = np.arange(9, dtype=np.float64)[None] / 10.0
    e = mlp.encode(raw)
    assert e.shape == (1, 320)
    assert mlp.N_ENC == 297
    assert np.count_nonzero(e[0, 299:]) == 0 and np.all(e[0, 198:200] == 0.0)
    assert np.allclose(e[0, :6], raw[0, :6]) and np.allclose(e[0, 200:203], raw[0, 6:])
    w3 = math.pi * 2 ** 1.5
    assert np.allclose(e[0, 6 + 36:12 + 36], np.sin(w3 * raw[0, :6]))
    assert np.allclose(e[0, 12 + 36:18 + 36], np.cos(w3 * raw[0, :6]))
    assert np.allclose(e[0, 203 + 18:206 + 18], np.sin(w3 * raw[0, 6:]))
    assert np.allclose(e[0, 206 + 18:209 + 18], np.cos(w3 * raw[0, 6:]))
    # the first 200 columns depend on position and normal only
    raw2 = raw.copy()
    raw2[0, 6:] = [0.3, -0.2, 0.9]
    assert np.array_equal(mlp.encode(raw2)[0, :200], e[0, :200])


def test_adam_first_step_moves_by_lr_times_sign():
    # with bias correction the first step is -lr * g / (|g| + eps) per element
    P = [(np.array([[1.0, -2.0]]), np.array([0.5]))]
    G = [(np.array([[0.3, -4.0]]), np.array([0.0]))]
    new, st = mlp.adam(P, G, {}, lr=0.01)
    assert np.allclose(new[0][0], [[0.99, -1.99]], atol=1e-9)
    assert new[0][1][0] == pytest.approx(0.5)
    assert st["t"] == 1


def test_output_layer_folds_into_shading():
    # sum_j (mu_j + s_j out_j) L_j  ==  (h W_out^T + b) folded with diag(s) L
    rng = np.random.default_rng(1)
    h = rng.standard_normal((4, 8))
    Wo = rng.standard_normal((5, 8))
    bo = rng.standard_normal(5)
    mu, sg = rng.standard_normal(5), rng.random(5) + 0.1
    L = rng.standard_normal((3, 5))
    direct = mlp.shade_from_outputs(h @ Wo.T + bo, mu, sg, L)
    Weff = (Wo * sg[:, None]).T @ L.T          # [8, 3]
    beff = (mu + sg * bo) @ L.T
    assert np.allclose(direct, h @ Weff + beff)
