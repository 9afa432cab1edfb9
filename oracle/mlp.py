"""Transport surrogate: FP64 forward, backward and Adam of the MLP (oracle).

Not part of the paper: a learned stand-in for stored transport.  It maps a
vertex's position, normal and view direction (9 numbers) to the Haar
transport coefficients at a fixed index set:

* encoding of the 9 inputs (position p, normal n, view direction w) with 16
  frequencies omega_f = pi * 2^(f/2), f = 0..15, laid out so that the part
  that depends on the vertex alone comes first:
  [p, n] (6), then per f: sin(omega_f [p, n]) (6), cos(omega_f [p, n]) (6),
  2 zeros (columns 0..199); w (3), then per f: sin(omega_f w) (3),
  cos(omega_f w) (3) (columns 200..298); zeros to 320 (297 features);
* 4 hidden layers of width 256 with GELU in its tanh form (Hendrycks and
  Gimpel 2016): gelu(z) = z (1 + tanh(sqrt(2/pi) (z + 0.044715 z^3))) / 2;
* a linear output layer of width 512 (standardised coefficients);
* loss: mean squared error over batch and outputs.

``bf16`` mirrors the storage roundings of the tensor-core path (weights,
encoded inputs, activations and back-propagated gradients rounded to
bfloat16 where that path stores them); everything else is FP64.

Test infrastructure only (see the package docstring).
"""
from __future__ import annotations

import math

import numpy as np

from .transport import to_bf16

N_RAW = 9
N_FREQ = 16
N_ENC = N_RAW + 2 * N_FREQ * N_RAW     # 297
N_VERTEX_COLS = 200                    # columns that depend on the vertex alone
N_IN = 320
WIDTH = 256
DEPTH = 4
N_OUT = 512
SIZES = (N_IN,) + (WIDTH,) * DEPTH + (N_OUT,)


def omegas() -> np.ndarray:
    return math.pi * 2.0 ** (np.arange(N_FREQ) / 2.0)


def encode(raw: np.ndarray) -> np.ndarray:
    """[B, 9] (p, n, w) -> [B, 320] in the layout of the module docstring."""
    raw = np.asarray(raw, dtype=np.float64)
    B = raw.shape[0]
    out = np.zeros((B, N_IN))
    pn, w = raw[:, :6], raw[:, 6:9]
    out[:, 0:6] = pn
    for f, om in enumerate(omegas()):
        out[:, 6 + 12 * f:12 + 12 * f] = np.sin(om * pn)
        out[:, 12 + 12 * f:18 + 12 * f] = np.cos(om * pn)
    out[:, 200:203] = w
    for f, om in enumerate(omegas()):
        out[:, 203 + 6 * f:206 + 6 * f] = np.sin(om * w)
        out[:, 206 + 6 * f:209 + 6 * f] = np.cos(om * w)
    return out


GELU_A = math.sqrt(2.0 / math.pi)
GELU_B = 0.044715


def gelu(z):
    return 0.5 * z * (1.0 + np.tanh(GELU_A * (z + GELU_B * z ** 3)))


def gelu_grad(z):
    t = np.tanh(GELU_A * (z + GELU_B * z ** 3))
    return 0.5 * (1.0 + t) + 0.5 * z * (1.0 - t * t) * GELU_A * (1.0 + 3.0 * GELU_B * z * z)


def init(rng: np.random.Generator):
    """[(W [out, in], b [out])] with W ~ N(0, 2/in) (hidden) and N(0, 1/in) (output)."""
    params = []
    for li in range(len(SIZES) - 1):
        fan_in, fan_out = SIZES[li], SIZES[li + 1]
        gain = 2.0 if li < len(SIZES) - 2 else 1.0
        W = rng.standard_normal((fan_out, fan_in)) * math.sqrt(gain / fan_in)
        params.append((W, np.zeros(fan_out)))
    return params


def _r(x, bf16):
    return to_bf16(x) if bf16 else x


def forward(params, X, bf16: bool = False):
    """Output [B, 512] and the cache for backward, from encoded inputs X [B, 320]."""
    h = _r(X, bf16)
    cache = {"h": [h], "z": []}
    n = len(params)
    for li, (W, b) in enumerate(params):
        z = h @ _r(W, bf16).T + b
        cache["z"].append(z)
        if li < n - 1:
            h = _r(gelu(z), bf16)
            cache["h"].append(h)
        else:
            h = z
    return h, cache


def mse(out, target):
    d = out - target
    return float((d * d).mean())


def backward(params, cache, out, target, bf16: bool = False):
    """Gradients [(dW, db)] of the mean squared error."""
    B = out.shape[0]
    g = 2.0 * (out - target) / (B * out.shape[1])
    grads = [None] * len(params)
    dz = _r(g, bf16)
    for li in range(len(params) - 1, -1, -1):
        W, _ = params[li]
        h = cache["h"][li]
        grads[li] = (dz.T @ h, dz.sum(axis=0))
        if li > 0:
            dh = dz @ _r(W, bf16)
            dz = _r(dh * gelu_grad(cache["z"][li - 1]), bf16)
    return grads


def adam(params, grads, state, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (bias-corrected); state = {'t', 'm', 'v'}."""
    t = state.get("t", 0) + 1
    m = state.get("m") or [(np.zeros_like(W), np.zeros_like(b)) for W, b in params]
    v = state.get("v") or [(np.zeros_like(W), np.zeros_like(b)) for W, b in params]
    new_p, new_m, new_v = [], [], []
    c1, c2 = 1.0 - b1 ** t, 1.0 - b2 ** t
    for (W, b), (gW, gb), (mW, mb), (vW, vb) in zip(params, grads, m, v):
        out = []
        for p, gp, mp, vp in ((W, gW, mW, vW), (b, gb, mb, vb)):
            mp = b1 * mp + (1 - b1) * gp
            vp = b2 * vp + (1 - b2) * gp * gp
            p = p - lr * (mp / c1) / (np.sqrt(vp / c2) + eps)
            out.append((p, mp, vp))
        new_p.append((out[0][0], out[1][0]))
        new_m.append((out[0][1], out[1][1]))
        new_v.append((out[0][2], out[1][2]))
    return new_p, {"t": t, "m": new_m, "v": new_v}


def shade_from_outputs(out, mu, sigma, lighting_at_idx):
    """radiance [B, C] = sum_j (mu_j + sigma_j out_j) L[c, idx_j] for
    lighting_at_idx [C, 512] (the lighting coefficients at the index set)."""
    T = mu[None, :] + sigma[None, :] * out
    return T @ np.asarray(lighting_at_idx, dtype=np.float64).T
