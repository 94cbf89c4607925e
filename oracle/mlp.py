"""FP64 numpy oracle for the triage surrogate network.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Paper Sec. 3.5 proposes predicting binding affinity from ligand features with
models ranging from regressions to deep networks, choosing by cost; the
surrogate here is a multilayer perceptron 256 -> 512 -> 512 -> 512 -> 1 with
ReLU on the hidden layers, trained by mean squared error with Adam
(Kingma & Ba 2015, Algorithm 1).  Every function is the textbook definition
written out with numpy matrix products as its only library step.

Parameter layout: ``params = [W1, b1, W2, b2, W3, b3, W4, b4]`` with
``W_l`` of shape [fan_in, fan_out] (row-major; y = x @ W + b).
"""
from __future__ import annotations

import numpy as np

DIMS = (256, 512, 512, 512, 1)


def bf16_round(x) -> np.ndarray:
    """Round FP32 values to the nearest BF16 (ties to even), returned as FP32.
    BF16 keeps the top 16 bits of the FP32 pattern; rounding adds half an ulp
    of the kept part plus the parity bit before truncating."""
    a = np.ascontiguousarray(x, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    bias = 0x7FFF + ((u >> 16) & 1)
    r = ((u + bias) & 0xFFFF0000).astype(np.uint32)
    out = r.view(np.float32).copy()
    nan = np.isnan(a)
    out[nan] = a[nan]
    return out


def _bf16(a):
    return bf16_round(np.asarray(a, np.float32)).astype(np.float64)


def forward(params, X, bf16_acts: bool = False):
    """Returns (y[B], cache) with cache = pre-activations and activations.

    ``bf16_acts`` applies the network's storage precision: the hidden
    activations are held in BF16, so each ReLU output is rounded to BF16
    before it feeds the next layer (all arithmetic stays FP64)."""
    X = np.asarray(X, np.float64)
    acts = [X]
    pres = []
    h = X
    n_layers = len(params) // 2
    for l in range(n_layers):
        W, b = np.asarray(params[2 * l], np.float64), np.asarray(params[2 * l + 1], np.float64)
        z = h @ W + b
        pres.append(z)
        if l < n_layers - 1:
            h = np.maximum(z, 0.0)
            if bf16_acts:
                h = _bf16(h)
        else:
            h = z
        acts.append(h)
    return h[:, 0], (acts, pres, bf16_acts)


def mse(y, t) -> float:
    y = np.asarray(y, np.float64)
    t = np.asarray(t, np.float64)
    return float(np.mean((y - t) ** 2))


def backward(params, cache, y, t):
    """Gradients of mse(y, t) with respect to every parameter (same layout).

    When the forward pass held activations in BF16, the gradients with
    respect to the hidden pre-activations are held in BF16 too (rounded
    after the ReLU mask), matching the network's storage precision."""
    acts, pres, bf16_acts = cache
    B = len(y)
    n_layers = len(params) // 2
    grads = [None] * len(params)
    d = (2.0 / B) * (np.asarray(y, np.float64) - np.asarray(t, np.float64))[:, None]
    for l in reversed(range(n_layers)):
        if l < n_layers - 1:
            d = d * (pres[l] > 0.0)
            if bf16_acts:
                d = _bf16(d)
        grads[2 * l] = acts[l].T @ d
        grads[2 * l + 1] = d.sum(axis=0)
        if l > 0:
            d = d @ np.asarray(params[2 * l], np.float64).T
    return grads


def adam_step(params, grads, m, v, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (step counts from 1); returns new (params, m, v)."""
    new_p, new_m, new_v = [], [], []
    for p, g, mi, vi in zip(params, grads, m, v):
        mi = beta1 * mi + (1.0 - beta1) * g
        vi = beta2 * vi + (1.0 - beta2) * g * g
        mhat = mi / (1.0 - beta1 ** step)
        vhat = vi / (1.0 - beta2 ** step)
        new_p.append(p - lr * mhat / (np.sqrt(vhat) + eps))
        new_m.append(mi)
        new_v.append(vi)
    return new_p, new_m, new_v


def standardize_stats(X):
    """Per-feature mean and standard deviation (population); features with
    zero spread get std 1 so they standardize to 0."""
    X = np.asarray(X, np.float64)
    mu = X.mean(axis=0)
    sd = X.std(axis=0)
    sd[sd == 0.0] = 1.0
    return mu, sd


def he_init(normal_draws, dims=DIMS):
    """He-normal weights (std sqrt(2 / fan_in)) from a flat array of standard
    normal draws, zero biases."""
    params = []
    off = 0
    for fi, fo in zip(dims[:-1], dims[1:]):
        w = np.asarray(normal_draws[off:off + fi * fo], np.float64).reshape(fi, fo)
        off += fi * fo
        params += [w * np.sqrt(2.0 / fi), np.zeros(fo)]
    return params


def n_weights(dims=DIMS) -> int:
    return sum(fi * fo for fi, fo in zip(dims[:-1], dims[1:]))
