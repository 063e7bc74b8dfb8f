"""FP64 oracle of the learned grain router (an MLP over query vectors).

TEST INFRASTRUCTURE ONLY (tests and the smoke check use it; the product
library does not).

The router is a multilayer perceptron d -> h1 -> h2 -> G with exact (erf)
GELU after the two hidden layers and a softmax over the G grains. It is
trained with soft-label cross-entropy against targets t_g = (number of the
query's brute-force top-10 neighbours stored in grain g) / 10, with AdamW.
The paper leaves learned grain partitioning to future work (sec. 4); these
choices are the build's own and are listed in the design notes.

The BF16 arithmetic of the GPU kernels is defined by where values are
rounded to BF16 before a matrix product; everything else is exact here
(FP64) and FP32 on the GPU:
  forward:  X_b = bf16(X); W_b = bf16(W) for each layer
            A1 = X_b W1_b^T + b1;  H1_b = bf16(gelu(A1))
            A2 = H1_b W2_b^T + b2; H2_b = bf16(gelu(A2))
            L  = H2_b W3_b^T + b3; P = softmax(L)
  loss:     -(1/B) sum_i sum_g T_ig log P_ig
  backward: dL = (P - T) / B, dL_b = bf16(dL)
            dW3 = dL_b^T H2_b, db3 = column sums of dL
            dH2 = dL_b W3_b;   dA2 = dH2 * gelu'(A2), dA2_b = bf16(dA2)
            dW2 = dA2_b^T H1_b, db2 = column sums of dA2
            dH1 = dA2_b W2_b;  dA1 = dH1 * gelu'(A1), dA1_b = bf16(dA1)
            dW1 = dA1_b^T X_b,  db1 = column sums of dA1
With round_bf16=False the same formulas run with no rounding at all (the
plain FP64 MLP), which is what the finite-difference pin checks.
"""
from __future__ import annotations

import math

import numpy as np

from . import hntl_oracle as O

_SQRT2 = math.sqrt(2.0)
_INV_SQRT_2PI = 1.0 / math.sqrt(2.0 * math.pi)


def _erf(x):
    return np.vectorize(math.erf, otypes=[np.float64])(x)


def gelu(x):
    return 0.5 * x * (1.0 + _erf(x / _SQRT2))


def gelu_grad(x):
    return 0.5 * (1.0 + _erf(x / _SQRT2)) + x * _INV_SQRT_2PI * np.exp(-0.5 * x * x)


def _r(x, on):
    if not on:
        return np.asarray(x, dtype=np.float64)
    return O.bf16_to_f32(O.bf16_round(np.asarray(x, dtype=np.float32))).reshape(np.shape(x)).astype(np.float64)


def forward(params, X, round_bf16=True):
    W1, b1, W2, b2, W3, b3 = (np.asarray(p, dtype=np.float64) for p in params)
    Xb = _r(X, round_bf16)
    A1 = Xb @ _r(W1, round_bf16).T + b1
    H1 = _r(gelu(A1), round_bf16)
    A2 = H1 @ _r(W2, round_bf16).T + b2
    H2 = _r(gelu(A2), round_bf16)
    L = H2 @ _r(W3, round_bf16).T + b3
    m = L.max(axis=1, keepdims=True)
    E = np.exp(L - m)
    P = E / E.sum(axis=1, keepdims=True)
    return dict(Xb=Xb, A1=A1, H1=H1, A2=A2, H2=H2, L=L, P=P)


def loss(P, T):
    B = P.shape[0]
    with np.errstate(divide="ignore"):
        lp = np.where(T > 0, np.log(np.maximum(P, 1e-300)), 0.0)
    return float(-(T * lp).sum() / B)


def backward(params, X, T, round_bf16=True):
    """Gradients (dW1, db1, dW2, db2, dW3, db3) and the loss, per the formulas above."""
    W1, b1, W2, b2, W3, b3 = (np.asarray(p, dtype=np.float64) for p in params)
    f = forward(params, X, round_bf16)
    B = X.shape[0]
    T = np.asarray(T, dtype=np.float64)
    dL = (f["P"] - T) / B
    dLb = _r(dL, round_bf16)
    dW3 = dLb.T @ f["H2"]
    db3 = dL.sum(0)
    dH2 = dLb @ _r(W3, round_bf16)
    dA2 = dH2 * gelu_grad(f["A2"])
    dA2b = _r(dA2, round_bf16)
    dW2 = dA2b.T @ f["H1"]
    db2 = dA2.sum(0)
    dH1 = dA2b @ _r(W2, round_bf16)
    dA1 = dH1 * gelu_grad(f["A1"])
    dA1b = _r(dA1, round_bf16)
    dW1 = dA1b.T @ f["Xb"]
    db1 = dA1.sum(0)
    return (dW1, db1, dW2, db2, dW3, db3), loss(f["P"], T)


def adamw(params, grads, m, v, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, wd=0.01):
    """One decoupled-weight-decay Adam step on FP64 copies (returns new params, m, v)."""
    out_p, out_m, out_v = [], [], []
    c1 = 1.0 - beta1 ** step
    c2 = 1.0 - beta2 ** step
    for p, g, mm, vv in zip(params, grads, m, v):
        p = np.asarray(p, dtype=np.float64)
        mm = beta1 * mm + (1.0 - beta1) * g
        vv = beta2 * vv + (1.0 - beta2) * g * g
        p = p - lr * ((mm / c1) / (np.sqrt(vv / c2) + eps) + wd * p)
        out_p.append(p)
        out_m.append(mm)
        out_v.append(vv)
    return out_p, out_m, out_v


def route(params, Q, nprobe, tau, centroid_probe, round_bf16=True):
    """Learned routing of each query: the nprobe grains of largest logit
    (ties to the lower grain id), kept when their softmax mass reaches tau,
    otherwise the query's centroid probes (centroid_probe [nq, nprobe]).
    Returns (probe i32 [nq, nprobe], fell_back bool [nq], mass f64 [nq],
    logits f64 [nq, G])."""
    L = forward(params, Q, round_bf16)["L"]
    nq, G = L.shape
    probe = np.zeros((nq, nprobe), dtype=np.int32)
    mass = np.zeros(nq)
    fell = np.zeros(nq, dtype=bool)
    for i in range(nq):
        order = sorted(range(G), key=lambda g: (-L[i, g], g))[:nprobe]
        m = L[i].max()
        e = np.exp(L[i] - m)
        mass[i] = e[order].sum() / e.sum()
        fell[i] = not (mass[i] >= tau)
        probe[i] = np.asarray(centroid_probe[i]) if fell[i] else np.asarray(order)
    return probe, fell, mass, L


def soft_targets(neighbour_ids, assign, G):
    """t_g = (# of a query's neighbour ids whose grain is g) / (# neighbours)."""
    nb = np.asarray(neighbour_ids)
    T = np.zeros((nb.shape[0], G), dtype=np.float64)
    k = nb.shape[1]
    for i in range(nb.shape[0]):
        for j in nb[i]:
            if j >= 0:
                T[i, assign[j]] += 1.0 / k
    return T


def init_params(d, h1, h2, G, seed):
    """Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights, zero biases (FP32)."""
    rng = np.random.default_rng(seed)
    out = []
    for fan_out, fan_in in ((h1, d), (h2, h1), (G, h2)):
        a = 1.0 / math.sqrt(fan_in)
        out.append(rng.uniform(-a, a, size=(fan_out, fan_in)).astype(np.float32))
        out.append(np.zeros(fan_out, dtype=np.float32))
    return out
