"""Pins of the router oracle: finite differences on a tiny MLP, the softmax
cross-entropy gradient in closed form, GELU against its definition, and
soft targets by hand."""
import math

import numpy as np

from oracle import router_oracle as R


def _tiny(seed=0):
    rng = np.random.default_rng(seed)
    d, h1, h2, G, B = 5, 7, 6, 4, 3
    params = R.init_params(d, h1, h2, G, seed)
    params = [p + (0.1 * rng.standard_normal(p.shape) if p.ndim == 1 else 0) for p in params]  # nonzero biases
    X = rng.standard_normal((B, d))
    T = rng.random((B, G))
    T /= T.sum(1, keepdims=True)
    return [np.asarray(p, dtype=np.float64) for p in params], X, T


def test_backward_matches_finite_differences():
    params, X, T = _tiny()
    grads, l0 = R.backward(params, X, T, round_bf16=False)
    h = 1e-6
    for pi, p in enumerate(params):
        flat = p.reshape(-1)
        for idx in range(0, flat.size, max(1, flat.size // 7)):
            old = flat[idx]
            flat[idx] = old + h
            lp = R.loss(R.forward(params, X, False)["P"], T)
            flat[idx] = old - h
            lm = R.loss(R.forward(params, X, False)["P"], T)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            an = grads[pi].reshape(-1)[idx]
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(fd)), (pi, idx, fd, an)


def test_softmax_ce_gradient_closed_form():
    # a one-layer view: dLoss/dlogits = (softmax - t) / B for soft targets summing to 1
    rng = np.random.default_rng(1)
    Lg = rng.standard_normal((4, 6))
    T = rng.random((4, 6))
    T /= T.sum(1, keepdims=True)
    P = np.exp(Lg - Lg.max(1, keepdims=True))
    P /= P.sum(1, keepdims=True)
    h = 1e-6
    for i in range(4):
        for j in range(6):
            Lp = Lg.copy()
            Lp[i, j] += h
            Pp = np.exp(Lp - Lp.max(1, keepdims=True))
            Pp /= Pp.sum(1, keepdims=True)
            Lm = Lg.copy()
            Lm[i, j] -= h
            Pm = np.exp(Lm - Lm.max(1, keepdims=True))
            Pm /= Pm.sum(1, keepdims=True)
            fd = (R.loss(Pp, T) - R.loss(Pm, T)) / (2 * h)
            assert abs(fd - (P[i, j] - T[i, j]) / 4) < 1e-8


def test_gelu_definition_and_derivative():
    xs = np.linspace(-6, 6, 41)
    for x in xs:
        assert abs(R.gelu(np.array([x]))[0] - 0.5 * x * (1 + math.erf(x / math.sqrt(2)))) < 1e-15
        h = 1e-6
        fd = (R.gelu(np.array([x + h]))[0] - R.gelu(np.array([x - h]))[0]) / (2 * h)
        assert abs(fd - R.gelu_grad(np.array([x]))[0]) < 1e-8
    assert R.gelu(np.array([0.0]))[0] == 0.0


def test_soft_targets_by_hand():
    nb = np.array([[0, 1, 2, 3], [4, 4 - 4, 1, -1]])
    assign = np.array([2, 0, 2, 1, 0])
    T = R.soft_targets(nb, assign, 3)
    np.testing.assert_allclose(T[0], [0.25, 0.25, 0.5])
    np.testing.assert_allclose(T[1], [0.5, 0.0, 0.25])  # the -1 pad contributes nothing


def test_adamw_first_step_is_sign_step():
    # with bias correction the first Adam step moves each weight by about lr * sign(g), plus decay
    p = [np.array([1.0, -2.0, 0.5])]
    g = [np.array([0.3, -0.01, 2.0])]
    newp, m, v = R.adamw(p, g, [np.zeros(3)], [np.zeros(3)], step=1, lr=0.1, wd=0.0, eps=0.0)
    np.testing.assert_allclose(newp[0], p[0] - 0.1 * np.sign(g[0]), rtol=1e-12)


def test_adamw_constant_gradient_closed_form_over_steps():
    """Under a gradient that never changes, the bias-corrected moments equal
    g and g^2 at every step t (m_t = (1 - b1^t) g, v_t = (1 - b2^t) g^2), so
    each step moves a weight by lr (g / (|g| + eps) + wd p): a wrong step
    count or bias-correction exponent breaks this from the second step on."""
    p0 = np.array([1.0, -2.0, 0.5, 3.0])
    g = np.array([0.3, -0.01, 2.0, -5.0])
    lr, wd, eps = 0.05, 0.1, 1e-3
    p, m, v = [p0.copy()], [np.zeros(4)], [np.zeros(4)]
    want = p0.copy()
    for t in range(1, 7):
        p, m, v = R.adamw(p, [g], m, v, step=t, lr=lr, wd=wd, eps=eps)
        want = (1.0 - lr * wd) * want - lr * g / (np.abs(g) + eps)
        np.testing.assert_allclose(m[0], (1.0 - 0.9 ** t) * g, rtol=1e-12)
        np.testing.assert_allclose(v[0], (1.0 - 0.999 ** t) * g * g, rtol=1e-12)
        np.testing.assert_allclose(p[0], want, rtol=1e-10, atol=1e-12)


def test_route_takes_largest_logits_and_falls_back_below_tau():
    """With W3 = 0 the logits are b3 for every input, so the probes, their
    softmax mass and the fallback decision follow by hand."""
    params = R.init_params(4, 8, 8, 6, seed=3)
    params[4] = np.zeros_like(params[4])
    params[5] = np.array([0.0, 2.0, 1.0, 2.0, -1.0, 0.5], dtype=np.float32)  # grains 1 and 3 tie
    Q = np.random.default_rng(1).standard_normal((3, 4))
    centroid = np.array([[5, 4], [0, 2], [4, 0]], dtype=np.int32)
    e = np.exp(params[5].astype(np.float64) - 2.0)
    mass = (e[1] + e[3]) / e.sum()  # top two: grains 1, 3 (the tie keeps both; lower id first)
    probe, fell, m, L = R.route(params, Q, 2, tau=0.0, centroid_probe=centroid)
    assert np.allclose(L, params[5][None, :])
    assert probe.tolist() == [[1, 3]] * 3 and not fell.any()
    assert np.allclose(m, mass)
    probe, fell, _, _ = R.route(params, Q, 2, tau=mass + 1e-9, centroid_probe=centroid)
    assert fell.all() and probe.tolist() == centroid.tolist()
    # the three largest: 1 and 3 (tied, lower id first), then 2
    probe, _, _, _ = R.route(params, Q, 3, tau=0.0, centroid_probe=np.zeros((3, 3), np.int32))
    assert probe[0].tolist() == [1, 3, 2]
