"""Pins of the oracle's decoupled appearance model (Sec. 4.1.1) and Adam."""
import numpy as np
import pytest
import torch

from oracle import appearance as app


def _flat(emb, W1, b1, W2, b2):
    return np.concatenate([np.ravel(emb), np.ravel(W1), np.ravel(b1), np.ravel(W2), np.ravel(b2)])


def test_zero_output_layer_is_the_identity():
    rng = np.random.default_rng(0)
    n, E, H = 3, 4, 5
    flat = _flat(rng.normal(size=(n, E)), rng.normal(size=(H, E)), rng.normal(size=H), np.zeros((12, H)), np.zeros(12))
    c = rng.uniform(0, 1, (3, 6, 7))
    _, _, _, corr = app.loss_and_grads(flat, n, E, H, [c], [c], [1])
    np.testing.assert_array_equal(corr[0], c)


def test_hand_computed_network_and_affine():
    # E = H = 2: e = (1, -2); W1 = [[1, 0.5], [2, 1]], b1 = (0.5, -0.5)
    # pre-activations: 1 - 1 + 0.5 = 0.5 and 2 - 2 - 0.5 = -0.5 -> h = (0.5, 0)
    E = H = 2
    W2 = np.zeros((12, 2))
    W2[0, 0] = 0.2    # a0 = 0.1
    W2[4, 0] = -0.4   # a4 = -0.2
    W2[4, 1] = 7.0    # multiplies the clipped unit: no effect
    W2[9, 0] = 0.1    # a9 = 0.05
    b2 = np.zeros(12)
    b2[8] = 0.3       # a8 = 0.3
    b2[11] = -0.1     # a11 = -0.1
    flat = _flat(np.array([[1.0, -2.0]]), np.array([[1.0, 0.5], [2.0, 1.0]]), np.array([0.5, -0.5]), W2, b2)
    M, t = app.affine(torch.tensor(flat), 1, E, H, 0)
    np.testing.assert_allclose(M.numpy(), np.diag([1.1, 0.8, 1.3]), atol=1e-15)
    np.testing.assert_allclose(t.numpy(), [0.05, 0.0, -0.1], atol=1e-15)
    c = np.array([0.2, 0.5, 0.8]).reshape(3, 1, 1)
    tgt = np.array([0.3, 0.4, 0.9]).reshape(3, 1, 1)
    loss, _, dcol, corr = app.loss_and_grads(flat, 1, E, H, [c], [tgt], [0])
    np.testing.assert_allclose(corr[0].ravel(), [0.27, 0.40, 0.94], atol=1e-15)
    # |0.27-0.3| + |0.4-0.4| + |0.94-0.9| over 3 channels; sign(0) = 0
    np.testing.assert_allclose(loss[0], (0.03 + 0.0 + 0.04) / 3, atol=1e-15)
    # dL/dc = M^T sign(r) / 3 = (1.1 * -1, 0, 1.3 * 1) / 3
    np.testing.assert_allclose(dcol[0].ravel(), [-1.1 / 3, 0.0, 1.3 / 3], atol=1e-15)


def test_gradients_match_central_differences():
    rng = np.random.default_rng(1)
    n, E, H = 2, 3, 4
    flat = rng.normal(0, 0.5, app.param_count(n, E, H))
    cols = [rng.uniform(0, 1, (3, 4, 5)), rng.uniform(0, 1, (3, 3, 4))]
    tgts = [rng.uniform(0, 1, (3, 4, 5)), rng.uniform(0, 1, (3, 3, 4))]
    idx = [1, 0]
    _, g, gc, corr = app.loss_and_grads(flat, n, E, H, cols, tgts, idx)
    assert min(np.abs(c - t).min() for c, t in zip(corr, tgts)) > 1e-4   # no kink within the step

    def L(f, cs):
        return app.loss_and_grads(f, n, E, H, cs, tgts, idx)[0].sum()
    h = 1e-6
    for i in range(len(flat)):
        a, b = flat.copy(), flat.copy()
        a[i] += h
        b[i] -= h
        fd = (L(a, cols) - L(b, cols)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 + 1e-5 * abs(g[i]), (i, fd, g[i])
    for v in range(2):
        for idx3 in [(0, 1, 2), (2, 2, 3), (1, 0, 0)]:
            a = [c.copy() for c in cols]
            b = [c.copy() for c in cols]
            a[v][idx3] += h
            b[v][idx3] -= h
            fd = (L(flat, a) - L(flat, b)) / (2 * h)
            assert abs(fd - gc[v][idx3]) <= 1e-6 + 1e-5 * abs(gc[v][idx3])


def test_adam_steps_of_a_constant_gradient_are_lr_sized():
    # with a constant gradient the bias-corrected moments are g and g^2 at every step
    p = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -4.0, 1e-3])
    m = v = np.zeros(3)
    for step in range(1, 6):
        q, m, v = app.adam(p, g, m, v, step, lr=0.01)
        np.testing.assert_allclose(p - q, 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-9)
        p = q


def test_training_recovers_per_view_exposure_and_white_balance():
    rng = np.random.default_rng(2)
    n, E, H = 4, 8, 16
    base = [rng.uniform(0.1, 0.9, (3, 8, 8)) for _ in range(n)]
    gains = rng.uniform(0.7, 1.3, (n, 3))
    offs = rng.uniform(-0.05, 0.05, (n, 3))
    tgts = [g[:, None, None] * c + o[:, None, None] for c, g, o in zip(base, gains, offs)]
    flat = np.concatenate([rng.normal(0, 0.1, n * E), rng.normal(0, 0.3, H * E), np.zeros(H),
                           np.zeros(12 * H), np.zeros(12)])
    m = v = np.zeros_like(flat)
    before = np.mean([app.psnr(c, t) for c, t in zip(base, tgts)])
    for step in range(1, 401):
        _, g, _, corr = app.loss_and_grads(flat, n, E, H, base, tgts, list(range(n)))
        flat, m, v = app.adam(flat, g, m, v, step, lr=1e-2)
    after = np.mean([app.psnr(c, t) for c, t in zip(corr, tgts)])
    assert after > before + 10, (before, after)
