"""Pins of the warm-start network oracle (oracle/learned.py), CPU only.

The convolution is checked against the convolution theorem (numpy FFT) and against
explicit index shifts that fix the tap order; its two derivatives against the exact
adjoint identities; the whole network's backward pass against central finite
differences; BF16 rounding against hand-worked ties and torch's conversion; Adam against
its closed form under a constant gradient.
"""
import numpy as np
import pytest

from oracle import learned as L
from synthetic import conv_net_parameters, normal_field, uniform_field


def _rand(shape, seed):
    return normal_field(int(np.prod(shape)), seed).reshape(shape)


def _grid(a, n):
    """voxel-major (N, C) -> (C, z, y, x)"""
    return np.asarray(a).T.reshape(-1, n, n, n)


def test_conv_matches_fft_cross_correlation():
    n, ci, co = 5, 3, 2
    x = _rand((n ** 3, ci), 1)
    W = _rand((27, co, ci), 2)
    b = _rand((co,), 3)
    y = L.conv3d(x, W, b, n)
    xg = _grid(x, n)
    for o in range(co):
        acc = np.zeros((n, n, n))
        for i in range(ci):
            k = np.zeros((n, n, n))                       # k[-d mod n] = W[t(d)]
            for t, (dx, dy, dz) in enumerate(L.tap_offsets()):
                k[(-dz) % n, (-dy) % n, (-dx) % n] += W[t, o, i]
            acc += np.real(np.fft.ifftn(np.fft.fftn(xg[i]) * np.fft.fftn(k)))
        assert np.abs(acc + b[o] - _grid(y, n)[o]).max() < 1e-12


def test_tap_order_and_orientation():
    """Tap 14 is d = (+1, 0, 0): y(x, y, z) = x((x+1) % n, y, z); tap 22 is d = (0, 0, +1);
    tap 10 is d = (0, -1, 0)."""
    n = 4
    x = _rand((n ** 3, 1), 4)
    xg = x[:, 0].reshape(n, n, n)
    for t, (ax, s) in ((14, (2, 1)), (22, (0, 1)), (10, (1, -1))):
        W = np.zeros((27, 1, 1))
        W[t] = 1.0
        y = L.conv3d(x, W, None, n)[:, 0].reshape(n, n, n)
        for z in range(n):
            for yy in range(n):
                for xx in range(n):
                    c = [z, yy, xx]
                    c[ax] = (c[ax] + s) % n
                    assert y[z, yy, xx] == xg[tuple(c)]
    W = np.zeros((27, 2, 1))                                  # centre tap = pointwise matrix
    W[13, :, 0] = (2.0, -3.0)
    assert np.array_equal(L.conv3d(x, W, None, n), x @ np.array([[2.0, -3.0]]))


def test_dgrad_is_the_adjoint_and_wgrad_the_weight_derivative():
    n, ci, co = 4, 3, 5
    x = _rand((n ** 3, ci), 5)
    dy = _rand((n ** 3, co), 6)
    W = _rand((27, co, ci), 7)
    lhs = float((L.conv3d(x, W, None, n) * dy).sum())
    assert abs(lhs - float((x * L.conv3d_dgrad(dy, W, n)).sum())) < 1e-11 * abs(lhs) + 1e-11
    V = _rand((27, co, ci), 8)
    c = _rand((co,), 9)
    dW, db = L.conv3d_wgrad(x, dy, n)
    got = float((V * dW).sum() + (c * db).sum())
    want = float((L.conv3d(x, V, c, n) * dy).sum())
    assert abs(got - want) < 1e-11 * abs(want) + 1e-11


def _small_net(seed, c_in0=4, C=4, nb=2):
    shapes = [(27, C, c_in0)] + [(27, C, C)] * (2 * nb) + [(27, C, C)]
    params = conv_net_parameters(shapes, seed, [1.0] * len(shapes))
    # nonzero biases so that every ReLU sees both signs
    return [(W.astype(np.float64), 0.1 * _rand((W.shape[1],), seed + 100 + l))
            for l, (W, _) in enumerate(params)]


def test_network_gradient_matches_central_differences():
    n, C = 3, 4
    params = _small_net(11, C=C)
    x = L.features(uniform_field(n ** 3, 12, 0.0, 1.0, np.float64), 4)
    T = _rand((n ** 3, 18), 13) * 0.1
    planes = 3                      # C = 4 output rows: the loss reads rows 0..2

    def loss(ps):
        y, _ = L.forward(ps, x, n, rounding=False)
        return L.mse_loss(y, T, planes)[0]

    y, cache = L.forward(params, x, n, rounding=False)
    _, dy = L.mse_loss(y, T, planes)
    grads = L.backward(params, cache, dy)
    for k in range(3):
        dirs = [(_rand(W.shape, 200 + 10 * k + l), _rand(b.shape, 300 + 10 * k + l))
                for l, (W, b) in enumerate(params)]
        eps = 1e-6
        plus = [(W + eps * dW, b + eps * db) for (W, b), (dW, db) in zip(params, dirs)]
        minus = [(W - eps * dW, b - eps * db) for (W, b), (dW, db) in zip(params, dirs)]
        fd = (loss(plus) - loss(minus)) / (2 * eps)
        an = sum(float((gW * dW).sum() + (gb * db).sum()) for (gW, gb), (dW, db) in zip(grads, dirs))
        assert abs(fd - an) <= 1e-6 * abs(an) + 1e-10, (fd, an)


def test_network_is_translation_equivariant():
    """Periodic convolutions commute with periodic shifts of the cell (rounding on)."""
    n = 5
    params = _small_net(21, c_in0=16, C=8, nb=1)
    rho = uniform_field(n ** 3, 22, 0.0, 1.0, np.float64)
    y, _ = L.forward(params, L.features(rho, 16), n)
    shift = (2, -1, 3)                                      # (dz, dy, dx)
    rho_s = np.roll(rho.reshape(n, n, n), shift, axis=(0, 1, 2)).ravel()
    ys, _ = L.forward(params, L.features(rho_s, 16), n)
    want = np.roll(y.reshape(n, n, n, -1), shift, axis=(0, 1, 2)).reshape(n ** 3, -1)
    assert np.array_equal(ys, want)


def test_bf16_rounding_ties_and_torch():
    one = 1.0
    assert L.bf16_round(one + 2.0 ** -8) == one                      # tie -> even (down)
    assert L.bf16_round(one + 3 * 2.0 ** -8) == one + 2.0 ** -6     # tie -> even (up)
    assert L.bf16_round(one + 2.0 ** -8 + 2.0 ** -20) == one + 2.0 ** -7
    assert L.bf16_round(-(one + 3 * 2.0 ** -8)) == -(one + 2.0 ** -6)
    assert L.bf16_round(3.0) == 3.0 and L.bf16_round(0.0) == 0.0
    torch = pytest.importorskip("torch")
    a = (normal_field(100000, 31) * np.exp(4 * normal_field(100000, 32))).astype(np.float32)
    want = torch.from_numpy(a).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(L.bf16_round(a), want)


def test_adam_closed_form_under_constant_gradient():
    """With a constant gradient g the bias-corrected moments are g and g^2 at every step,
    so each step moves w by -lr g / (|g| + eps)."""
    g = np.array([0.5, -2.0, 1e-3, 0.0])
    w = np.array([1.0, 2.0, 3.0, 4.0])
    m = v = np.zeros(4)
    lr, eps = 1e-2, 1e-8
    cur = w
    for step in range(1, 6):
        cur, m, v = L.adam_step(cur, g, m, v, step, lr, eps=eps)
    want = w - 5 * lr * g / (np.abs(g) + eps)
    assert np.abs(cur - want).max() < 1e-12


def test_mse_loss_gradient_and_displacement_maps():
    N = 7
    y = _rand((N, 32), 41)
    T = _rand((N, 18), 42)
    l0, g = L.mse_loss(y, T)
    assert np.all(g[:, 18:] == 0)
    d = _rand((N, 32), 43)
    eps = 1e-6
    fd = (L.mse_loss(y + eps * d, T)[0] - L.mse_loss(y - eps * d, T)[0]) / (2 * eps)
    assert abs(fd - float((g * d).sum())) < 1e-8
    n, s = 2, np.array([0.05, 0.1, 0.2, 0.03, 0.07, 0.5])
    u = _rand((18, n ** 3), 44)
    T2 = L.displacement_target(u, n, s)
    assert np.allclose(T2[:, 4], u[4] / (n * s[1])) and np.allclose(T2[:, 17], u[17] / (n * s[5]))
    assert np.allclose(L.displacement_from_output(np.hstack([T2, np.zeros((n ** 3, 14))]), n, s), u)


def test_pool_by_brute_force():
    n, f = 6, 3
    rho = uniform_field(n ** 3, 51, 0.0, 1.0, np.float64)
    got = L.pool(rho, n, f)
    g = rho.reshape(n, n, n)                                 # (z, y, x)
    for k in range(2):
        for j in range(2):
            for i in range(2):
                want = np.mean([g[f * k + c, f * j + b, f * i + a]
                                for a in range(f) for b in range(f) for c in range(f)])
                assert abs(got[i + 2 * (j + 2 * k)] - want) < 1e-15


def test_features_hand_values():
    x = L.features(np.array([0.0, 1.0, 0.5, 0.2]), 16)
    assert x.shape == (4, 16) and np.all(x[:, 3:] == 0)
    assert np.array_equal(x[0, :3], [0.0, 0.0, 0.0]) and np.array_equal(x[1, :3], [1.0, 1.0, 1.0])
    assert np.array_equal(x[2, :3], [0.5, 0.25, 0.125])
    assert np.allclose(x[3, :3], [0.2, 0.04, 0.008], rtol=1e-15, atol=0)
