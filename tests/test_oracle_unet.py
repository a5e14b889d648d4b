"""Pins of the U-Net oracle (oracle/unet.py): closed forms of convolution,
pooling and upsampling, and the hand-written backward pass against central
finite differences of the loss.  CPU only."""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def un():
    from oracle import unet
    return unet


def test_parameter_count(un):
    assert un.num_params() == 27 * 13088 + 16 + (16 + 16 + 32 + 32 + 64 + 64 + 32 + 32 + 16 + 16 + 1)


def test_delta_kernel_shifts_with_zero_fill(un):
    rng = np.random.default_rng(0)
    x = rng.standard_normal((1, 5, 6, 7))
    W = np.zeros((1, 1, 3, 3, 3))
    W[0, 0, 2, 1, 0] = 1.0      # picks x[v + (1, 0, -1)]
    y = un.conv(x, W, np.zeros(1))
    want = np.zeros_like(x)
    want[:, :-1, :, 1:] = x[:, 1:, :, :-1]
    assert np.array_equal(y, want)


def test_box_kernel_counts_in_domain_neighbours(un):
    x = np.ones((2, 4, 5, 6))
    W = np.ones((1, 2, 3, 3, 3))
    y = un.conv(x, W, np.array([0.5]))[0]
    cnt = lambda n: np.minimum(np.arange(n) + 1, n - np.arange(n)).clip(max=2) + 1
    want = 2 * cnt(4)[:, None, None] * cnt(5)[None, :, None] * cnt(6)[None, None, :] + 0.5
    assert np.array_equal(y, want)


def test_pool_and_up(un):
    rng = np.random.default_rng(1)
    x = rng.standard_normal((3, 2, 4, 6))
    assert np.allclose(un.pool(un.up(x)), x)
    c = np.full((1, 4, 4, 4), 2.5)
    assert np.array_equal(un.pool(c), np.full((1, 2, 2, 2), 2.5))
    # adjointness: <pool(a), b> = <a, pool_backward(b)>, <up(a), b> = <a, up_backward(b)>
    a = rng.standard_normal((2, 4, 4, 8))
    b = rng.standard_normal((2, 2, 2, 4))
    assert np.isclose(np.sum(un.pool(a) * b), np.sum(a * un.pool_backward(b)))
    assert np.isclose(np.sum(un.up(b) * a), np.sum(b * un.up_backward(a)))


def test_backward_matches_finite_differences(un):
    rng = np.random.default_rng(2)
    shape = (8, 8, 8)
    x = rng.standard_normal((2,) + shape)
    t = rng.standard_normal((1,) + shape)
    mask = (rng.uniform(size=(1,) + shape) > 0.2).astype(np.float64)
    p = un.init_params(3) * 0.5 + 0.01 * rng.standard_normal(un.num_params())
    y, a = un.forward(p, x)
    L, dy = un.loss(y, t, mask)
    g, dx = un.backward(p, a, dy)
    h = 1e-6
    # a spread of parameters: every layer's weights and biases
    offs, o = [], 0
    for ci, co, k in un.LAYERS:
        n = co * ci * k ** 3
        offs += [o, o + n // 3, o + n - 1, o + n, o + n + co - 1]
        o += n + co
    for q in offs:
        e = np.zeros_like(p)
        e[q] = h
        lp = un.loss(un.forward(p + e, x)[0], t, mask)[0]
        lm = un.loss(un.forward(p - e, x)[0], t, mask)[0]
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[q]) <= 1e-5 * max(1.0, abs(fd)) + 1e-7, (q, fd, g[q])
    for idx in ((0, 1, 2, 3), (1, 7, 0, 5), (0, 4, 4, 4)):
        e = np.zeros_like(x)
        e[idx] = h
        lp = un.loss(un.forward(p, x + e)[0], t, mask)[0]
        lm = un.loss(un.forward(p, x - e)[0], t, mask)[0]
        assert abs((lp - lm) / (2 * h) - dx[idx]) <= 1e-5 * max(1.0, abs(dx[idx])) + 1e-7


def test_adam_first_step_moves_by_lr(un):
    p = np.array([1.0, -2.0, 3.0])
    g = np.array([0.5, -4.0, 0.0])
    q, m, v = un.adam(p, np.zeros(3), np.zeros(3), g, 1, 0.1)
    assert np.allclose(q, p - 0.1 * np.sign(g), atol=1e-6)
