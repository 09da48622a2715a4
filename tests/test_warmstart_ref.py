"""Pins of the float64 warm-start network reference (oracle/warmstart_ref.py):
the convolution against a brute-force loop over its definition, the
analytic backward pass against central finite differences of the loss, and
the bfloat16 rounding against hand-checked values."""
import numpy as np

from oracle import warmstart_ref as ref


def brute_conv(A, W, b, d):
    n, R, _, ci = A.shape
    co = W.shape[1]
    Y = np.zeros((n, R, R, co))
    for k in range(n):
        for y in range(R):
            for x in range(R):
                for o in range(co):
                    s = b[o]
                    for t in range(9):
                        dy, dx = t // 3 - 1, t % 3 - 1
                        yy, xx = y + d * dy, x + d * dx
                        if 0 <= yy < R and 0 <= xx < R:
                            s += sum(A[k, yy, xx, c] * W[t, o, c] for c in range(ci))
                    Y[k, y, x, o] = s
    return Y


def test_conv_matches_brute_force():
    rng = np.random.default_rng(0)
    for d in (1, 2, 3):
        A = rng.standard_normal((2, 5, 5, 2))
        W = rng.standard_normal((9, 3, 2))
        b = rng.standard_normal(3)
        assert np.allclose(ref.conv(A, W, b, d), brute_conv(A, W, b, d), rtol=0, atol=1e-12)


def test_conv_center_tap_is_a_pointwise_product():
    rng = np.random.default_rng(1)
    A = rng.standard_normal((1, 4, 4, 3))
    W = np.zeros((9, 2, 3))
    W[4] = rng.standard_normal((2, 3))
    assert np.allclose(ref.conv(A, W, np.zeros(2), 2), A @ W[4].T, atol=1e-14)


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(2)
    io, C, L, dil = 3, 4, 2, [1, 2]
    n = ref.param_count(io, C, L)
    theta = 0.3 * rng.standard_normal(n)
    X = rng.standard_normal((2, 6, 6, io))
    T = rng.standard_normal((2, 6, 6, io))
    w = rng.random((2, 6, 6))
    loss, g = ref.loss_and_grad(theta, X, T, w, 2, io, C, L, dil)
    h = 1e-6
    for k in rng.choice(n, 60, replace=False):
        e = np.zeros(n)
        e[k] = h
        lp, _ = ref.loss_and_grad(theta + e, X, T, w, 2, io, C, L, dil)
        lm, _ = ref.loss_and_grad(theta - e, X, T, w, 2, io, C, L, dil)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(fd)), (k, fd, g[k])


def test_loss_is_zero_at_the_target_and_ignores_unused_channels():
    rng = np.random.default_rng(3)
    io, C, L = 3, 4, 1
    theta = 0.3 * rng.standard_normal(ref.param_count(io, C, L))
    X = rng.standard_normal((1, 5, 5, io))
    Y, _ = ref.forward(theta, X, io, C, L, [1])
    T = Y.copy()
    T[..., 2] += 5.0          # channel 2 does not enter when out_ch = 2
    loss, g = ref.loss_and_grad(theta, X, T, np.ones((1, 5, 5)), 2, io, C, L, [1])
    assert loss == 0.0 and not g.any()


def test_round_bf16():
    v = np.array([1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, -2.5, 1 + 2 ** -7])
    assert list(ref.round_bf16(v)) == [1.0, 1.0, 1 + 2 ** -6, -2.5, 1 + 2 ** -7]
