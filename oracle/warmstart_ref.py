"""Plain float64 reference of the warm-start network (test infrastructure).

The paper has no network; this is the reference for the learned warm start
of the library (include/maclab_ws.h), written from its definition there:

    H_1     = conv(X; W_0, b_0)
    H_{l+1} = H_l + conv_{d_l}(relu(H_l); W_l, b_l)      l = 1..L
    Y       = conv(relu(H_{L+1}); W_out, b_out)
    loss    = sum_p w_p sum_{c < out_ch} (Y[p, c] - T[p, c])^2

conv is a 3 x 3 cross-correlation with dilation d and zero padding on NHWC
arrays; weights W[tap][c_out][c_in], tap = 3 (dy + 1) + (dx + 1), input pixel
(y + d dy, x + d dx).  The parameter vector is W_0, b_0, W_1, b_1, ...,
W_out, b_out, flattened in that order.

Only tests/ and the benchmark's baseline leg may import this module.  It is
pinned by tests/test_warmstart_ref.py: the convolution against a brute-force
loop, the backward pass against central finite differences.
"""
from __future__ import annotations

import numpy as np

TAPS = [(t // 3 - 1, t % 3 - 1) for t in range(9)]


def layer_shapes(io: int, channels: int, blocks: int):
    """(c_in, c_out) of the lift, the blocks and the head."""
    return [(io, channels)] + [(channels, channels)] * blocks + [(channels, io)]


def param_count(io: int, channels: int, blocks: int) -> int:
    return sum(9 * ci * co + co for ci, co in layer_shapes(io, channels, blocks))


def unpack(theta: np.ndarray, io: int, channels: int, blocks: int):
    """Parameter vector -> list of (W [9][co][ci], b [co])."""
    out, k = [], 0
    for ci, co in layer_shapes(io, channels, blocks):
        W = theta[k:k + 9 * co * ci].reshape(9, co, ci)
        k += 9 * co * ci
        b = theta[k:k + co]
        k += co
        out.append((W, b))
    assert k == theta.size
    return out


def conv(A: np.ndarray, W: np.ndarray, b: np.ndarray, d: int) -> np.ndarray:
    """Y[n, y, x, o] = b[o] + sum_{t, c} A[n, y + d dy_t, x + d dx_t, c] W[t, o, c]."""
    n, R, _, _ = A.shape
    P = np.pad(A, ((0, 0), (d, d), (d, d), (0, 0)))
    Y = np.broadcast_to(b, A.shape[:3] + (W.shape[1],)).copy()
    for t, (dy, dx) in enumerate(TAPS):
        S = P[:, d + d * dy:d + d * dy + R, d + d * dx:d + d * dx + R, :]
        Y += S @ W[t].T
    return Y


def conv_backward(A: np.ndarray, W: np.ndarray, d: int, dY: np.ndarray):
    """Gradients of sum(dY * conv(A, W, b, d)) w.r.t. A, W and b."""
    n, R, _, _ = A.shape
    P = np.pad(A, ((0, 0), (d, d), (d, d), (0, 0)))
    dP = np.zeros_like(P)
    dW = np.zeros_like(W)
    for t, (dy, dx) in enumerate(TAPS):
        sy, sx = d + d * dy, d + d * dx
        S = P[:, sy:sy + R, sx:sx + R, :]
        dW[t] = np.einsum("nyxo,nyxc->oc", dY, S)
        dP[:, sy:sy + R, sx:sx + R, :] += dY @ W[t]
    return dP[:, d:d + R, d:d + R, :], dW, dY.sum(axis=(0, 1, 2))


def relu(x):
    return np.maximum(x, 0.0)


def forward(theta, X, io, channels, blocks, dilations):
    """Output Y and the residual stream H_1 .. H_{L+1}."""
    layers = unpack(theta, io, channels, blocks)
    H = [conv(X, *layers[0], 1)]
    for l in range(blocks):
        H.append(H[-1] + conv(relu(H[-1]), *layers[1 + l], dilations[l]))
    Y = conv(relu(H[-1]), *layers[-1], 1)
    return Y, H


def loss_and_grad(theta, X, T, w, out_ch, io, channels, blocks, dilations):
    """Loss and its gradient with respect to the parameter vector."""
    layers = unpack(theta, io, channels, blocks)
    Y, H = forward(theta, X, io, channels, blocks, dilations)
    diff = (Y - T)[..., :out_ch]
    loss = float(np.sum(w[..., None] * diff ** 2))
    dY = np.zeros_like(Y)
    dY[..., :out_ch] = 2.0 * w[..., None] * diff
    grads = [None] * len(layers)
    dA, dW, db = conv_backward(relu(H[-1]), layers[-1][0], 1, dY)
    grads[-1] = (dW, db)
    dH = dA * (H[-1] > 0)
    for l in range(blocks - 1, -1, -1):
        dA, dW, db = conv_backward(relu(H[l]), layers[1 + l][0], dilations[l], dH)
        grads[1 + l] = (dW, db)
        dH = dH + dA * (H[l] > 0)
    _, dW, db = conv_backward(X, layers[0][0], 1, dH)
    grads[0] = (dW, db)
    g = np.concatenate([np.concatenate([dW.ravel(), db.ravel()]) for dW, db in grads])
    return loss, g


def round_bf16(x: np.ndarray) -> np.ndarray:
    """Round float values to the nearest bfloat16 (ties to even), returned as
    float64: the precision in which the library stores weights and inputs."""
    f = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (f >> 16) & 1
    r = ((f + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)
