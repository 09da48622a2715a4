"""The learned warm start at the benchmark's network shape (64 x 64 cells,
128 channels, the default 12 residual blocks, batch 16), layer by layer and
element by element against the float64 reference, within bounds derived
from the arithmetic the library does.

Every layer is checked on its own stored inputs (maclab_ws_inspect): the
reference recomputes the layer's output from the bfloat16 tensors the
library kept, so the only differences left are the library's own roundings:

  * products of two bfloat16 values are exact in float; summing n of them
    in float errs by at most  n_acc * 2^-22 * S,  S = sum of |terms| of the
    output (the bias and residual included), n_acc the longest chain of
    float additions any term goes through in that kernel (9 C_in / 16
    tensor-core accumulations of 16 products each plus the epilogue; for
    the weight gradient, the pixel chunks of one split plus the splits).
    2^-22 is four times float's unit roundoff: the tensor cores' internal
    accumulation is not specified as round-to-nearest;
  * an output stored in bfloat16 (H_l and its gradient) is rounded once
    more, by at most u = 2^-8 of its value.

So |got - ref| <= u |ref| + (1 + u) n_acc 2^-22 S  for every element, at
every pixel, borders included.  The bound is about 0.4 % of a typical
output; a transposed, flipped or shifted tap, a lost halo row or a wrong
zero fill moves an output by several per cent of S, which the planted
mistake below confirms.
"""
import multiprocessing
import os

import numpy as np
import pytest

from oracle import warmstart_ref as ref

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

IO = 16
U_BF16 = 2.0 ** -8
U_ACC = 2.0 ** -22
BATCH = 16


def setup(net, seed):
    rng = np.random.default_rng(seed)
    C, blocks = net.channels, len(net.dilations)
    theta = np.zeros(net.nparam)
    k = 0
    for ci, co in ref.layer_shapes(IO, C, blocks):
        theta[k:k + 9 * ci * co] = rng.standard_normal(9 * ci * co) * np.sqrt(1.0 / (9 * ci))
        k += 9 * ci * co
        theta[k:k + co] = 0.1 * rng.standard_normal(co)
        k += co
    theta = ref.round_bf16(theta.astype(np.float32))
    X = ref.round_bf16(rng.standard_normal((BATCH, 64, 64, IO)).astype(np.float32))
    T = rng.standard_normal(X.shape).astype(np.float32).astype(np.float64)
    w = rng.random(X.shape[:3])
    return theta, X, T, (w / w.sum()).astype(np.float32).astype(np.float64)


def conv_chain(cin):
    """Float additions on the longest path of one convolution output: 9 cin
    / 16 accumulations of 16-product sums, then the bias and the residual."""
    return 9 * cin // 16 + 16 + 2


def wgrad_chain(cin, cout, pixels):
    """Float additions on the longest path of one weight-gradient entry, the
    longer of the two kernels' (then 16 inside a 16-product accumulation):
    mma.sync, the 32-pixel chunks one split takes, two accumulations each,
    then the splits' sums in order; tcgen05, the 64-pixel segments of one of
    at most 50 splits, four accumulations each, then the splits' sums."""
    chunks = pixels // 32
    mt = 64 if cout % 64 == 0 else 16
    nt = 64 if cin % 64 == 0 else 16
    splits = max(1, min(chunks, 304 // max(1, (cout // mt) * (cin // nt) * 9) + 1))
    mma_sync = 2 * (-(-chunks // splits)) + splits
    segs = pixels // 64
    s5 = max(1, min(segs, 50))
    tc5 = 4 * (-(-segs // s5)) + s5
    return max(mma_sync, tc5) + 16


def bias_chain(pixels, channels):
    """Float additions of one bias-gradient entry: a thread's share of one
    of 256 blocks' pixels (256 / (channels / 8) threads share a channel),
    the block's threads in order, the 256 block sums."""
    lanes = 256 // (channels // 8)
    return -(-(-(-pixels // 256)) // lanes) + lanes + 256


def abs_input_grad(G, W, d):
    """sum over taps of |G| shifted by the tap times |W|^T: the magnitude
    sum of the input gradient's terms (a convolution of |G| with the taps
    mirrored and the channels transposed)."""
    return ref.conv(np.abs(G), np.abs(W)[::-1].transpose(0, 2, 1), np.zeros(W.shape[2]), d)


def abs_weight_grad(A, G, d):
    """sum over pixels of |G[p]| |A[p + d tap]|: the magnitude sum of each
    weight-gradient entry, [9][c_out][c_in]."""
    n, R, _, ci = A.shape
    Pd = np.pad(np.abs(A), ((0, 0), (d, d), (d, d), (0, 0)))
    aG = np.abs(G).reshape(-1, G.shape[3])
    out = np.empty((9, G.shape[3], ci))
    for t, (dy, dx) in enumerate(ref.TAPS):
        S = Pd[:, d + d * dy:d + d * dy + R, d + d * dx:d + d * dx + R, :].reshape(-1, ci)
        out[t] = aG.T @ S
    return out


def backward_references(tasks):
    """ref.conv_backward of every layer, in parallel processes (spawned, so
    that they share nothing with this process's CUDA context; one BLAS
    thread each)."""
    keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
    saved = {k: os.environ.get(k) for k in keys}
    os.environ.update({k: "1" for k in keys})
    try:
        ctx = multiprocessing.get_context("spawn")
        with ctx.Pool(min(len(tasks), os.cpu_count() or 1)) as pool:
            return pool.starmap(ref.conv_backward, tasks)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


def check(name, got, want, S, n_acc, stored_bf16, report):
    bound = (U_BF16 * np.abs(want) if stored_bf16 else 0.0) + (1 + U_BF16) * n_acc * U_ACC * S
    err = np.abs(got - want)
    ratio = float((err / np.maximum(bound, 1e-300)).max())
    typical = float(np.median(np.abs(want)))
    report.append("%-28s max err/bound %.3f  max err %.3g  median |ref| %.3g" % (name, ratio, err.max(), typical))
    assert np.isfinite(got).all(), name
    assert (err <= bound).all(), (name, ratio, np.unravel_index(np.argmax(err / np.maximum(bound, 1e-300)),
                                                                err.shape))


@pytest.mark.parametrize("path", [0, 1, 2])
def test_full_shape_every_layer_elementwise(path):
    from paper_1902_02999_gb300.warmstart import WarmStartNet
    net = WarmStartNet(max_batch=BATCH, tensor_path=path)
    C, dil, L = net.channels, list(net.dilations), len(net.dilations)
    assert (C, L) == (128, 12)
    theta, X, T, w = setup(net, 5)
    net.set_params(theta)
    net.keep_gradients(True)
    dev = lambda a: torch.tensor(a, dtype=torch.float32, device="cuda")
    loss, g = net.gradients(dev(X), dev(T), dev(w), out_ch=3)
    torch.cuda.synchronize()
    get = lambda what, k: net.inspect(what, k, BATCH).cpu().numpy().astype(np.float64)
    layers = ref.unpack(theta, IO, C, L)
    P = BATCH * 64 * 64
    report = []
    # offsets of each layer's weights and bias in the parameter vector
    offs, k = [], 0
    for ci, co in ref.layer_shapes(IO, C, L):
        offs.append((k, k + 9 * ci * co))
        k += 9 * ci * co + co

    H = [get(0, k) for k in range(L + 1)]  # H_1 .. H_{L+1}
    Y = get(3, 0)
    dY = get(2, 0)
    for k in range(L + 2):
        Wk, bk = layers[k]
        d = 1 if k in (0, L + 1) else dil[k - 1]
        ci = Wk.shape[2]
        A = X if k == 0 else ref.relu(H[k - 1])
        # forward: H[k] = H[k-1] + conv(A) (blocks), conv(X) (lift), Y = conv (head)
        want = ref.conv(A, Wk, bk, d)
        S = ref.conv(np.abs(A), np.abs(Wk), np.abs(bk), d)
        if 1 <= k <= L:
            want = want + H[k - 1]
            S = S + np.abs(H[k - 1])
        got = Y if k == L + 1 else H[k]
        check("forward layer %d (d=%d)" % (k, d), got, want, S, conv_chain(ci), k <= L, report)

    # the loss and its output gradient from the library's own Y
    diff = (Y - T)[..., :3]
    want_loss = float(np.sum(w[..., None] * diff ** 2))
    report.append("loss %.9g vs %.9g" % (loss, want_loss))
    assert abs(loss - want_loss) <= 4 * 2.0 ** -24 * want_loss
    want_dY = np.zeros_like(Y)
    want_dY[..., :3] = 2.0 * w[..., None] * diff
    assert (dY[..., 3:] == 0).all()
    check("dY", dY, want_dY, np.abs(want_dY), 2, True, report)

    # backward, layer by layer from the stored output gradients
    dil_of = lambda k: 1 if k in (0, L + 1) else dil[k - 1]
    inputs = [X] + [ref.relu(H[k - 1]) for k in range(1, L + 2)]
    grads = [get(1, k) for k in range(L + 1)] + [dY]
    refs = backward_references([(inputs[k], layers[k][0], dil_of(k), grads[k]) for k in range(L + 2)])
    for k in range(L + 1, -1, -1):
        Wk, bk = layers[k]
        d = dil_of(k)
        ci, co = Wk.shape[2], Wk.shape[1]
        A, G = inputs[k], grads[k]
        dA, dW, db = refs[k]
        SdA = abs_input_grad(G, Wk, d)
        SdW = abs_weight_grad(A, G, d)
        Sdb = np.abs(G).sum(axis=(0, 1, 2))
        w0, b0 = offs[k]
        check("weight grad layer %d" % k, g[w0:b0].astype(np.float64), dW.ravel(), SdW.ravel(),
              wgrad_chain(ci, co, P), False, report)
        check("bias grad layer %d" % k, g[b0:b0 + co].astype(np.float64), db, Sdb, bias_chain(P, co), False, report)
        if k == 0:
            continue
        want = dA * (H[k - 1] > 0)
        S = SdA
        if k <= L:
            want = want + G
            S = S + np.abs(G)
        check("input grad layer %d" % k, get(1, k - 1), want, S, conv_chain(co), True, report)
    print("\npath %d\n  " % path + "\n  ".join(report))
    net.close()


def test_bound_catches_a_transposed_tap():
    """The same bound against a reference with one layer's taps mirrored
    (W[t] -> W[8 - t], a flipped kernel) fails: the check has the power to
    see a mistake of that kind.  The mistake is planted in the reference."""
    from paper_1902_02999_gb300.warmstart import WarmStartNet
    net = WarmStartNet(max_batch=BATCH, tensor_path=0)
    C, L = net.channels, len(net.dilations)
    theta, X, _, _ = setup(net, 5)
    net.set_params(theta)
    net.forward(torch.tensor(X, dtype=torch.float32, device="cuda"))
    H0 = net.inspect(0, 0, BATCH).cpu().numpy().astype(np.float64)
    H1 = net.inspect(0, 1, BATCH).cpu().numpy().astype(np.float64)
    Wk, bk = ref.unpack(theta, IO, C, L)[1]
    A = ref.relu(H0)
    S = ref.conv(np.abs(A), np.abs(Wk), np.abs(bk), 1) + np.abs(H0)
    bound = U_BF16 * np.abs(H1) + (1 + U_BF16) * conv_chain(C) * U_ACC * S
    flipped = H0 + ref.conv(A, Wk[::-1], bk, 1)
    ok = H0 + ref.conv(A, Wk, bk, 1)
    assert (np.abs(H1 - ok) <= bound).all()
    frac = float(np.mean(np.abs(H1 - flipped) > bound))
    print("flipped kernel: %.1f %% of the outputs out of bound" % (100 * frac))
    assert frac > 0.9
    net.close()
