"""The learned warm start on the GPU (include/maclab_ws.h) against the
float64 network reference (oracle/warmstart_ref.py), and what it gains.

Tolerances: the library stores activations in bfloat16 (8 significant
bits) and sums products in float.  The reference gets the same bfloat16
inputs and weights, so what remains is the rounding of the stored
activations and gradients, a few parts in a thousand per layer; relative
L2 errors of 3e-2 (outputs) and 6e-2 (gradients, per layer) leave room for
that and still catch a transposed, flipped or misplaced tap, which errs by
O(1).
"""
import numpy as np
import pytest

import inputs
from oracle import warmstart_ref as ref

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

IO = 16


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def make(C, dil, batch, seed=0, tensor_path=0):
    from paper_1902_02999_gb300.warmstart import WarmStartNet
    return WarmStartNet(res=64, channels=C, dilations=dil, max_batch=batch, seed=seed, tensor_path=tensor_path)


def random_setup(net, C, dil, batch, seed):
    rng = np.random.default_rng(seed)
    n = ref.param_count(IO, C, len(dil))
    assert n == net.nparam
    theta = np.zeros(n)
    k = 0
    for ci, co in ref.layer_shapes(IO, C, len(dil)):
        theta[k:k + 9 * ci * co] = rng.standard_normal(9 * ci * co) * np.sqrt(1.0 / (9 * ci))
        k += 9 * ci * co
        theta[k:k + co] = 0.1 * rng.standard_normal(co)
        k += co
    theta = ref.round_bf16(theta.astype(np.float32))
    X = ref.round_bf16(rng.standard_normal((batch, 64, 64, IO)).astype(np.float32))
    T = rng.standard_normal((batch, 64, 64, IO))
    w = rng.random((batch, 64, 64))
    w /= w.sum()
    return theta, X, T, w


@pytest.mark.parametrize("C,dil,path", [(128, (1, 2), 0), (128, (1, 2), 1), (128, (1, 2), 2), (64, (3,), 0)])
def test_forward_matches_reference(C, dil, path):
    net = make(C, dil, 2, tensor_path=path)
    theta, X, _, _ = random_setup(net, C, dil, 2, 1)
    net.set_params(theta)
    y = net.forward(torch.tensor(X, dtype=torch.float32, device="cuda")).cpu().numpy()
    want, _ = ref.forward(theta, X, IO, C, len(dil), list(dil))
    assert rel(y, want) <= 3e-2, rel(y, want)
    net.close()


@pytest.mark.parametrize("C,dil,path", [(128, (1, 4), 0), (128, (1, 4), 1), (128, (1, 4), 2), (64, (2,), 0)])
def test_gradients_match_reference(C, dil, path):
    net = make(C, dil, 2, tensor_path=path)
    theta, X, T, w = random_setup(net, C, dil, 2, 2)
    net.set_params(theta)
    dev = lambda a: torch.tensor(a, dtype=torch.float32, device="cuda")
    loss, g = net.gradients(dev(X), dev(T), dev(w), out_ch=3)
    want_loss, want_g = ref.loss_and_grad(theta, X, T, w, 3, IO, C, len(dil), list(dil))
    assert abs(loss - want_loss) <= 3e-2 * want_loss
    k = 0
    for ci, co in ref.layer_shapes(IO, C, len(dil)):
        for size in (9 * ci * co, co):
            e = rel(g[k:k + size], want_g[k:k + size])
            assert e <= 6e-2, (ci, co, size, e)
            k += size
    net.close()


@pytest.mark.parametrize("path", [0, 1])
def test_tcgen05_and_mma_sync_paths_agree(path):
    """The 128 -> 128 convolutions on tcgen05 (operands staged by TMA, the
    default, or by cp.async) and on mma.sync give the same outputs and
    gradients up to the order of float summation and the rounding of the
    stored bfloat16 activations."""
    C, dil = 128, (1, 2, 4)
    nets = [make(C, dil, 2, tensor_path=t) for t in (2, path)]
    theta, X, T, w = random_setup(nets[0], C, dil, 2, 4)
    dev = lambda a: torch.tensor(a, dtype=torch.float32, device="cuda")
    outs, grads = [], []
    for net in nets:
        net.set_params(theta)
        outs.append(net.forward(dev(X)).cpu().numpy())
        grads.append(net.gradients(dev(X), dev(T), dev(w))[1])
        net.close()
    assert rel(outs[0], outs[1]) <= 1e-2, rel(outs[0], outs[1])
    assert rel(grads[0], grads[1]) <= 2e-2, rel(grads[0], grads[1])


def test_training_fits_a_small_set():
    C, dil = 64, (1, 2)
    net = make(C, dil, 4)
    rng = np.random.default_rng(3)
    X = torch.tensor(rng.standard_normal((4, 64, 64, IO)), dtype=torch.float32, device="cuda")
    # targets: a smooth function of the inputs
    T = torch.zeros_like(X)
    T[..., 0] = torch.tanh(X[..., 0] + 0.5 * X[..., 1])
    T[..., 1] = 0.5 * X[..., 2]
    w = torch.full((4, 64, 64), 1.0 / (4 * 64 * 64), device="cuda")
    first = net.train_step(X, T, w, 3e-3)
    for _ in range(150):
        last = net.train_step(X, T, w, 3e-3)
    assert last < 0.2 * first, (first, last)
    net.close()


def test_encode_and_decode_constant_fields():
    from paper_1902_02999_gb300.warmstart import lake_fields
    net = make(64, (1,), 1)
    case = inputs.dish_lake(256, seed=5)
    D, M = lake_fields(case, torch.device("cuda"))
    pitch = 256
    eta = torch.full((256, pitch), 0.25, dtype=torch.float32, device="cuda")
    u = torch.full_like(eta, -0.5)
    v = torch.full_like(eta, 2.0)
    scale = (2.0, 0.5, 1.0, 4.0)
    x, t, w = net.encode(D, M, case, scale, state=(eta.data_ptr(), u.data_ptr(), v.data_ptr(), pitch))
    frac = (case.mask != 0).reshape(64, 4, 64, 4).mean(axis=(1, 3))
    wn = w.cpu().numpy()
    assert np.allclose(wn, frac)
    tn = t.cpu().numpy()
    live = frac > 0
    assert np.allclose(tn[live, 0], 0.5) and np.allclose(tn[live, 1], -0.5) and np.allclose(tn[live, 2], 0.5)
    xn = x.cpu().numpy()
    assert np.allclose(xn[..., 0], frac) and np.allclose(xn[..., 2], case.wind_u / 5, atol=1e-6)
    assert np.allclose(xn[..., 7], case.dx / 2, rtol=1e-6)
    y = torch.zeros((64, 64, IO), dtype=torch.float32, device="cuda")
    y[..., 0], y[..., 1], y[..., 2] = 0.5, -0.5, 0.5
    h, uu, vv = (a.cpu().numpy() for a in net.decode(y, D, M, scale))
    Dn = case.h_ref - case.zb
    fl = case.mask == inputs.FLUID
    assert np.allclose(h[fl], Dn[fl] + 0.25, atol=1e-6)
    assert np.allclose(uu[fl], -0.5) and np.allclose(vv[fl], 2.0)
    assert (uu[case.mask == inputs.NOSLIP] == 0).all() and (uu[case.mask == 0] == 0).all()
    # volume constraint: eta shifted by one constant to sum to the target
    live = case.mask != 0
    Df = D.cpu().numpy().astype(np.float64)
    for target in (0.0, 3.0):
        h2 = net.decode(y, D, M, scale, target)[0].cpu().numpy()
        assert abs((h2 - Df)[live].sum() - target) <= 1e-9 * live.sum()
        d = (h2 - h)[live]
        assert np.allclose(d, d[0], rtol=0, atol=1e-12)
        assert (h2[~live] == h[~live]).all()
    net.close()


def test_warm_start_reaches_the_plain_accuracy_in_fewer_steps():
    """Train on 256 seeded lakes; on 8 unseen lakes the plain iteration from
    the network's proposal gets as close to the FP64 steady state (residual
    1e-11) as the iteration from rest gets at residual 1e-8, in fewer steps."""
    from paper_1902_02999_gb300.warmstart import WarmStartNet, compare, make_dataset, train
    net = WarmStartNet(res=64, channels=64, dilations=(1, 2, 4, 8, 16, 1), max_batch=16, seed=0)
    cases = [inputs.dish_lake(256, seed=2000 + k) for k in range(256)]
    X, T, W, scale, _ = make_dataset(net, cases, tol=1e-7, max_steps=80000, chunk=256)
    losses = train(net, X, T, W, epochs=12, batch=16, lr=2e-3)
    assert losses[-1] < 0.3 * losses[0]
    res = compare(net, [inputs.dish_lake(256, seed=k) for k in range(8)], scale, max_steps=200000)
    assert (res["plain_steps"] > 0).all() and (res["matched_steps"] > 0).all(), res
    assert np.median(res["matched_steps"]) < np.median(res["plain_steps"]), res
    assert (res["proposal_error"].max(axis=0) < 1.0).all()
    net.close()


def test_training_is_deterministic():
    """Split-K and block partial sums are added in a fixed order, so two
    networks trained from the same seed on the same data end bitwise equal,
    and a gradient evaluated twice is the same."""
    C, dil = 128, (1, 2)
    rng = np.random.default_rng(11)
    X = torch.tensor(rng.standard_normal((4, 64, 64, IO)), dtype=torch.float32, device="cuda")
    T = torch.tensor(rng.standard_normal((4, 64, 64, IO)), dtype=torch.float32, device="cuda")
    w = torch.full((4, 64, 64), 1.0 / (4 * 64 * 64), device="cuda")
    nets = [make(C, dil, 4, seed=5) for _ in range(2)]
    losses = []
    for net in nets:
        losses.append([net.train_step(X, T, w, 1e-3) for _ in range(4)])
    assert losses[0] == losses[1]
    assert np.array_equal(nets[0].get_params(), nets[1].get_params())
    g1 = nets[0].gradients(X, T, w)
    g2 = nets[0].gradients(X, T, w)
    assert g1[0] == g2[0] and np.array_equal(g1[1], g2[1])
    for net in nets:
        net.close()
